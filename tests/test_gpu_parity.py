"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element.

Tolerances (relative, ‖gpu − oracle‖₂/‖oracle‖₂ unless stated):
  FP64 grid arithmetic  1e-12 for one application (FFT rounding is O(log N · 1e-16) and the
                        operator norm is O(1)); 1e-10 for solves (the FP64 bound the method's
                        accuracy target states).
  FP32 grid arithmetic  2e-5 for one application (single-precision FFT rounding O(log N · 6e-8)
                        amplified by the O(10) ratio of ‖S̃‖‖L⁻¹‖‖S*‖ to ‖A‖).
  Float-float           1e-12 for one application, the FP64 bound (its FFT rounding is
                        O(log N · 2^−47), the point work is FP64).
Every comparison bounds both the relative 2-norm and the element-wise error max|Δ|/max|ref|.
  Mixed-precision solve 1e-8 against the oracle solution (refinement drives the FP64 residual
                        below rtol·‖U_b‖ with rtol chosen so that the error bound holds).
"""
import numpy as np
import pytest

import ibdl_inputs as I
from oracle import ibdl_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_07403_gb300 import build as b
    from paper_2210_07403_gb300 import ibdl

    b.build()
    ibdl.load()


def _rel(a, b):
    """The larger of the relative 2-norm error ‖a − b‖₂/‖b‖₂ and the element-wise error
    max|a − b|/max|b|, so every tolerance below bounds both (an error at a few points cannot hide
    in the norm)."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    d = np.abs(a - b)
    return float(max(np.linalg.norm(d) / np.linalg.norm(b), d.max() / np.abs(b).max()))


def _geom(p):
    from paper_2210_07403_gb300 import Geometry

    return Geometry.from_problem(p)


def _scalar_problem(N, M, delta="cos", dipole="analytic", symbol="spectral", lam=0.0, center=(0.5, 0.5),
                    R=0.25, box=1.0, origin=(0.0, 0.0)):
    bd = I.circle(M, R, center)
    Ub = I.harmonic_cubic(bd.X[0], bd.X[1], z0=center)[None, :]
    return I.Problem("t", 2, N, box, origin, bd, Ub, "scalar", lam=lam, delta=delta, dipole=dipole, symbol=symbol)


def _stokes_problem(N, M, delta="cos", dipole="analytic", symbol="spectral"):
    p = I.star_stokes(N, M, delta=delta, dipole=dipole, symbol=symbol)
    return p


SCALAR_CASES = [
    # N, M, delta, dipole, symbol, lam
    (16, 25, "cos", "analytic", "spectral", 0.0),
    (64, 100, "cos", "analytic", "spectral", 0.0),
    (64, 100, "sqrt", "analytic", "fd2", 3.0),
    (64, 137, "sqrt", "spectral_div", "spectral", 0.0),
    (128, 201, "cos", "spectral_div", "fd2", 50.0),
    (256, 403, "sqrt", "analytic", "spectral", 7.0),
]


@pytest.mark.parametrize("case", SCALAR_CASES)
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32x2", 1e-12), ("fp32", 2e-5)])
def test_scalar_apply(case, precision, tol):
    N, M, delta, dipole, symbol, lam = case
    p = _scalar_problem(N, M, delta, dipole, symbol, lam)
    g = _geom(p)
    og = O.geometry_from_problem(p)
    rng = np.random.default_rng(N + M)
    for _ in range(2):
        q = rng.standard_normal(M)
        y = g.apply(torch.from_numpy(q).cuda(), precision=precision).cpu().numpy()
        assert _rel(y, O.apply(og, q)) < tol


@pytest.mark.parametrize("dipole", ["analytic", "spectral_div"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32x2", 1e-12), ("fp32", 2e-5)])
def test_stokes_apply(dipole, precision, tol):
    p = _stokes_problem(128, 200, dipole=dipole)
    g = _geom(p)
    og = O.geometry_from_problem(p)
    q = np.random.default_rng(1).standard_normal(2 * p.bd.M)
    y = g.apply(torch.from_numpy(q).cuda(), precision=precision).cpu().numpy()
    assert _rel(y, O.apply(og, q)) < tol


def test_apply_wraps_periodically_and_ragged_point_counts():
    """Boundaries that cross the periodic box edge, a single point, and many points per cell."""
    for center, M in [((0.02, 0.97), 90), ((0.5, 0.5), 1), ((0.3, 0.6), 1000)]:
        p = _scalar_problem(32, M, "sqrt", "analytic", "spectral", 1.0, center=center, R=0.2)
        g = _geom(p)
        og = O.geometry_from_problem(p)
        q = np.random.default_rng(M).standard_normal(M)
        y = g.apply(torch.from_numpy(q).cuda()).cpu().numpy()
        assert _rel(y, O.apply(og, q)) < 1e-12


def test_apply_box_and_origin():
    """A non-unit box with the paper's centred origin (Sec. 2.2.1: [−L/2, L/2]²)."""
    bd = I.circle(150, 0.6, (0.0, 0.0))
    p = I.Problem("t", 2, 64, 2.0, (-1.0, -1.0), bd, np.sin(2 * bd.t)[None, :], "scalar", lam=1.0,
                  delta="sqrt", dipole="spectral_div", symbol="fd2")
    g = _geom(p)
    q = np.random.default_rng(3).standard_normal(150)
    y = g.apply(torch.from_numpy(q).cuda()).cpu().numpy()
    assert _rel(y, O.apply(O.geometry_from_problem(p), q)) < 1e-12


@pytest.mark.parametrize("pde", ["scalar", "stokes"])
def test_evaluate_field(pde):
    p = _scalar_problem(64, 100) if pde == "scalar" else _stokes_problem(64, 120)
    g = _geom(p)
    og = O.geometry_from_problem(p)
    q = np.random.default_rng(2).standard_normal(p.ncomp * p.bd.M)
    u = g.evaluate_field(torch.from_numpy(q).cuda()).cpu().numpy()
    ref = O.grid_field(og, q)
    assert u.shape == ref.shape
    assert _rel(u, ref) < 1e-12


@pytest.mark.parametrize("dipole", ["analytic", "spectral_div"])
def test_adjoint(dipole):
    p = _scalar_problem(64, 100, "sqrt", dipole, "spectral", 2.0)
    g = _geom(p)
    og = O.geometry_from_problem(p)
    w = np.random.default_rng(4).standard_normal(100)
    z = g.adjoint(torch.from_numpy(w).cuda()).cpu().numpy()
    assert _rel(z, O.adjoint_apply(og, w)) < 1e-12
    z32 = g.adjoint(torch.from_numpy(w).cuda(), precision="fp32").cpu().numpy()
    assert _rel(z32, O.adjoint_apply(og, w)) < 2e-5


def test_solve_circle_laplace_fp64():
    """The 64² circle workload: GMRES to 1e-10, same iteration count and Q as the oracle."""
    p = I.circle_laplace(64, 100)
    g = _geom(p)
    ref = O.solve(O.geometry_from_problem(p), p.Ub, 1e-10)
    Q, info, _ = g.solve(torch.from_numpy(p.Ub.reshape(-1)).cuda(), rtol=1e-10)
    assert info["iterations"] == ref.iterations
    assert _rel(Q.cpu().numpy(), ref.x) < 1e-10
    assert info["rel_residual"] <= 1e-10


def test_solve_paper_iteration_count():
    """The paper's circle Helmholtz problem (Sec. 5.4.1) needs 4 GMRES iterations at N = 256."""
    p = I.paper_circle_helmholtz(256, 1.0)
    g = _geom(p)
    Q, info, _ = g.solve(torch.from_numpy(p.Ub.reshape(-1)).cuda(), rtol=1e-8)
    assert info["iterations"] == 4
    ref = O.solve(O.geometry_from_problem(p), p.Ub, 1e-8)
    assert _rel(Q.cpu().numpy(), ref.x) < 1e-10


def test_solve_stokes_full_size_fp64_and_mixed():
    """The 512² Stokes star workload at full size: FP64 plain GMRES and mixed precision
    (FP32 applies, FP64 Arnoldi and refinement) against the oracle's solution."""
    p = I.star_stokes()
    g = _geom(p)
    g.autotune()  # the launch shapes bench.py times
    og = O.geometry_from_problem(p)
    ref = O.solve(og, p.Ub, 1e-12, maxit=80)
    ub = torch.from_numpy(p.Ub.reshape(-1)).cuda()
    Q64, info64, _ = g.solve(ub, rtol=1e-12, maxit=80)
    assert _rel(Q64.cpu().numpy(), ref.x) < 1e-10
    # mixed precision with the float-float refinement residual (the default) and with the FP64 one
    for residual in ("fp32x2", "fp64"):
        Qm, infom, _ = g.solve(ub, rtol=1e-10, precision="mixed", maxit=200, residual=residual)
        assert infom["rel_residual"] <= 1e-10
        assert _rel(Qm.cpu().numpy(), ref.x) < 1e-8
        assert infom["fp32_applies"] > infom["fp64_applies"] + infom["fp32x2_applies"]
        assert infom["fp32x2_applies" if residual == "fp32x2" else "fp64_applies"] == infom["sweeps"]
    # sampled operator outputs at full size, FP64 and float-float
    q = np.random.default_rng(5).standard_normal(2 * p.bd.M)
    for precision in ("fp64", "fp32x2"):
        y = g.apply(torch.from_numpy(q).cuda(), precision=precision).cpu().numpy()
        assert _rel(y, O.apply(og, q)) < 1e-12


def test_solve_host_driven_loop_matches_graph():
    """With stage timing on, GMRES runs from the host (one launch per kernel, events around
    each); the result must match the captured-graph cycle, and the stage record must count the
    kernels of every application."""
    p = I.star_stokes(128, 200)
    g = _geom(p)
    ub = torch.from_numpy(p.Ub.reshape(-1)).cuda()
    for prec in ("fp64", "mixed"):
        Qg, infog, _ = g.solve(ub, rtol=1e-10, precision=prec)
        g.set_stage_timing(True)
        g.stage_times()
        Qh, infoh, _ = g.solve(ub, rtol=1e-10, precision=prec)
        st = g.stage_times()
        g.set_stage_timing(False)
        assert infoh["iterations"] == infog["iterations"]
        # FP32 applications sum shared-memory atomics in a run-dependent order (~1e-7 relative
        # per application); two mixed solves each reach a residual ≤ 1e-10, so they agree to
        # κ(A)·1e-10 with κ(A) = O(10). FP64 applications differ at rounding level only.
        tol = 1e-12 if prec == "fp64" else 1e-9
        assert _rel(Qh.cpu().numpy(), Qg.cpu().numpy()) < tol
        assert st["arnoldi"][1] >= infoh["iterations"]
    ref = O.solve(O.geometry_from_problem(p), p.Ub, 1e-10)
    assert _rel(Qg.cpu().numpy(), ref.x) < 1e-8


def test_solve_restart_cycles():
    """A restart length shorter than the iteration count: several graph cycles, same answer."""
    p = I.star_stokes(128, 200)
    g = _geom(p)
    ub = torch.from_numpy(p.Ub.reshape(-1)).cuda()
    Q, info, _ = g.solve(ub, rtol=1e-10, restart=6, maxit=400)
    assert info["sweeps"] > 1
    ref = O.solve(O.geometry_from_problem(p), p.Ub, 1e-12)
    assert _rel(Q.cpu().numpy(), ref.x) < 1e-8


def test_mixed_solve_short_restart():
    """Mixed precision with a restart length shorter than an inner solve: a sweep whose inner cycle
    stops at the restart length is followed by a residual restart and does not count against
    max_refine, so the solve still reaches rtol (graph-driven and host-driven alike)."""
    p = I.star_stokes(128, 200)
    g = _geom(p)
    ub = torch.from_numpy(p.Ub.reshape(-1)).cuda()
    ref = O.solve(O.geometry_from_problem(p), p.Ub, 1e-12)
    for timing in (False, True):
        g.set_stage_timing(timing)
        Q, info, _ = g.solve(ub, rtol=1e-10, precision="mixed", restart=5, maxit=400, max_refine=3)
        assert info["rel_residual"] <= 1e-10
        assert info["sweeps"] > 3
        assert info["fp32x2_applies"] == info["sweeps"] and info["fp64_applies"] == 0
        assert _rel(Q.cpu().numpy(), ref.x) < 1e-8
    g.set_stage_timing(False)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_zero_rhs(precision):
    """U_b = 0: Q = 0 with a zero relative residual and no error, the norm of U_b taken from the
    first cycle on the device."""
    p = I.circle_laplace(64, 100)
    g = _geom(p)
    Q, info, st = g.solve(torch.zeros(100, dtype=torch.float64, device="cuda"), rtol=1e-10, precision=precision)
    assert st == 0 and info["rel_residual"] == 0.0
    assert float(Q.abs().max()) == 0.0


@pytest.mark.parametrize("N,pde,precision,tol", [(8192, "scalar", "fp64", 1e-12), (8192, "scalar", "fp32", 2e-5),
                                                   (4096, "scalar", "fp32x2", 1e-12), (4096, "stokes", "fp64", 1e-12),
                                                   (4096, "stokes", "fp32x2", 1e-12), (8192, "stokes", "fp32", 2e-5)])
def test_large_grids(N, pde, precision, tol):
    """The largest grids of each precision (one padded column or row pair per field in shared
    memory; threads holding several lanes): applications against the oracle at full size."""
    from paper_2210_07403_gb300 import Geometry

    M = I.points_for_spacing(2 * np.pi * 0.25, 1.0 / N, 1.0)
    bd = I.circle(M)
    og = O.Geometry(O.Grid(2, N), bd.X, bd.n, bd.w, "cos", "analytic", "spectral", pde, 0.0)
    g = Geometry(bd.X, bd.n, bd.w, N, pde=pde)
    q = np.random.default_rng(N).standard_normal(og.ncomp * M)
    y = g.apply(torch.from_numpy(q).cuda(), precision=precision).cpu().numpy()
    assert _rel(y, O.apply(og, q)) < tol
    g.close()


def test_grid_limits_are_refused():
    """Float-float is built to 4096²: at 8192² its applications return IBDL_ERR_UNSUPPORTED and
    no launch is made (FP64 and FP32 run there, one field per launch where the fields do not fit
    shared memory together: test_gpu_split.py)."""
    from paper_2210_07403_gb300 import Geometry, IbdlError

    N = 8192
    bd = I.circle(I.points_for_spacing(2 * np.pi * 0.25, 1.0 / N, 1.0))
    for pde, precision in (("stokes", "fp32x2"), ("scalar", "fp32x2")):
        g = Geometry(bd.X, bd.n, bd.w, N, pde=pde)
        q = torch.zeros(g.nd, dtype=torch.float64, device="cuda")
        with pytest.raises(IbdlError, match="UNSUPPORTED"):
            g.apply(q, precision=precision)
        g.close()


@pytest.mark.parametrize("case", ["star 512", "cylinder c=0.5", "star 256 restart 64", "circle restart 4"])
def test_true_residual_matches_the_estimate(case):
    """The Arnoldi basis stays orthonormal: an FP64 solve to rtol 1e-13 has a true relative residual
    ‖U_b − A Q‖/‖U_b‖ (recomputed with ibdl_apply) within 3e-13, so the GMRES residual estimate,
    which assumes an orthonormal basis, is not drifting. Covers long cycles and restarts."""
    if case == "star 512":
        p, kw = I.star_stokes(), {}
    elif case == "cylinder c=0.5":
        p, kw = I.cylinder_array(512, 0.5), {}
    elif case == "star 256 restart 64":
        p, kw = I.star_stokes(256, 400), {"restart": 64}
    else:
        p, kw = I.circle_laplace(64, 100), {"restart": 4}
    g = _geom(p)
    b = p.Ub.reshape(-1)
    if p.eta > 0:
        b = np.concatenate([b, p.meta["rhs_aug"]])
    bd = torch.from_numpy(b).cuda()
    Q, info, st = g.solve(bd, rtol=1e-13, maxit=400, **kw)
    assert st == 0 and info["rel_residual"] <= 1e-13
    r = bd - g.apply(Q)
    assert float(r.norm() / bd.norm()) < 3e-13, (info, float(r.norm() / bd.norm()))


def test_solve_host_buffers():
    p = I.circle_laplace(64, 100)
    g = _geom(p)
    Q, info, _ = g.solve(p.Ub.reshape(-1), rtol=1e-10)
    ref = O.solve(O.geometry_from_problem(p), p.Ub, 1e-10)
    assert not Q.is_cuda
    assert _rel(Q.numpy(), ref.x) < 1e-10


def test_error_paths():
    from paper_2210_07403_gb300 import ibdl

    p = I.circle_laplace(32, 50)
    g = _geom(p)
    q_host = torch.zeros(50, dtype=torch.float64)
    with pytest.raises(ibdl.IbdlError) as e:
        ibdl.ibdl_apply(g.handle, ibdl.IBDL_FP64, q_host.data_ptr(), q_host.data_ptr())
    assert e.value.status == ibdl.IBDL_ERR_INVALID_ARG
    ub = torch.from_numpy(p.Ub.reshape(-1)).cuda()
    bad = ub.clone()
    bad[3] = float("nan")
    _, _, st = g.solve(bad, check=False)
    assert st == ibdl.IBDL_ERR_NONFINITE
    Q, info, st = g.solve(ub, rtol=1e-12, maxit=1, check=False)
    assert st == ibdl.IBDL_ERR_NOT_CONVERGED and info["iterations"] == 1
    # the geometry is still usable afterwards
    Q, info, st = g.solve(ub, rtol=1e-8)
    assert st == ibdl.IBDL_OK
    with pytest.raises(ibdl.IbdlError):
        ibdl.ibdl_apply(g.handle, 7, ub.data_ptr(), Q.data_ptr())


# ----------------------------------------------------------------------------------------
# 3-D (scalar operator)
# ----------------------------------------------------------------------------------------


def _sphere_problem(N, delta="cos", dipole="analytic", lam=0.0, M=None):
    M = M or int(round(4 * np.pi * 0.25 ** 2 * N * N))
    return I.sphere_poisson(N, M, delta=delta, dipole=dipole, lam=lam)


@pytest.mark.parametrize("N,delta,dipole,lam", [(16, "cos", "analytic", 0.0), (32, "sqrt", "analytic", 5.0),
                                                (32, "cos", "spectral_div", 0.0), (16, "sqrt", "spectral_div", 2.0)])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32x2", 1e-12), ("fp32", 2e-5)])
def test_3d_apply(N, delta, dipole, lam, precision, tol):
    p = _sphere_problem(N, delta, dipole, lam)
    g = _geom(p)
    og = O.geometry_from_problem(p)
    q = np.random.default_rng(N).standard_normal(p.bd.M)
    y = g.apply(torch.from_numpy(q).cuda(), precision=precision).cpu().numpy()
    assert _rel(y, O.apply(og, q)) < tol
    # the Euclidean transpose Aᵀ = W A* W⁻¹ in the same arithmetic
    z = g.apply_transpose(torch.from_numpy(q).cuda(), precision=precision).cpu().numpy()
    assert _rel(z, O.transpose_apply(og, q)) < tol


def test_3d_field_and_adjoint():
    for dipole in ("analytic", "spectral_div"):
        p = _sphere_problem(16, "sqrt", dipole, 1.0)
        g = _geom(p)
        og = O.geometry_from_problem(p)
        q = np.random.default_rng(7).standard_normal(p.bd.M)
        u = g.evaluate_field(torch.from_numpy(q).cuda()).cpu().numpy()
        assert _rel(u, O.grid_field(og, q)) < 1e-12
        z = g.adjoint(torch.from_numpy(q).cuda()).cpu().numpy()
        assert _rel(z, O.adjoint_apply(og, q)) < 1e-12


def test_3d_solve_sphere():
    p = _sphere_problem(32)
    g = _geom(p)
    og = O.geometry_from_problem(p)
    ref = O.solve(og, p.Ub, 1e-10)
    Q, info, _ = g.solve(torch.from_numpy(p.Ub.reshape(-1)).cuda(), rtol=1e-10)
    assert info["iterations"] == ref.iterations
    assert _rel(Q.cpu().numpy(), ref.x) < 1e-10
    Qm, infom, _ = g.solve(torch.from_numpy(p.Ub.reshape(-1)).cuda(), rtol=1e-10, precision="mixed")
    assert _rel(Qm.cpu().numpy(), ref.x) < 1e-8
    assert infom["fp32x2_applies"] > 0 and infom["fp64_applies"] == 0  # the float-float residual


def test_3d_full_size_apply():
    """The 128³ sphere workload with 12 000 Fibonacci points: one FP64 and one float-float
    application."""
    p = I.sphere_poisson()
    g = _geom(p)
    q = np.random.default_rng(11).standard_normal(p.bd.M)
    ref = O.apply(O.geometry_from_problem(p), q)
    for prec in ("fp64", "fp32x2"):
        y = g.apply(torch.from_numpy(q).cuda(), precision=prec).cpu().numpy()
        assert _rel(y, ref) < 1e-12


@pytest.mark.parametrize("pde", ["scalar", "stokes"])
def test_autotune_keeps_parity(pde):
    """After the autotuner picks launch shapes, applications and solves still match the oracle."""
    p = _scalar_problem(128, 201, "sqrt", "analytic", "spectral", 2.0) if pde == "scalar" else _stokes_problem(128, 200)
    g = _geom(p)
    g.autotune()
    og = O.geometry_from_problem(p)
    q = np.random.default_rng(9).standard_normal(p.ncomp * p.bd.M)
    for prec, tol in (("fp64", 1e-12), ("fp32", 2e-5)):
        y = g.apply(torch.from_numpy(q).cuda(), precision=prec).cpu().numpy()
        assert _rel(y, O.apply(og, q)) < tol
    Q, info, _ = g.solve(torch.from_numpy(p.Ub.reshape(-1)).cuda(), rtol=1e-10)
    assert _rel(Q.cpu().numpy(), O.solve(og, p.Ub, 1e-12, maxit=80).x) < 1e-9


def test_applications_repeat():
    """Run to run: the spread sums shared-memory atomics and the gather adds partial sums with
    global atomics, in an order that varies between runs. Repeated applications of the 512² Stokes
    star still agree to rounding: 1e-13 in FP64 and float-float, 1e-6 in FP32 (relative 2-norm
    and element-wise)."""
    p = _stokes_problem(512, 800)
    g = _geom(p)
    q = torch.from_numpy(np.random.default_rng(11).standard_normal(2 * p.bd.M)).cuda()
    for precision, tol in (("fp64", 1e-13), ("fp32x2", 1e-13), ("fp32", 1e-6)):
        ys = [g.apply(q, precision=precision).cpu().numpy() for _ in range(4)]
        for y in ys[1:]:
            assert _rel(y, ys[0]) < tol, precision
