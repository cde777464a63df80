"""GPU parity of the differentiation path (transposed operator, transposed solve, boundary
derivatives, autograd) against the FP64 oracle, and against central finite differences of the
GPU solve itself.

Tolerances (relative, ‖gpu − oracle‖₂/‖oracle‖₂):
  Aᵀ application           1e-12 FP64, 2e-5 FP32 (the arithmetic of A's application, see the
                           operator parity tests).
  transposed solve         1e-10 FP64 (both sides solve to rtol 1e-13; the operator is well
                           conditioned, second kind); 1e-8 mixed (refinement to rtol 1e-11).
  boundary derivatives     1e-11 from the same (Q, λ): direct FP64 grid fields and gathers, whose
                           rounding is FFT rounding O(log N · 1e-16) times the O(1/h²) size of
                           ∇∇δ_h relative to the result.
  full gradient            1e-9 FP64 against the oracle's gradient (two solves at rtol 1e-13).
  finite differences       1e-6 relative (central differences, step 1e-6: truncation O(1e-12)
                           times third derivatives of size O(1/h³) ~ 1e-7 at h = 1/64, plus
                           solve tolerance 1e-13 / step 1e-6 = 1e-7).
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


def _perturbed_circle(N, M, delta, lam, seed, symbol="spectral", dipole="analytic"):
    """Circle points moved off grid lines (φ'' jumps there), tilted normals and uneven weights,
    so that every term of the boundary derivatives matters."""
    rng = np.random.default_rng(seed)
    bd = I.circle(M)
    h = 1.0 / N
    X = bd.X + 0.1 * h * rng.uniform(-1, 1, bd.X.shape)
    n = bd.n + 0.2 * rng.standard_normal(bd.n.shape)
    n = n / np.linalg.norm(n, axis=0)
    w = bd.w * (1 + 0.2 * rng.uniform(-1, 1, M))
    og = O.Geometry(O.Grid(2, N), X, n, w, delta, dipole, symbol, "scalar", lam)
    Ub = I.harmonic_cubic(X[0], X[1])
    return og, Ub, rng


def _gpu_geom(og):
    from paper_2210_07403_gb300 import Geometry

    return Geometry(og.X, og.n, og.w, og.grid.N, box=og.grid.box, origin=og.grid.origin, lam=og.lam,
                    delta=og.delta, dipole=og.dipole, symbol=og.symbol)


def _cuda(v):
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).cuda()


TRANSPOSE_CASES = [
    # N, M, delta, dipole, symbol, lam
    (16, 25, "cos", "analytic", "spectral", 0.0),
    (64, 100, "sqrt", "analytic", "fd2", 3.0),
    (64, 137, "sqrt", "spectral_div", "spectral", 0.0),
    (256, 403, "cos", "analytic", "spectral", 7.0),
]


@pytest.mark.parametrize("case", TRANSPOSE_CASES)
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32x2", 1e-12), ("fp32", 2e-5)])
def test_transpose_apply(case, precision, tol):
    N, M, delta, dipole, symbol, lam = case
    og, _, rng = _perturbed_circle(N, M, delta, lam, N + M, symbol, dipole)
    g = _gpu_geom(og)
    for _ in range(2):
        v = rng.standard_normal(M)
        z = g.apply_transpose(_cuda(v), precision=precision).cpu().numpy()
        assert _rel(z, O.transpose_apply(og, v)) < tol


def test_transpose_apply_is_transpose_of_apply():
    """⟨a, A b⟩ = ⟨Aᵀa, b⟩ on the GPU alone, at a size the oracle would take long to densify."""
    og, _, rng = _perturbed_circle(512, 800, "cos", 0.0, 5)
    g = _gpu_geom(og)
    a, b = rng.standard_normal(800), rng.standard_normal(800)
    Ab = g.apply(_cuda(b)).cpu().numpy()
    Ata = g.apply_transpose(_cuda(a)).cpu().numpy()
    assert abs(a @ Ab - Ata @ b) < 1e-12 * np.linalg.norm(a) * np.linalg.norm(Ab)


@pytest.mark.parametrize("precision,rtol,tol", [("fp64", 1e-13, 1e-10), ("mixed", 1e-11, 1e-8)])
def test_transpose_solve(precision, rtol, tol):
    og, _, rng = _perturbed_circle(64, 100, "sqrt", 2.0, 11)
    G = rng.standard_normal(100)
    ref = O.solve_transpose(og, G, 1e-13, maxit=200).x
    g = _gpu_geom(og)
    lam, info, _ = g.solve_transpose(_cuda(G), rtol=rtol, precision=precision, inner_rtol=1e-5)
    assert info["rel_residual"] <= rtol
    assert _rel(lam.cpu().numpy(), ref) < tol
    # graph path and host-driven path agree
    g.set_stage_timing(True)
    lam2, _, _ = g.solve_transpose(_cuda(G), rtol=rtol, precision=precision, inner_rtol=1e-5)
    g.set_stage_timing(False)
    assert _rel(lam2.cpu().numpy(), lam.cpu().numpy()) < (1e-12 if precision == "fp64" else 1e-9)


@pytest.mark.parametrize("delta,lam", [("sqrt", 2.0), ("cos", 0.0)])
def test_boundary_vjp_2d(delta, lam):
    og, Ub, rng = _perturbed_circle(64, 100, delta, lam, 3)
    Q = rng.standard_normal(100)
    L = rng.standard_normal(100)
    dX, dn, dw = O.param_gradient(og, Q, L)
    g = _gpu_geom(og)
    gX, gn, gw = g.solve_vjp(_cuda(Q), _cuda(L))
    # the entry point returns ∂J/∂p = −∂(λᵀAQ)/∂p
    assert _rel(gX.cpu().numpy(), -dX) < 1e-11
    assert _rel(gn.cpu().numpy(), -dn) < 1e-11
    assert _rel(gw.cpu().numpy(), -dw) < 1e-11
    # outputs not asked for are skipped; the spread accumulates with shared-memory atomics, so
    # two calls agree to rounding, not bit for bit
    gX2, gn2, gw2 = g.solve_vjp(_cuda(Q), _cuda(L), want=(True, False, False))
    assert gn2 is None and gw2 is None
    assert _rel(gX2.cpu().numpy(), gX.cpu().numpy()) < 1e-13


def test_boundary_vjp_3d():
    p = I.sphere_poisson(32, 700, delta="cos", lam=1.0)
    og = O.geometry_from_problem(p)
    rng = np.random.default_rng(4)
    og.X = og.X + 0.1 * og.grid.h * rng.uniform(-1, 1, og.X.shape)
    Q, L = rng.standard_normal(og.M), rng.standard_normal(og.M)
    dX, dn, dw = O.param_gradient(og, Q, L)
    from paper_2210_07403_gb300 import Geometry

    g = Geometry(og.X, og.n, og.w, 32, lam=1.0, delta="cos")
    gX, gn, gw = g.solve_vjp(_cuda(Q), _cuda(L))
    assert _rel(gX.cpu().numpy(), -dX) < 1e-11
    assert _rel(gn.cpu().numpy(), -dn) < 1e-11
    assert _rel(gw.cpu().numpy(), -dw) < 1e-11
    z = g.apply_transpose(_cuda(L)).cpu().numpy()
    assert _rel(z, O.transpose_apply(og, L)) < 1e-12


def _autograd_grads(og, Ub, gvec, precision="fp64", rtol=1e-13):
    from paper_2210_07403_gb300 import autograd as AG

    t = [_cuda(a).requires_grad_(True) for a in (Ub, og.X, og.n, og.w)]
    Q = AG.solve(*t, og.grid.N, lam=og.lam, delta=og.delta, symbol=og.symbol, rtol=rtol, precision=precision,
                 inner_rtol=1e-5)
    J = (Q * _cuda(gvec)).sum()
    J.backward()
    return Q.detach().cpu().numpy(), [a.grad.cpu().numpy() for a in t]


@pytest.mark.parametrize("delta,lam", [("sqrt", 2.0), ("cos", 0.0)])
def test_autograd_against_oracle_gradient(delta, lam):
    og, Ub, rng = _perturbed_circle(64, 100, delta, lam, 21)
    gvec = rng.standard_normal(100)
    Q, (dUb, dX, dn, dw) = _autograd_grads(og, Ub, gvec)
    Qr, dUr, dXr, dnr, dwr = O.solve_gradient(og, Ub, gvec)
    assert _rel(Q, Qr) < 1e-10
    assert _rel(dUb, dUr) < 1e-9
    assert _rel(dX, dXr) < 1e-9
    assert _rel(dn, dnr) < 1e-9
    assert _rel(dw, dwr) < 1e-9


def test_autograd_mixed_precision():
    og, Ub, rng = _perturbed_circle(64, 100, "cos", 1.0, 22)
    gvec = rng.standard_normal(100)
    _, (dUb, dX, dn, dw) = _autograd_grads(og, Ub, gvec, precision="mixed", rtol=1e-11)
    _, dUr, dXr, dnr, dwr = O.solve_gradient(og, Ub, gvec)
    for a, b in ((dUb, dUr), (dX, dXr), (dn, dnr), (dw, dwr)):
        assert _rel(a, b) < 1e-8


def test_autograd_against_finite_differences():
    """Central differences (step 1e-6) of J = gᵀQ computed by the GPU solve alone."""
    from paper_2210_07403_gb300 import Geometry

    og, Ub, rng = _perturbed_circle(64, 100, "sqrt", 2.0, 23)
    gvec = rng.standard_normal(100)
    _, (dUb, dX, dn, dw) = _autograd_grads(og, Ub, gvec)

    def J(ub=Ub, X=og.X, n=og.n, w=og.w):
        g = Geometry(X, n, w, og.grid.N, lam=og.lam, delta=og.delta)
        Q, _, _ = g.solve(_cuda(ub), rtol=1e-13, maxit=300)
        g.close()
        return float(gvec @ Q.cpu().numpy())

    e = 1e-6
    for i in rng.choice(100, 4, replace=False):
        d = np.zeros(100)
        d[i] = e
        assert (J(ub=Ub + d) - J(ub=Ub - d)) / (2 * e) == pytest.approx(dUb[i], rel=1e-6, abs=1e-9)
        assert (J(w=og.w + d) - J(w=og.w - d)) / (2 * e) == pytest.approx(dw[i], rel=1e-6, abs=1e-8)
        for m in range(2):
            D = np.zeros_like(og.X)
            D[m, i] = e
            assert (J(X=og.X + D) - J(X=og.X - D)) / (2 * e) == pytest.approx(dX[m, i], rel=1e-6, abs=1e-8)
        # the library takes unit normals only: rotate n_i by ±e, whose derivative is dn_i · t_i
        # with t_i = (−n_y, n_x) (the normal component of dn is covered by the oracle gradient)
        def rotated(th):
            n = og.n.copy()
            c, s_ = np.cos(th), np.sin(th)
            n[:, i] = (c * og.n[0, i] - s_ * og.n[1, i], s_ * og.n[0, i] + c * og.n[1, i])
            return n

        t = np.array([-og.n[1, i], og.n[0, i]])
        assert (J(n=rotated(e)) - J(n=rotated(-e))) / (2 * e) == pytest.approx(dn[:, i] @ t, rel=1e-6, abs=1e-8)


def test_gradient_error_paths():
    from paper_2210_07403_gb300 import Geometry, IbdlError

    og, _, rng = _perturbed_circle(64, 100, "cos", 0.0, 30, dipole="spectral_div")
    g = _gpu_geom(og)
    v = _cuda(rng.standard_normal(100))
    with pytest.raises(IbdlError, match="UNSUPPORTED"):
        g.solve_vjp(v, v)
    p = I.star_stokes(64, 100, dipole="spectral_div")
    gs = Geometry.from_problem(p)
    w = _cuda(rng.standard_normal(200))
    with pytest.raises(IbdlError, match="UNSUPPORTED"):
        gs.apply_transpose(w)
    with pytest.raises(IbdlError, match="UNSUPPORTED"):
        gs.solve_transpose(w)
    with pytest.raises(IbdlError, match="UNSUPPORTED"):
        gs.probe_vjp(np.full((2, 3), 0.5), w, _cuda(np.ones(6)))
    # overlapping outputs are rejected before any launch
    from paper_2210_07403_gb300 import ibdl

    og2, _, _ = _perturbed_circle(64, 100, "cos", 0.0, 31)
    g2 = _gpu_geom(og2)
    buf = torch.zeros(400, dtype=torch.float64, device="cuda")
    q = _cuda(rng.standard_normal(100))
    with pytest.raises(IbdlError, match="overlaps"):
        ibdl.ibdl_solve_vjp(g2.handle, q.data_ptr(), q.data_ptr(), buf.data_ptr(), buf.data_ptr() + 8 * 100, 0)


# ----------------------------------------------------------------------------------------
# Stokes and probes
# ----------------------------------------------------------------------------------------


def _perturbed_star(N, M, seed, tilt=0.2):
    p = I.star_stokes(N, M)
    og = O.geometry_from_problem(p)
    rng = np.random.default_rng(seed)
    og.X = og.X + 0.1 * og.grid.h * rng.uniform(-1, 1, og.X.shape)
    nn = og.n + tilt * rng.standard_normal(og.n.shape)
    og.n = nn / np.linalg.norm(nn, axis=0)
    og.w = og.w * (1 + 0.2 * rng.uniform(-1, 1, og.M))
    return og, p.Ub.reshape(-1), rng


def _gpu_stokes(og):
    from paper_2210_07403_gb300 import Geometry

    return Geometry(og.X, og.n, og.w, og.grid.N, pde="stokes", delta=og.delta, symbol=og.symbol)


@pytest.mark.parametrize("N,M,symbol", [(64, 100, "spectral"), (128, 230, "fd2"), (512, 800, "spectral")])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32x2", 1e-12), ("fp32", 2e-5)])
def test_stokes_transpose_apply(N, M, symbol, precision, tol):
    og, _, rng = _perturbed_star(N, M, N)
    og.symbol = symbol
    g = _gpu_stokes(og)
    v = rng.standard_normal(2 * M)
    z = g.apply_transpose(_cuda(v), precision=precision).cpu().numpy()
    assert _rel(z, O.transpose_apply(og, v)) < tol


@pytest.mark.parametrize("precision,rtol,tol", [("fp64", 1e-13, 1e-10), ("mixed", 1e-11, 1e-8)])
def test_stokes_transpose_solve(precision, rtol, tol):
    og, _, rng = _perturbed_star(64, 100, 12, tilt=0.0)
    G = rng.standard_normal(200)
    ref = O.solve_transpose(og, G, 1e-13, maxit=300).x
    g = _gpu_stokes(og)
    lam, info, _ = g.solve_transpose(_cuda(G), rtol=rtol, precision=precision, inner_rtol=1e-5, maxit=300)
    assert info["rel_residual"] <= rtol
    assert _rel(lam.cpu().numpy(), ref) < tol


def test_stokes_solve_vjp():
    og, _, rng = _perturbed_star(64, 100, 13)
    Q, L = rng.standard_normal(200), rng.standard_normal(200)
    dX, dn, dw = O.stokes_param_gradient(og, Q, L)
    gX, gn, gw = _gpu_stokes(og).solve_vjp(_cuda(Q), _cuda(L))
    assert _rel(gX.cpu().numpy(), -dX) < 1e-11
    assert _rel(gn.cpu().numpy(), -dn) < 1e-11
    assert _rel(gw.cpu().numpy(), -dw) < 1e-11


@pytest.mark.parametrize("pde", ["scalar", "stokes"])
def test_probe_evaluate_and_vjp(pde):
    if pde == "stokes":
        og, _, rng = _perturbed_star(64, 100, 14)
        g = _gpu_stokes(og)
        P = I.star_probes(9, 64, min_dist_h=2.0, seed=5)
    else:
        og, _, rng = _perturbed_circle(64, 100, "sqrt", 3.0, 14)
        g = _gpu_geom(og)
        P = 0.5 + 0.15 * rng.uniform(-1, 1, (2, 9))
    P[:, 0] = (0.25, 1.1)  # one probe outside the box: wraps periodically
    c = og.ncomp
    Q = rng.standard_normal(c * og.M)
    nu = rng.standard_normal((c, P.shape[1]))
    U = g.probe_evaluate(P, _cuda(Q)).cpu().numpy()
    assert _rel(U, O.probe_evaluate(og, P, Q)) < 1e-12
    ref = O.probe_vjp(og, P, Q, nu)
    got = g.probe_vjp(P, _cuda(Q), _cuda(nu))
    for a, b in zip(got, ref):
        assert _rel(a.cpu().numpy().reshape(-1), b.reshape(-1)) < 1e-11


def _probe_objective_grads(og, Ub, P, pde, rtol=1e-13, precision="fp64"):
    from paper_2210_07403_gb300 import autograd as AG

    t = [_cuda(a).requires_grad_(True) for a in (Ub, og.X, og.n, og.w)]
    b = AG.Boundary(*t[1:], og.grid.N, pde=pde, lam=og.lam, delta=og.delta, symbol=og.symbol)
    Q = b.solve(t[0], rtol=rtol, precision=precision, maxit=300)
    J = (b.probe(Q, P) ** 2).sum()
    J.backward()
    b.close()
    return float(J.detach()), [a.grad.cpu().numpy() for a in t]


def _oracle_probe_objective_grads(og, Ub, P):
    Q = O.solve(og, Ub, 1e-13, maxit=300).x
    U = O.probe_evaluate(og, P, Q)
    dQ, pX, pn, pw = O.probe_vjp(og, P, Q, 2 * U)
    _, dUb, sX, sn, sw = O.solve_gradient(og, Ub, dQ.reshape(-1))
    return float(np.sum(U ** 2)), [dUb, pX + sX, pn + sn, pw + sw]


@pytest.mark.parametrize("pde", ["scalar", "stokes"])
def test_probe_objective_autograd_against_oracle(pde):
    if pde == "stokes":
        og, Ub, rng = _perturbed_star(64, 100, 15)
        P = I.star_probes(8, 64, min_dist_h=2.0, seed=5)
    else:
        og, Ub, rng = _perturbed_circle(64, 100, "cos", 1.0, 15)
        P = 0.5 + 0.15 * rng.uniform(-1, 1, (2, 8))
    J, grads = _probe_objective_grads(og, Ub, P, pde)
    Jr, ref = _oracle_probe_objective_grads(og, Ub, P)
    assert J == pytest.approx(Jr, rel=1e-10)
    for a, b in zip(grads, ref):
        assert _rel(a.reshape(-1), b.reshape(-1)) < 1e-9


def test_stokes_probe_objective_against_finite_differences():
    """J = Σ_p |u(p)|² through the GPU solve alone: central differences (step 1e-6) in U_b and X."""
    from paper_2210_07403_gb300 import Geometry

    og, Ub, rng = _perturbed_star(64, 100, 16)
    P = I.star_probes(8, 64, min_dist_h=2.0, seed=5)
    _, (dUb, dX, dn, dw) = _probe_objective_grads(og, Ub, P, "stokes")

    def J(ub=Ub, X=og.X, n=og.n, w=og.w):
        g = Geometry(X, n, w, og.grid.N, pde="stokes", delta=og.delta)
        Q, _, _ = g.solve(_cuda(ub), rtol=1e-13, maxit=300)
        U = g.probe_evaluate(P, Q).cpu().numpy()
        g.close()
        return float(np.sum(U ** 2))

    e = 1e-6
    for i in rng.choice(100, 3, replace=False):
        for m in range(2):
            d = np.zeros(200)
            d[m * 100 + i] = e
            assert (J(ub=Ub + d) - J(ub=Ub - d)) / (2 * e) == pytest.approx(dUb[m * 100 + i], rel=1e-6, abs=1e-9)
            D = np.zeros_like(og.X)
            D[m, i] = e
            assert (J(X=og.X + D) - J(X=og.X - D)) / (2 * e) == pytest.approx(dX[m, i], rel=1e-6, abs=1e-8)
        d = np.zeros(100)
        d[i] = e
        assert (J(w=og.w + d) - J(w=og.w - d)) / (2 * e) == pytest.approx(dw[i], rel=1e-6, abs=1e-8)


def _normals_weights_torch(X):
    """Normals from centred differences of a closed counter-clockwise curve (Sec. 5.3.1) and
    Δs_i = ½(|X_{i+1} − X_i| + |X_i − X_{i−1}|), differentiable in torch."""
    d = torch.roll(X, -1, 1) - torch.roll(X, 1, 1)
    n = torch.stack([d[1], -d[0]]) / torch.linalg.norm(d, dim=0)
    fw = torch.linalg.norm(torch.roll(X, -1, 1) - X, dim=0)
    w = 0.5 * (fw + torch.roll(fw, 1, 0))
    return n, w


def test_total_derivative_with_normals_and_weights_from_points():
    """n and Δs computed from X in torch: autograd chains them into ∂J/∂X; checked against central
    differences of the whole pipeline (points → normals, weights → GPU solve → probes)."""
    from paper_2210_07403_gb300 import Geometry
    from paper_2210_07403_gb300 import autograd as AG

    rng = np.random.default_rng(17)
    bd = I.star(100)
    X0 = bd.X + 0.1 / 64 * rng.uniform(-1, 1, bd.X.shape)
    Ub = I.star_stokes(64, 100).Ub.reshape(-1)
    P = I.star_probes(8, 64, min_dist_h=2.0, seed=5)

    X = _cuda(X0).requires_grad_(True)
    n, w = _normals_weights_torch(X)
    b = AG.Boundary(X, n, w, 64, pde="stokes")
    J = (b.probe(b.solve(_cuda(Ub), rtol=1e-13, maxit=300), P) ** 2).sum()
    J.backward()
    dX = X.grad.cpu().numpy()

    def Jx(Xp):
        t = torch.from_numpy(Xp)
        nn, ww = _normals_weights_torch(t)
        g = Geometry(Xp, nn.numpy(), ww.numpy(), 64, pde="stokes")
        Q, _, _ = g.solve(_cuda(Ub), rtol=1e-13, maxit=300)
        v = float((g.probe_evaluate(P, Q) ** 2).sum())
        g.close()
        return v

    e = 1e-6
    for i in rng.choice(100, 3, replace=False):
        for m in range(2):
            D = np.zeros_like(X0)
            D[m, i] = e
            assert (Jx(X0 + D) - Jx(X0 - D)) / (2 * e) == pytest.approx(dX[m, i], rel=1e-6, abs=1e-8)


def test_stokes_probe_objective_full_size():
    """The 1024² star with 1600 points and 64 probes at ≥ 8h: GPU gradient against the oracle
    gradient on every entry (1e-8) and against central differences of the GPU solve on a sample.
    At h = 1/1024 the step e = 1e-6 is 1e-3 of a cell, and the central difference itself carries
    a relative truncation error of order (e/h)² ≈ 1e-6 times the third-derivative constant of δ_h
    (the oracle's own central differences here are off by up to 5.5e-6, the same at solve
    tolerances 1e-13 and 1e-15). So the plain difference is held to 1e-5, and the Richardson
    value (4D(e) − D(2e))/3, whose truncation is O((e/h)⁴), to 1e-6."""
    from paper_2210_07403_gb300 import Geometry

    p, P = I.star_stokes_probes()
    og = O.geometry_from_problem(p)
    Ub = p.Ub.reshape(-1)
    J, (dUb, dX, dn, dw) = _probe_objective_grads(og, Ub, P, "stokes", rtol=1e-12)
    Jr, ref = _oracle_probe_objective_grads(og, Ub, P)
    assert J == pytest.approx(Jr, rel=1e-9)
    for a, b in zip((dUb, dX, dn, dw), ref):
        assert _rel(a.reshape(-1), b.reshape(-1)) < 1e-8

    g = Geometry.from_problem(p)

    def Jx(X):
        gg = Geometry(X, og.n, og.w, 1024, pde="stokes", delta=og.delta)
        Q, _, _ = gg.solve(_cuda(Ub), rtol=1e-13, maxit=400)
        v = float((gg.probe_evaluate(P, Q) ** 2).sum())
        gg.close()
        return v

    rng = np.random.default_rng(6)
    e = 1e-6
    for i in rng.choice(og.M, 2, replace=False):
        for m in range(2):
            D = np.zeros_like(og.X)
            D[m, i] = e
            d1 = (Jx(og.X + D) - Jx(og.X - D)) / (2 * e)
            d2 = (Jx(og.X + 2 * D) - Jx(og.X - 2 * D)) / (4 * e)
            assert d1 == pytest.approx(dX[m, i], rel=1e-5, abs=1e-9)
            assert (4 * d1 - d2) / 3 == pytest.approx(dX[m, i], rel=1e-6, abs=1e-9)
    g.close()
