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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


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
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
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
    p = I.star_stokes(64, 100)
    gs = Geometry.from_problem(p)
    w = _cuda(rng.standard_normal(200))
    with pytest.raises(IbdlError, match="UNSUPPORTED"):
        gs.apply_transpose(w)
    with pytest.raises(IbdlError, match="UNSUPPORTED"):
        gs.solve_transpose(w)
    # overlapping outputs are rejected before any launch
    from paper_2210_07403_gb300 import ibdl

    og2, _, _ = _perturbed_circle(64, 100, "cos", 0.0, 31)
    g2 = _gpu_geom(og2)
    buf = torch.zeros(400, dtype=torch.float64, device="cuda")
    q = _cuda(rng.standard_normal(100))
    with pytest.raises(IbdlError, match="overlaps"):
        ibdl.ibdl_solve_vjp(g2.handle, q.data_ptr(), q.data_ptr(), buf.data_ptr(), buf.data_ptr() + 8 * 100, 0)
