"""GPU parity of the source term g̃ (Sec. 5.1.2, Eq. "ibdl schur again"; Sec. 6.1.1) against the
FP64 oracle, through the C ABI (2-D scalar, Stokes and Brinkman; 3-D scalar): the forced field (ibdl_evaluate_field_forced) and the forced solve
(ibdl_solve_forced). Tolerances as for the operator: fields and right-hand sides 1e-12, FP64
solves 1e-10, mixed solves 1e-8."""
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


def _cuda(v):
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).cuda()


def _geom(p):
    from paper_2210_07403_gb300 import Geometry

    return Geometry.from_problem(p)


def _smooth_source(og, seed, mean=0.4):
    """A smooth periodic source on the box: a few random Fourier modes (|m| ≤ 4) plus a mean."""
    rng = np.random.default_rng(seed)
    x, y = og.grid.coords()
    L = og.grid.box
    out = []
    for _ in range(og.ncomp):
        f = np.full(x.shape, mean)
        for _ in range(6):
            mx, my = rng.integers(-4, 5, 2)
            a, ph = rng.standard_normal(), rng.uniform(0, 2 * np.pi)
            f = f + a * np.cos(2 * np.pi * (mx * x + my * y) / L + ph)
        out.append(f)
    return np.stack(out) if og.ncomp > 1 else out[0]


CASES = [
    ("scalar spectral", lambda: I.circle_laplace(64, 100)),
    ("scalar fd2 sqrt", lambda: I.circle_laplace(128, 200, delta="sqrt", symbol="fd2")),
    ("scalar screened", lambda: I.circle_laplace(64, 100, lam=7.0)),
    ("scalar spectral_div", lambda: I.circle_laplace(64, 100, dipole="spectral_div")),
    ("stokes", lambda: I.star_stokes(128, 200)),
    ("stokes spectral_div", lambda: I.star_stokes(64, 100, dipole="spectral_div")),
    ("brinkman", lambda: I.circle_brinkman(128, 200, lam=30.0, mu=0.7)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_forced_field(name, make):
    p = make()
    g, og = _geom(p), O.geometry_from_problem(p)
    src = _smooth_source(og, 11)
    rng = np.random.default_rng(3)
    Q = rng.standard_normal(og.ncomp * og.M)
    u = g.evaluate_field(_cuda(Q), g=_cuda(src)).cpu().numpy()
    assert _rel(u, O.forced_field(og, Q, src)) < 1e-12
    # without a source the call is the unforced one
    u0 = g.evaluate_field(_cuda(Q)).cpu().numpy()
    assert _rel(u0, O.grid_field(og, Q)) < 1e-12


@pytest.mark.parametrize("name,make", [CASES[0], CASES[2], CASES[4], CASES[6]], ids=["scalar", "screened", "stokes", "brinkman"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-8)])
def test_forced_solve(name, make, precision, tol):
    p = make()
    g, og = _geom(p), O.geometry_from_problem(p)
    src = _smooth_source(og, 12)
    ub = p.Ub.reshape(-1)
    ref = O.solve(og, O.forced_rhs(og, ub, src), 1e-13, maxit=200).x
    Q, info, st = g.solve(_cuda(ub), rtol=1e-12 if precision == "fp64" else 1e-10, precision=precision,
                          inner_rtol=1e-5, maxit=300, g=_cuda(src))
    assert st == 0
    assert _rel(Q.cpu().numpy(), ref) < tol


def test_forced_solve_host_buffers_and_field():
    """U_b and Q in host memory (io_on_host) with g̃ on the device; the forced field of the result
    against the oracle's."""
    p = I.circle_laplace(64, 100, lam=2.0)
    g, og = _geom(p), O.geometry_from_problem(p)
    src = _smooth_source(og, 13)
    ub = p.Ub.reshape(-1)
    Q, info, _ = g.solve(ub, rtol=1e-12, g=_cuda(src))
    assert not Q.is_cuda
    ref = O.solve(og, O.forced_rhs(og, ub, src), 1e-13).x
    assert _rel(Q.numpy(), ref) < 1e-10
    u = g.evaluate_field(Q.cuda(), g=_cuda(src)).cpu().numpy()
    assert _rel(u, O.forced_field(og, ref, src)) < 1e-10


def test_completed_body_force_through_the_source():
    """The cylinder array driven by its body force as a grid source (g̃ = (−1, 0) everywhere): the
    constraint rows come from h^d Σ g̃ and the drag equals the one from the hand-built right-hand
    side of the completed method."""
    p = I.cylinder_array(256, 0.2)
    g, og = _geom(p), O.geometry_from_problem(p)
    src = np.zeros((2,) + og.grid.shape)
    src[0] = -1.0
    b = np.concatenate([p.Ub.reshape(-1), p.meta["rhs_aug"]])
    x1, _, _ = g.solve(_cuda(b), rtol=1e-12, maxit=300)
    x2, _, _ = g.solve(_cuda(np.concatenate([p.Ub.reshape(-1), [5.0, 5.0]])), rtol=1e-12, maxit=300, g=_cuda(src))
    assert _rel(x2.cpu().numpy(), x1.cpu().numpy()) < 1e-10
    ref = O.solve(og, O.forced_rhs(og, b, src), 1e-12, maxit=300).x
    assert _rel(x2.cpu().numpy(), ref) < 1e-9


def _smooth_source_3d(og, seed, mean=0.3):
    rng = np.random.default_rng(seed)
    x, y, z = og.grid.coords()
    f = np.full(x.shape, mean)
    for _ in range(6):
        m = rng.integers(-3, 4, 3)
        f = f + rng.standard_normal() * np.cos(2 * np.pi * (m[0] * x + m[1] * y + m[2] * z) + rng.uniform(0, 6.3))
    return f


@pytest.mark.parametrize("lam", [0.0, 2.0])
def test_forced_3d(lam):
    """The scalar 3-D operator with a source: field 1e-12 and solve 1e-10 against the oracle."""
    p = I.sphere_poisson(32, 700, delta="cos", lam=lam)
    g, og = _geom(p), O.geometry_from_problem(p)
    src = _smooth_source_3d(og, 21)
    Q = np.random.default_rng(4).standard_normal(og.M)
    u = g.evaluate_field(_cuda(Q), g=_cuda(src)).cpu().numpy()
    assert _rel(u, O.forced_field(og, Q, src)) < 1e-12
    ub = p.Ub.reshape(-1)
    ref = O.solve(og, O.forced_rhs(og, ub, src), 1e-13, maxit=100).x
    x, info, st = g.solve(_cuda(ub), rtol=1e-12, g=_cuda(src))
    assert st == 0 and _rel(x.cpu().numpy(), ref) < 1e-10


def test_source_error_paths():
    from paper_2210_07403_gb300 import IbdlError, ibdl

    g2 = _geom(I.circle_laplace(32, 50))
    u = torch.zeros(32, 32, dtype=torch.float64, device="cuda")
    q = torch.zeros(50, dtype=torch.float64, device="cuda")
    with pytest.raises(IbdlError, match="INVALID_ARG"):  # u_grid aliases g_grid
        ibdl.ibdl_evaluate_field_forced(g2.handle, q.data_ptr(), u.data_ptr(), u.data_ptr())
    with pytest.raises(IbdlError, match="INVALID_ARG"):  # g_grid in host memory
        h = np.zeros(32 * 32)
        ibdl.ibdl_evaluate_field_forced(g2.handle, q.data_ptr(), h.ctypes.data, u.data_ptr())
