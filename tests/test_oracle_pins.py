"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics (CPU only).

Each test checks the oracle against something other than itself: closed forms of the delta
kernels, discrete identities the paper states, brute-force evaluation on tiny inputs, an
independently assembled saddle-point system, manufactured solutions, and the GMRES iteration
counts the paper prints. A plausible slip anywhere in the oracle (a dropped term, a sign, an
index or transposition error) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import ibdl_inputs as I
from oracle import ibdl_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                a, b, c = line.split()
                rows.append((int(a), float(b), int(c)))
    return rows


# ----------------------------------------------------------------------------------------
# δ_h kernels (Sec. 2.2.2)
# ----------------------------------------------------------------------------------------

FRAC = np.linspace(0, 1, 97)[:-1]


@pytest.mark.parametrize("kind", ["sqrt", "cos"])
def test_phi_partition_moments(kind):
    phi, _ = O.KERNELS[kind]
    j = np.arange(-4, 5)[:, None]
    r = FRAC[None, :] - j
    v = phi(r)
    assert np.allclose(v.sum(0), 1.0, atol=1e-15)  # partition of unity
    even = v[(j[:, 0] % 2) == 0].sum(0)
    odd = v[(j[:, 0] % 2) == 1].sum(0)
    assert np.allclose(even, 0.5, atol=1e-15) and np.allclose(odd, 0.5, atol=1e-15)
    assert np.allclose((v * v).sum(0), 3.0 / 8.0, atol=1e-15)  # Σφ² = 3/8
    m1 = (r * v).sum(0)
    if kind == "sqrt":
        assert np.allclose(m1, 0.0, atol=1e-15)  # first moment vanishes
    else:
        # cosine kernel: Σ (r−j) φ(r−j) = f − ½ + ½(cos(πf/2) − sin(πf/2)), f = frac(r)
        ref = FRAC - 0.5 + 0.5 * (np.cos(np.pi * FRAC / 2) - np.sin(np.pi * FRAC / 2))
        assert np.allclose(m1, ref, atol=1e-15)
        assert 0.02 < np.abs(m1).max() < 0.022
    assert np.all(v >= 0)
    assert np.all(phi(np.array([2.0, -2.0, 2.5, 7.0])) == 0)


def test_phi_sqrt_values():
    # Closed-form values of the √-Peskin kernel.
    assert O.phi_sqrt(np.array([0.0]))[0] == pytest.approx(0.5, abs=1e-16)
    assert O.phi_sqrt(np.array([1.0]))[0] == pytest.approx(0.25, abs=1e-16)
    assert O.phi_sqrt(np.array([0.5]))[0] == pytest.approx((2 + math.sqrt(2)) / 8, abs=1e-16)
    assert O.phi_sqrt(np.array([1.5]))[0] == pytest.approx((2 - math.sqrt(2)) / 8, abs=1e-16)


@pytest.mark.parametrize("kind", ["sqrt", "cos"])
def test_dphi_is_derivative_and_c1(kind):
    phi, dphi = O.KERNELS[kind]
    r = np.linspace(-2.2, 2.2, 881)
    r = r[np.min(np.abs(r[:, None] - np.array([-2, -1, 0, 1, 2])[None, :]), 1) > 1e-3]
    e = 1e-6
    fd = (phi(r + e) - phi(r - e)) / (2 * e)
    assert np.allclose(dphi(r), fd, atol=1e-8)
    for k in (0.0, 1.0, 2.0):  # continuity of φ' at the piece boundaries
        for s in (1, -1):
            x = s * k
            assert dphi(np.array([x - 1e-9]))[0] == pytest.approx(dphi(np.array([x + 1e-9]))[0], abs=1e-6)
    assert dphi(np.array([0.0]))[0] == 0.0


# ----------------------------------------------------------------------------------------
# S, S*, S̃ (Sec. 2.2.2, Sec. 5.3.1)
# ----------------------------------------------------------------------------------------


def _tiny_geom(dim=2, N=12, M=17, delta="cos", seed=0, box=1.3, origin=None, **kw):
    rng = np.random.default_rng(seed)
    origin = origin if origin is not None else tuple(rng.uniform(-0.5, 0.5, dim))
    X = np.asarray(origin)[:, None] + rng.uniform(-0.5, 1.5, (dim, M)) * box  # some wrap around
    n = rng.standard_normal((dim, M))
    n /= np.linalg.norm(n, axis=0)
    w = rng.uniform(0.5, 1.5, M) * box / N
    return O.Geometry(O.Grid(dim, N, box, origin), X, n, w, delta, **kw)


def _brute_delta(geom, which="phi"):
    """Dense matrix D[g, i] = δ_h(x_g − X_i) (or ∂_m δ_h) evaluated over every node with the
    periodic minimum image: independent of the oracle's stencil bookkeeping."""
    g = geom.grid
    phi, dphi = O.KERNELS[geom.delta]
    coords = [c.reshape(-1) for c in g.coords()]
    L = g.box
    diffs = []
    for j in range(g.dim):
        dj = coords[j][:, None] - geom.X[j][None, :]
        dj = dj - L * np.round(dj / L)
        diffs.append(dj / g.h)
    if which == "phi":
        out = np.ones_like(diffs[0])
        for j in range(g.dim):
            out = out * phi(diffs[j])
        return out / g.h ** g.dim
    grads = []
    for m in range(g.dim):
        out = np.ones_like(diffs[0])
        for j in range(g.dim):
            out = out * (dphi(diffs[j]) / g.h if j == m else phi(diffs[j]))
        grads.append(out / g.h ** g.dim)
    return grads


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("delta", ["sqrt", "cos"])
def test_spread_interp_bruteforce(dim, delta):
    geom = _tiny_geom(dim=dim, N=10 if dim == 2 else 7, M=13, delta=delta, seed=dim)
    D = _brute_delta(geom)
    rng = np.random.default_rng(7)
    F = rng.standard_normal(geom.M)
    u = rng.standard_normal(geom.grid.shape)
    assert np.allclose(O.spread(geom, F).reshape(-1), D @ (F * geom.w), rtol=1e-13, atol=1e-12)
    assert np.allclose(O.interp(geom, u), geom.grid.h ** dim * (D.T @ u.reshape(-1)), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_spread_grad_bruteforce(dim):
    geom = _tiny_geom(dim=dim, N=9 if dim == 2 else 7, M=11, delta="sqrt", seed=5)
    G = _brute_delta(geom, "grad")
    rng = np.random.default_rng(8)
    V = rng.standard_normal((dim, geom.M))
    ref = sum(G[m] @ (V[m] * geom.w) for m in range(dim))
    assert np.allclose(O.spread_grad(geom, V).reshape(-1), ref, rtol=1e-12, atol=1e-10)
    u = rng.standard_normal(geom.grid.shape)
    ref2 = np.stack([geom.grid.h ** dim * (G[m].T @ u.reshape(-1)) for m in range(dim)])
    assert np.allclose(O.interp_grad(geom, u), ref2, rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("delta", ["sqrt", "cos"])
def test_dipole_is_derivative_in_point_position(delta):
    """∇_x δ_h(x − X) = −∇_X δ_h(x − X): S̃Q = ∇·S(Qn) equals minus the derivative of the
    ordinary spread of Q when every point moves along its normal (central difference)."""
    geom = _tiny_geom(N=16, M=21, delta=delta, seed=3)
    rng = np.random.default_rng(4)
    Q = rng.standard_normal(geom.M)
    eps = 1e-5 * geom.grid.h

    def moved(s):
        gg = O.Geometry(geom.grid, geom.X + s * eps * geom.n, geom.n, geom.w, delta)
        return O.spread(gg, Q)

    fd = -(moved(1) - moved(-1)) / (2 * eps)
    an = O.dipole_field(geom, Q)
    assert np.allclose(an, fd, rtol=1e-6, atol=1e-6 * np.abs(an).max())


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("delta", ["sqrt", "cos"])
def test_adjointness_and_conservation(dim, delta):
    """⟨SF, u⟩_h = ⟨F, S*u⟩_w (Sec. 2.1; discrete form Sec. 2.2.4), S*1 = 1, ∫SF = Σ Δs F."""
    geom = _tiny_geom(dim=dim, N=16 if dim == 2 else 8, M=40, delta=delta, seed=11)
    rng = np.random.default_rng(12)
    F = rng.standard_normal(geom.M)
    u = rng.standard_normal(geom.grid.shape)
    h = geom.grid.h
    lhs = h ** dim * np.sum(O.spread(geom, F) * u)
    rhs = np.sum(geom.w * F * O.interp(geom, u))
    assert lhs == pytest.approx(rhs, rel=1e-13)
    assert np.allclose(O.interp(geom, np.ones(geom.grid.shape)), 1.0, atol=1e-14)
    assert h ** dim * O.spread(geom, F).sum() == pytest.approx(np.sum(geom.w * F), rel=1e-13)
    V = rng.standard_normal((dim, geom.M))
    lhs = h ** dim * np.sum(O.spread_grad(geom, V) * u)
    rhs = np.sum(geom.w * V * O.interp_grad(geom, u))
    assert lhs == pytest.approx(rhs, rel=1e-12)


# ----------------------------------------------------------------------------------------
# Fourier symbols and the periodic solve (Sec. 2.2.1, Sec. 2.2.4, Sec. 2.3.1)
# ----------------------------------------------------------------------------------------


def _lap5(u, h):
    """5-point Laplacian (Sec. 2.2.1) by periodic shifts, any dimension."""
    out = -2 * u.ndim * u
    for ax in range(u.ndim):
        out = out + np.roll(u, 1, ax) + np.roll(u, -1, ax)
    return out / h ** 2


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("lam", [0.0, 7.5])
def test_fd2_solve_inverts_five_point_stencil(dim, lam):
    g = O.Grid(dim, 16 if dim == 2 else 8, 1.7, (0.1,) * dim)
    geom = O.Geometry(g, np.zeros((dim, 1)), np.ones((dim, 1)), np.ones(1), symbol="fd2", lam=lam)
    rng = np.random.default_rng(1)
    f = rng.standard_normal(g.shape)
    if lam == 0.0:
        f -= f.mean()  # solvability for the periodic Laplacian
    v = O.minus_Linv(geom, f)
    # −(Δ − λ) v = f  ⇔  v = −L⁻¹ f
    assert np.allclose(-(_lap5(v, g.h) - lam * v), f, atol=1e-10 * np.abs(f).max())
    if lam == 0.0:
        assert abs(v.mean()) < 1e-13  # Δ₀⁻¹ returns the mean-zero solution


@pytest.mark.parametrize("lam", [0.0, 3.0])
def test_spectral_solve_single_modes(lam):
    """On a Fourier mode cos(k·x + c) the spectral solve divides by |k|² + λ exactly."""
    g = O.Grid(2, 16, 2.0, (-1.0, -1.0))
    geom = O.Geometry(g, np.zeros((2, 1)), np.ones((2, 1)), np.ones(1), lam=lam)
    x, y = g.coords()
    for mx, my in [(1, 0), (0, 3), (2, -5), (7, 7), (3, 1)]:
        kx, ky = 2 * np.pi * mx / g.box, 2 * np.pi * my / g.box
        f = np.cos(kx * x + ky * y + 0.3)
        assert np.allclose(O.minus_Linv(geom, f), f / (kx * kx + ky * ky + lam), atol=1e-14)
    assert np.allclose(O.minus_Linv(geom, np.ones(g.shape)), 0.0 if lam == 0 else 1.0 / max(lam, 1))


def test_derivative_symbols():
    """Spectral ∂_x of sin(kx) is k cos(kx) except at the Nyquist mode (set to zero);
    the fd2 symbol reproduces the centred difference."""
    g = O.Grid(2, 16, 1.0)
    x, y = g.coords()
    _, der = O.symbols(g, "spectral")
    for m in (1, 3, 7):
        k = 2 * np.pi * m
        got = np.real(np.fft.ifftn(der[0] * np.fft.fftn(np.sin(k * x + 0.2))))
        assert np.allclose(got, k * np.cos(k * x + 0.2), atol=1e-11)
        got = np.real(np.fft.ifftn(der[1] * np.fft.fftn(np.sin(k * y))))
        assert np.allclose(got, k * np.cos(k * y), atol=1e-11)
    nyq = np.cos(np.pi * 16 * x)  # the m = N/2 mode
    assert np.allclose(np.real(np.fft.ifftn(der[0] * np.fft.fftn(nyq))), 0.0, atol=1e-12)
    _, derf = O.symbols(g, "fd2")
    u = np.random.default_rng(0).standard_normal(g.shape)
    cd = (np.roll(u, -1, 1) - np.roll(u, 1, 1)) / (2 * g.h)
    assert np.allclose(np.real(np.fft.ifftn(derf[0] * np.fft.fftn(u))), cd, atol=1e-12)


# ----------------------------------------------------------------------------------------
# operator-level pins (Sec. 3, Sec. 5.3)
# ----------------------------------------------------------------------------------------


def _circle_geom(N, delta="sqrt", lam=0.0, dipole="analytic", symbol="spectral", alpha=1.0):
    M = I.points_for_spacing(2 * np.pi * 0.25, 1.0 / N, alpha)
    bd = I.circle(M)
    return O.Geometry(O.Grid(2, N), bd.X, bd.n, bd.w, delta, dipole, symbol, "scalar", lam), bd


@pytest.mark.parametrize("delta", ["sqrt", "cos"])
def test_constant_density_jump(delta):
    """Q ≡ 1: u = −Δ₀⁻¹S̃1 approximates χ_Ω − |Ω|/|C| (the indicator construction of
    Sec. 5.3.5 via the Green's-derivative identity of Sec. 3), so S*u → ½ − |Ω|/|C| and
    A·1 → 1 − |Ω|/|C| (= 1 − π/16 for the circle), at first order in h."""
    target = 1 - math.pi / 16
    errs = []
    for N in (32, 64, 128):
        geom, bd = _circle_geom(N, delta)
        errs.append(abs(O.apply(geom, np.ones(bd.M)).mean() - target))
        if N == 128:
            u = O.field_scalar(geom, np.ones(bd.M))
            x, y = geom.grid.coords()
            r = np.hypot(x - 0.5, y - 0.5)
            # the cosine kernel's non-zero first moment shifts the plateaus by O(h)
            tol = 1e-3 if delta == "sqrt" else 2e-2
            assert np.allclose(u[r < 0.15], 1 - math.pi / 16, atol=tol)
            assert np.allclose(u[r > 0.4], -math.pi / 16, atol=tol)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.015
    assert O.fitted_order([1 / 32, 1 / 64, 1 / 128], errs) > 0.7


def test_circle_mode_one_periodic_correction():
    """For Q = cos θ on the circle, the free-space double layer gives A Q = ½Q (the PV
    integral of ∇G·n is constant on a circle, Sec. 3). The mean-zero periodic Green's function
    adds |x|²/(4|C|), whose double-layer potential on the circle is (|Ω|/(2|C|)) cos θ, so the
    cos θ coefficient of A Q tends to ½ + π/32; the m = 3 diagonal tends to ½."""
    e1, e3 = [], []
    for N in (64, 128, 256):
        geom, bd = _circle_geom(N)
        th = bd.t
        c1 = 2 * np.mean(O.apply(geom, np.cos(th)) * np.cos(th))
        c3 = 2 * np.mean(O.apply(geom, np.cos(3 * th)) * np.cos(3 * th))
        e1.append(abs(c1 - (0.5 + math.pi / 32)))
        e3.append(abs(c3 - 0.5))
    assert e1[0] > e1[1] > e1[2] and e1[2] < 6e-3
    assert e3[0] > e3[1] > e3[2] and e3[2] < 6e-3


@pytest.mark.parametrize("delta,lam,dipole", [("sqrt", 0.0, "analytic"), ("cos", 3.0, "analytic"),
                                              ("cos", 0.0, "spectral_div")])
def test_gmres_matches_dense_lu(delta, lam, dipole):
    geom, bd = _circle_geom(32, delta, lam, dipole)
    Ub = I.harmonic_cubic(bd.X[0], bd.X[1])
    A = O.dense_operator(geom)
    q_lu = np.linalg.solve(A, Ub)
    res = O.solve(geom, Ub, 1e-14, maxit=bd.M)
    assert np.linalg.norm(res.x - q_lu) <= 1e-11 * np.linalg.norm(q_lu)
    assert res.true_rel_residual < 1e-12


@pytest.mark.parametrize("dipole", ["analytic", "spectral_div"])
def test_saddle_system_dense(dipole):
    """Assemble the un-reduced IBDL system [[L, S̃], [S*, ½I]] (Sec. 5.3.2) densely on a 16²
    grid from stencils and brute-force kernel evaluations (5-point Laplacian, centred
    differences; no FFT), solve it by LU, and compare Q and u with the oracle's GMRES on the
    Schur operator and its grid field."""
    N, lam = 16, 2.0
    geom, bd = _circle_geom(N, "sqrt", lam, dipole, "fd2", alpha=1.5)
    g = geom.grid
    n2 = N * N
    eye = np.eye(n2).reshape((n2,) + g.shape)
    Lmat = np.stack([(_lap5(e, g.h) - lam * e).reshape(-1) for e in eye], axis=1)
    D = _brute_delta(geom)  # (n2, M)
    if dipole == "analytic":
        G = _brute_delta(geom, "grad")
        St = sum(G[m] * (geom.w * geom.n[m])[None, :] for m in range(2))
    else:
        def cdiff(u, ax):
            return (np.roll(u, -1, ax) - np.roll(u, 1, ax)) / (2 * g.h)
        St = np.zeros((n2, bd.M))
        for m, ax in ((0, 1), (1, 0)):
            cols = (D * (geom.w * geom.n[m])[None, :]).T.reshape((bd.M,) + g.shape)
            St += np.stack([cdiff(c, ax).reshape(-1) for c in cols], axis=1)
    Sstar = g.h ** 2 * D.T
    K = np.block([[Lmat, St], [Sstar, 0.5 * np.eye(bd.M)]])
    Ub = np.sin(2 * bd.t)
    sol = np.linalg.solve(K, np.concatenate([np.zeros(n2), Ub]))
    u_lu, q_lu = sol[:n2], sol[n2:]
    res = O.solve(geom, Ub, 1e-14, maxit=bd.M)
    assert np.allclose(res.x, q_lu, rtol=0, atol=1e-10 * np.abs(q_lu).max())
    assert np.allclose(O.field_scalar(geom, res.x).reshape(-1), u_lu, atol=1e-10 * np.abs(u_lu).max())


def test_null_vector_of_unreduced_system():
    """(u, Q) = (χ_{C∖Ω}, −1) is in the null space of [[Δ, S̃], [S*, ½I]] (Sec. 5.3.3): with the
    mean-zero inverse, u = −Δ₀⁻¹S̃(−1) equals χ_{C∖Ω} up to a constant and the regularisation
    error, and S*(χ_{C∖Ω}) + ½(−1) ≈ 0 on Γ."""
    geom, bd = _circle_geom(128)
    u = O.field_scalar(geom, -np.ones(bd.M))
    x, y = geom.grid.coords()
    r = np.hypot(x - 0.5, y - 0.5)
    outside = u[r > 0.4].mean()
    inside = u[r < 0.15].mean()
    assert outside - inside == pytest.approx(1.0, abs=5e-3)
    chi = u - inside  # ≈ χ_{C∖Ω}
    assert np.allclose(O.interp(geom, chi) - 0.5, 0.0, atol=2e-2)


@pytest.mark.parametrize("dipole", ["analytic", "spectral_div"])
def test_adjoint_identity(dipole):
    geom, bd = _circle_geom(32, "cos", 2.0, dipole)
    rng = np.random.default_rng(3)
    Q, W = rng.standard_normal(bd.M), rng.standard_normal(bd.M)
    lhs = np.sum(bd.w * O.apply(geom, Q) * W)
    rhs = np.sum(bd.w * Q * O.adjoint_apply(geom, W))
    assert lhs == pytest.approx(rhs, rel=1e-12)


# ----------------------------------------------------------------------------------------
# the paper's printed numbers and manufactured solutions
# ----------------------------------------------------------------------------------------


@pytest.mark.parametrize("row", _golden("ibdl_iterations_circle_helmholtz.txt"))
def test_paper_iteration_table(row):
    N, alpha, its = row
    p = I.paper_circle_helmholtz(N, alpha)
    res = O.solve(O.geometry_from_problem(p), p.Ub, 1e-8)
    assert res.iterations == its


@pytest.mark.parametrize("row", _golden("ibdl_iterations_tol1e-10.txt"))
def test_paper_iterations_tight_tolerance(row):
    N, alpha, its = row
    p = I.paper_circle_helmholtz(N, alpha)
    res = O.solve(O.geometry_from_problem(p), p.Ub, 1e-10)
    assert abs(res.iterations - its) <= 1


def test_first_order_convergence_paper_helmholtz():
    """u = I₂(r) sin 2θ / I₂(0.25) solves the paper's circle Helmholtz problem (Sec. 5.4.1);
    away from Γ the IBDL grid solution converges at first order."""
    special = pytest.importorskip("scipy.special")
    errs, hs = [], []
    for N in (64, 128, 256):
        p = I.paper_circle_helmholtz(N, 1.0)
        geom = O.geometry_from_problem(p)
        q = O.solve(geom, p.Ub, 1e-10).x
        u = O.field_scalar(geom, q)
        x, y = geom.grid.coords()
        r = np.hypot(x, y)
        ex = special.iv(2, r) * np.sin(2 * np.arctan2(y, x)) / special.iv(2, 0.25)
        errs.append(np.abs(u - ex)[r < 0.15].max())
        hs.append(1.0 / N)
    assert O.fitted_order(hs, errs) > 0.85


@pytest.mark.parametrize("delta", ["cos", "sqrt"])
def test_harmonic_cubic_converges(delta):
    """The workload's Laplace problem, u = Re((z − z0)^3): interior error decreases with h."""
    errs = []
    for N in (32, 64, 128):
        p = I.circle_laplace(N, I.points_for_spacing(2 * np.pi * 0.25, 1.0 / N), delta=delta)
        geom = O.geometry_from_problem(p)
        res = O.solve(geom, p.Ub, 1e-10)
        assert res.iterations <= 8
        u = O.field_scalar(geom, res.x)
        x, y = geom.grid.coords()
        r = np.hypot(x - 0.5, y - 0.5)
        errs.append(np.abs(u - I.harmonic_cubic(x, y))[r < 0.15].max())
    assert errs[0] > errs[1] > errs[2]
    assert O.fitted_order([1 / 32, 1 / 64, 1 / 128], errs) > 0.4


# ----------------------------------------------------------------------------------------
# Stokes (Sec. 6.1, Sec. 6.3.3)
# ----------------------------------------------------------------------------------------


def _stokes_geom(N, delta="sqrt", dipole="analytic", symbol="spectral"):
    M = I.points_for_spacing(2 * np.pi * 0.25, 1.0 / N)
    bd = I.circle(M)
    return O.Geometry(O.Grid(2, N), bd.X, bd.n, bd.w, delta, dipole, symbol, "stokes"), bd


@pytest.mark.parametrize("dipole", ["analytic", "spectral_div"])
def test_stokes_velocity_satisfies_pde(dipole):
    """The velocity returned for a density satisfies, mode by mode away from Nyquist, the
    discrete equations of Sec. 6.1.1: ∇·u + S(Q·n) = 0 and Δu + ∇·(S A) = ∇p for some p
    (a gradient ⇔ zero discrete curl), with mean-zero u."""
    geom, bd = _stokes_geom(32, dipole=dipole)
    g = geom.grid
    rng = np.random.default_rng(9)
    Q = rng.standard_normal((2, bd.M))
    u = O.stokes_velocity(geom, Q.reshape(-1))
    lap, der = O.symbols(g, "spectral")
    Uh = [np.fft.fftn(u[0]), np.fft.fftn(u[1])]
    sh = np.fft.fftn(O.spread(geom, np.sum(Q * bd.n, 0)))
    A = [[Q[l] * bd.n[m] + Q[m] * bd.n[l] for m in range(2)] for l in range(2)]
    if dipole == "analytic":
        gh = [np.fft.fftn(O.spread_grad(geom, np.array(A[l]))) for l in range(2)]
    else:
        gh = [sum(der[m] * np.fft.fftn(O.spread(geom, A[l][m])) for m in range(2)) for l in range(2)]
    kx = np.broadcast_to(np.fft.fftfreq(32, 1 / 32)[None, :], g.shape)
    ky = np.broadcast_to(np.fft.fftfreq(32, 1 / 32)[:, None], g.shape)
    ok = (np.abs(kx) != 16) & (np.abs(ky) != 16) & (lap != 0)
    div = der[0] * Uh[0] + der[1] * Uh[1] + sh
    assert np.abs(div[ok]).max() < 1e-9 * np.abs(sh).max()
    mom = [-lap * Uh[l] + gh[l] for l in range(2)]
    curl = der[0] * mom[1] - der[1] * mom[0]
    assert np.abs(curl[ok]).max() < 1e-9 * np.abs(gh[0]).max() * 2 * np.pi * 16
    assert abs(u[0].mean()) < 1e-14 and abs(u[1].mean()) < 1e-14


@pytest.mark.parametrize("flow", ["poly", "rotation"])
def test_stokes_first_order(flow):
    fn = I.stokes_poly if flow == "poly" else I.rigid_rotation
    errs = []
    for N in (64, 128, 256):
        geom, bd = _stokes_geom(N)
        Ub = fn(bd.X[0], bd.X[1])
        res = O.solve(geom, Ub, 1e-10, maxit=60)
        assert res.iterations <= 14  # Sec. 6.4.1 reports 9-10 for the Brinkman analogue
        u = O.stokes_velocity(geom, res.x)
        x, y = geom.grid.coords()
        r = np.hypot(x - 0.5, y - 0.5)
        errs.append(np.abs(u - fn(x, y)).max(0)[r < 0.15].max())
    assert O.fitted_order([1 / 64, 1 / 128, 1 / 256], errs) > 0.85


def test_stokes_gmres_matches_dense_lu():
    geom, bd = _stokes_geom(32)
    Ub = I.stokes_poly(bd.X[0], bd.X[1]).reshape(-1)
    A = O.dense_operator(geom)
    q_lu = np.linalg.solve(A, Ub)
    res = O.solve(geom, Ub, 1e-13, maxit=2 * bd.M)
    assert np.linalg.norm(res.x - q_lu) <= 1e-9 * np.linalg.norm(q_lu)


# ----------------------------------------------------------------------------------------
# 3-D
# ----------------------------------------------------------------------------------------


def test_sphere_harmonic_converges():
    """The 3-D workload's problem on coarse grids: x² − y² + z(x − 0.5) is harmonic, and the
    interior error of the IBDL solution decreases as the grid is refined."""
    errs = []
    for N in (16, 24, 32):
        M = int(round(4 * np.pi * 0.25 ** 2 * N * N))
        p = I.sphere_poisson(N, M)
        geom = O.geometry_from_problem(p)
        res = O.solve(geom, p.Ub, 1e-8)
        assert res.iterations <= 10
        u = O.field_scalar(geom, res.x)
        x, y, z = geom.grid.coords()
        r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
        errs.append(np.abs(u - I.harmonic_3d(x, y, z))[r < 0.12].max())
    assert errs[0] > errs[1] > errs[2]


# ----------------------------------------------------------------------------------------
# gradients (adjoint solve and boundary derivatives)
# ----------------------------------------------------------------------------------------


@pytest.mark.parametrize("kind", ["sqrt", "cos"])
def test_ddphi_is_second_derivative(kind):
    _, dphi = O.KERNELS[kind]
    d2 = O.KERNELS2[kind]
    r = np.linspace(-2.2, 2.2, 881)
    r = r[np.min(np.abs(r[:, None] - np.array([-2, -1, 0, 1, 2])[None, :]), 1) > 1e-3]
    e = 1e-6
    assert np.allclose(d2(r), (dphi(r + e) - dphi(r - e)) / (2 * e), atol=1e-7)


def test_transpose_is_matrix_transpose():
    geom, bd = _circle_geom(16, "sqrt", 2.0)
    geom.w = geom.w * (1 + 0.3 * np.sin(np.arange(bd.M)))  # non-uniform weights
    A = O.dense_operator(geom)
    At = O.dense_operator(geom, O.transpose_apply)
    assert np.allclose(At, A.T, atol=1e-12 * np.abs(A).max())


@pytest.mark.parametrize("delta,lam,dim", [("sqrt", 2.0, 2), ("cos", 0.0, 2), ("cos", 1.0, 3)])
def test_gradient_against_finite_differences(delta, lam, dim):
    """J = gᵀQ(U_b, X, n, w) with Q the solve: the adjoint gradients against central differences
    in every argument (step 1e-6), perturbing one input at a time."""
    if dim == 2:
        geom, bd = _circle_geom(32, delta, lam)
        Ub = I.harmonic_cubic(bd.X[0], bd.X[1])
    else:
        p = I.sphere_poisson(12, 120, delta=delta, lam=lam)
        geom = O.geometry_from_problem(p)
        Ub = p.Ub.reshape(-1)
    rng = np.random.default_rng(17)
    gvec = rng.standard_normal(geom.M)
    # non-uniform weights and tilted normals make every term of the formulas matter; the jitter
    # keeps points off grid lines, where φ'' jumps and A has a kink in X
    geom.X = geom.X + 0.1 * geom.grid.h * rng.uniform(-1, 1, geom.X.shape)
    geom.w = geom.w * (1 + 0.2 * rng.uniform(-1, 1, geom.M))
    nn = geom.n + 0.2 * rng.standard_normal(geom.n.shape)
    geom.n = nn / np.linalg.norm(nn, axis=0)
    Q, dUb, dX, dn, dw = O.solve_gradient(geom, Ub, gvec)

    def J(ub=Ub, X=geom.X, n=geom.n, w=geom.w):
        g2 = O.Geometry(geom.grid, X, n, w, geom.delta, geom.dipole, geom.symbol, geom.pde, geom.lam)
        return float(gvec @ O.solve(g2, ub, 1e-13, maxit=200).x)

    e = 1e-6
    for i in rng.choice(geom.M, 3, replace=False):
        d = np.zeros(geom.M)
        d[i] = e
        assert (J(ub=Ub + d) - J(ub=Ub - d)) / (2 * e) == pytest.approx(dUb[i], rel=1e-6, abs=1e-9)
        assert (J(w=geom.w + d) - J(w=geom.w - d)) / (2 * e) == pytest.approx(dw[i], rel=1e-5, abs=1e-8)
        for m in range(dim):
            D = np.zeros_like(geom.X)
            D[m, i] = e
            assert (J(X=geom.X + D) - J(X=geom.X - D)) / (2 * e) == pytest.approx(dX[m, i], rel=1e-5, abs=1e-8)
            assert (J(n=geom.n + D) - J(n=geom.n - D)) / (2 * e) == pytest.approx(dn[m, i], rel=1e-5, abs=1e-8)


def _star_geom(N, M, seed, tilt=0.2):
    """Small Stokes star with points off grid lines, tilted normals and uneven weights."""
    p = I.star_stokes(N, M)
    g = O.geometry_from_problem(p)
    rng = np.random.default_rng(seed)
    g.X = g.X + 0.1 * g.grid.h * rng.uniform(-1, 1, g.X.shape)
    nn = g.n + tilt * rng.standard_normal(g.n.shape)
    g.n = nn / np.linalg.norm(nn, axis=0)
    g.w = g.w * (1 + 0.2 * rng.uniform(-1, 1, g.M))
    return g, p.Ub.reshape(-1), rng


def test_stokes_transpose_is_matrix_transpose():
    geom, _, _ = _star_geom(16, 30, 1)
    A = O.dense_operator(geom)
    At = O.dense_operator(geom, O.transpose_apply)
    assert np.allclose(At, A.T, atol=1e-12 * np.abs(A).max())


@pytest.mark.parametrize("pde", ["scalar", "stokes"])
def test_probe_transpose_is_matrix_transpose(pde):
    """Eᵀν from probe_vjp against the dense matrix of Q ↦ E Q assembled column by column."""
    if pde == "stokes":
        geom, _, rng = _star_geom(16, 30, 2)
    else:
        geom, bd = _circle_geom(16, "sqrt", 1.0)
        rng = np.random.default_rng(2)
    P = 0.5 + 0.1 * rng.uniform(-1, 1, (2, 5))
    nd = geom.ncomp * geom.M
    E = np.stack([O.probe_evaluate(geom, P, np.eye(nd)[j]).reshape(-1) for j in range(nd)], axis=1)
    nu = rng.standard_normal(E.shape[0])
    dQ, _, _, _ = O.probe_vjp(geom, P, np.zeros(nd), nu)
    assert np.allclose(dQ.reshape(-1), E.T @ nu, atol=1e-12 * np.abs(E).max() * np.abs(nu).sum())


def _fd_check(J, args, grads, idx, rng, e=1e-6, rel=1e-5, abs_=1e-8):
    """Central differences of J in entries (component m, point i) of each named argument."""
    for name, a in args.items():
        g = grads[name]
        for i in idx:
            for m in range(a.shape[0] if a.ndim == 2 else 1):
                D = np.zeros_like(a)
                if a.ndim == 2:
                    D[m, i] = e
                else:
                    D[i] = e
                fd = (J(**{name: a + D}) - J(**{name: a - D})) / (2 * e)
                ref = g[m, i] if a.ndim == 2 else g[i]
                assert fd == pytest.approx(ref, rel=rel, abs=abs_), (name, m, i)


def test_stokes_gradient_against_finite_differences():
    geom, Ub, rng = _star_geom(32, 60, 3)
    gvec = rng.standard_normal(2 * geom.M)
    Q, dUb, dX, dn, dw = O.solve_gradient(geom, Ub, gvec)

    def J(ub=Ub, X=geom.X, n=geom.n, w=geom.w):
        g2 = O.Geometry(geom.grid, X, n, w, geom.delta, geom.dipole, geom.symbol, geom.pde, geom.lam, geom.mu)
        return float(gvec @ O.solve(g2, ub, 1e-13, maxit=300).x)

    idx = rng.choice(geom.M, 3, replace=False)
    for i in idx:
        for m in range(2):
            d = np.zeros(2 * geom.M)
            d[m * geom.M + i] = 1e-6
            assert (J(ub=Ub + d) - J(ub=Ub - d)) / 2e-6 == pytest.approx(dUb[m * geom.M + i], rel=1e-6, abs=1e-9)
    _fd_check(J, {"X": geom.X, "n": geom.n, "w": geom.w}, {"X": dX, "n": dn, "w": dw}, idx, rng)


@pytest.mark.parametrize("pde", ["scalar", "stokes"])
def test_probe_objective_gradient_against_finite_differences(pde):
    """J = Σ_p |u(p)|² with Q = A⁻¹U_b: the gradient assembled from probe_vjp (ν = 2u(p)) and the
    adjoint solve with ∂J/∂Q = Eᵀν, against central differences in U_b, X, n and Δs."""
    if pde == "stokes":
        geom, Ub, rng = _star_geom(32, 60, 4)
        P = I.star_probes(6, 32, min_dist_h=2.0, seed=5)
    else:
        geom, bd = _circle_geom(32, "cos", 2.0)
        rng = np.random.default_rng(4)
        geom.X = geom.X + 0.1 * geom.grid.h * rng.uniform(-1, 1, geom.X.shape)
        Ub = I.harmonic_cubic(geom.X[0], geom.X[1])
        P = 0.5 + 0.12 * rng.uniform(-1, 1, (2, 6))

    def J(ub=Ub, X=geom.X, n=geom.n, w=geom.w):
        g2 = O.Geometry(geom.grid, X, n, w, geom.delta, geom.dipole, geom.symbol, geom.pde, geom.lam, geom.mu)
        Q = O.solve(g2, ub, 1e-13, maxit=300).x
        return float(np.sum(O.probe_evaluate(g2, P, Q) ** 2))

    Q = O.solve(geom, Ub, 1e-13, maxit=300).x
    nu = 2 * O.probe_evaluate(geom, P, Q)
    dQ, pX, pn, pw = O.probe_vjp(geom, P, Q, nu)
    _, dUb, sX, sn, sw = O.solve_gradient(geom, Ub, dQ.reshape(-1))
    c = geom.ncomp
    idx = rng.choice(geom.M, 3, replace=False)
    for i in idx:
        for m in range(c):
            d = np.zeros(c * geom.M)
            d[m * geom.M + i] = 1e-6
            assert (J(ub=Ub + d) - J(ub=Ub - d)) / 2e-6 == pytest.approx(dUb[m * geom.M + i], rel=1e-5, abs=1e-9)
    _fd_check(J, {"X": geom.X, "n": geom.n, "w": geom.w}, {"X": pX + sX, "n": pn + sn, "w": pw + sw}, idx, rng)


# ----------------------------------------------------------------------------------------
# Brinkman (Sec. 6.3.2) and Neumann (Sec. 5.2)
# ----------------------------------------------------------------------------------------


@pytest.mark.parametrize("lam,mu", [(10.0, 1.0), (40.0, 0.5)])
def test_brinkman_velocity_satisfies_pde(lam, mu):
    """Mode by mode away from Nyquist: ∇·u + S(Q·n) = 0 and μΔu − λu + μ∇·(S A) = ∇p for some p
    (zero discrete curl), the interior Brinkman system of Sec. 6.3.2 with η = 0."""
    geom, bd = _stokes_geom(32)
    geom.lam, geom.mu = lam, mu
    g = geom.grid
    rng = np.random.default_rng(10)
    Q = rng.standard_normal((2, bd.M))
    u = O.stokes_velocity(geom, Q.reshape(-1))
    lap, der = O.symbols(g, "spectral")
    Uh = [np.fft.fftn(u[0]), np.fft.fftn(u[1])]
    sh = np.fft.fftn(O.spread(geom, np.sum(Q * bd.n, 0)))
    A = [[Q[l] * bd.n[m] + Q[m] * bd.n[l] for m in range(2)] for l in range(2)]
    gh = [np.fft.fftn(O.spread_grad(geom, np.array(A[l]))) for l in range(2)]
    kx = np.broadcast_to(np.fft.fftfreq(32, 1 / 32)[None, :], g.shape)
    ky = np.broadcast_to(np.fft.fftfreq(32, 1 / 32)[:, None], g.shape)
    ok = (np.abs(kx) != 16) & (np.abs(ky) != 16) & (lap != 0)
    div = der[0] * Uh[0] + der[1] * Uh[1] + sh
    assert np.abs(div[ok]).max() < 1e-9 * np.abs(sh).max()
    mom = [-(mu * lap + lam) * Uh[l] + mu * gh[l] for l in range(2)]
    curl = der[0] * mom[1] - der[1] * mom[0]
    assert np.abs(curl[ok]).max() < 1e-9 * np.abs(gh[0]).max() * 2 * np.pi * 16
    # the same velocity is not a Stokes one: the λ term matters
    mom0 = [-lap * Uh[l] + gh[l] for l in range(2)]
    assert np.abs((der[0] * mom0[1] - der[1] * mom0[0])[ok]).max() > 1e-3 * np.abs(gh[0]).max()


def test_brinkman_tends_to_stokes():
    geom, bd = _stokes_geom(32)
    Q = np.random.default_rng(11).standard_normal(2 * bd.M)
    ref = O.apply(geom, Q)
    geom.lam = 1e-6
    assert np.linalg.norm(O.apply(geom, Q) - ref) < 1e-5 * np.linalg.norm(ref)


def test_brinkman_first_order():
    """Interior velocity against the exact unforced Brinkman flow (λ = 100, μ = 1), r < 0.15,
    relative to its maximum: first order. The Stokes operator on the same data does not approach
    it (the flow is not a Stokes flow), so the λ term of the symbol is what converges."""
    errs = []
    for N in (64, 128, 256):
        M = I.points_for_spacing(2 * np.pi * 0.25, 1.0 / N, 1.2)
        p = I.circle_brinkman(N, M, lam=100.0, delta="sqrt")
        geom = O.geometry_from_problem(p)
        res = O.solve(geom, p.Ub.reshape(-1), 1e-10, maxit=80)
        assert res.iterations <= 16
        u = O.stokes_velocity(geom, res.x)
        x, y = geom.grid.coords()
        r = np.hypot(x - 0.5, y - 0.5)
        exact = I.brinkman_flow(x, y, 100.0)
        scale = np.abs(exact).max(0)[r < 0.15].max()
        errs.append(np.abs(u - exact).max(0)[r < 0.15].max() / scale)
    assert O.fitted_order([1 / 64, 1 / 128, 1 / 256], errs) > 0.85
    geom.lam = 0.0
    u0 = O.stokes_velocity(geom, O.solve(geom, p.Ub.reshape(-1), 1e-10, maxit=80).x)
    assert np.abs(u0 - exact).max(0)[r < 0.15].max() / scale > 5 * errs[-1]


def test_neumann_operator_is_dirichlet_minus_identity():
    geom, bd = _circle_geom(32, "sqrt", 1.0)
    Q = np.random.default_rng(12).standard_normal(bd.M)
    ref = O.apply(geom, Q)
    geom.bc = "neumann"
    assert np.allclose(O.apply(geom, Q), ref - Q, atol=1e-14)


def test_single_layer_weighted_symmetric():
    """W·S*(−L⁻¹)S is symmetric (S* is the adjoint of S under the weighted products, −L⁻¹ is
    symmetric), and positive for λ > 0 (−L⁻¹ has a positive symbol)."""
    geom, bd = _circle_geom(16, "cos", 2.0)
    geom.w = geom.w * (1 + 0.3 * np.sin(np.arange(bd.M)))
    SL = np.stack([O.single_layer(geom, e) for e in np.eye(bd.M)], axis=1)
    WS = geom.w[:, None] * SL
    assert np.allclose(WS, WS.T, atol=1e-12 * np.abs(WS).max())
    assert np.linalg.eigvalsh(0.5 * (WS + WS.T)).min() > -1e-12 * np.abs(WS).max()


def test_neumann_first_order():
    """The Neumann solve (Sec. 5.2) on the paper's circle: U_b → u|Γ = sin 2θ at first order, in a
    few GMRES iterations (the paper reports 4-6 for its Neumann test, Sec. 5.7)."""
    errs = []
    for N in (64, 128, 256):
        p = I.paper_circle_neumann(N)
        geom = O.geometry_from_problem(p)
        res = O.solve(geom, O.neumann_rhs(geom, p.Ub.reshape(-1)), 1e-10, maxit=60)
        assert res.iterations <= 12
        errs.append(np.abs(res.x - p.meta["exact_Ub"].reshape(-1)).max())
    assert O.fitted_order([1 / 64, 1 / 128, 1 / 256], errs) > 0.8


# ----------------------------------------------------------------------------------------
# completed method (Sec. 5.3.3, Sec. 6.1.3, Sec. 6.3.3)
# ----------------------------------------------------------------------------------------


def _drag_table():
    out = {}
    with open(os.path.join(GOLDEN, "cylinder_drag.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                c, ibdl, gk = line.split()
                out[float(c)] = (float(ibdl), float(gk))
    return out


@pytest.mark.parametrize("c,N,tol", [(0.05, 256, 0.01), (0.2, 512, 0.01), (0.4, 512, 0.03)])
def test_cylinder_drag_against_published(c, N, tol):
    """Exterior Stokes flow past a periodic array of cylinders with the completed method
    (η = 10, Δs ≈ Δx): the net force is the body force exactly (the constraint rows), and the
    dimensionless drag D = B₁/(μU) is within first-order distance of the boundary-integral
    values the paper quotes (its own IBDL values at N = 2^13 are within 0.1 % of them)."""
    ref = _drag_table()[c][1]
    p = I.cylinder_array(N, c)
    geom = O.geometry_from_problem(p)
    b = np.concatenate([p.Ub.reshape(-1), p.meta["rhs_aug"]])
    res = O.solve(geom, b, 1e-10, maxit=200)
    assert res.iterations <= 20
    B = O.net_force(geom, res.x)
    assert abs(B[0] - 1.0) < 1e-9 and abs(B[1]) < 1e-9
    D = B[0] / O.mean_inflow(geom, res.x)
    assert abs(D - ref) < tol * ref


def test_completed_interior_laplace_first_order():
    """The completed scalar method (λ = 0, η = 10) on an interior circle still converges at first
    order to the harmonic cubic inside (the single-layer term and the mean ū only change what
    the density represents outside Ω)."""
    errs = []
    for N in (64, 128, 256):
        geom, bd = _circle_geom(N, "sqrt", 0.0)
        geom.eta = 10.0
        Ub = I.harmonic_cubic(bd.X[0], bd.X[1])
        b = np.concatenate([Ub, [0.0]])
        res = O.solve(geom, b, 1e-11, maxit=80)
        assert res.iterations <= 20
        u = O.grid_field(geom, res.x)
        x, y = geom.grid.coords()
        r = np.hypot(x - 0.5, y - 0.5)
        errs.append(np.abs(u - I.harmonic_cubic(x, y))[r < 0.15].max())
    assert O.fitted_order([1 / 64, 1 / 128, 1 / 256], errs) > 0.8


def test_completed_rejects_screening():
    geom, bd = _circle_geom(16, "cos", 1.0)
    geom.eta = 1.0
    with pytest.raises(NotImplementedError):
        O.apply(geom, np.ones(bd.M + 1))


# ----------------------------------------------------------------------------------------
# post-processing: indicator flagging (Sec. 5.3.5), near-boundary interpolation (Sec. 5.3.4)
# ----------------------------------------------------------------------------------------


def _three_shapes(N, alpha=0.75):
    """A circle, a rotated ellipse and a star in one box, as in the indicator illustration of
    Sec. 5.3.5, with their exact membership tests."""
    h = 1.0 / N
    c = I.circle(I.points_for_spacing(2 * np.pi * 0.12, h, alpha), R=0.12, center=(0.25, 0.27))
    e = I.ellipse(I.points_for_spacing(2 * np.pi * 0.12, h, alpha), 0.16, 0.08, rot=0.6, center=(0.72, 0.3))
    s = I.star(I.points_for_spacing(2 * np.pi * 0.17, h, alpha), a=0.17, eps=0.2, k=5, center=(0.5, 0.72))

    def inside(x, y):
        in_c = np.hypot(x - 0.25, y - 0.27) < 0.12
        xr, yr = x - 0.72, y - 0.3
        u, v = np.cos(0.6) * xr + np.sin(0.6) * yr, -np.sin(0.6) * xr + np.cos(0.6) * yr
        in_e = (u / 0.16) ** 2 + (v / 0.08) ** 2 < 1
        th = np.arctan2(y - 0.72, x - 0.5)
        in_s = np.hypot(x - 0.5, y - 0.72) < 0.17 * (1 + 0.2 * np.cos(5 * th))
        return in_c | in_e | in_s

    X = np.concatenate([c.X, e.X, s.X], axis=1)
    n = np.concatenate([c.n, e.n, s.n], axis=1)
    w = np.concatenate([c.w, e.w, s.w])
    return X, n, w, inside


def _dist_to(X_dense, x, y):
    pts = np.stack([x.ravel(), y.ravel()], 1)
    d = np.full(pts.shape[0], np.inf)
    for i in range(0, X_dense.shape[1], 512):
        blk = X_dense[:, i:i + 512].T
        d = np.minimum(d, np.sqrt(((pts[:, None, :] - blk[None]) ** 2).sum(-1)).min(1))
    return d.reshape(x.shape)


@pytest.mark.parametrize("delta,symbol", [("sqrt", "fd2"), ("cos", "spectral")])
def test_indicator_flags_three_shapes(delta, symbol):
    """χ → 1 inside the curves and 0 outside (the jump of the double layer of a unit density,
    Sec. 3), so the flags equal exact membership at every node farther than 2h from Γ, for
    three shapes at once; reversed normals give χ → −1 inside and the same flags."""
    N = 128
    X, n, w, inside = _three_shapes(N)
    geom = O.Geometry(O.Grid(2, N), X, n, w, delta, "analytic", symbol, "scalar", 0.0)
    chi, flags = O.indicator(geom)
    x, y = geom.grid.coords()
    Xd, _, _, _ = _three_shapes(2048, alpha=1.0)
    far = _dist_to(Xd, x, y) > 2.0 / N
    exact = inside(x, y)
    assert np.array_equal(flags[far], exact[far])
    deep = _dist_to(Xd, x, y) > 8.0 / N
    assert np.abs(chi[deep & exact] - 1).max() < 0.02
    assert np.abs(chi[deep & ~exact]).max() < 0.02
    assert abs(chi.flat[0]) == 0.0
    geom_in = O.Geometry(O.Grid(2, N), X, -n, w, delta, "analytic", symbol, "scalar", 0.0)
    chi2, flags2 = O.indicator(geom_in)
    assert np.array_equal(flags2, flags)
    assert np.allclose(chi2, -chi, atol=1e-12)


def test_indicator_ignores_the_geometry_pde():
    """The indicator solves the Laplace problem whatever PDE, λ or η the geometry carries."""
    N = 64
    bd = I.circle(I.points_for_spacing(2 * np.pi * 0.25, 1 / N, 0.75))
    g0 = O.Geometry(O.Grid(2, N), bd.X, bd.n, bd.w, "cos", "analytic", "spectral", "scalar", 0.0)
    g1 = O.Geometry(O.Grid(2, N), bd.X, bd.n, bd.w, "cos", "analytic", "spectral", "stokes", 5.0, 2.0)
    assert np.array_equal(O.indicator(g0)[0], O.indicator(g1)[0])


def test_nearest_three_against_brute_force():
    """Nearest boundary points under periodic wrap: brute force over the nine periodic images."""
    rng = np.random.default_rng(11)
    L = 2.0
    X = rng.uniform(-1, 1, (2, 40))
    geom = O.Geometry(O.Grid(2, 32, L, (-1.0, -1.0)), X, np.zeros_like(X), np.ones(40))
    for _ in range(50):
        p = rng.uniform(-1, 1, 2)
        three, d, d2 = O.nearest_three(geom, p)
        best = [min((X[0, i] + sx * L - p[0]) ** 2 + (X[1, i] + sy * L - p[1]) ** 2
                    for sx in (-1, 0, 1) for sy in (-1, 0, 1)) for i in range(40)]
        assert list(three) == list(np.argsort(best, kind="stable")[:3])
        assert np.allclose(d2, best, rtol=1e-13, atol=1e-15)


def test_chord_foot_is_the_closest_point():
    """x_A is the point of the chord's line closest to x_p (brute force along the line)."""
    rng = np.random.default_rng(12)
    for _ in range(30):
        d = rng.standard_normal((2, 2))
        xA, t = O.chord_foot(d, 0, 1)
        s = np.linspace(t - 1, t + 1, 20001)
        line = d[:, 1:2] + s * (d[:, 0:1] - d[:, 1:2])
        assert abs(s[np.argmin(np.hypot(*line))] - t) < 2e-4
        assert abs((xA @ (d[:, 0] - d[:, 1]))) < 1e-12


@pytest.mark.parametrize("shape", ["circle", "star"])
def test_near_boundary_reproduces_linear_fields(shape):
    """Linear data are reproduced exactly: u_A (linear along the chord), u_B (bilinear) and the
    blend along x_A–x_B are each exact for linear functions, so every replaced node takes the
    exact value although the grid values within the band and outside Ω are garbage; a Stokes
    geometry carries two components with different slopes."""
    N, m1, m2 = 128, 6.0, 8.0
    M = I.points_for_spacing(2 * np.pi * 0.25, 1 / N, 0.75)
    bd = I.circle(M) if shape == "circle" else I.star(M)
    geom = O.Geometry(O.Grid(2, N), bd.X, bd.n, bd.w, "cos", "analytic", "spectral", "stokes")
    x, y = geom.grid.coords()
    if shape == "circle":
        omega = np.hypot(x - 0.5, y - 0.5) < 0.25
    else:
        th = np.arctan2(y - 0.5, x - 0.5)
        omega = np.hypot(x - 0.5, y - 0.5) < 0.25 * (1 + 0.2 * np.cos(5 * th))
    lin = [lambda x, y: 0.3 + 1.7 * x - 0.9 * y, lambda x, y: -1.1 + 0.4 * x + 2.3 * y]
    dist = _dist_to(I.circle(4096).X if shape == "circle" else I.star(4096).X, x, y)
    rng = np.random.default_rng(3)
    u = np.stack([np.where(omega & (dist > (m1 + 0.3) / N), f(x, y), rng.standard_normal(x.shape)) for f in lin])
    Ub = np.stack([f(bd.X[0], bd.X[1]) for f in lin])
    out = O.near_boundary_interp(geom, Ub, u, omega, m1, m2)
    band = omega & (dist < (m1 - 0.3) / N)
    for c, f in enumerate(lin):
        assert np.abs(out[c][band] - f(x, y)[band]).max() < 1e-12
    keep = ~omega | (dist > (m1 + 0.3) / N)
    assert np.array_equal(out[:, keep], u[:, keep])


def _bessel_exact(x, y):
    """u = I₂(r) sin 2θ / I₂(0.25): the exact solution of the paper's circle problem (Δu − u = 0,
    U_b = sin 2θ on r = 0.25, Sec. 5.4.1)."""
    from scipy.special import iv

    r, th = np.hypot(x, y), np.arctan2(y, x)
    return iv(2, r) / iv(2, 0.25) * np.sin(2 * th)


@pytest.mark.parametrize("symbol,delta", [("fd2", "sqrt"), ("spectral", "cos")])
def test_near_boundary_restores_pointwise_convergence(symbol, delta):
    """Sec. 5.3.4 and its max-norm study, on the paper's circle problem (Δu − u = 0, U_b = sin 2θ,
    Δs ≈ 0.75Δx): the raw max-norm error over Ω stays O(1) (the density's jump smeared over the
    delta's support), while the interpolated one converges (finite differences: m1 = 6, m2 = 8;
    spectral: m1 = 2(log₂N − 4), m2 = m1 + 2)."""
    raw, fixed, hs = [], [], []
    for N in (64, 128, 256):
        # finite differences take the paper's divergence of the spread Q n; spectral the analytic dipole
        p = I.paper_circle_helmholtz(N, 0.75, delta, symbol, dipole="spectral_div" if symbol == "fd2" else "analytic")
        geom = O.geometry_from_problem(p)
        Q = O.solve(geom, p.Ub.reshape(-1), 1e-12, maxit=200).x
        u = O.field_scalar(geom, Q)
        _, flags = O.indicator(geom)
        x, y = geom.grid.coords()
        exact = _bessel_exact(x, y)
        m1 = 6.0 if symbol == "fd2" else 2.0 * (math.log2(N) - 4)
        m2 = 8.0 if symbol == "fd2" else m1 + 2
        ui = O.near_boundary_interp(geom, p.Ub.reshape(-1), u, flags, m1, m2)
        raw.append(np.abs(u - exact)[flags].max())
        fixed.append(np.abs(ui - exact)[flags].max())
        hs.append(1 / N)
    assert min(raw) > 0.5
    assert fixed[-1] < raw[-1] / 10
    assert O.fitted_order(hs, fixed) > (1.0 if symbol == "fd2" else 0.6)


# ----------------------------------------------------------------------------------------
# source term g̃ (Sec. 5.1.2, Eq. "ibdl schur again"; Sec. 6.1.1)
# ----------------------------------------------------------------------------------------


def _lap_fd(u, h):
    """5-point Laplacian by shifts (Sec. 2.2.1), periodic."""
    return (np.roll(u, 1, 0) + np.roll(u, -1, 0) + np.roll(u, 1, 1) + np.roll(u, -1, 1) - 4 * u) / h ** 2


def _dx_fd(u, h, axis):
    """centred first difference by shifts (axis 1 = x, axis 0 = y)."""
    return (np.roll(u, -1, axis) - np.roll(u, 1, axis)) / (2 * h)


def _empty_geom(N, pde, lam=0.0, mu=1.0, symbol="spectral"):
    z = np.zeros((2, 3))
    return O.Geometry(O.Grid(2, N), z, z, np.ones(3), "cos", "analytic", symbol, pde, lam, mu)


@pytest.mark.parametrize("symbol", ["spectral", "fd2"])
@pytest.mark.parametrize("lam", [0.0, 3.0])
def test_source_field_recovers_periodic_solutions(symbol, lam):
    """A periodic u with g̃ = L u (and, for Stokes, g̃ = μΔu − λu − ∇p with ∇·u = 0) must come back
    from the source alone: u_g = u. For the spectral symbols L is applied by derivatives of the
    Fourier modes; for finite differences by the 5-point stencil applied by shifts, so the check
    is independent of the oracle's symbol code."""
    N, mu = 32, 0.7
    x, y = O.Grid(2, N).coords()
    h = 1.0 / N
    u = np.cos(2 * np.pi * (2 * x + y)) + 0.3 * np.sin(2 * np.pi * (x - 3 * y))
    if symbol == "spectral":
        Lu = -(2 * np.pi) ** 2 * (5 * np.cos(2 * np.pi * (2 * x + y)) + 0.3 * 10 * np.sin(2 * np.pi * (x - 3 * y)))
    else:
        Lu = _lap_fd(u, h)
    geom = _empty_geom(N, "scalar", lam, symbol=symbol)
    ref = u - u.mean() if lam == 0.0 else u
    assert np.abs(O.source_field(geom, Lu - lam * u) - ref).max() < 1e-12
    # Stokes / Brinkman: a divergence-free cellular flow with a pressure
    s2, c2 = np.sin(2 * np.pi * x), np.cos(2 * np.pi * x)
    sy, cy = np.sin(2 * np.pi * y), np.cos(2 * np.pi * y)
    U = np.stack([s2 * cy, -c2 * sy])
    p = np.sin(2 * np.pi * (x + 2 * y))
    if symbol == "spectral":
        LU = -(2 * np.pi) ** 2 * 2 * U
        gp = np.stack([2 * np.pi * np.cos(2 * np.pi * (x + 2 * y)), 4 * np.pi * np.cos(2 * np.pi * (x + 2 * y))])
    else:
        # U is divergence free under the centred difference, so the operator's projection (the
        # literal I − ∇Δ₀⁻¹∇· with the 5-point Δ₀) keeps it; that projection does not remove a
        # centred-difference gradient exactly (its ∇·∇ is not the 5-point Laplacian), so the
        # finite-difference case carries no pressure
        LU = np.stack([_lap_fd(U[0], h), _lap_fd(U[1], h)])
        gp = 0.0 * U
    g = mu * LU - lam * U - gp
    geom = _empty_geom(N, "stokes", lam, mu, symbol=symbol)
    assert np.abs(O.source_field(geom, g) - U).max() < 1e-12


def test_forced_solve_converges_scalar():
    """Laplace with a source: u = Re((z − z0)³) + sin 2πx sin 2πy inside the circle, g̃ = Δu =
    −8π² sin 2πx sin 2πy on all of C (periodic, mean zero), U_b = u on Γ. The forced solve
    converges to u inside Ω at first order; without g̃ it does not approach u."""
    errs, unforced = [], []
    for N in (64, 128, 256):
        geom, bd = _circle_geom(N, "sqrt", 0.0, symbol="fd2", alpha=0.75)
        x, y = geom.grid.coords()
        per = lambda x, y: np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
        ub = I.harmonic_cubic(bd.X[0], bd.X[1]) + per(bd.X[0], bd.X[1])
        g = -8 * np.pi ** 2 * per(x, y)
        Q = O.solve(geom, O.forced_rhs(geom, ub, g), 1e-12, maxit=80).x
        u = O.forced_field(geom, Q, g)
        r = np.hypot(x - 0.5, y - 0.5)
        exact = I.harmonic_cubic(x, y) + per(x, y)
        errs.append(np.abs(u - exact)[r < 0.15].max())
        Q0 = O.solve(geom, ub, 1e-12, maxit=80).x
        unforced.append(np.abs(O.grid_field(geom, Q0) - exact)[r < 0.15].max())
    assert O.fitted_order([1 / 64, 1 / 128, 1 / 256], errs) > 0.8
    assert min(unforced) > 20 * errs[-1]


def test_forced_solve_converges_stokes():
    """Stokes with a body force: u = (polynomial interior flow) + (cellular flow U with pressure p),
    g̃ = μΔU − ∇p on C (the polynomial flow needs none), U_b = u on the star. The forced solve
    converges to u inside Ω at first order."""
    mu = 1.0
    errs = []
    for N in (64, 128, 256):
        p = I.star_stokes(N, I.points_for_spacing(1.9124, 1 / N, 1.0))
        geom = O.geometry_from_problem(p)
        x, y = geom.grid.coords()

        def cell(x, y):
            return np.stack([np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y), -np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y)])

        X = p.bd.X
        ub = (I.stokes_poly(X[0], X[1]) + cell(X[0], X[1])).reshape(-1)
        ub, _ = I.remove_normal_flux(ub.reshape(2, -1), p.bd)
        pr = np.cos(2 * np.pi * x) * np.cos(2 * np.pi * y)
        gp = np.stack([-2 * np.pi * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y),
                       -2 * np.pi * np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y)])
        g = mu * (-(2 * np.pi) ** 2 * 2) * cell(x, y) - gp
        Q = O.solve(geom, O.forced_rhs(geom, ub.reshape(-1), g), 1e-12, maxit=120).x
        u = O.forced_field(geom, Q, g)
        th = np.arctan2(y - 0.5, x - 0.5)
        inside = np.hypot(x - 0.5, y - 0.5) < 0.6 * 0.25 * (1 + 0.2 * np.cos(5 * th))
        exact = I.stokes_poly(x, y) + cell(x, y)
        errs.append(np.abs(u - exact)[:, inside].max())
    assert O.fitted_order([1 / 64, 1 / 128, 1 / 256], errs) > 0.8


def test_forced_rhs_completed_constraint_rows():
    """Completed method: a constant body force has no mean-free part, so the boundary rows keep
    U_b and the constraint rows become h^d Σ g̃, the values the cylinder-array drag pin uses."""
    p = I.cylinder_array(64, 0.2)
    geom = O.geometry_from_problem(p)
    g = np.zeros((2,) + geom.grid.shape)
    g[0] = -1.0
    rhs = O.forced_rhs(geom, np.concatenate([p.Ub.reshape(-1), [9.0, 9.0]]), g)
    assert np.abs(rhs[: 2 * geom.M] - p.Ub.reshape(-1)).max() < 1e-12
    assert np.allclose(rhs[2 * geom.M:], p.meta["rhs_aug"], atol=1e-12)


# ----------------------------------------------------------------------------------------
# normals and weights from the points (Sec. 5.3.1)
# ----------------------------------------------------------------------------------------


def test_estimated_normals_and_weights_on_a_circle():
    """On an equispaced circle the centred chord is perpendicular to the radius, so the estimated
    normal is the exact radial normal; the weight is the chord 2R sin(π/M). A clockwise ordering
    gives the inward normals, and a circle crossing the periodic edge gives the same values."""
    M, R = 37, 0.25
    bd = I.circle(M, R)
    n = O.estimate_normals(bd.X, 1.0)
    assert np.abs(n - bd.n).max() < 1e-14
    assert np.abs(O.estimate_weights(bd.X, 1.0) - 2 * R * np.sin(np.pi / M)).max() < 1e-15
    assert np.abs(O.estimate_normals(bd.X[:, ::-1], 1.0) + bd.n[:, ::-1]).max() < 1e-14
    wrapped = np.mod(bd.X + np.array([[0.4], [0.45]]), 1.0)  # centre (0.9, 0.95): crosses both edges
    assert np.abs(O.estimate_normals(wrapped, 1.0) - bd.n).max() < 1e-13
    assert np.abs(O.estimate_weights(wrapped, 1.0) - 2 * R * np.sin(np.pi / M)).max() < 1e-13


def test_estimated_geometry_keeps_first_order_accuracy():
    """The paper's claim for the estimates: the solution stays first-order accurate. Star curve
    (normals not radial), harmonic data, estimated normals and chord weights."""
    errs = []
    for N in (64, 128, 256):
        M = I.points_for_spacing(1.9124, 1 / N, 1.0)
        bd = I.star(M)
        n, w = O.estimate_normals(bd.X, 1.0), O.estimate_weights(bd.X, 1.0)
        assert np.abs(np.sum(n * bd.n, axis=0) - 1).max() < 0.02  # close to the exact normals
        geom = O.Geometry(O.Grid(2, N), bd.X, n, w, "cos", "analytic", "spectral", "scalar", 0.0)
        ub = I.harmonic_cubic(bd.X[0], bd.X[1])
        Q = O.solve(geom, ub, 1e-12, maxit=80).x
        x, y = geom.grid.coords()
        u = O.field_scalar(geom, Q)
        r = np.hypot(x - 0.5, y - 0.5)
        errs.append(np.abs(u - I.harmonic_cubic(x, y))[r < 0.12].max())
    assert O.fitted_order([1 / 64, 1 / 128, 1 / 256], errs) > 0.8
