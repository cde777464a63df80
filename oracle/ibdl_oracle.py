"""FP64 CPU oracle of the IBDL operator hot path (Leathers 2022, arXiv 2210.07403).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module. The CUDA product path never calls it, and this
module shares no code with it (no kernels, headers, tables or helpers): the only common
dependency is the seeded input generator ``ibdl_inputs``, which holds no method arithmetic.

Everything here is a plain, slow, literal transcription of the discrete operators, written
for a reader to check against the paper by eye:

  δ_h         regularised delta, Sec. 2.2.2 (√-Peskin 4-point) and its cosine variant
  S, S*       spread / interpolation, Sec. 2.2.2
  S̃Q          dipole spread ∇·(S(Q n)), Sec. 5.1.1 and Sec. 5.3.1
  -L⁻¹        periodic Fourier solve, Sec. 2.2.1, Sec. 2.2.4 (Δ₀⁻¹: mean-zero inverse)
  A Q         −S* L⁻¹ S̃ Q + ½Q, Sec. 5.3.2 (Eq. "ibdl schur again")
  A Q Stokes  −S*Δ₀⁻¹∇Δ₀⁻¹Δ S(Q·n) − S*Δ₀⁻¹ P ∇·(S A) + ½Q, Sec. 6.3.3 (interior, η = 0)
  GMRES       unrestarted, zero initial guess, Sec. 5.3.2
  χ, flags    indicator of the enclosed region, Sec. 5.3.5
  interp      near-boundary linear interpolation, Sec. 5.3.4
  u_g         the grid response to a source g̃ (scalar L⁻¹g̃, Stokes −P̂ĝ/(μ|k|²+λ)), Sec. 5.1.2, Sec. 6.1.1
  n, Δs       normals and weights estimated from the points, Sec. 5.3.1

Readings of points the paper leaves open are listed with each function; all are the same
readings the CUDA path takes.

Array conventions: a grid field of dimension d has shape (N,)*d indexed [..., y, x]
(x fastest); boundary arrays are SoA, X and n of shape (d, M), densities (c, M).

Parity status: every function below is pinned by ``tests/test_oracle_pins.py`` against
closed forms, invariants, brute force on tiny inputs or the paper's printed iteration counts.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np

# ----------------------------------------------------------------------------------------
# δ_h: one-dimensional kernels φ and their derivatives (Sec. 2.2.2)
# ----------------------------------------------------------------------------------------


def phi_sqrt(r):
    """Peskin 4-point kernel (Sec. 2.2.2):
    φ(r) = (3 − 2|r| + √(1 + 4|r| − 4r²))/8 for |r| ≤ 1,
           (5 − 2|r| − √(−7 + 12|r| − 4r²))/8 for 1 ≤ |r| ≤ 2, 0 beyond."""
    a = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(a)
    m1 = a <= 1
    m2 = (a > 1) & (a < 2)
    out[m1] = (3 - 2 * a[m1] + np.sqrt(1 + 4 * a[m1] - 4 * a[m1] ** 2)) / 8
    out[m2] = (5 - 2 * a[m2] - np.sqrt(-7 + 12 * a[m2] - 4 * a[m2] ** 2)) / 8
    return out


def dphi_sqrt(r):
    """dφ/dr of the √-Peskin kernel, differentiated piece by piece (C¹ at |r| = 0, 1, 2)."""
    r = np.asarray(r, dtype=np.float64)
    a = np.abs(r)
    out = np.zeros_like(a)
    m1 = a <= 1
    m2 = (a > 1) & (a < 2)
    out[m1] = (-2 + (2 - 4 * a[m1]) / np.sqrt(1 + 4 * a[m1] - 4 * a[m1] ** 2)) / 8
    out[m2] = (-2 - (6 - 4 * a[m2]) / np.sqrt(-7 + 12 * a[m2] - 4 * a[m2] ** 2)) / 8
    return np.sign(r) * out


def phi_cos(r):
    """Cosine 4-point kernel φ(r) = (1 + cos(πr/2))/4 for |r| < 2 (the workloads' delta)."""
    r = np.asarray(r, dtype=np.float64)
    return np.where(np.abs(r) < 2, 0.25 * (1 + np.cos(0.5 * np.pi * r)), 0.0)


def dphi_cos(r):
    r = np.asarray(r, dtype=np.float64)
    return np.where(np.abs(r) < 2, -0.125 * np.pi * np.sin(0.5 * np.pi * r), 0.0)


KERNELS = {"sqrt": (phi_sqrt, dphi_sqrt), "cos": (phi_cos, dphi_cos)}

# ----------------------------------------------------------------------------------------
# grid and boundary
# ----------------------------------------------------------------------------------------


@dataclass
class Grid:
    """Periodic box [origin, origin + box)^d with N nodes per axis, x_i = origin + i h
    (Sec. 2.2.1, which uses origin −L/2)."""

    dim: int
    N: int
    box: float = 1.0
    origin: tuple = None

    def __post_init__(self):
        if self.origin is None:
            self.origin = (0.0,) * self.dim
        self.origin = tuple(float(o) for o in self.origin)

    @property
    def h(self) -> float:
        return self.box / self.N

    @property
    def shape(self):
        return (self.N,) * self.dim

    def coords(self):
        """Node coordinates as a list [x, y(, z)] of arrays of the grid's shape."""
        ax = [self.origin[j] + self.h * np.arange(self.N) for j in range(self.dim)]
        mesh = np.meshgrid(*ax[::-1], indexing="ij")  # [.., y, x] ordering
        return mesh[::-1]


@dataclass
class Geometry:
    """The discrete immersed boundary and the operator options."""

    grid: Grid
    X: np.ndarray  # (d, M)
    n: np.ndarray  # (d, M) outward unit normals
    w: np.ndarray  # (M,) quadrature weights Δs_i
    delta: str = "cos"
    dipole: str = "analytic"  # "analytic" | "spectral_div"
    symbol: str = "spectral"  # "spectral" | "fd2"
    pde: str = "scalar"  # "scalar" (L = Δ − λ) | "stokes" (L = μΔ − λ: Stokes λ = 0, Brinkman λ = k² > 0)
    lam: float = 0.0
    mu: float = 1.0
    bc: str = "dirichlet"  # "dirichlet" (jump +½) | "neumann" (jump −½, Sec. 5.2; scalar)
    eta: float = 0.0  # completed method (Sec. 5.3.3, Sec. 6.1.3): ηSQ added to the sources

    @property
    def jump(self) -> float:
        return -0.5 if self.bc == "neumann" else 0.5

    @property
    def naug(self) -> int:
        """Extra unknowns ū of the completed method (λ = 0): one mean per velocity component."""
        return self.ncomp if self.eta > 0 else 0

    def split(self, x):
        """(Q (c, M), ū (c,)) from a flat vector of the (possibly augmented) system."""
        x = np.asarray(x, dtype=np.float64).reshape(-1)
        c, M = self.ncomp, self.M
        return x[: c * M].reshape(c, M), x[c * M:]

    @property
    def M(self) -> int:
        return self.X.shape[1]

    @property
    def ncomp(self) -> int:
        return self.grid.dim if self.pde == "stokes" else 1


def geometry_from_problem(p) -> Geometry:
    """Build a Geometry from an ``ibdl_inputs.Problem``."""
    return Geometry(Grid(p.dim, p.N, p.box, p.origin), p.bd.X, p.bd.n, p.bd.w, p.delta,
                    p.dipole, p.symbol, p.pde, p.lam, p.mu, getattr(p, "bc", "dirichlet"),
                    getattr(p, "eta", 0.0))


def _stencil(geom: Geometry):
    """For each point and axis, the four node indices touched by the 4-point kernel and the
    scaled offsets r = (x_node − X)/h. The first node is floor((X − origin)/h) − 1, so the
    four nodes straddle X; indices wrap periodically."""
    g = geom.grid
    xi = (geom.X - np.asarray(g.origin)[:, None]) / g.h  # (d, M)
    base = np.floor(xi).astype(np.int64) - 1
    a = np.arange(4)
    idx = (base[:, :, None] + a) % g.N  # (d, M, 4)
    r = (base[:, :, None] + a) - xi[:, :, None]  # (d, M, 4)
    return idx, r


def _offsets(dim):
    return itertools.product(range(4), repeat=dim)


def _node_index(idx, off):
    """Tuple of index arrays in [..., y, x] order for stencil offset ``off``."""
    d = len(off)
    return tuple(idx[j, :, off[j]] for j in reversed(range(d)))


# ----------------------------------------------------------------------------------------
# S, S*, S̃ (Sec. 2.2.2, Sec. 5.3.1)
# ----------------------------------------------------------------------------------------


def spread(geom: Geometry, F: np.ndarray) -> np.ndarray:
    """(S F)(x_g) = Σ_i F_i δ_h(x_g − X_i) Δs_i, δ_h = h^{−d} Π_j φ(x_j/h) (Sec. 2.2.2)."""
    g = geom.grid
    phi, _ = KERNELS[geom.delta]
    idx, r = _stencil(geom)
    out = np.zeros(g.shape)
    for off in _offsets(g.dim):
        wt = np.ones(geom.M)
        for j in range(g.dim):
            wt = wt * phi(r[j, :, off[j]])
        np.add.at(out, _node_index(idx, off), F * geom.w * wt / g.h ** g.dim)
    return out


def interp(geom: Geometry, u: np.ndarray) -> np.ndarray:
    """(S* u)(X_i) = Σ_g u_g δ_h(x_g − X_i) h^d (Sec. 2.2.2); at most 4^d terms per point."""
    g = geom.grid
    phi, _ = KERNELS[geom.delta]
    idx, r = _stencil(geom)
    out = np.zeros(geom.M)
    for off in _offsets(g.dim):
        wt = np.ones(geom.M)
        for j in range(g.dim):
            wt = wt * phi(r[j, :, off[j]])
        out += u[_node_index(idx, off)] * wt
    return out


def spread_grad(geom: Geometry, V: np.ndarray) -> np.ndarray:
    """Σ_i Δs_i Σ_m V_{m,i} ∂_m δ_h(x_g − X_i): the analytic divergence of S(V) for a
    boundary vector field V of shape (d, M). With V = Q n this is S̃Q = ∇·(S(Q n))
    (Sec. 5.1.1), the dipole spread with the exact gradient of δ_h."""
    g = geom.grid
    phi, dphi = KERNELS[geom.delta]
    idx, r = _stencil(geom)
    out = np.zeros(g.shape)
    for off in _offsets(g.dim):
        ph = [phi(r[j, :, off[j]]) for j in range(g.dim)]
        dph = [dphi(r[j, :, off[j]]) / g.h for j in range(g.dim)]
        val = np.zeros(geom.M)
        for m in range(g.dim):
            term = V[m].copy()
            for j in range(g.dim):
                term = term * (dph[j] if j == m else ph[j])
            val += term
        np.add.at(out, _node_index(idx, off), geom.w * val / g.h ** g.dim)
    return out


def interp_grad(geom: Geometry, u: np.ndarray) -> np.ndarray:
    """(S*∇u)-like gather with the analytic kernel gradient: G_{m,i} = Σ_g u_g ∂_m δ_h(x_g − X_i) h^d.
    This is the transpose partner of ``spread_grad`` (used by the adjoint operator)."""
    g = geom.grid
    phi, dphi = KERNELS[geom.delta]
    idx, r = _stencil(geom)
    out = np.zeros((g.dim, geom.M))
    for off in _offsets(g.dim):
        ph = [phi(r[j, :, off[j]]) for j in range(g.dim)]
        dph = [dphi(r[j, :, off[j]]) / g.h for j in range(g.dim)]
        ug = u[_node_index(idx, off)]
        for m in range(g.dim):
            term = ug.copy()
            for j in range(g.dim):
                term = term * (dph[j] if j == m else ph[j])
            out[m] += term
    return out


# ----------------------------------------------------------------------------------------
# Fourier symbols and the periodic solve (Sec. 2.2.1, Sec. 2.3.1, Sec. 2.2.4)
# ----------------------------------------------------------------------------------------


def wavenumbers(grid: Grid):
    """k = 2π m / box with m = 0, 1, …, N/2 − 1, −N/2, …, −1 (np.fft ordering)."""
    return 2 * np.pi * np.fft.fftfreq(grid.N, d=1.0 / grid.N) / grid.box


def symbols(grid: Grid, kind: str):
    """Per-axis symbols of the Laplacian and of the first derivative, broadcast to the grid.

    spectral: −Δ ↦ Σ k_j², ∂_j ↦ i k_j, with the first-derivative symbol set to 0 at the
              Nyquist index m = −N/2 (reading: that mode has no real counterpart; zeroing it
              makes the discrete ∇· exactly minus the adjoint of ∇).
    fd2:      5-point Laplacian −Δ ↦ Σ (4/h²) sin²(k_j h/2) (Sec. 2.2.1) and the centred
              difference ∂_j ↦ i sin(k_j h)/h (Sec. 5.3.1), zero at Nyquist by itself.
    Returns (lap, [deriv_j]) with lap real (the symbol of −Δ) and deriv_j imaginary."""
    k = wavenumbers(grid)
    h = grid.h
    d = grid.dim
    if kind == "spectral":
        lap1 = k * k
        kd = k.copy()
        kd[grid.N // 2] = 0.0
        der1 = 1j * kd
    elif kind == "fd2":
        lap1 = 4.0 / h ** 2 * np.sin(k * h / 2) ** 2
        der1 = 1j * np.sin(k * h) / h
    else:
        raise ValueError(kind)
    shape = grid.shape
    lap = np.zeros(shape)
    der = []
    for j in range(d):
        bshape = [1] * d
        bshape[d - 1 - j] = grid.N  # axis j lives at array position d−1−j
        lap = lap + lap1.reshape(bshape)
        der.append(np.broadcast_to(der1.reshape(bshape), shape))
    return lap, der


def minus_Linv(geom: Geometry, f: np.ndarray) -> np.ndarray:
    """u = −L⁻¹ f for L = Δ − λ on the periodic box: û = f̂ / (|k|²_sym + λ). When λ = 0 the
    k = 0 mode is set to zero, i.e. Δ₀⁻¹ returns the mean-zero solution (Sec. 2.2.4)."""
    lap, _ = symbols(geom.grid, geom.symbol)
    F = np.fft.fftn(f)
    den = lap + geom.lam
    U = np.zeros_like(F)
    nz = den != 0
    U[nz] = F[nz] / den[nz]
    return np.real(np.fft.ifftn(U))


def dipole_field(geom: Geometry, Q: np.ndarray) -> np.ndarray:
    """S̃Q = ∇·(S(Q n)) on the grid (Sec. 5.3.1). ``analytic``: the exact gradient of δ_h;
    ``spectral_div``: spread the vector Q n, then take the divergence with the same Fourier
    symbol family as the Laplacian (the paper's choice: match the PDE discretisation)."""
    if geom.dipole == "analytic":
        return spread_grad(geom, Q[None, :] * geom.n)
    _, der = symbols(geom.grid, geom.symbol)
    acc = np.zeros(geom.grid.shape, dtype=complex)
    for j in range(geom.grid.dim):
        acc += der[j] * np.fft.fftn(spread(geom, Q * geom.n[j]))
    return np.real(np.fft.ifftn(acc))


# ----------------------------------------------------------------------------------------
# the IBDL Schur operator (scalar: Sec. 5.3.2; Stokes: Sec. 6.3.3)
# ----------------------------------------------------------------------------------------


def field_scalar(geom: Geometry, Q: np.ndarray) -> np.ndarray:
    """u = −L⁻¹ S̃ Q on the grid (step 2 of the method in Sec. 5.1.2 with g̃ = 0); completed
    method (Sec. 5.3.3): u₀ = −Δ₀⁻¹(S̃ + ηS)Q, the mean ū added by the caller."""
    f = dipole_field(geom, Q)
    if geom.eta > 0:
        f = f + geom.eta * spread(geom, Q)
    return minus_Linv(geom, f)


def stokes_velocity(geom: Geometry, Q: np.ndarray) -> np.ndarray:
    """Velocity of the interior Stokes IBDL system (Sec. 6.1.1, Eq. "ibdl stokes"; Sec. 6.3.3
    with η = 0, g̃ = 0) on the grid, shape (d, N, …):

        u = −Δ₀⁻¹∇Δ₀⁻¹Δ S(Q·n) − Δ₀⁻¹ P ∇·(S A),   A_lm = Q_l n_m + Q_m n_l,
        P = I − ∇Δ₀⁻¹∇·.

    In Fourier space with k̃ the first-derivative symbol's wave vector and |k|² the
    Laplacian's: û = (i k̃ ŝ + P̂ ĝ)/|k|², P̂ = I − k̃k̃ᵀ/|k|², û(0) = 0, where s = S(Q·n) and
    g = ∇·(S A) (μ cancels because η = 0). Reading: Δ₀⁻¹Δ only removes the mean, which ∇
    annihilates, so the source term is −∇Δ₀⁻¹ s, the same as the Brinkman form of Sec. 6.3.2.
    ``analytic`` takes g_l = Σ_m ∂_m S(A_lm) with the exact gradient of δ_h;
    ``spectral_div`` spreads A_lm and applies the derivative symbols."""
    g = geom.grid
    d = g.dim
    Q = Q.reshape(d, geom.M)
    n = geom.n
    s_hat = np.fft.fftn(spread(geom, np.sum(Q * n, axis=0)))
    lap, der = symbols(g, geom.symbol)
    A = np.array([[Q[l] * n[m] + Q[m] * n[l] for m in range(d)] for l in range(d)])
    g_hat = []
    for l in range(d):
        if geom.dipole == "analytic":
            gl = spread_grad(geom, A[l])
            if geom.eta > 0:
                # completed method (Sec. 6.3.3, Eq. "discrete operator for Q"): (η/μ)SQ joins
                # the projected source, P((η/μ)SQ + ∇·(SA))
                gl = gl + (geom.eta / geom.mu) * spread(geom, Q[l])
            g_hat.append(np.fft.fftn(gl))
        else:
            acc = np.zeros(g.shape, dtype=complex)
            for m in range(d):
                acc += der[m] * np.fft.fftn(spread(geom, A[l, m]))
            g_hat.append(acc)
    nz = lap != 0
    inv = np.zeros(g.shape)
    inv[nz] = 1.0 / lap[nz]
    # k̃ k̃ᵀ with i k̃_l = der[l]  ⇒  k̃_l k̃_m = −der[l] der[m]
    kdotg = sum(-1j * der[m] * g_hat[m] for m in range(d))  # k̃·ĝ
    u = np.zeros((d,) + g.shape)
    for l in range(d):
        Pg = g_hat[l] - (-1j * der[l]) * kdotg * inv
        if geom.lam > 0:
            # Brinkman (Sec. 6.3.2, Eq. "brink ibdl eqn", η = 0): L = μΔ − λ, so the projected
            # dipole term is μ P̂ĝ/(μ|k|² + λ) (defined at k = 0); the source term is unchanged
            U = der[l] * s_hat * inv + Pg * (geom.mu / (geom.mu * lap + geom.lam))
        else:
            U = (der[l] * s_hat + Pg) * inv
            U[~nz] = 0.0
        u[l] = np.real(np.fft.ifftn(U))
    return u


def grid_field(geom: Geometry, Q: np.ndarray) -> np.ndarray:
    """The grid solution from a density: scalar u (shape grid) or Stokes velocity (d, grid);
    for the completed method Q carries ū after the density and u = u₀ + ū."""
    if geom.naug:
        Qd, ub = geom.split(Q)
        if geom.pde == "stokes":
            return stokes_velocity(geom, Qd.reshape(-1)) + ub[:, None, None]
        return field_scalar(geom, Qd.reshape(-1)) + ub[0]
    if geom.pde == "stokes":
        return stokes_velocity(geom, Q)
    return field_scalar(geom, Q.reshape(-1))


def apply(geom: Geometry, Q: np.ndarray) -> np.ndarray:
    """A Q = S* u + ½ Q with u the grid field of Q: scalar A Q = −S*L⁻¹S̃Q + ½Q (Sec. 5.3.2),
    Stokes A Q = S* u(Q) + ½Q (Sec. 6.3.3). Q and the result are flat SoA arrays (c·M,).
    Neumann (Sec. 5.2, Eq. "Neumann saddle point"): the jump term is −½Q and the unknown is U_b.
    Completed method (λ = 0; Sec. 5.3.3 and Sec. 6.3.3, Eq. "discrete operator for Q"): the
    unknowns are (Q, ū), the boundary rows gain ū·1 and the c constraint rows are η Σ_i Δs_i Q_i."""
    Q = np.asarray(Q, dtype=np.float64).reshape(-1)
    if geom.naug:
        if geom.lam > 0 or geom.dipole != "analytic" or geom.bc != "dirichlet":
            raise NotImplementedError("completed method: λ = 0, analytic dipole, Dirichlet data")
        Qd, ub = geom.split(Q)
        flat = Qd.reshape(-1)
        if geom.pde == "stokes":
            u = stokes_velocity(geom, flat)
            rows = np.concatenate([interp(geom, u[l]) for l in range(geom.grid.dim)]) + geom.jump * flat
        else:
            rows = interp(geom, field_scalar(geom, flat)) + geom.jump * flat
        rows = rows + np.repeat(ub, geom.M)
        return np.concatenate([rows, geom.eta * (Qd @ geom.w)])
    if geom.pde == "stokes":
        d = geom.grid.dim
        u = stokes_velocity(geom, Q)
        return np.concatenate([interp(geom, u[l]) for l in range(d)]) + geom.jump * Q
    return interp(geom, field_scalar(geom, Q)) + geom.jump * Q


def dipole_adjoint(geom: Geometry, u: np.ndarray) -> np.ndarray:
    """(S̃)* u: the adjoint of the dipole spread under ⟨f, u⟩_h = h^d Σ_g f_g u_g and
    ⟨a, b⟩_w = Σ_i Δs_i a_i b_i. analytic: Σ_m n_m Σ_g u_g ∂_m δ_h(x_g − X_i) h^d (the
    kernel-gradient gather); spectral_div: −Σ_m n_m S*(∂_m u), because the derivative symbol
    is imaginary and odd, i.e. anti-self-adjoint."""
    if geom.dipole == "analytic":
        return np.sum(geom.n * interp_grad(geom, u), axis=0)
    _, der = symbols(geom.grid, geom.symbol)
    U = np.fft.fftn(u)
    return -sum(geom.n[m] * interp(geom, np.real(np.fft.ifftn(der[m] * U)))
                for m in range(geom.grid.dim))


def adjoint_apply(geom: Geometry, W: np.ndarray) -> np.ndarray:
    """A* W for the scalar operator, adjoint with respect to the Δs-weighted boundary inner
    product. S is adjoint to S* under the weighted products (Sec. 2.1, Sec. 2.2.4), and −L⁻¹
    has a real even symbol, so it is self-adjoint; hence A* W = ½W + (S̃)*(−L⁻¹)(S W)."""
    if geom.pde != "scalar":
        raise NotImplementedError("adjoint implemented for the scalar operator")
    W = np.asarray(W, dtype=np.float64).reshape(-1)
    return geom.jump * W + dipole_adjoint(geom, minus_Linv(geom, spread(geom, W)))


def dense_operator(geom: Geometry, fn=apply) -> np.ndarray:
    """Assemble the operator column by column (c·M applications)."""
    nd = geom.ncomp * geom.M
    A = np.zeros((nd, nd))
    e = np.zeros(nd)
    for j in range(nd):
        e[:] = 0
        e[j] = 1
        A[:, j] = fn(geom, e)
    return A


# ----------------------------------------------------------------------------------------
# GMRES (Sec. 5.3.2: the Schur operator is not symmetric, so "gmres" is used)
# ----------------------------------------------------------------------------------------


@dataclass
class GmresResult:
    x: np.ndarray
    iterations: int
    history: list  # relative residual after each iteration (least-squares value)
    true_rel_residual: float


def gmres(op, b: np.ndarray, rtol: float, maxit: int = 50, x0=None) -> GmresResult:
    """Unrestarted GMRES from the definition: after k steps, x_k = x0 + V_k y_k where V_k is an
    orthonormal basis of the Krylov space K_k(A, r0) built by Arnoldi (modified Gram–Schmidt)
    and y_k = argmin ‖β e₁ − H̄_k y‖₂ (solved by a library least-squares routine). Stops at the
    first k with ‖β e₁ − H̄_k y_k‖₂ ≤ rtol·‖b‖₂ (relative Euclidean residual; reading of the
    paper's "gmres, tolerance 1e-8")."""
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    x0 = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=np.float64).reshape(-1)
    r0 = b - (op(x0) if np.any(x0) else 0.0)
    beta = float(np.linalg.norm(r0))
    bnorm = float(np.linalg.norm(b))
    if beta == 0.0:
        return GmresResult(x0, 0, [], 0.0)
    V = [r0 / beta]
    H = np.zeros((maxit + 1, maxit))
    hist = []
    y = np.zeros(0)
    k = 0
    for k in range(maxit):
        w = op(V[k])
        for j in range(k + 1):
            H[j, k] = float(np.dot(V[j], w))
            w = w - H[j, k] * V[j]
        H[k + 1, k] = float(np.linalg.norm(w))
        e1 = np.zeros(k + 2)
        e1[0] = beta
        y = np.linalg.lstsq(H[:k + 2, :k + 1], e1, rcond=None)[0]
        res = float(np.linalg.norm(e1 - H[:k + 2, :k + 1] @ y))
        hist.append(res / bnorm)
        if res <= rtol * bnorm or H[k + 1, k] == 0.0:
            break
        V.append(w / H[k + 1, k])
    x = x0 + np.stack(V[:k + 1], axis=1) @ y
    true = float(np.linalg.norm(b - op(x))) / bnorm
    return GmresResult(x, k + 1, hist, true)


def solve(geom: Geometry, Ub: np.ndarray, rtol: float, maxit: int = 50) -> GmresResult:
    """Q solving A Q = U_b (g̃ = 0, so the right-hand side is U_b; Sec. 5.1.2 step 1)."""
    return gmres(lambda q: apply(geom, q), np.asarray(Ub, dtype=np.float64).reshape(-1),
                 rtol, maxit)


def fitted_order(hs, errs) -> float:
    """Least-squares slope of log(err) against log(h)."""
    return float(np.polyfit(np.log(hs), np.log(errs), 1)[0])


def domain_norms(u_err: np.ndarray, mask: np.ndarray, h: float, dim: int, omega: float):
    """L1, L2 and max norms scaled by the area of Ω (Sec. 2.2.1)."""
    e = np.abs(u_err[mask])
    return (h ** dim / omega * e.sum(), math.sqrt(h ** dim / omega * (e * e).sum()),
            float(e.max()) if e.size else 0.0)


# ----------------------------------------------------------------------------------------
# gradients of a solve with respect to the data and the boundary (scalar operator, analytic
# dipole): for Q = A(X, n, w)⁻¹ U_b and an objective J(Q) with g = ∂J/∂Q,
#   λ = A⁻ᵀ g,  ∂J/∂U_b = λ,  ∂J/∂p = −λᵀ (∂A/∂p) Q  for p = X, n, w.
# ----------------------------------------------------------------------------------------


def ddphi_sqrt(r):
    """φ'' of the √-Peskin kernel on each piece (even in r; jumps at |r| = 0, 1, 2 are harmless
    almost everywhere)."""
    a = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(a)
    m1 = a <= 1
    m2 = (a > 1) & (a < 2)
    s = np.sqrt(1 + 4 * a[m1] - 4 * a[m1] ** 2)
    out[m1] = (-4 / s - (2 - 4 * a[m1]) * (4 - 8 * a[m1]) / (2 * s ** 3)) / 8
    t = np.sqrt(-7 + 12 * a[m2] - 4 * a[m2] ** 2)
    out[m2] = (4 / t + (6 - 4 * a[m2]) * (12 - 8 * a[m2]) / (2 * t ** 3)) / 8
    return out


def ddphi_cos(r):
    r = np.asarray(r, dtype=np.float64)
    return np.where(np.abs(r) < 2, -(np.pi ** 2 / 16) * np.cos(0.5 * np.pi * r), 0.0)


KERNELS2 = {"sqrt": ddphi_sqrt, "cos": ddphi_cos}


def transpose_apply(geom: Geometry, G: np.ndarray) -> np.ndarray:
    """Aᵀ G (Euclidean transpose). Scalar: W A* W⁻¹ G with W = diag(Δs) and A* the Δs-weighted
    adjoint; Stokes: ``stokes_transpose_apply``."""
    if geom.pde == "stokes":
        return stokes_transpose_apply(geom, G)
    G = np.asarray(G, dtype=np.float64).reshape(-1)
    return geom.w * adjoint_apply(geom, G / geom.w)


def solve_transpose(geom: Geometry, G: np.ndarray, rtol: float, maxit: int = 50) -> GmresResult:
    """λ with Aᵀ λ = G, by GMRES on the transposed operator."""
    return gmres(lambda v: transpose_apply(geom, v), np.asarray(G, dtype=np.float64).reshape(-1), rtol, maxit)


def _stencil_weights(geom: Geometry):
    """Per stencil offset: node index tuple, and per axis φ, φ', φ'' at r (φ'/h, φ''/h² in x)."""
    g = geom.grid
    phi, dphi = KERNELS[geom.delta]
    ddphi = KERNELS2[geom.delta]
    idx, r = _stencil(geom)
    for off in _offsets(g.dim):
        rr = [r[j, :, off[j]] for j in range(g.dim)]
        yield (_node_index(idx, off), [phi(x) for x in rr], [dphi(x) / g.h for x in rr],
               [ddphi(x) / g.h ** 2 for x in rr])


def spread_unweighted(geom: Geometry, c: np.ndarray) -> np.ndarray:
    """ψ_g = Σ_i c_i Φ(x_g − X_i) with Φ = Π_j φ(x_j/h) (no Δs, no h^−d)."""
    out = np.zeros(geom.grid.shape)
    for node, ph, _, _ in _stencil_weights(geom):
        np.add.at(out, node, c * np.prod(ph, axis=0))
    return out


def gather_derivatives(geom: Geometry, u: np.ndarray):
    """At every point: G_m = Σ_g u_g ∂_m Φ(x_g − X_i) and H_ml = Σ_g u_g ∂_m ∂_l Φ(x_g − X_i)
    (derivatives with respect to the argument x_g − X_i). Shapes (d, M) and (d, d, M)."""
    d, M = geom.grid.dim, geom.M
    G = np.zeros((d, M))
    H = np.zeros((d, d, M))
    for node, ph, dph, ddph in _stencil_weights(geom):
        ug = u[node]
        for m in range(d):
            G[m] += ug * np.prod([dph[j] if j == m else ph[j] for j in range(d)], axis=0)
            for l in range(d):
                if l == m:
                    f = [ddph[j] if j == m else ph[j] for j in range(d)]
                else:
                    f = [dph[j] if j in (m, l) else ph[j] for j in range(d)]
                H[m, l] += ug * np.prod(f, axis=0)
    return G, H


def param_gradient(geom: Geometry, Q: np.ndarray, lam: np.ndarray):
    """Derivatives of L = λᵀ A(X, n, w) Q (scalar operator, analytic dipole spread):
        (S*u)_j = Σ_g u_g Φ(x_g − X_j), u = −L⁻¹ f, f_g = Σ_k Δs_k Q_k n_k·∇δ_h(x_g − X_k).
    With ψ = Σ_j λ_j Φ(x_g − X_j) and v = −L⁻¹ ψ (−L⁻¹ is symmetric), λᵀS*u = vᵀ f, so
        ∂L/∂X_i = −λ_i Σ_g u_g ∇Φ(x_g − X_i) − Δs_i Q_i Σ_g v_g ∇∇δ_h(x_g − X_i) n_i,
        ∂L/∂n_i = Δs_i Q_i Σ_g v_g ∇δ_h(x_g − X_i),
        ∂L/∂Δs_i = Q_i n_i · Σ_g v_g ∇δ_h(x_g − X_i).
    φ'' jumps where a node sits at a whole-number offset (√-Peskin |r| = 1 and 2, cosine
    |r| = 2), so A is not differentiable in X_i for a point exactly on a grid line; the gradient
    there takes the value of the piece that contains the offset (a set of measure zero).
    Returns (dX (d, M), dn (d, M), dw (M,))."""
    if geom.pde != "scalar" or geom.dipole != "analytic":
        raise NotImplementedError("gradients are implemented for the scalar operator with the analytic dipole")
    Q = np.asarray(Q, dtype=np.float64).reshape(-1)
    lam = np.asarray(lam, dtype=np.float64).reshape(-1)
    hd = geom.grid.h ** geom.grid.dim
    u = field_scalar(geom, Q)
    v = minus_Linv(geom, spread_unweighted(geom, lam))
    Gu, _ = gather_derivatives(geom, u)
    Gv, Hv = gather_derivatives(geom, v)
    Gv, Hv = Gv / hd, Hv / hd
    dX = -lam[None, :] * Gu - (geom.w * Q)[None, :] * np.einsum("mli,li->mi", Hv, geom.n)
    dn = (geom.w * Q)[None, :] * Gv
    dw = Q * np.sum(geom.n * Gv, axis=0)
    return dX, dn, dw


def solve_gradient(geom: Geometry, Ub: np.ndarray, dJdQ: np.ndarray, rtol: float = 1e-13):
    """Q = A⁻¹U_b and the gradients of J with ∂J/∂Q = dJdQ: returns (Q, dUb, dX, dn, dw)."""
    Q = solve(geom, Ub, rtol, maxit=200).x
    lam = solve_transpose(geom, dJdQ, rtol, maxit=200).x
    grad = param_gradient if geom.pde == "scalar" else stokes_param_gradient
    dX, dn, dw = grad(geom, Q, lam)
    return Q, lam, -dX, -dn, -dw


# ----------------------------------------------------------------------------------------
# Stokes: transpose and boundary derivatives; values and derivatives at probe points
# ----------------------------------------------------------------------------------------
# Both operators are A Q = S*(K[s(Q); g(Q)]) + ½Q with K a Fourier multiplier and the spread
# sources linear in Q:
#   scalar  f = Σ_i w_i Q_i n_i·∇δ_h(x − X_i),                         K = −L⁻¹ (Sec. 5.3.2)
#   Stokes  s = Σ_i w_i (Q_i·n_i) δ_h,  g_m = Σ_i w_i Σ_k A_mk,i ∂_kδ_h,   A = Q nᵀ + n Qᵀ,
#           K[s; g] = F⁻¹[(i k̃ ŝ + P̂ ĝ)/|k|²],  P̂ = I − k̃k̃ᵀ/|k|²    (Sec. 6.3.3, η = 0)
# With the plain grid sum as inner product, the transpose of a real multiplier with symbol σ(k)
# has symbol conj σ(k); the transpose of S* is the unweighted spread ψ = Σ_i μ_i Φ(x − X_i).


def _multiplier_T(geom: Geometry, psi):
    """Kᵀψ for ψ of shape (c, grid): scalar → [v] with v = −L⁻¹ψ (real even symbol);
    Stokes → [v_s, v_g1, …, v_gd] with v̂_s = −i k̃·ψ̂/|k|², v̂_g = P̂ψ̂/|k|²."""
    if geom.pde == "scalar":
        return [minus_Linv(geom, psi[0])]
    g = geom.grid
    d = g.dim
    lap, der = symbols(g, geom.symbol)
    nz = lap != 0
    inv = np.zeros(g.shape)
    inv[nz] = 1.0 / lap[nz]
    kt = [-1j * der[l] for l in range(d)]  # k̃_l (real values), i k̃_l = der[l]
    P = [np.fft.fftn(psi[l]) for l in range(d)]
    kp = sum(kt[l] * P[l] for l in range(d))
    vs = np.real(np.fft.ifftn(-1j * kp * inv))
    ginv = geom.mu / (geom.mu * lap + geom.lam) if geom.lam > 0 else inv  # Brinkman: μ/(μ|k|² + λ)
    vg = [np.real(np.fft.ifftn((P[m] - kt[m] * kp * inv) * ginv)) for m in range(d)]
    return [vs] + vg


def _spread_terms(geom: Geometry, Q: np.ndarray, v):
    """For the spread sources of Q (analytic dipole) and adjoint grid fields v = Kᵀψ, the
    pieces of ⟨v, sources(Q)⟩:
        dQ = ∂/∂Q (the spread transpose), dX, dn, dw = ∂/∂X, ∂/∂n, ∂/∂Δs at fixed Q.
    Shapes: dQ (c, M), dX and dn (d, M), dw (M,)."""
    if geom.dipole != "analytic":
        raise NotImplementedError("derivatives are implemented for the analytic dipole spread")
    d, M = geom.grid.dim, geom.M
    hd = geom.grid.h ** d
    ws = geom.w / hd
    n = geom.n
    if geom.pde == "scalar":
        q = Q.reshape(M)
        G, H = gather_derivatives(geom, v[0])
        dQ = (ws * np.sum(n * G, axis=0))[None, :]
        dX = -(ws * q)[None, :] * np.einsum("mli,li->mi", H, n)
        dn = (ws * q)[None, :] * G
        dw = q * np.sum(n * G, axis=0) / hd
        return dQ, dX, dn, dw
    Q = Q.reshape(d, M)
    c = np.sum(Q * n, axis=0)
    A = np.array([[Q[m] * n[k] + Q[k] * n[m] for k in range(d)] for m in range(d)])  # (d, d, M)
    a_s = interp(geom, v[0])
    Gs, _ = gather_derivatives(geom, v[0])
    G, H = zip(*[gather_derivatives(geom, v[1 + m]) for m in range(d)])
    G, H = np.array(G), np.array(H)  # G[m, k] = Σ v_gm ∂_kΦ, H[m, k, j] = Σ v_gm ∂_k∂_jΦ
    dQ = np.array([ws * (n[l] * a_s + sum(n[k] * (G[l, k] + G[k, l]) for k in range(d))) for l in range(d)])
    dX = -ws[None, :] * (c[None, :] * Gs + np.einsum("mki,mkji->ji", A, H))
    dn = ws[None, :] * np.array([Q[j] * a_s + sum(Q[m] * G[m, j] for m in range(d))
                                 + sum(Q[k] * G[j, k] for k in range(d)) for j in range(d)])
    dw = (c * a_s + np.einsum("mki,mki->i", A, G)) / hd
    return dQ, dX, dn, dw


def stokes_transpose_apply(geom: Geometry, mu: np.ndarray) -> np.ndarray:
    """Aᵀμ for the Stokes operator: ½μ + (spread transpose)(Kᵀ Σ_i μ_i Φ(x − X_i))."""
    d, M = geom.grid.dim, geom.M
    mu = np.asarray(mu, dtype=np.float64).reshape(d, M)
    psi = [spread_unweighted(geom, mu[l]) for l in range(d)]
    dQ, _, _, _ = _spread_terms(geom, np.zeros(d * M), _multiplier_T(geom, psi))
    return (geom.jump * mu + dQ).reshape(-1)


def stokes_param_gradient(geom: Geometry, Q: np.ndarray, mu: np.ndarray):
    """Derivatives of L = μᵀ A(X, n, w) Q for the Stokes operator (analytic dipole):
    the interpolation term −Σ_l μ_{l,i} Σ_g u_l ∇Φ(x_g − X_i) with u the velocity of Q, plus the
    spread terms of ⟨Kᵀψ, sources(Q)⟩ with ψ_l = Σ_j μ_{l,j} Φ(x − X_j)."""
    d, M = geom.grid.dim, geom.M
    Q = np.asarray(Q, dtype=np.float64).reshape(d, M)
    mu = np.asarray(mu, dtype=np.float64).reshape(d, M)
    u = stokes_velocity(geom, Q.reshape(-1))
    dX = np.zeros((d, M))
    for l in range(d):
        Gu, _ = gather_derivatives(geom, u[l])
        dX -= mu[l][None, :] * Gu
    psi = [spread_unweighted(geom, mu[l]) for l in range(d)]
    _, sX, sn, sw = _spread_terms(geom, Q, _multiplier_T(geom, psi))
    return dX + sX, sn, sw


def mean_inflow(geom: Geometry, x: np.ndarray) -> float:
    """U = ∫ u(x₀, y) dy along the left edge x₀ of the box (Sec. 6.5.3: the average horizontal
    velocity on the left side), by the grid sum over that column of nodes."""
    u = grid_field(geom, x)
    return float(u[0][:, 0].sum() * geom.grid.h)


def net_force(geom: Geometry, x: np.ndarray) -> np.ndarray:
    """B = −η ∫_Γ Q ds of the completed Stokes method (Sec. 6.1.3)."""
    Qd, _ = geom.split(x)
    return -geom.eta * (Qd @ geom.w)


def single_layer(geom: Geometry, V: np.ndarray) -> np.ndarray:
    """S*(−L⁻¹)(S V): the single-layer operator of the scalar method (the IBSL Schur complement up
    to sign, Sec. 2.2.3), which carries the Neumann data into the right-hand side."""
    if geom.pde != "scalar":
        raise NotImplementedError("single layer: scalar operator")
    return interp(geom, minus_Linv(geom, spread(geom, np.asarray(V, dtype=np.float64).reshape(-1))))


def neumann_rhs(geom: Geometry, Vb: np.ndarray) -> np.ndarray:
    """Right-hand side S*L⁻¹SV_b of the Neumann equation (Sec. 5.2, Eq. "Neumann saddle point",
    g̃ = 0) for the normal derivative V_b: −single_layer(V_b)."""
    return -single_layer(geom, Vb)


def probe_geometry(geom: Geometry, P: np.ndarray) -> Geometry:
    """The probe points P (d, n_p) as a point set on the same grid (normals and weights unused)."""
    P = np.asarray(P, dtype=np.float64)
    nrm = np.zeros_like(P)
    nrm[0] = 1.0
    return Geometry(geom.grid, P, nrm, np.ones(P.shape[1]), geom.delta, geom.dipole, geom.symbol, geom.pde,
                    geom.lam, geom.mu)


def probe_evaluate(geom: Geometry, P: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """E Q: the grid solution of Q (Sec. 5.1.2 step 2) interpolated at the probes with δ_h,
    u(p) = Σ_g u_g δ_h(x_g − p) h^d. Shape (c, n_p)."""
    pg = probe_geometry(geom, P)
    u = grid_field(geom, np.asarray(Q, dtype=np.float64))
    if geom.pde == "scalar":
        return interp(pg, u)[None, :]
    return np.array([interp(pg, u[l]) for l in range(geom.grid.dim)])


def probe_vjp(geom: Geometry, P: np.ndarray, Q: np.ndarray, nu: np.ndarray):
    """For ν of shape (c, n_p): (Eᵀν, ∂(νᵀ E Q)/∂X, ∂/∂n, ∂/∂Δs) with E = E(X, n, Δs) and the
    probes fixed. Eᵀν spreads ν at the probes (unweighted), applies Kᵀ and the spread transpose."""
    pg = probe_geometry(geom, P)
    c = geom.ncomp
    nu = np.asarray(nu, dtype=np.float64).reshape(c, -1)
    psi = [spread_unweighted(pg, nu[l]) for l in range(c)]
    return _spread_terms(geom, np.asarray(Q, dtype=np.float64), _multiplier_T(geom, psi))


# ----------------------------------------------------------------------------------------
# solution post-processing: indicator flagging (Sec. 5.3.5) and near-boundary interpolation
# (Sec. 5.3.4)
# ----------------------------------------------------------------------------------------


def indicator(geom: Geometry):
    """The regularised indicator of the region enclosed by the discrete curve(s), Sec. 5.3.5:
    χ solves Δχ = −S̃1 (the IBDL grid field of the unit density for the Laplacian, mean-zero
    inverse, whatever PDE the geometry carries; its δ_h, dipole spread and symbol are kept),
    shifted so that χ = 0 at the box corner (grid node 0), and the flags |χ| > ½.

    Reading: the paper thresholds χ itself at ½ for outward normals; |χ| flags the enclosed
    nodes for either orientation of the normals (χ ≈ −1 inside when the normals point inward,
    as for an exterior problem). Returns (χ, flags) on the grid."""
    g0 = Geometry(geom.grid, geom.X, geom.n, geom.w, geom.delta, geom.dipole, geom.symbol, "scalar", 0.0)
    chi = field_scalar(g0, np.ones(geom.M))
    chi = chi - chi.flat[0]
    return chi, np.abs(chi) > 0.5


def min_image(d, L):
    """Minimum-image offset in a periodic box of side L: d − L·round(d/L) (ties to even)."""
    return d - L * np.round(d / L)


def nearest_three(geom: Geometry, p):
    """The three boundary points nearest to the point p (2-D), ordered by the squared
    minimum-image distance dx·dx + dy·dy in FP64, equal distances by index. Returns the indices
    and the offsets X_i − p of all points."""
    d = min_image(geom.X - np.asarray(p, dtype=np.float64)[:, None], geom.grid.box)
    d2 = d[0] * d[0] + d[1] * d[1]
    order = np.lexsort((np.arange(geom.M), d2))
    return order[:3], d, d2


def chord_foot(d, i1, i2):
    """x_A − x_p on the chord from x_1 to x_2 (offsets d relative to x_p), Sec. 5.3.4: the point of
    the line through x_1, x_2 closest to x_p, x_A = x_2 + t(x_1 − x_2) with
    t = (x_p − x_2)·(x_1 − x_2)/|x_1 − x_2|². Reading: the printed projection has the sign of
    (x_2 − x_p) reversed against the text, which asks for the closest point; the text decides.
    Returns (x_A − x_p, t)."""
    x1, x2 = d[:, i1], d[:, i2]
    seg = x1 - x2
    t = float(-(x2 @ seg) / (seg @ seg))
    return x2 + t * seg, t


def near_boundary_interp(geom: Geometry, Ub, u, omega, m1: float = 6.0, m2: float = 8.0) -> np.ndarray:
    """Sec. 5.3.4 (2-D), per component of u ((c, N, N) or (N, N)): every node x_p of the mask
    ``omega`` whose nearest boundary point lies closer than m1·h gets
        u(x_p) = u_A |x_B − x_p|/|x_B − x_A| + u_B |x_A − x_p|/|x_B − x_A|,
    x_A the foot of x_p on the chord of its two nearest boundary points x_1, x_2 (when t falls
    outside [0, 1]: on the chord of the two outermost of the three nearest points, i.e. the
    pair farthest apart, t then clamped to [0, 1]), u_A = U_b(x_1)|x_A − x_2|/|x_2 − x_1| +
    U_b(x_2)|x_A − x_1|/|x_2 − x_1|, x_B = x_A + m2·h (x_p − x_A)/|x_p − x_A| and u_B the bilinear
    interpolation of the four grid values around x_B. A node on the chord (x_A = x_p) takes u_A.
    Other nodes keep their values. Distances by minimum image; the node set, the neighbours and
    the fallback are decided on squared FP64 distances. The paper's settings: m1 = 6, m2 = 8
    (finite differences); m1 = 2(log₂N − 4), m2 = m1 + 2 (spectral)."""
    grid = geom.grid
    if grid.dim != 2:
        raise NotImplementedError("near-boundary interpolation: 2-D")
    h, N = grid.h, grid.N
    c = geom.ncomp
    U = np.asarray(u, dtype=np.float64).reshape((c, N, N))
    Ubc = np.asarray(Ub, dtype=np.float64).reshape(-1)[: c * geom.M].reshape(c, geom.M)
    out = U.copy()
    xs, ys = grid.coords()
    r1 = m1 * h
    for iy, ix in zip(*np.nonzero(np.asarray(omega).reshape(N, N))):
        p = np.array([xs[iy, ix], ys[iy, ix]])
        three, d, d2 = nearest_three(geom, p)
        if not d2[three[0]] < r1 * r1:
            continue
        i1, i2 = three[0], three[1]
        xA, t = chord_foot(d, i1, i2)
        if t < 0.0 or t > 1.0:
            pairs = [(three[0], three[1]), (three[0], three[2]), (three[1], three[2])]
            sep = [np.sum((d[:, a] - d[:, b]) ** 2) for a, b in pairs]
            i1, i2 = pairs[int(np.argmax(sep))]
            xA, t = chord_foot(d, i1, i2)
            t = min(1.0, max(0.0, t))
            xA = d[:, i2] + t * (d[:, i1] - d[:, i2])
        lseg = math.hypot(*(d[:, i1] - d[:, i2]))
        wa1 = math.hypot(*(xA - d[:, i2])) / lseg  # weight of U_b(x_1)
        wa2 = math.hypot(*(xA - d[:, i1])) / lseg  # weight of U_b(x_2)
        rA = math.hypot(*xA)  # |x_A − x_p|
        if rA == 0.0:
            out[:, iy, ix] = Ubc[:, i1] * wa1 + Ubc[:, i2] * wa2
            continue
        xB = xA - xA / rA * (m2 * h)  # x_p is the origin: x_B − x_p
        gx = (p[0] + xB[0] - grid.origin[0]) / h
        gy = (p[1] + xB[1] - grid.origin[1]) / h
        jx, jy = int(math.floor(gx)), int(math.floor(gy))
        ax, ay = gx - jx, gy - jy
        rB = math.hypot(*xB)  # |x_B − x_p|
        for comp in range(c):
            uA = Ubc[comp, i1] * wa1 + Ubc[comp, i2] * wa2
            F = U[comp]
            uB = ((1 - ax) * (1 - ay) * F[jy % N, jx % N] + ax * (1 - ay) * F[jy % N, (jx + 1) % N]
                  + (1 - ax) * ay * F[(jy + 1) % N, jx % N] + ax * ay * F[(jy + 1) % N, (jx + 1) % N])
            out[comp, iy, ix] = (uA * rB + uB * rA) / (m2 * h)
    return out.reshape(np.shape(u))


# ----------------------------------------------------------------------------------------
# source term g̃ (Sec. 5.1.2 and Eq. "ibdl schur again"; Sec. 6.1.1, Eq. "ibdl stokes")
# ----------------------------------------------------------------------------------------


def source_field(geom: Geometry, g: np.ndarray) -> np.ndarray:
    """u_g, the grid response to the source g̃ on C alone, with the geometry's symbols.

    Scalar, L u + S̃Q = g̃: u = −L⁻¹S̃Q + L⁻¹g̃, so u_g = L⁻¹g̃, û_g = −ĝ/(|k|² + λ); for λ = 0 the
    mean of g̃ is dropped (Δ₀⁻¹; reading: the mean enters only the completed method's constraint).
    Stokes/Brinkman, L u − ∇p + μ∇·(SA) = g̃ with L = μΔ − λ and ∇·u = −S(Q·n): the g̃ part is the
    divergence-free solution of L u − ∇p = g̃, û_g = −P̂ĝ/(μ|k|² + λ) with the projection P̂ of the
    operator's own Stokes term; û_g(0) = 0 when λ = 0, −ĝ(0)/λ otherwise."""
    grid = geom.grid
    if geom.pde != "stokes":
        return -minus_Linv(geom, np.asarray(g, dtype=np.float64).reshape(grid.shape))
    d = grid.dim
    G = [np.fft.fftn(np.asarray(g, dtype=np.float64).reshape((d,) + grid.shape)[l]) for l in range(d)]
    lap, der = symbols(grid, geom.symbol)
    nz = lap != 0
    inv = np.zeros(grid.shape)
    inv[nz] = 1.0 / lap[nz]
    kdotg = sum(-1j * der[m] * G[m] for m in range(d))
    den = geom.mu * lap + geom.lam
    u = np.zeros((d,) + grid.shape)
    for l in range(d):
        PG = G[l] - (-1j * der[l]) * kdotg * inv
        U = np.zeros_like(PG)
        ok = den != 0
        U[ok] = -PG[ok] / den[ok]
        u[l] = np.real(np.fft.ifftn(U))
    return u


def forced_rhs(geom: Geometry, Ub: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Right-hand side of the Schur system with a source: U_b − S*u_g (Eq. "ibdl schur again":
    −S*L⁻¹S̃Q + ½Q = U_b − S*L⁻¹g̃; the Stokes system alike). Completed method (Sec. 5.3.3,
    Sec. 6.3.3): its c constraint rows are h^d Σ_g g̃_l, replacing whatever U_b held there."""
    c, M = geom.ncomp, geom.M
    ug = source_field(geom, g).reshape((c,) + geom.grid.shape)
    rows = np.asarray(Ub, dtype=np.float64).reshape(-1)[: c * M] - np.concatenate(
        [interp(geom, ug[l]) for l in range(c)])
    if geom.naug:
        gs = np.asarray(g, dtype=np.float64).reshape(c, -1)
        return np.concatenate([rows, geom.grid.h ** geom.grid.dim * gs.sum(axis=1)])
    return rows


def forced_field(geom: Geometry, Q: np.ndarray, g: np.ndarray) -> np.ndarray:
    """The grid solution with a source: the field of Q plus u_g (Sec. 5.1.2 step 2)."""
    u = grid_field(geom, Q)
    return u + source_field(geom, g).reshape(u.shape)


# ----------------------------------------------------------------------------------------
# normals and weights estimated from the points (Sec. 5.3.1)
# ----------------------------------------------------------------------------------------


def estimate_normals(X: np.ndarray, box: float) -> np.ndarray:
    """Unit normals of one closed 2-D curve from its ordered points, Sec. 5.3.1 (Eq. "normal vector
    approximations"): n_i = (Y_{i+1} − Y_{i−1}, −(X_{i+1} − X_{i−1}))/‖X_{i+1} − X_{i−1}‖, differences by
    minimum image. The normal points to the right of the direction of travel: outward for a
    counter-clockwise curve (interior domain), inward for a clockwise one (exterior domain)."""
    X = np.asarray(X, dtype=np.float64)
    d = min_image(np.roll(X, -1, axis=1) - np.roll(X, 1, axis=1), box)
    n = np.stack([d[1], -d[0]])
    return n / np.hypot(d[0], d[1])


def estimate_weights(X: np.ndarray, box: float) -> np.ndarray:
    """Δs_i ≈ ‖X_{i+1} − X_i‖ (Sec. 5.3.1), minimum image, one closed curve."""
    X = np.asarray(X, dtype=np.float64)
    d = min_image(np.roll(X, -1, axis=1) - X, box)
    return np.hypot(d[0], d[1])
