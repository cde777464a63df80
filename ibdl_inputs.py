"""Seeded synthetic inputs for the IBDL operator: boundary curves/surfaces and boundary data.

This module is shared by the FP64 oracle, the CUDA path's tests, ``bench.py`` and the smoke
check. It holds none of the IBDL method's arithmetic (no delta kernel, spread, Fourier solve
or Krylov step): it only places boundary points, their outward unit normals and quadrature
weights on the shapes the paper and the workloads use, and evaluates boundary data.

Conventions (shared by both sides):
  * points ``X`` are SoA arrays of shape ``(d, M)``; normals ``n`` the same; weights ``w`` ``(M,)``.
  * Curves are traversed counter-clockwise and sampled equispaced in arclength, so every
    weight equals ``perimeter / M`` (Sec. 2.2.2 and Sec. 5.3.1: equally spaced points,
    ``Δs = L_IB / N_IB``).
  * Normals point out of the interior domain Ω (Sec. 5.1.1).
  * The periodic box is ``[origin, origin + box)^d``; the workloads use the unit box.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------------------
# closed curves sampled equispaced in arclength
# ----------------------------------------------------------------------------------------


@dataclass
class Boundary:
    """Discrete boundary: points, outward unit normals, quadrature weights, curve parameter."""

    X: np.ndarray  # (d, M)
    n: np.ndarray  # (d, M)
    w: np.ndarray  # (M,)
    t: np.ndarray  # (M,) arclength parameter mapped to [0, 2π) (curves) or point index (surfaces)
    measure: float  # perimeter (2-D) or area (3-D) of Γ
    enclosed: float  # area (2-D) or volume (3-D) of Ω
    meta: dict = field(default_factory=dict)

    @property
    def M(self) -> int:
        return int(self.X.shape[1])

    @property
    def dim(self) -> int:
        return int(self.X.shape[0])


def _curve_by_arclength(radius_fn, M: int, center, rot: float = 0.0, nq: int = 4096) -> Boundary:
    """Sample a star-shaped curve ``c + Rot(rot) r(θ)(cos θ, sin θ)`` at M points equispaced in
    arclength. ``radius_fn(θ)`` returns ``(r, dr/dθ)``. The speed |X'(θ)| is expanded in a
    Fourier series (spectrally accurate for smooth periodic curves), integrated term by term,
    and the arclength map is inverted by Newton's method."""
    th = 2 * np.pi * np.arange(nq) / nq
    r, dr = radius_fn(th)
    speed = np.sqrt(r * r + dr * dr)
    c = np.fft.rfft(speed) / nq  # speed ≈ c0 + 2 Re Σ_{k≥1} c_k e^{ikθ}
    # keep the modes above the FFT's round-off floor (≈ 1e-16 |c0|)
    big = np.nonzero(np.abs(c[1:]) > 1e-15 * abs(c[0]))[0]
    kmax = min(max(int(big[-1]) + 2 if big.size else 16, 16), len(c) - 1)
    ck = c[1:kmax + 1]
    kk = np.arange(1, kmax + 1)
    perimeter = 2 * np.pi * c[0].real

    def s_of(theta):
        e = np.exp(1j * np.outer(theta, kk))
        return c[0].real * theta + 2 * np.real(((e - 1) / (1j * kk)) @ ck)

    def speed_of(theta):
        rr, dd = radius_fn(theta)
        return np.sqrt(rr * rr + dd * dd)

    target = perimeter * np.arange(M) / M
    theta = 2 * np.pi * np.arange(M) / M
    for _ in range(60):
        step = (s_of(theta) - target) / speed_of(theta)
        theta = theta - step
        if np.max(np.abs(step)) < 1e-15:
            break
    r, dr = radius_fn(theta)
    ct, st = np.cos(theta), np.sin(theta)
    x = r * ct
    y = r * st
    tx = dr * ct - r * st
    ty = dr * st + r * ct
    tn = np.sqrt(tx * tx + ty * ty)
    tx, ty = tx / tn, ty / tn
    nx, ny = ty, -tx  # outward for a counter-clockwise curve
    cr, sr = math.cos(rot), math.sin(rot)
    X = np.stack([center[0] + cr * x - sr * y, center[1] + sr * x + cr * y])
    n = np.stack([cr * nx - sr * ny, sr * nx + cr * ny])
    # enclosed area = ½ ∫ r² dθ
    area = 0.5 * np.mean(radius_fn(th)[0] ** 2) * 2 * np.pi
    w = np.full(M, perimeter / M)
    return Boundary(X=X, n=n, w=w, t=2 * np.pi * np.arange(M) / M, measure=perimeter,
                    enclosed=area, meta={"theta": theta})


def circle(M: int, R: float = 0.25, center=(0.5, 0.5)) -> Boundary:
    """Circle of radius R, M points at θ_i = 2πi/M, normals (cos θ, sin θ), Δs = 2πR/M."""
    th = 2 * np.pi * np.arange(M) / M
    X = np.stack([center[0] + R * np.cos(th), center[1] + R * np.sin(th)])
    n = np.stack([np.cos(th), np.sin(th)])
    w = np.full(M, 2 * np.pi * R / M)
    return Boundary(X=X, n=n, w=w, t=th, measure=2 * np.pi * R, enclosed=np.pi * R * R,
                    meta={"theta": th, "R": R, "center": tuple(center)})


def star(M: int, a: float = 0.25, eps: float = 0.2, k: int = 5, center=(0.5, 0.5)) -> Boundary:
    """Star r(θ) = a(1 + eps cos kθ), equispaced in arclength (the Stokes workload's curve)."""

    def rf(th):
        return a * (1 + eps * np.cos(k * th)), -a * eps * k * np.sin(k * th)

    b = _curve_by_arclength(rf, M, center)
    b.meta.update({"a": a, "eps": eps, "k": k, "center": tuple(center)})
    return b


def ellipse(M: int, a: float, b: float, rot: float = 0.0, center=(0.5, 0.5)) -> Boundary:
    """Ellipse with semi-axes a, b rotated by ``rot``, equispaced in arclength."""

    def rf(th):
        c, s = np.cos(th), np.sin(th)
        q = (c / a) ** 2 + (s / b) ** 2
        r = 1 / np.sqrt(q)
        dq = 2 * c * s * (1 / b ** 2 - 1 / a ** 2)
        return r, -0.5 * dq * q ** -1.5

    out = _curve_by_arclength(rf, M, center, rot=rot)
    out.enclosed = math.pi * a * b
    out.meta.update({"a": a, "b": b, "rot": rot, "center": tuple(center)})
    return out


def fibonacci_sphere(M: int, R: float = 0.25, center=(0.5, 0.5, 0.5)) -> Boundary:
    """Quasi-uniform Fibonacci lattice on a sphere; radial normals; equal area weights 4πR²/M."""
    i = np.arange(M)
    z = 1 - (2 * i + 1) / M
    rho = np.sqrt(1 - z * z)
    ga = np.pi * (3 - math.sqrt(5))
    ph = i * ga
    n = np.stack([rho * np.cos(ph), rho * np.sin(ph), z])
    X = np.asarray(center, dtype=float)[:, None] + R * n
    w = np.full(M, 4 * np.pi * R * R / M)
    return Boundary(X=X, n=n, w=w, t=i.astype(float), measure=4 * np.pi * R * R,
                    enclosed=4 / 3 * np.pi * R ** 3, meta={"R": R, "center": tuple(center)})


def points_for_spacing(measure: float, h: float, alpha: float = 1.0) -> int:
    """Number of points giving Δs ≈ alpha·h on a curve of the given perimeter."""
    return max(8, int(round(measure / (alpha * h))))


# ----------------------------------------------------------------------------------------
# boundary data and exact solutions (test data, evaluated pointwise)
# ----------------------------------------------------------------------------------------


def harmonic_cubic(x, y, z0=(0.5, 0.5)):
    """Re((x + iy − z0)^3), harmonic in the plane."""
    xp, yp = x - z0[0], y - z0[1]
    return xp ** 3 - 3 * xp * yp * yp


def harmonic_3d(x, y, z):
    """x² − y² + z(x − 0.5), harmonic in space."""
    return x * x - y * y + z * (x - 0.5)


def stokes_poly(x, y, c=(0.5, 0.5)):
    """Polynomial Stokes flow from the stream function ψ = r²x' (μ = 1):
    u = (2x'y', −(3x'² + y'²)), p = −8y'. Divergence free and μΔu = ∇p."""
    xp, yp = x - c[0], y - c[1]
    return np.stack([2 * xp * yp, -(3 * xp * xp + yp * yp)])


def rigid_rotation(x, y, c=(0.5, 0.5), omega=1.0):
    xp, yp = x - c[0], y - c[1]
    return np.stack([-omega * yp, omega * xp])


def random_modes(t, K: int, amp: float, rng: np.random.Generator, ncomp: int, decay: bool = False):
    """Smooth random periodic data Σ_{m=0}^{K} (a_m cos mt + b_m sin mt) per component,
    a_m, b_m ~ N(0,1)·amp/√(2K+1) (times 1/(1+m) when ``decay``)."""
    out = np.zeros((ncomp, t.size))
    m = np.arange(K + 1)
    scale = amp / math.sqrt(2 * K + 1) * (1.0 / (1 + m) if decay else np.ones(K + 1))
    for c in range(ncomp):
        a = rng.standard_normal(K + 1) * scale
        b = rng.standard_normal(K + 1) * scale
        out[c] = np.cos(np.outer(t, m)) @ a + np.sin(np.outer(t, m)) @ b
    return out


def remove_normal_flux(U: np.ndarray, bd: Boundary) -> tuple[np.ndarray, float]:
    """Make vector boundary data flux free: U ← U − (Σ w U·n / Σ w) n. Interior Stokes
    Dirichlet data must carry no net flux through Γ (incompressibility). Returns the
    corrected data and the removed flux Σ w U·n."""
    flux = float(np.sum(bd.w * np.sum(U * bd.n, axis=0)))
    return U - (flux / float(np.sum(bd.w))) * bd.n, flux


# ----------------------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------------------


@dataclass
class Problem:
    """One boundary-value problem: grid, boundary, data and operator options."""

    name: str
    dim: int
    N: int
    box: float
    origin: tuple
    bd: Boundary
    Ub: np.ndarray  # (c, M)
    pde: str  # "scalar" | "stokes"
    lam: float = 0.0
    mu: float = 1.0
    delta: str = "cos"  # "cos" | "sqrt"
    dipole: str = "analytic"  # "analytic" | "spectral_div"
    symbol: str = "spectral"  # "spectral" | "fd2"
    rtol: float = 1e-10
    meta: dict = field(default_factory=dict)
    bc: str = "dirichlet"  # "dirichlet": Ub holds U_b; "neumann": Ub holds V_b = ∂u/∂n (Sec. 5.2)
    eta: float = 0.0  # completed method (η > 0, λ = 0): the unknowns gain one mean per component

    @property
    def h(self) -> float:
        return self.box / self.N

    @property
    def ncomp(self) -> int:
        return self.dim if self.pde == "stokes" else 1


def circle_laplace(N: int = 64, M: int = 100, delta: str = "cos", dipole: str = "analytic",
                   symbol: str = "spectral", lam: float = 0.0) -> Problem:
    """2-D Laplace Dirichlet on the unit periodic box: circle R = 0.25 about (0.5, 0.5),
    boundary data Re((z − z0)^3), GMRES to 1e-10 (the 64² / 100-point circle workload)."""
    bd = circle(M)
    Ub = harmonic_cubic(bd.X[0], bd.X[1])[None, :]
    return Problem("circle_laplace", 2, N, 1.0, (0.0, 0.0), bd, Ub, "scalar", lam=lam,
                   delta=delta, dipole=dipole, symbol=symbol, rtol=1e-10)


def star_stokes(N: int = 512, M: int = 800, seed: int = 2, delta: str = "cos",
                dipole: str = "analytic", symbol: str = "spectral", K: int = 8,
                amp: float = 0.1) -> Problem:
    """2-D steady Stokes (μ = 1) on the unit periodic box: star r(θ) = 0.25(1 + 0.2 cos 5θ)
    about (0.5, 0.5); rigid rotation plus seeded smooth random modes |m| ≤ K, amplitude amp,
    made flux free. The 512² / 800-point star is the Stokes workload."""
    bd = star(M)
    rng = np.random.default_rng(seed)
    U = rigid_rotation(bd.X[0], bd.X[1]) + random_modes(bd.t, K, amp, rng, 2)
    U, flux = remove_normal_flux(U, bd)
    return Problem("star_stokes", 2, N, 1.0, (0.0, 0.0), bd, U, "stokes", mu=1.0,
                   delta=delta, dipole=dipole, symbol=symbol, rtol=1e-8,
                   meta={"removed_flux": flux, "seed": seed})


def star_probes(n_probes: int = 64, N: int = 1024, min_dist_h: float = 8.0, seed: int = 5,
                a: float = 0.25, eps: float = 0.2, k: int = 5, center=(0.5, 0.5)) -> np.ndarray:
    """Probe points inside the star r(θ) = a(1 + eps cos kθ), uniform in area, at distance at
    least min_dist_h·h (h = 1/N) from the curve (distance to 2¹⁶ samples of the curve).
    Shape (2, n_probes)."""
    rng = np.random.default_rng(seed)
    th = np.linspace(0, 2 * np.pi, 1 << 16, endpoint=False)
    rc = a * (1 + eps * np.cos(k * th))
    curve = np.stack([center[0] + rc * np.cos(th), center[1] + rc * np.sin(th)])
    rmax = a * (1 + eps)
    out = []
    while len(out) < n_probes:
        x = center[0] + rmax * rng.uniform(-1, 1)
        y = center[1] + rmax * rng.uniform(-1, 1)
        t = np.arctan2(y - center[1], x - center[0])
        if np.hypot(x - center[0], y - center[1]) >= a * (1 + eps * np.cos(k * t)):
            continue
        if np.min(np.hypot(curve[0] - x, curve[1] - y)) < min_dist_h / N:
            continue
        out.append((x, y))
    return np.array(out).T


def star_stokes_probes(N: int = 1024, M: int = 1600, n_probes: int = 64, probe_seed: int = 5,
                       **kw) -> tuple[Problem, np.ndarray]:
    """The differentiation workload: the Stokes star problem at N², M points (same data recipe
    as ``star_stokes``) and n_probes probes inside the star at ≥ 8h from it. The objective is
    J = Σ_p |u(p)|² with u(p) the δ_h interpolation of the grid velocity."""
    return star_stokes(N, M, **kw), star_probes(n_probes, N, seed=probe_seed)


def sphere_poisson(N: int = 128, M: int = 12000, delta: str = "cos", lam: float = 0.0,
                   dipole: str = "analytic", symbol: str = "spectral") -> Problem:
    """3-D Laplace on the unit periodic box: sphere R = 0.25 about (0.5,0.5,0.5), Fibonacci
    points, boundary data x² − y² + z(x − 0.5)."""
    bd = fibonacci_sphere(M)
    Ub = harmonic_3d(bd.X[0], bd.X[1], bd.X[2])[None, :]
    return Problem("sphere_poisson", 3, N, 1.0, (0.0, 0.0, 0.0), bd, Ub, "scalar", lam=lam,
                   delta=delta, dipole=dipole, symbol=symbol, rtol=1e-8)


def ellipse_batch(B: int = 256, seed: int = 3, grids=(128, 256, 512)) -> list[Problem]:
    """Batch of independent screened-Poisson problems: N ~ U{grids}, λ ~ U[0, 100], ellipse
    semi-axes ~ U[0.1, 0.3], orientation ~ U[0, π), centre (0.5, 0.5), Δs ≈ h, smooth random
    data |m| ≤ 6 with 1/(1+m) decay."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(B):
        N = int(rng.choice(grids))
        lam = float(rng.uniform(0, 100))
        a, b = rng.uniform(0.1, 0.3, size=2)
        rot = float(rng.uniform(0, np.pi))
        # perimeter via the arclength sampler at a fine resolution, then Δs ≈ h
        probe = ellipse(64, a, b, rot)
        M = points_for_spacing(probe.measure, 1.0 / N)
        bd = ellipse(M, a, b, rot)
        Ub = random_modes(bd.t, 6, 1.0, rng, 1, decay=True)
        out.append(Problem(f"ellipse_{i}", 2, N, 1.0, (0.0, 0.0), bd, Ub, "scalar", lam=lam,
                           rtol=1e-8, meta={"a": a, "b": b, "rot": rot}))
    return out


def paper_circle_helmholtz(N: int, alpha: float, delta: str = "sqrt", symbol: str = "fd2",
                           dipole: str = "spectral_div") -> Problem:
    """The paper's circle test (Sec. 5.4.1): Δu − u = 0 inside r = 0.25 centred in the box
    [−0.5, 0.5]², U_b = sin 2θ, Δs ≈ alpha·Δx, finite differences, √-Peskin delta."""
    h = 1.0 / N
    M = points_for_spacing(2 * np.pi * 0.25, h, alpha)
    bd = circle(M, 0.25, (0.0, 0.0))
    th = bd.meta["theta"]
    Ub = np.sin(2 * th)[None, :]
    return Problem("paper_circle_helmholtz", 2, N, 1.0, (-0.5, -0.5), bd, Ub, "scalar",
                   lam=1.0, delta=delta, dipole=dipole, symbol=symbol, rtol=1e-8,
                   meta={"alpha": alpha})


def paper_circle_neumann(N: int, alpha: float = 0.75, lam: float = 1.0, delta: str = "sqrt",
                         symbol: str = "fd2", dipole: str = "analytic") -> Problem:
    """Neumann problem on the paper's circle (Sec. 5.2; geometry of Sec. 5.6): Δu − λu = 0 inside
    r = 0.25 centred in [−0.5, 0.5]², u = I₂(√λ r) sin 2θ / I₂(√λ R), so the unknown U_b = u|Γ is
    sin 2θ and the data are V_b = ∂u/∂n = √λ I₂'(√λ R)/I₂(√λ R) sin 2θ. Δs ≈ alpha·Δx."""
    from scipy.special import iv, ivp

    h = 1.0 / N
    R = 0.25
    M = points_for_spacing(2 * np.pi * R, h, alpha)
    bd = circle(M, R, (0.0, 0.0))
    th = bd.meta["theta"]
    k = math.sqrt(lam)
    Vb = (k * ivp(2, k * R) / iv(2, k * R) * np.sin(2 * th))[None, :]
    return Problem("paper_circle_neumann", 2, N, 1.0, (-0.5, -0.5), bd, Vb, "scalar", lam=lam,
                   delta=delta, dipole=dipole, symbol=symbol, rtol=1e-10, bc="neumann",
                   meta={"alpha": alpha, "exact_Ub": np.sin(2 * th)[None, :]})


def brinkman_flow(x, y, lam: float, mu: float = 1.0, angle: float = 0.3):
    """A Brinkman flow without forcing: stream function ψ = e^{κ(x cos a + y sin a)}, κ = √(λ/μ),
    u = (∂_y ψ, −∂_x ψ) with constant pressure, so μΔu − λu = 0 and ∇·u = 0 (not a Stokes flow)."""
    k = math.sqrt(lam / mu)
    e = np.exp(k * ((x - 0.5) * math.cos(angle) + (y - 0.5) * math.sin(angle)))
    return np.stack([k * math.sin(angle) * e, -k * math.cos(angle) * e])


def circle_brinkman(N: int = 128, M: int = 200, lam: float = 10.0, mu: float = 1.0, delta: str = "cos",
                    symbol: str = "spectral", dipole: str = "analytic") -> Problem:
    """Interior Brinkman problem (Sec. 6.3.2, η = 0): circle R = 0.25 about (0.5, 0.5) in the unit
    box, L = μΔ − λ, boundary data the exact flow ``brinkman_flow`` (flux removed, rounding level)."""
    bd = circle(M, 0.25, (0.5, 0.5))
    U = brinkman_flow(bd.X[0], bd.X[1], lam, mu)
    U, flux = remove_normal_flux(U, bd)
    return Problem("circle_brinkman", 2, N, 1.0, (0.0, 0.0), bd, U, "stokes", lam=lam, mu=mu,
                   delta=delta, dipole=dipole, symbol=symbol, rtol=1e-10, meta={"removed_flux": flux})


def cylinder_array(N: int, c: float, eta: float = 10.0, alpha: float = 1.0, delta: str = "cos",
                   symbol: str = "spectral") -> Problem:
    """Stokes flow past a periodic array of cylinders (Sec. 6.5.3): the box [−0.5, 0.5]², a disk
    of area fraction c (radius √(c/π)) at the origin, u = 0 on its boundary, forcing g = (−1, 0),
    completed method with η; the fluid is exterior, so the normals point into the disk. The
    constant forcing has no mean-free part, so it enters only the constraint rows:
    η Σ Δs Q = h² Σ g̃ = (−1, 0) (box area 1)."""
    r = math.sqrt(c / math.pi)
    h = 1.0 / N
    M = points_for_spacing(2 * np.pi * r, h, alpha)
    bd = circle(M, r, (0.0, 0.0))
    bd.n = -bd.n
    p = Problem("cylinder_array", 2, N, 1.0, (-0.5, -0.5), bd, np.zeros((2, M)), "stokes", mu=1.0,
                delta=delta, dipole="analytic", symbol=symbol, rtol=1e-10,
                meta={"c": c, "radius": r, "rhs_aug": np.array([-1.0, 0.0])}, eta=eta)
    return p

