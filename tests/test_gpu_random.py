"""Seeded random sweep of operator configurations against the FP64 oracle, through the C ABI.

Each case draws a grid (32² to 256²), a curve (circle, ellipse or star, possibly crossing the
periodic edges, dense enough that a row band holds many more than 32 points so every thread of
the spread and gather kernels handles several work items), the delta kernel, the dipole spread,
the symbol, the PDE and its parameters, the boundary condition, and a random density. FP64
applications must agree with the oracle to 1e-12 and FP32 ones to 2e-5 (the operator tolerances
of the other parity tests)."""
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


def _case(seed):
    rng = np.random.default_rng(1000 + seed)
    N = int(rng.choice([32, 64, 128, 256]))
    kind = rng.choice(["circle", "ellipse", "star"])
    spacing = float(rng.choice([0.1, 0.3, 0.75, 1.5]))  # Δs/h: 0.1 packs ~10 points per cell
    centre = tuple(rng.uniform(0.0, 1.0, 2))  # anywhere in the box: curves cross the edges
    if kind == "circle":
        R = rng.uniform(0.1, 0.3)
        bd = I.circle(I.points_for_spacing(2 * np.pi * R, 1.0 / N, spacing), R=R, center=centre)
    elif kind == "ellipse":
        a, b = rng.uniform(0.1, 0.3, 2)
        per = np.pi * (3 * (a + b) - np.sqrt((3 * a + b) * (a + 3 * b)))
        bd = I.ellipse(I.points_for_spacing(per, 1.0 / N, spacing), a, b, rot=rng.uniform(0, np.pi), center=centre)
    else:
        a = rng.uniform(0.12, 0.25)
        bd = I.star(I.points_for_spacing(2 * np.pi * a * 1.1, 1.0 / N, spacing), a=a, center=centre)
    pde = rng.choice(["scalar", "scalar", "stokes"])
    lam = float(rng.choice([0.0, 0.0, rng.uniform(0.5, 60.0)]))
    mu = float(rng.uniform(0.5, 2.0)) if pde == "stokes" else 1.0
    delta = rng.choice(["cos", "sqrt"])
    dipole = rng.choice(["analytic", "spectral_div"])
    symbol = rng.choice(["spectral", "fd2"])
    bc = "neumann" if pde == "scalar" and rng.random() < 0.25 else "dirichlet"
    og = O.Geometry(O.Grid(2, N), bd.X, bd.n, bd.w, delta, dipole, symbol, pde, lam, mu, bc)
    q = rng.standard_normal(og.ncomp * og.M)
    return og, q


@pytest.mark.parametrize("seed", range(24))
def test_random_configuration(seed):
    from paper_2210_07403_gb300 import Geometry

    og, q = _case(seed)
    g = Geometry(og.X, og.n, og.w, og.grid.N, pde=og.pde, lam=og.lam, mu=og.mu, delta=og.delta,
                 dipole=og.dipole, symbol=og.symbol, bc=og.bc)
    ref = O.apply(og, q)
    qd = torch.from_numpy(q).cuda()
    for precision, tol in (("fp64", 1e-12), ("fp32x2", 1e-12), ("fp32", 2e-5)):
        y = g.apply(qd, precision=precision).cpu().numpy()
        err = max(np.linalg.norm(y - ref) / np.linalg.norm(ref), np.abs(y - ref).max() / np.abs(ref).max())
        assert err < tol, (seed, precision, err, og.grid.N, og.M, og.pde, og.delta, og.dipole, og.symbol, og.bc, og.lam)
    g.close()
