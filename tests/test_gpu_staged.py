"""GPU parity of the staged FP32 column pass: persistent CTAs whose column units are copied into
shared memory by the tensor memory accelerator a few units ahead of their transforms.

IBDL_COL_STAGED (read when a geometry or batch is created) forces it on ("1") or off ("0"); unset,
the direct pass runs until the autotuner picks the faster of the two. Here it is forced on for
single problems of every operator form (each CTA walks several units, the packed kx = 0 column
among them) and for a batch (units of different problems and sizes), and off for the same batch.
Tolerances as in test_gpu_parity.py: FP32 applications 2e-5 against the FP64 oracle (relative
2-norm and element-wise), mixed solves 1e-8."""
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
    """max of the relative 2-norm error and the element-wise error max|a − b|/max|b|"""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    d = np.abs(a - b)
    return float(max(np.linalg.norm(d) / np.linalg.norm(b), d.max() / np.abs(b).max()))


def _scalar(N, M, delta, dipole, symbol, lam):
    bd = I.circle(M, 0.25, (0.5, 0.5))
    Ub = I.harmonic_cubic(bd.X[0], bd.X[1])[None, :]
    return I.Problem("t", 2, N, 1.0, (0.0, 0.0), bd, Ub, "scalar", lam=lam, delta=delta, dipole=dipole, symbol=symbol)


CASES = [
    # N, M, delta, dipole, symbol, lam
    (16, 25, "cos", "analytic", "spectral", 0.0),
    (64, 137, "sqrt", "spectral_div", "spectral", 0.0),
    (128, 201, "cos", "spectral_div", "fd2", 50.0),
    (256, 403, "sqrt", "analytic", "fd2", 7.0),
    (512, 800, "cos", "analytic", "spectral", 0.0),
]


@pytest.mark.parametrize("case", CASES)
def test_staged_scalar_apply_adjoint_single_layer(case, monkeypatch):
    """A, A*, Aᵀ and the single layer in FP32 with the staged column pass, twice in a row."""
    from paper_2210_07403_gb300 import Geometry

    monkeypatch.setenv("IBDL_COL_STAGED", "1")
    N, M, delta, dipole, symbol, lam = case
    p = _scalar(N, M, delta, dipole, symbol, lam)
    g = Geometry.from_problem(p)
    og = O.geometry_from_problem(p)
    rng = np.random.default_rng(N + 7)
    for _ in range(2):
        q = rng.standard_normal(M)
        qd = torch.from_numpy(q).cuda()
        assert _rel(g.apply(qd, precision="fp32").cpu().numpy(), O.apply(og, q)) < 2e-5
        assert _rel(g.adjoint(qd, precision="fp32").cpu().numpy(), O.adjoint_apply(og, q)) < 2e-5
        assert _rel(g.apply_transpose(qd, precision="fp32").cpu().numpy(), O.transpose_apply(og, q)) < 2e-5
        if lam > 0:
            assert _rel(g.single_layer(qd, precision="fp32").cpu().numpy(), O.single_layer(og, q)) < 2e-5
    g.close()


@pytest.mark.parametrize("N,M", [(128, 200), (512, 800)])
@pytest.mark.parametrize("dipole", ["analytic", "spectral_div"])
def test_staged_stokes_apply(N, M, dipole, monkeypatch):
    """The Stokes operator (three or four fields in, two out) and, for the analytic dipole, its
    transpose (two in, three out) in FP32 with the staged column pass."""
    from paper_2210_07403_gb300 import Geometry

    monkeypatch.setenv("IBDL_COL_STAGED", "1")
    p = I.star_stokes(N, M, dipole=dipole)
    g = Geometry.from_problem(p)
    og = O.geometry_from_problem(p)
    q = np.random.default_rng(N).standard_normal(2 * p.bd.M)
    qd = torch.from_numpy(q).cuda()
    assert _rel(g.apply(qd, precision="fp32").cpu().numpy(), O.apply(og, q)) < 2e-5
    if dipole == "analytic":
        assert _rel(g.apply_transpose(qd, precision="fp32").cpu().numpy(), O.transpose_apply(og, q)) < 2e-5
    g.close()


def test_staged_matches_direct(monkeypatch):
    """The staged and the direct column pass give the same FP32 application (both run the same
    transforms and symbol; only the order of the spread's and the gather's atomic additions may
    differ)."""
    from paper_2210_07403_gb300 import Geometry

    p = I.star_stokes(512, 800)
    q = torch.from_numpy(np.random.default_rng(5).standard_normal(2 * p.bd.M)).cuda()
    ys = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("IBDL_COL_STAGED", mode)
        g = Geometry.from_problem(p)
        ys[mode] = g.apply(q, precision="fp32").cpu().numpy()
        g.close()
    assert _rel(ys["1"], ys["0"]) < 1e-6


def test_staged_mixed_solve(monkeypatch):
    """The mixed-precision solve of the 512² Stokes star with every FP32 application staged: the
    column pass inside the captured GMRES cycles (programmatic launch, stop flag) against the
    oracle solution."""
    from paper_2210_07403_gb300 import Geometry

    monkeypatch.setenv("IBDL_COL_STAGED", "1")
    p = I.star_stokes(512, 800)
    g = Geometry.from_problem(p)
    og = O.geometry_from_problem(p)
    ub = p.Ub.reshape(-1)
    Q, info, _ = g.solve(torch.from_numpy(ub.copy()).cuda(), rtol=1e-10, precision="mixed")
    ref = O.solve(og, p.Ub, 1e-12)
    assert _rel(Q.cpu().numpy(), ref.x) < 1e-8
    assert info["fp32_applies"] > 0
    g.close()


@pytest.mark.parametrize("mode", ["0", "1"])
def test_batch_column_pass_modes(mode, monkeypatch):
    """A batch of problems of three grid sizes and several column units per size, FP32, with the
    column pass staged ("1") and direct ("0"), against the oracle per problem."""
    from paper_2210_07403_gb300.ibdl import Batch

    monkeypatch.setenv("IBDL_COL_STAGED", mode)
    rng = np.random.default_rng(31)
    probs = []
    for i, (N, delta, symbol, lam) in enumerate([(64, "cos", "spectral", 0.0), (128, "sqrt", "fd2", 3.0),
                                                  (256, "cos", "spectral", 40.0), (128, "cos", "spectral", 0.0),
                                                  (64, "sqrt", "spectral", 99.0), (256, "sqrt", "fd2", 10.0)]):
        a, b = rng.uniform(0.1, 0.3, 2)
        M = I.points_for_spacing(I.ellipse(64, a, b).measure, 1.0 / N)
        bd = I.ellipse(M, a, b, rot=float(rng.uniform(0, np.pi)))
        Ub = I.random_modes(bd.t, 6, 1.0, rng, 1, decay=True)
        probs.append(I.Problem(f"p{i}", 2, N, 1.0, (0.0, 0.0), bd, Ub, "scalar", lam=lam, delta=delta,
                               dipole="analytic", symbol=symbol))
    B = Batch(probs)
    q = np.random.default_rng(4).standard_normal(B.total)
    for _ in range(2):
        y = B.apply(torch.from_numpy(q).cuda(), precision="fp32").cpu().numpy()
        for b, p in enumerate(probs):
            sl = slice(B.offsets[b], B.offsets[b + 1])
            assert _rel(y[sl], O.apply(O.geometry_from_problem(p), q[sl])) < 2e-5
    B.close()
