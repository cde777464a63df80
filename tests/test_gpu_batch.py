"""GPU parity of batched launches: many independent 2-D problems of different grid sizes, point
counts, λ, deltas and symbols in one launch per stage, against the FP64 oracle per problem
(same tolerances as the single-problem tests)."""
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


def _mixed_batch(dipole="analytic"):
    rng = np.random.default_rng(21)
    probs = []
    for i, (N, delta, symbol, lam) in enumerate([(32, "cos", "spectral", 0.0), (64, "sqrt", "fd2", 3.0),
                                                  (128, "cos", "spectral", 40.0), (64, "cos", "spectral", 0.0),
                                                  (32, "sqrt", "spectral", 99.0)]):
        a, b = rng.uniform(0.1, 0.3, 2)
        M = I.points_for_spacing(I.ellipse(64, a, b).measure, 1.0 / N)
        bd = I.ellipse(M, a, b, rot=float(rng.uniform(0, np.pi)))
        Ub = I.random_modes(bd.t, 6, 1.0, rng, 1, decay=True)
        probs.append(I.Problem(f"p{i}", 2, N, 1.0, (0.0, 0.0), bd, Ub, "scalar", lam=lam, delta=delta,
                               dipole=dipole, symbol=symbol))
    return probs


@pytest.mark.parametrize("dipole", ["analytic", "spectral_div"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32x2", 1e-12), ("fp32", 2e-5)])
def test_batch_apply(dipole, precision, tol):
    from paper_2210_07403_gb300.ibdl import Batch

    probs = _mixed_batch(dipole)
    B = Batch(probs)
    q = np.random.default_rng(3).standard_normal(B.total)
    y = B.apply(torch.from_numpy(q).cuda(), precision=precision).cpu().numpy()
    for b, p in enumerate(probs):
        sl = slice(B.offsets[b], B.offsets[b + 1])
        assert _rel(y[sl], O.apply(O.geometry_from_problem(p), q[sl])) < tol


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32x2", 1e-12), ("fp32", 2e-5)])
def test_batch_apply_persistent_column_pass(precision, tol, monkeypatch):
    """The persistent batched column pass (IBDL_BATCH_PERSISTENT=1, read when the batch is
    created): CTAs that walk their size's units match the oracle as the one-CTA-per-unit launches
    do, and a batched mixed solve with it converges to the oracle's solution."""
    from paper_2210_07403_gb300.ibdl import Batch

    monkeypatch.setenv("IBDL_BATCH_PERSISTENT", "1")
    probs = _mixed_batch()
    B = Batch(probs)
    q = np.random.default_rng(4).standard_normal(B.total)
    y = B.apply(torch.from_numpy(q).cuda(), precision=precision).cpu().numpy()
    for b, p in enumerate(probs):
        sl = slice(B.offsets[b], B.offsets[b + 1])
        assert _rel(y[sl], O.apply(O.geometry_from_problem(p), q[sl])) < tol
    if precision == "fp32":
        ub = torch.from_numpy(np.concatenate([p.Ub.reshape(-1) for p in probs])).cuda()
        Q, _, _ = B.solve(ub, rtol=1e-10, precision="mixed")
        Q = Q.cpu().numpy()
        for b, p in enumerate(probs):
            sl = slice(B.offsets[b], B.offsets[b + 1])
            assert _rel(Q[sl], O.solve(O.geometry_from_problem(p), p.Ub, 1e-12).x) < 1e-8


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_solve(precision):
    from paper_2210_07403_gb300.ibdl import Batch

    probs = _mixed_batch()
    B = Batch(probs)
    ub = torch.from_numpy(np.concatenate([p.Ub.reshape(-1) for p in probs])).cuda()
    Q, infos, st = B.solve(ub, rtol=1e-10, precision=precision)
    Q = Q.cpu().numpy()
    for b, p in enumerate(probs):
        ref = O.solve(O.geometry_from_problem(p), p.Ub, 1e-12)
        sl = slice(B.offsets[b], B.offsets[b + 1])
        assert infos[b]["rel_residual"] <= 1e-10
        assert _rel(Q[sl], ref.x) < (1e-10 if precision == "fp64" else 1e-8)


def test_batch_ellipse_workload_sampled():
    """The 256-problem ellipse batch (grids 128²…512²): mixed-precision batched solve; every
    problem reaches the residual tolerance, and sampled problems match the oracle."""
    from paper_2210_07403_gb300.ibdl import Batch

    probs = I.ellipse_batch(256)
    B = Batch(probs)
    ub = torch.from_numpy(np.concatenate([p.Ub.reshape(-1) for p in probs])).cuda()
    Q, infos, st = B.solve(ub, rtol=1e-9, precision="mixed", inner_rtol=1e-5)
    assert st == 0
    assert max(i["rel_residual"] for i in infos) <= 1e-9
    Q = Q.cpu().numpy()
    for b in (0, 77, 255):
        ref = O.solve(O.geometry_from_problem(probs[b]), probs[b].Ub, 1e-12)
        sl = slice(B.offsets[b], B.offsets[b + 1])
        assert _rel(Q[sl], ref.x) < 1e-8


def test_batch_autotune_keeps_parity():
    from paper_2210_07403_gb300.ibdl import Batch

    probs = _mixed_batch()
    B = Batch(probs)
    B.autotune()
    q = np.random.default_rng(5).standard_normal(B.total)
    for prec, tol in (("fp64", 1e-12), ("fp32", 2e-5)):
        y = B.apply(torch.from_numpy(q).cuda(), precision=prec).cpu().numpy()
        for b, p in enumerate(probs):
            sl = slice(B.offsets[b], B.offsets[b + 1])
            assert _rel(y[sl], O.apply(O.geometry_from_problem(p), q[sl])) < tol
    ub = torch.from_numpy(np.concatenate([p.Ub.reshape(-1) for p in probs])).cuda()
    Q, infos, st = B.solve(ub, rtol=1e-10, precision="mixed")
    assert st == 0
