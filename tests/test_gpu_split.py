"""GPU parity of 2-D applications that run one field per launch.

Such an application is a spread + row FFT launch per input field, the column transforms of each
field, one pointwise symbol launch, and an inverse row FFT + interpolation launch per output
field. The library uses it where a band's or a column's fields do not fit shared memory
together: the Stokes operator in FP64 at 8192², and the divergence-dipole forms (four fields)
from 4096² in FP64. IBDL_SPLIT_FIELDS=1, read when a geometry is created, forces it for every
multi-field operator. Here it is forced at small sizes, in every precision and operator form,
and runs by itself at the full sizes.

Tolerances as in test_gpu_parity.py: FP64 and float-float applications 1e-12, FP32 2e-5
(relative 2-norm and element-wise against the FP64 oracle), mixed solves 1e-8."""
import numpy as np
import pytest

import ibdl_inputs as I
from oracle import ibdl_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-12, "fp32x2": 1e-12, "fp32": 2e-5}


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


@pytest.mark.parametrize("N,M", [(64, 120), (256, 400)])
@pytest.mark.parametrize("dipole", ["analytic", "spectral_div"])
@pytest.mark.parametrize("precision", ["fp64", "fp32x2", "fp32"])
def test_split_stokes(N, M, dipole, precision, monkeypatch):
    """The Stokes operator (three or four fields in, two out), and for the analytic dipole its
    transpose (two in, three out), one field per launch."""
    from paper_2210_07403_gb300 import Geometry

    monkeypatch.setenv("IBDL_SPLIT_FIELDS", "1")
    p = I.star_stokes(N, M, dipole=dipole)
    g = Geometry.from_problem(p)
    assert g.launch_plan(precision)["split"] == 1
    og = O.geometry_from_problem(p)
    rng = np.random.default_rng(N + M)
    for _ in range(2):
        q = rng.standard_normal(2 * p.bd.M)
        qd = torch.from_numpy(q).cuda()
        assert _rel(g.apply(qd, precision=precision).cpu().numpy(), O.apply(og, q)) < TOL[precision]
        if dipole == "analytic":
            z = g.apply_transpose(qd, precision=precision).cpu().numpy()
            assert _rel(z, O.transpose_apply(og, q)) < TOL[precision]
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32x2", "fp32"])
def test_split_scalar_spectral_divergence(precision, monkeypatch):
    """The scalar operator with the spectral divergence (two fields in), its adjoint and
    transpose (two fields out), one field per launch."""
    from paper_2210_07403_gb300 import Geometry

    monkeypatch.setenv("IBDL_SPLIT_FIELDS", "1")
    bd = I.circle(201)
    Ub = I.harmonic_cubic(bd.X[0], bd.X[1])[None, :]
    p = I.Problem("t", 2, 128, 1.0, (0.0, 0.0), bd, Ub, "scalar", lam=5.0, delta="sqrt", dipole="spectral_div",
                  symbol="fd2")
    g = Geometry.from_problem(p)
    og = O.geometry_from_problem(p)
    q = np.random.default_rng(8).standard_normal(201)
    qd = torch.from_numpy(q).cuda()
    assert _rel(g.apply(qd, precision=precision).cpu().numpy(), O.apply(og, q)) < TOL[precision]
    assert _rel(g.apply_transpose(qd, precision=precision).cpu().numpy(), O.transpose_apply(og, q)) < TOL[precision]
    if precision != "fp32x2":
        assert _rel(g.adjoint(qd, precision=precision).cpu().numpy(), O.adjoint_apply(og, q)) < TOL[precision]
    g.close()


@pytest.mark.parametrize("pde", ["scalar", "stokes"])
def test_split_field_evaluation(pde, monkeypatch):
    """Grid output (the solution field on the grid), one field per launch, FP64."""
    from paper_2210_07403_gb300 import Geometry

    monkeypatch.setenv("IBDL_SPLIT_FIELDS", "1")
    if pde == "stokes":
        p = I.star_stokes(64, 120)
    else:
        bd = I.circle(100)
        p = I.Problem("t", 2, 64, 1.0, (0.0, 0.0), bd, I.harmonic_cubic(bd.X[0], bd.X[1])[None, :], "scalar",
                      dipole="spectral_div")
    g = Geometry.from_problem(p)
    og = O.geometry_from_problem(p)
    q = np.random.default_rng(2).standard_normal(p.ncomp * p.bd.M)
    u = g.evaluate_field(torch.from_numpy(q).cuda()).cpu().numpy()
    assert _rel(u, O.grid_field(og, q)) < 1e-12
    g.close()


def test_split_mixed_solve(monkeypatch):
    """The 512² Stokes star solved in mixed precision with every application (FP32 inner,
    float-float residual) one field per launch, against the oracle solution."""
    from paper_2210_07403_gb300 import Geometry

    monkeypatch.setenv("IBDL_SPLIT_FIELDS", "1")
    p = I.star_stokes(512, 800)
    g = Geometry.from_problem(p)
    og = O.geometry_from_problem(p)
    Q, info, _ = g.solve(torch.from_numpy(p.Ub.reshape(-1).copy()).cuda(), rtol=1e-10, precision="mixed")
    assert _rel(Q.cpu().numpy(), O.solve(og, p.Ub, 1e-12).x) < 1e-8
    assert info["fp32x2_applies"] > 0
    g.close()


@pytest.mark.parametrize("N,dipole", [(8192, "analytic"), (4096, "spectral_div")])
def test_split_full_size_fp64(N, dipole):
    """Where the fields do not fit together, one field per launch is chosen by itself: the Stokes
    operator in FP64 at 8192² (three fields, 442 KB per column) and the four-field
    divergence-dipole form at 4096², against the oracle at full size."""
    from paper_2210_07403_gb300 import Geometry

    M = I.points_for_spacing(2 * np.pi * 0.25, 1.0 / N, 1.0)
    bd = I.circle(M)
    og = O.Geometry(O.Grid(2, N), bd.X, bd.n, bd.w, "cos", dipole, "spectral", "stokes", 0.0)
    g = Geometry(bd.X, bd.n, bd.w, N, pde="stokes", dipole=dipole)
    assert g.launch_plan("fp64")["split"] == 1
    q = np.random.default_rng(N).standard_normal(2 * M)
    y = g.apply(torch.from_numpy(q).cuda(), precision="fp64").cpu().numpy()
    assert _rel(y, O.apply(og, q)) < 1e-12
    g.close()
