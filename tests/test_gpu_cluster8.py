"""The Arnoldi step on an 8-CTA cluster: the launch on devices that cannot place a 16-CTA cluster
(a GB300 always takes 16). IBDL_ARNOLDI_CLUSTER=8 selects it in a child process, which solves
the 64² circle (FP64, checked against the oracle), the 512² Stokes star (FP64 and mixed, checked
against this process's 16-CTA solves) and a batch of four ellipses (FP64, against the 16-CTA
batch). The two cluster sizes sum the slices' dot products in different orders, so solutions
agree to rounding and the iteration counts to within one."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import ibdl_inputs as I
from oracle import ibdl_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, json
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import ibdl_inputs as I
from paper_2210_07403_gb300 import Geometry, ibdl
from paper_2210_07403_gb300.ibdl import Batch
ibdl.load()
out = sys.argv[2]
its = {}
p = I.circle_laplace()
g = Geometry.from_problem(p)
Q, info, st = g.solve(torch.from_numpy(p.Ub.reshape(-1).copy()).cuda(), rtol=1e-10)
np.save(out + "/circle.npy", Q.cpu().numpy()); its["circle"] = info["iterations"]
p = I.star_stokes()
g = Geometry.from_problem(p)
ub = torch.from_numpy(p.Ub.reshape(-1).copy()).cuda()
for prec in ("fp64", "mixed"):
    Q, info, st = g.solve(ub, rtol=1e-9, precision=prec, inner_rtol=1e-5)
    np.save(out + "/star_" + prec + ".npy", Q.cpu().numpy()); its["star_" + prec] = info["iterations"]
probs = I.ellipse_batch(4)
B = Batch(probs)
ubb = torch.from_numpy(np.concatenate([q.Ub.reshape(-1) for q in probs])).cuda()
Q, infos, st = B.solve(ubb, rtol=1e-10, precision="fp64")
np.save(out + "/batch.npy", Q.cpu().numpy()); its["batch"] = max(i["iterations"] for i in infos)
json.dump(its, open(out + "/its.json", "w"))
"""


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


def test_arnoldi_on_an_8_cta_cluster(tmp_path):
    from paper_2210_07403_gb300 import Geometry
    from paper_2210_07403_gb300.ibdl import Batch

    env = dict(os.environ, IBDL_ARNOLDI_CLUSTER="8")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(tmp_path)], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    its = json.load(open(tmp_path / "its.json"))

    p = I.circle_laplace()
    og = O.geometry_from_problem(p)
    ref = O.solve(og, p.Ub.reshape(-1), 1e-13).x
    assert _rel(np.load(tmp_path / "circle.npy"), ref) < 1e-10

    p = I.star_stokes()
    g = Geometry.from_problem(p)
    ub = torch.from_numpy(p.Ub.reshape(-1).copy()).cuda()
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-8)):
        Q, info, st = g.solve(ub, rtol=1e-9, precision=prec, inner_rtol=1e-5)
        assert st == 0
        assert _rel(np.load(tmp_path / f"star_{prec}.npy"), Q.cpu().numpy()) < tol
        assert abs(its["star_" + prec] - info["iterations"]) <= 1

    probs = I.ellipse_batch(4)
    B = Batch(probs)
    ubb = torch.from_numpy(np.concatenate([q.Ub.reshape(-1) for q in probs])).cuda()
    Q, infos, st = B.solve(ubb, rtol=1e-10, precision="fp64")
    assert st == 0
    assert _rel(np.load(tmp_path / "batch.npy"), Q.cpu().numpy()) < 1e-9
    assert abs(its["batch"] - max(i["iterations"] for i in infos)) <= 1
