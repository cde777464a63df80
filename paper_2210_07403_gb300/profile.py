"""Run operator applications of a named workload inside a profiler range, for ncu.

    python -m paper_2210_07403_gb300.profile --workload star512 --precision fp32 --repeat 1

builds the workload's geometry (or batch), autotunes its launch shapes as bench.py does, warms up
with three applications, then runs `--repeat` applications between cudaProfilerStart and
cudaProfilerStop, so that `ncu --profile-from-start off` captures exactly those kernels.

Workloads (synthetic, seeded, as in ibdl_inputs):
    star512      2-D Stokes, 512² grid, star with 800 points (the bench's workload)
    batch256     256 ellipses, N ∈ {128, 256, 512}, screened Poisson (one batched application)
    circle<N>    the size sweep's circle (scalar Laplace, Δs ≈ 0.75h) at N², e.g. circle4096
    sphere128    3-D Laplace, 128³ grid, Fibonacci sphere with 12 000 points
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np


def _build(workload: str, dev):
    import torch

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import ibdl_inputs as I

    from . import Geometry
    from .ibdl import Batch

    if workload == "batch256":
        probs = I.ellipse_batch(256)
        B = Batch(probs)
        B.autotune()
        q = torch.from_numpy(np.concatenate([p.Ub.reshape(-1) for p in probs])).to(dev)
        return B, q
    if workload == "star512":
        p = I.star_stokes(512, 800)
    elif workload == "sphere128":
        p = I.sphere_poisson()
    elif workload.startswith("circle"):
        N = int(workload[len("circle"):])
        bd = I.circle(I.points_for_spacing(2 * np.pi * 0.25, 1.0 / N, 0.75))
        ub = I.harmonic_cubic(bd.X[0], bd.X[1])
        p = I.Problem(workload, 2, N, 1.0, (0.0, 0.0), bd, ub[None, :], "scalar", delta="cos")
    else:
        raise SystemExit(f"unknown workload {workload!r}")
    g = Geometry.from_problem(p)
    g.autotune()
    return g, torch.from_numpy(p.Ub.reshape(-1).copy()).to(dev)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", default="star512")
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "fp32x2"])
    ap.add_argument("--repeat", type=int, default=1)
    args = ap.parse_args(argv)
    import torch

    from . import build as b
    from . import ibdl

    b.build()
    ibdl.load()
    dev = torch.device("cuda", 0)
    obj, q = _build(args.workload, dev)
    y = torch.empty_like(q)
    for _ in range(3):
        obj.apply(q, y, precision=args.precision)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    for _ in range(args.repeat):
        obj.apply(q, y, precision=args.precision)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(f"{args.workload} {args.precision}: {args.repeat} application(s), |y|_1 = {float(y.abs().sum()):.6e}")


if __name__ == "__main__":
    main()
