"""Benchmark of the IBDL operator hot path on GB300 (one JSON line on rank 0).

Workload: 2-D steady Stokes IBDL solve on the unit periodic box, 512² grid, star
r(θ) = 0.25(1 + 0.2 cos 5θ) with 800 points equispaced in arclength, cosine 4-point delta,
analytic dipole spread, spectral symbols; boundary data = rigid rotation + seeded random modes
|m| ≤ 8, amplitude 0.1, made flux free (synthetic, seed 2).

A step is one mixed-precision solve (FP32 operator applications inside GMRES, FP64 Arnoldi,
refinement residual from a float-float application with FP64 subtraction) to the relative
residual that keeps the solution within 1e-8 of the FP64 plain GPU solve and of the FP64 oracle. `value` is solves/s over all ranks (each rank solves its own replica:
weak scaling, no collective). L2 is flushed (a 256 MiB write) before every timed step and the
flush is outside the per-step CUDA-event timing.

Also reported: FP32/FP64 operator applications per second, the FP64 plain GPU solve rate, the
per-kernel device times (stage timing events), the roofline of the dominant kernel, SM clocks
sampled during the timed region, the end-to-end rate through the C ABI with host buffers, and
the FP64 CPU oracle timed on this host on one core and on all cores (`cpu_baseline`), and the
error of every workload's solution against the FP64 oracle's (solved in a background process
while the GPU runs).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IBDL operator applies/s & solves/s at 1e-8 vs FP64 plain GPU; % HBM roofline"
WORKLOAD = "stokes_star_512"
N_GRID, N_POINTS = 512, 800
SOLVE_RTOL = 1e-9          # residual tolerance of the timed solves (error ≤ 1e-8 checked below)
INNER_RTOL = 1e-5          # relative tolerance of each inner FP32-apply GMRES (two refinement sweeps)
REF_RTOL = 1e-13           # the FP64 plain GPU reference solution
ACCURACY = 1e-8


def _workload():
    return {"workload": WORKLOAD, "grid": f"{N_GRID}x{N_GRID}", "n_points": N_POINTS, "pde": "stokes",
            "delta": "cos", "dipole": "analytic", "symbol": "spectral", "solve_rtol": SOLVE_RTOL, "seed": 2}


def _config():
    return dict(_workload(),
                precision="mixed: fp32 applies, fp64 arnoldi, float-float refinement residual (fp64 subtraction)",
                inner_rtol=INNER_RTOL, gmres="restart 50, each cycle one CUDA graph with a device-side while loop",
                launch_shapes="autotuned on the GPU before the warm-up",
                l2="flushed before each timed step (256 MiB write, untimed)")


def _reference_config():
    return dict(_workload(), precision="fp64 throughout (numpy oracle)",
                gmres="full GMRES from the definition: modified Gram-Schmidt, least squares by numpy",
                transforms="numpy.fft", where="host CPU, one process, single-threaded BLAS")


def _problem():
    import ibdl_inputs as I

    return I.star_stokes(N_GRID, N_POINTS)


# ------------------------------------------------------------------------------------------
# the FP64 CPU oracle (cpu_baseline and --impl reference)
# ------------------------------------------------------------------------------------------

_ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import ibdl_inputs as I
from oracle import ibdl_oracle as O
p = I.star_stokes({n}, {m})
g = O.geometry_from_problem(p)
t_start = {t_start!r}
if t_start:
    while time.time() < t_start:
        time.sleep(0.005)
t_end = time.time() + {budget}
times, stamps = [], []
while len(times) < {max_solves} and (not times or time.time() < t_end):
    t0 = time.perf_counter()
    r = O.solve(g, p.Ub, {rtol}, maxit=100)
    times.append(time.perf_counter() - t0)
    stamps.append(time.time())
print(json.dumps({{"times": times, "iterations": r.iterations, "last": stamps[-1]}}))
"""

_BLAS1 = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}


def _oracle_cmd(budget_s, max_solves, rtol, t_start=0.0):
    code = _ORACLE_SNIPPET.format(root=ROOT, n=N_GRID, m=N_POINTS, budget=budget_s, max_solves=max_solves,
                                  rtol=rtol, t_start=t_start)
    return [sys.executable, "-c", code]


def run_oracle(budget_s: float, max_solves: int, rtol: float = SOLVE_RTOL):
    """Time the oracle's FP64 solve of the workload in a fresh single-threaded process."""
    out = subprocess.run(_oracle_cmd(budget_s, max_solves, rtol), capture_output=True, text=True,
                         env=dict(os.environ, **_BLAS1), check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_oracle_all_cores(budget_s: float, procs: int, rtol: float = SOLVE_RTOL):
    """The oracle on every host core: `procs` single-threaded processes solve the workload from a
    common start time for `budget_s` seconds; throughput = all completed solves / (last finish −
    start)."""
    t_start = time.time() + 4.0  # every process has imported numpy and built its geometry by then
    ps = [subprocess.Popen(_oracle_cmd(budget_s, 1000, rtol, t_start), stdout=subprocess.PIPE, text=True,
                           env=dict(os.environ, **_BLAS1)) for _ in range(procs)]
    res = [json.loads(p.communicate()[0].strip().splitlines()[-1]) for p in ps]
    n = sum(len(r["times"]) for r in res)
    span = max(r["last"] for r in res) - t_start
    return {"solves": n, "seconds": span, "value": n / span, "procs": procs}


# Oracle solutions of the workloads the bench solves on the GPU, for their errors against the
# oracle: the 512² star, three problems of the ellipse batch, the 128³ sphere, the 1024² circle
# of the size sweep and the cylinder array at c = 0.2 (1024²), each to rtol 1e-12.
_REFERENCE_SNIPPET = r"""
import sys
import numpy as np
sys.path.insert(0, {root!r})
import ibdl_inputs as I
from oracle import ibdl_oracle as O
out = {{}}
p = I.star_stokes({n}, {m})
out["star"] = O.solve(O.geometry_from_problem(p), p.Ub, 1e-12, maxit=100).x
probs = I.ellipse_batch(256)
for b in (0, 77, 255):
    q = probs[b]
    out["batch%d" % b] = O.solve(O.geometry_from_problem(q), q.Ub, 1e-12, maxit=100).x
p = I.sphere_poisson()
out["sphere"] = O.solve(O.geometry_from_problem(p), p.Ub, 1e-12, maxit=100).x
N = 1024
bd = I.circle(I.points_for_spacing(2 * np.pi * 0.25, 1.0 / N, 0.75))
ub = I.harmonic_cubic(bd.X[0], bd.X[1])
q = I.Problem("sweep", 2, N, 1.0, (0.0, 0.0), bd, ub[None, :], "scalar", delta="cos")
out["sweep1024"] = O.solve(O.geometry_from_problem(q), ub, 1e-12, maxit=100).x
p = I.cylinder_array(1024, 0.2)
b = np.concatenate([p.Ub.reshape(-1), p.meta["rhs_aug"]])
out["cyl0.2"] = O.solve(O.geometry_from_problem(p), b, 1e-12, maxit=200).x
np.savez({path!r}, **out)
"""


def start_oracle_references(path: str):
    """Start the oracle solutions of the workloads in a background single-threaded process."""
    code = _REFERENCE_SNIPPET.format(root=ROOT, n=N_GRID, m=N_POINTS, path=path)
    return subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.DEVNULL, stderr=subprocess.PIPE,
                            env=dict(os.environ, **_BLAS1))


def _err(x, ref) -> float:
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    ref = np.asarray(ref, dtype=np.float64).reshape(-1)
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------

_SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"ibdl_bench_clocks_{os.getpid()}_{index}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={_SMI_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------

# the sources of the 2-D kernels: a traffic record is valid for the kernels built from these
KERNEL_SOURCES = ("apply2d_kernels.cuh", "fft8.cuh", "fft.cuh", "ff.cuh", "tma.cuh", "ibdl_internal.cuh")


def _stored_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu capture summary, if that capture
    was taken on the current kernel source (the file records a hash of KERNEL_SOURCES)."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for name in KERNEL_SOURCES:
            with open(os.path.join(ROOT, "paper_2210_07403_gb300", "csrc", name), "rb") as f:
                h.update(f.read())
        if rec.get("source_sha256") != h.hexdigest():
            return None
        entry = rec.get("kernels", {}).get(kernel)
        return None if entry is None else float(entry["dram_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# algorithmic HBM bytes per launch of each kernel of the 2-D Stokes application (analytic
# dipole: 3 fields spread, 2 interpolated), w bytes per real, grid N²: the packed half
# spectrum of one real field is N²·w bytes.
def _kernel_bytes(stage: str, n: int, m: int) -> float:
    w = 8 if stage.endswith("fp64") else 4
    grid = n * n * w
    pts = m * (2 * 4 * 4 + 4) * w / 2  # point tables read per pass (small)
    if stage.startswith("spread_rowfft"):
        return 3 * grid + pts
    if stage.startswith("column"):
        return 5 * grid
    if stage.startswith("rowifft_gather"):
        return 2 * grid + pts
    return 0.0


def _event_ms(fn, K, flush, stream):
    """K device-timed calls of fn, each after an untimed L2 flush; returns (median ms, last result)."""
    import torch

    ms, out = [], None
    for _ in range(K):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return float(np.median(ms)), out


def extra_workloads(dev, flush, stream, sols, K=5):
    """The other workload shapes (context, not the headline): the 64² circle, the 256-problem
    ellipse batch (with its HBM roofline: the batch does not fit in L2) and the 128³ sphere.
    `sols` receives the GPU solutions compared with the oracle's at the end (sols[key][prec])."""
    import torch

    import ibdl_inputs as I
    from paper_2210_07403_gb300 import Geometry
    from paper_2210_07403_gb300.ibdl import Batch

    out = {}
    peak, _ = _peaks()
    # 64² circle, Laplace, GMRES to 1e-10 (FP64)
    p = I.circle_laplace(64, 100)
    g = Geometry.from_problem(p)
    ub = torch.from_numpy(p.Ub.reshape(-1).copy()).to(dev)
    for _ in range(3):
        g.solve(ub, rtol=1e-10)
    t, (Q, info, _) = _event_ms(lambda: g.solve(ub, rtol=1e-10), K, flush, stream)
    out["circle_laplace_64"] = {"fp64_solves_per_s": round(1e3 / t, 1), "iterations": info["iterations"],
                                "rel_residual": info["rel_residual"]}
    g.close()
    # 256 ellipses, N ∈ {128, 256, 512}, λ ∈ [0, 100]: batched
    probs = I.ellipse_batch(256)
    B = Batch(probs)
    B.autotune()
    cells = sum(q.N ** 2 for q in probs)
    ub = torch.from_numpy(np.concatenate([q.Ub.reshape(-1) for q in probs])).to(dev)
    y = torch.empty_like(ub)
    res = {"problems": len(probs), "grid_cells": cells, "points": B.total}
    for prec in ("fp32", "fp64"):
        for _ in range(3):
            B.apply(ub, y, precision=prec)
        t, _ = _event_ms(lambda: B.apply(ub, y, precision=prec), K, flush, stream)
        w = 4 if prec == "fp32" else 8
        achieved = 4 * cells * w / (t * 1e-3) / 1e9
        res["apply_" + prec] = {"us": round(t * 1e3, 1), "algorithmic_bytes": 4 * cells * w,
                                "achieved_GBps": round(achieved, 1), "frac_of_measured_hbm": round(achieved / peak, 4)}
    offs = np.cumsum([0] + [q.ncomp * q.bd.M for q in probs])
    sols["batch"] = {}
    for prec in ("fp64", "mixed"):
        def run():
            return B.solve(ub, rtol=SOLVE_RTOL, precision=prec, inner_rtol=INNER_RTOL)
        for _ in range(2):
            run()
        t, (Q, infos, st) = _event_ms(run, K, flush, stream)
        Qh = Q.cpu().numpy()
        sols["batch"][prec] = {b: Qh[offs[b]:offs[b + 1]] for b in (0, 77, 255)}
        res["solve_" + prec] = {"problems_per_s": round(len(probs) / (t * 1e-3), 1), "ms_per_batch": round(t, 3),
                                "max_iterations": max(i["iterations"] for i in infos),
                                "max_rel_residual": max(i["rel_residual"] for i in infos), "status": st}
    res["speedup_mixed_vs_fp64"] = round(res["solve_mixed"]["problems_per_s"] / res["solve_fp64"]["problems_per_s"], 3)
    out["ellipse_batch_256"] = res
    B.close()
    # 128³ sphere, 12 000 points
    p = I.sphere_poisson()
    g = Geometry.from_problem(p)
    ub = torch.from_numpy(p.Ub.reshape(-1).copy()).to(dev)
    y = torch.empty_like(ub)
    res = {}
    for prec in ("fp32", "fp64"):
        for _ in range(3):
            g.apply(ub, y, precision=prec)
        t, _ = _event_ms(lambda: g.apply(ub, y, precision=prec), K, flush, stream)
        res["apply_" + prec + "_us"] = round(t * 1e3, 1)
    sols["sphere"] = {}
    for prec in ("fp64", "mixed"):
        def run():
            return g.solve(ub, rtol=SOLVE_RTOL, precision=prec, inner_rtol=INNER_RTOL)
        for _ in range(2):
            run()
        t, (Q, info, st) = _event_ms(run, K, flush, stream)
        sols["sphere"][prec] = Q.cpu().numpy()
        res["solve_" + prec] = {"solves_per_s": round(1e3 / t, 1), "iterations": info["iterations"],
                                "fp64_applies": info["fp64_applies"], "rel_residual": info["rel_residual"]}
    res["speedup_mixed_vs_fp64"] = round(res["solve_mixed"]["solves_per_s"] / res["solve_fp64"]["solves_per_s"], 3)
    out["sphere_128"] = res
    g.close()
    out["stokes_star_probes_1024"] = differentiation_workload(dev, flush, stream, K)
    out["cylinder_array_drag_1024"] = cylinder_drag_workload(dev, flush, stream, sols=sols)
    out["cylinder_array_drag_2048"] = cylinder_drag_workload(dev, flush, stream, N=2048)
    # the paper's own resolution: FP64 applications one field per launch (three FP64 fields of a
    # column do not fit shared memory together at 8192²)
    out["cylinder_array_drag_8192"] = cylinder_drag_workload(dev, flush, stream, K=1, N=8192, cs=(0.05, 0.2, 0.4))
    out["postprocess"] = postprocess_workload(dev, flush, stream)
    out["size_sweep"] = size_sweep_workload(dev, flush, stream, sols=sols)
    return out


def oracle_errors(out: dict, sols: dict, ref: dict, headline: dict):
    """Errors of the GPU solutions against the oracle's (relative 2-norm), into the result."""
    headline["error_vs_oracle"] = {k: _err(v, ref["star"]) for k, v in sols["star"].items()}
    if not out:
        return
    w = out
    w["ellipse_batch_256"]["error_vs_oracle"] = {
        prec: {f"problem_{b}": _err(x, ref[f"batch{b}"]) for b, x in per.items()} for prec, per in sols["batch"].items()}
    w["sphere_128"]["error_vs_oracle"] = {prec: _err(x, ref["sphere"]) for prec, x in sols["sphere"].items()}
    w["size_sweep"]["N=1024"]["error_vs_oracle"] = {prec: _err(x, ref["sweep1024"])
                                                    for prec, x in sols["sweep1024"].items()}
    w["cylinder_array_drag_1024"]["c=0.2"]["error_vs_oracle"] = {prec: _err(x, ref["cyl0.2"])
                                                                 for prec, x in sols["cyl0.2"].items()}


def differentiation_workload(dev, flush, stream, K=5):
    """Forward + backward of J = Σ_p |u(p)|² on the 1024² Stokes star (1600 points, 64 probes at
    ≥ 8h): the solve, the probe values, the transposed solve and the boundary derivatives, with
    gradients to U_b, X, n and Δs. "step" includes building the geometry from the points (what a
    shape-optimisation step pays); "fwd_bwd" reuses a built geometry."""
    import torch

    import ibdl_inputs as I
    from paper_2210_07403_gb300 import autograd as AG

    p, P = I.star_stokes_probes()
    base = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
            for a in (p.Ub.reshape(-1), p.bd.X, p.bd.n, p.bd.w)]
    Pd = torch.from_numpy(np.ascontiguousarray(P)).to(dev)
    res = {"grid": p.N, "points": int(p.bd.X.shape[1]), "probes": int(P.shape[1]), "objective": "sum |u(p)|^2"}
    grads = {}
    for prec, rtol in (("fp64", 1e-10), ("mixed", SOLVE_RTOL)):
        leaves = [a.clone().requires_grad_(True) for a in base]

        def fwd_bwd(b):
            for a in leaves:
                a.grad = None
            J = (b.probe(b.solve(leaves[0], rtol=rtol, precision=prec, inner_rtol=INNER_RTOL), Pd) ** 2).sum()
            J.backward()
            return J

        def step():
            b = AG.Boundary(*leaves[1:], p.N, pde="stokes", delta=p.delta, symbol=p.symbol)
            J = fwd_bwd(b)
            b.close()
            return J

        for _ in range(2):
            step()
        t_step, _ = _event_ms(step, K, flush, stream)
        b = AG.Boundary(*leaves[1:], p.N, pde="stokes", delta=p.delta, symbol=p.symbol)
        fwd_bwd(b)
        t_fb, J = _event_ms(lambda: fwd_bwd(b), K, flush, stream)
        t_fwd, _ = _event_ms(lambda: (b.probe(b.solve(leaves[0].detach(), rtol=rtol, precision=prec,
                                                      inner_rtol=INNER_RTOL), Pd) ** 2).sum(), K, flush, stream)
        b.close()
        grads[prec] = [a.grad.detach().cpu().numpy().reshape(-1) for a in leaves]
        res[prec] = {"rtol": rtol, "step_ms": round(t_step, 3), "fwd_bwd_ms": round(t_fb, 3),
                     "forward_ms": round(t_fwd, 3), "J": float(J.detach())}
    res["mixed_grad_rel_diff_vs_fp64"] = {
        k: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        for k, a, b in zip(("Ub", "X", "n", "w"), grads["mixed"], grads["fp64"])}
    return res


def _published_drag():
    """The paper's drag table (Sec. 6.5.3), as stored in the golden file: c -> (IBDL at 8192², G&K)."""
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", "cylinder_drag.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                c, ibdl, gk = line.split()
                out[float(c)] = (float(ibdl), float(gk))
    return out


def cylinder_drag_workload(dev, flush, stream, K=3, N=1024, cs=(0.05, 0.1, 0.2, 0.3, 0.4, 0.5), sols=None):
    """The paper's Stokes flow past a periodic array of cylinders (Sec. 6.5.3) at N², completed
    method (η = 10, Δs ≈ Δx): the dimensionless drag D = B₁/(μU) per area fraction c against the
    published values, and the solve rate in FP64 (rtol 1e-10) and mixed precision (rtol 1e-9)."""
    import torch

    import ibdl_inputs as I
    from paper_2210_07403_gb300 import Geometry

    pub = _published_drag()
    res = {"grid": N, "eta": 10.0, "spacing": "ds ~ dx"}
    for c in cs:
        p = I.cylinder_array(N, c)
        g = Geometry.from_problem(p)
        b = torch.from_numpy(np.concatenate([p.Ub.reshape(-1), p.meta["rhs_aug"]])).to(dev)
        w = torch.from_numpy(p.bd.w).to(dev)
        row = {"points": int(p.bd.X.shape[1])}
        for prec, rtol in (("fp64", 1e-10), ("mixed", SOLVE_RTOL)):
            def run():
                return g.solve(b, rtol=rtol, precision=prec, inner_rtol=INNER_RTOL, maxit=400)
            run()
            t, (x, info, st) = _event_ms(run, K, flush, stream)
            if sols is not None and c == 0.2:
                sols.setdefault("cyl0.2", {})[prec] = x.cpu().numpy()
            u = g.evaluate_field(x)
            U = float(u[0][:, 0].sum()) / N
            D = float(-p.eta * (x[: g.M] * w).sum()) / U
            row[prec] = {"D": D, "iterations": info["iterations"], "solves_per_s": round(1e3 / t, 1)}
        ibdl_ref, gk = pub.get(c, (None, None))
        row["D_published_ibdl_8192"] = ibdl_ref
        row["D_greengard_kropinski"] = gk
        if gk:
            row["rel_diff_vs_gk"] = (row["fp64"]["D"] - gk) / gk
        res[f"c={c}"] = row
        g.close()
    return res


def postprocess_workload(dev, flush, stream, K=5, Ns=(256, 512, 1024, 2048)):
    """Post-processing (Sec. 5.3.4, Sec. 5.3.5). The paper's max-norm study on its circle problem
    (Δu − u = 0 inside r = 0.25, U_b = sin 2θ, Δs ≈ 0.75Δx, finite differences, m1 = 6, m2 = 8):
    GPU solve → field → indicator → near-boundary interpolation, max error over Ω without and with
    the interpolation against u = I₂(r) sin 2θ / I₂(0.25). Then the device time of each step on the
    1024² Stokes star (spectral settings m1 = 12, m2 = 14)."""
    import torch
    from scipy.special import iv

    import ibdl_inputs as I
    from paper_2210_07403_gb300 import Geometry

    res = {"problem": "circle r=0.25, Delta u - u = 0, U_b = sin 2theta, fd2, sqrt delta, m1=6, m2=8"}
    raw, fixed = [], []
    for N in Ns:
        p = I.paper_circle_helmholtz(N, 0.75, "sqrt", "fd2")
        g = Geometry.from_problem(p)
        ub = torch.from_numpy(p.Ub.reshape(-1).copy()).to(dev)
        Q, info, _ = g.solve(ub, rtol=1e-10, maxit=200)
        u = g.evaluate_field(Q)
        _, flags = g.indicator()
        ui = g.near_boundary(ub, u, flags, 6.0, 8.0)
        xs = p.origin[0] + np.arange(N) / N
        x, y = np.meshgrid(xs, xs)
        exact = iv(2, np.hypot(x, y)) / iv(2, 0.25) * np.sin(2 * np.arctan2(y, x))
        m = flags.cpu().numpy().astype(bool)
        raw.append(float(np.abs(u.cpu().numpy() - exact)[m].max()))
        fixed.append(float(np.abs(ui.cpu().numpy() - exact)[m].max()))
        g.close()
    res["grids"] = list(Ns)
    res["max_err_raw"] = raw
    res["max_err_interpolated"] = fixed
    res["order_interpolated"] = round(float(np.polyfit(np.log([1.0 / N for N in Ns]), np.log(fixed), 1)[0]), 3)
    p = I.star_stokes(1024, 1600)
    g = Geometry.from_problem(p)
    ub = torch.from_numpy(p.Ub.reshape(-1).copy()).to(dev)
    Q, info, _ = g.solve(ub, rtol=1e-10, maxit=200)
    u = g.evaluate_field(Q)
    _, flags = g.indicator()
    out = torch.empty_like(u)
    for _ in range(3):
        g.indicator()
        g.near_boundary(ub, u, flags, 12.0, 14.0, out=out)
    t_ind, _ = _event_ms(lambda: g.indicator(), K, flush, stream)
    t_nb, _ = _event_ms(lambda: g.near_boundary(ub, u, flags, 12.0, 14.0, out=out), K, flush, stream)
    res["stokes_star_1024"] = {"indicator_us": round(t_ind * 1e3, 1), "near_boundary_us": round(t_nb * 1e3, 1),
                               "nodes_replaced": int((out != u).any(0).sum()), "m1": 12, "m2": 14}
    g.close()
    return res


def size_sweep_workload(dev, flush, stream, Ns=(512, 1024, 2048, 4096, 8192), napply=50, sols=None):
    """The 64² circle problem's geometry on finer grids (Δs ≈ 0.75h, the paper's spacing; its
    studies run N = 2^6 … 2^14): scalar Laplace, analytic dipole, spectral symbol. Per N and
    precision: applications/s from CUDA events over `napply` back-to-back applications after an
    L2 flush, the algorithmic bytes 4N²w (+ boundary vectors) per application against the measured
    HBM bandwidth, whether the grid fields fit in L2, and FP64 and mixed solve rates to 1e-9 (the
    mixed solves' refinement residual is float-float to 4096², FP64 at 8192²)."""
    import torch

    import ibdl_inputs as I
    from paper_2210_07403_gb300 import Geometry, IbdlError

    hbm, _ = _peaks()
    res = {"geometry": "circle R=0.25 at (0.5,0.5), ds ~ 0.75h, Re((z-z0)^3) data, scalar Laplace"}
    for N in Ns:
        M = I.points_for_spacing(2 * np.pi * 0.25, 1.0 / N, 0.75)
        bd = I.circle(M)
        ub = torch.from_numpy(I.harmonic_cubic(bd.X[0], bd.X[1])).to(dev)
        g = Geometry(bd.X, bd.n, bd.w, N, delta="cos")
        row = {"points": M}
        g.autotune(7)  # FP64, FP32 and float-float (the mixed solves' residual; to 4096²)
        for prec, w in (("fp32", 4), ("fp64", 8)):
            try:
                y = torch.empty_like(ub)
                for _ in range(5):
                    g.apply(ub, y, precision=prec)
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(napply):
                    g.apply(ub, y, precision=prec)
                e1.record(stream)
                e1.synchronize()
                us = e0.elapsed_time(e1) / napply * 1e3
                alg = 4 * N * N * w + 3 * M * 8
                row["apply_" + prec] = {"us": round(us, 2), "algorithmic_bytes": alg,
                                        "achieved_GBps": round(alg / us / 1e3, 1),
                                        "frac_of_measured_hbm": round(alg / us / 1e3 / hbm, 4) if hbm else None,
                                        # one scalar field (the packed half spectrum) against the 129 MB L2
                                        "l2_resident": N * N * w < 100e6}
            except IbdlError as e:
                row["apply_" + prec] = {"unsupported": str(e).split(":")[0]}
        for prec in ("fp64", "mixed"):
            try:
                def run():
                    return g.solve(ub, rtol=SOLVE_RTOL, precision=prec, inner_rtol=INNER_RTOL)
                run()
                t, (Q, info, st) = _event_ms(run, 3, flush, stream)
                if sols is not None and N == 1024:
                    sols.setdefault("sweep1024", {})[prec] = Q.cpu().numpy()
                row["solve_" + prec] = {"solves_per_s": round(1e3 / t, 2), "iterations": info["iterations"],
                                        "rel_residual": info["rel_residual"]}
                if prec == "mixed":
                    row["solve_mixed"]["residual"] = "fp32x2" if info["fp32x2_applies"] else "fp64"
            except IbdlError as e:
                row["solve_" + prec] = {"unsupported": str(e).split(":")[0]}
        res[f"N={N}"] = row
        g.close()
    return res


def cufft_compare(dev, stream):
    """cuFFT (torch.fft) time for the transforms alone of one 512² Stokes application."""
    import torch

    res = {}
    for name, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
        x = torch.randn(3, N_GRID, N_GRID, dtype=dt, device=dev)
        for _ in range(5):
            torch.fft.irfft2(torch.fft.rfft2(x)[:2], s=(N_GRID, N_GRID))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(50):
            torch.fft.irfft2(torch.fft.rfft2(x)[:2], s=(N_GRID, N_GRID))
        e1.record(stream)
        e1.synchronize()
        res[name + "_us"] = round(e0.elapsed_time(e1) / 50 * 1e3, 1)
    res["what"] = "torch.fft rfft2 of 3 fields + irfft2 of 2 fields at 512² (no spread, symbol or interpolation)"
    return res


def aggregate_over_ranks(local_seconds, steps: int, world: int, device=None):
    """Whole-job throughput of weak-scaled replicas: every rank solved `steps` problems; the job
    took as long as the slowest rank. local_seconds: this rank's timed seconds (a list: timed
    region, then e2e). Returns (values per entry = world·steps / max seconds, max seconds)."""
    import torch

    t = torch.tensor(list(local_seconds), dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist

        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    mx = [float(v) for v in t.tolist()]
    return [world * steps / v for v in mx], mx


def run_ours(args, rank: int, world: int, local_rank: int):
    import torch
    import torch.distributed as dist

    from paper_2210_07403_gb300 import Geometry, build as b
    from paper_2210_07403_gb300 import ibdl

    b.build()
    # oracle solutions of the workloads, in the background while the GPU runs (rank 0 only)
    ref_path = os.path.join(tempfile.gettempdir(), f"ibdl_bench_oracle_{os.getpid()}.npz")
    ref_proc = start_oracle_references(ref_path) if rank == 0 and not args.no_oracle_errors else None
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    p = _problem()
    geom = Geometry.from_problem(p)
    geom.autotune()  # launch shapes timed on this GPU (the parity tests run the same shapes)
    nd = 2 * p.bd.M
    ub = torch.from_numpy(p.Ub.reshape(-1).copy()).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def l2_flush():
        flush.fill_(1.0)

    # FP64 plain GPU reference solution (tight tolerance)
    q_ref, info_ref, _ = geom.solve(ub, rtol=REF_RTOL, maxit=100)

    def solve(precision, host=False):
        src = ub_host if host else ub
        return geom.solve(src, rtol=SOLVE_RTOL, precision=precision, maxit=200, inner_rtol=INNER_RTOL)

    ub_host = torch.from_numpy(p.Ub.reshape(-1).copy()).pin_memory()

    for _ in range(args.warmup):
        solve("mixed")
        solve("fp64")
        geom.apply(ub, precision="fp32")
        geom.apply(ub, precision="fp64")
    torch.cuda.synchronize()

    def timed(fn, K):
        """K device-timed calls of fn with an untimed L2 flush before each; returns ms list."""
        ms = []
        outs = []
        for _ in range(K):
            l2_flush()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            outs.append(fn())
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms, outs

    K = args.steps
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if args.host_driven:
        geom.set_stage_timing(True)
    with ClockSampler(local_rank) as clocks:
        t_wall0 = time.perf_counter()
        ms_mixed, outs = timed(lambda: solve("mixed"), K)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if args.host_driven:
        geom.set_stage_timing(False)

    err_mixed = max(float(torch.linalg.norm(q - q_ref) / torch.linalg.norm(q_ref)) for q, _, _ in outs)
    info_m = outs[-1][1]
    sols = {"star": {"mixed": outs[-1][0].cpu().numpy()}}
    launches = int(sum(o[1]["kernel_launches"] for o in outs))

    # FP64 plain GPU solves (the comparison path)
    ms_fp64, outs64 = timed(lambda: solve("fp64"), K)
    err_fp64 = max(float(torch.linalg.norm(q - q_ref) / torch.linalg.norm(q_ref)) for q, _, _ in outs64)
    sols["star"]["fp64"] = outs64[-1][0].cpu().numpy()

    # per-stage device time of a mixed solve (a separate pass: stage timing records an event
    # around every kernel and drives GMRES from the host, so it is kept out of the timed steps)
    geom.set_stage_timing(True)
    geom.stage_times()
    for _ in range(K):
        solve("mixed")
    stages_mixed = geom.stage_times()

    # operator applications, per-kernel device times for the roofline
    Y = torch.empty_like(ub)
    geom.stage_times()
    ms_a32, _ = timed(lambda: geom.apply(ub, Y, precision="fp32"), max(K, 20))
    st32 = geom.stage_times()
    ms_a64, _ = timed(lambda: geom.apply(ub, Y, precision="fp64"), max(K, 20))
    st64 = geom.stage_times()
    geom.set_stage_timing(False)

    # back-to-back applications as the solves run them (programmatic launch between kernels, no
    # event between kernels): 20 warm-ups, then 200 applications in 10 event-timed chunks of 20
    def back_to_back(prec):
        for _ in range(20):
            geom.apply(ub, Y, precision=prec)
        per = []
        for _ in range(10):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(20):
                geom.apply(ub, Y, precision=prec)
            e1.record(stream)
            e1.synchronize()
            per.append(e0.elapsed_time(e1) / 20 * 1e3)
        return {"us_median": round(float(np.median(per)), 2), "us_p10": round(float(np.percentile(per, 10)), 2),
                "us_p90": round(float(np.percentile(per, 90)), 2),
                "per_s": round(1e6 / float(np.median(per)), 1)}

    b2b = {prec: back_to_back(prec) for prec in ("fp32", "fp32x2", "fp64")}

    # end to end through the C ABI with host buffers (copies inside the call)
    ms_e2e, outs_e2e = timed(lambda: solve("mixed", host=True), K)
    err_e2e = max(float(torch.linalg.norm(q.to(dev) - q_ref) / torch.linalg.norm(q_ref)) for q, _, _ in outs_e2e)

    # max over ranks: every rank solved K replicas of the problem
    (value, e2e_value), (t_mixed, t_e2e) = aggregate_over_ranks([sum(ms_mixed) / 1e3, sum(ms_e2e) / 1e3], K,
                                                                 world, dev)
    if rank != 0:
        return None
    extras = None if args.no_extras else extra_workloads(dev, flush, stream, sols)
    cufft = None if args.no_extras else cufft_compare(dev, stream)

    # dominant kernel of the timed mixed solves, and its average launch from the apply loop
    per_stage = {k: v for k, v in stages_mixed.items()}
    dom = max((k for k in per_stage if k != "arnoldi" and k != "other"), key=lambda k: per_stage[k][0])
    loop = st32 if dom.endswith("fp32") else st64
    dom_ms = loop[dom][0] / loop[dom][1]
    bytes_dom = _kernel_bytes(dom, N_GRID, N_POINTS)
    peak, peak_src = _peaks()
    achieved = bytes_dom / (dom_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": _stored_traffic(dom), "peak_source": peak_src,
            "avg_launch_us": round(dom_ms * 1e3, 2), "algorithmic_bytes": int(bytes_dom),
            "note": "grid fields are L2-resident between kernels of one application (6 MB FP32)"}

    # errors against the oracle (its solutions were computed in the background meanwhile)
    mixed_block = {}
    if ref_proc is not None:
        _, err_txt = ref_proc.communicate()
        if ref_proc.returncode == 0:
            with np.load(ref_path) as z:
                ref = {k: z[k] for k in z.files}
            os.remove(ref_path)
            oracle_errors(extras or {}, sols, ref, mixed_block)
        else:
            mixed_block["error_vs_oracle"] = {"unavailable": err_txt.strip().splitlines()[-1] if err_txt else "failed"}

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        o = run_oracle(budget_s=12.0, max_solves=8)
        tm = float(np.mean(o["times"]))
        procs = host_cores()
        allc = run_oracle_all_cores(budget_s=10.0, procs=procs)
        cpu = {"value": round(allc["value"], 4), "unit": "solves/s", "cores": procs, "kind": "oracle",
               "sample": f"{allc['solves']} FP64 numpy oracle solves of the 512² Stokes star to rtol {SOLVE_RTOL:g} "
                         f"({o['iterations']} GMRES iterations each) by {procs} single-threaded processes, one per "
                         f"host core, in {allc['seconds']:.1f} s",
               "single_core": {"value": round(1.0 / tm, 4), "unit": "solves/s", "cores": 1,
                               "sample": f"{len(o['times'])} solves in one single-threaded process"}}

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "solves/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(t_mixed / K * 1e3, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 applies + f64 arnoldi + f32x2 refinement residual",
        "data": "synthetic (seeded star boundary and Fourier-mode boundary data)", "config": _config(),
        "applies_per_s": {"fp32": round(1e3 / float(np.mean(ms_a32)), 1),
                          "fp64": round(1e3 / float(np.mean(ms_a64)), 1),
                          "how": "one application at a time, L2 flushed before each, events around every kernel"},
        "applies_back_to_back": dict(b2b, how="200 applications after 20 warm-ups, 10 chunks of 20 "
                                              "timed with CUDA events, programmatic launch between kernels"),
        "fp64_plain": {"solves_per_s": round(K / (sum(ms_fp64) / 1e3), 3), "error_vs_ref": err_fp64,
                       "iterations": outs64[-1][1]["iterations"]},
        "mixed": dict({"error_vs_fp64_plain": err_mixed, "iterations": info_m["iterations"],
                       "fp32_applies": info_m["fp32_applies"], "fp64_applies": info_m["fp64_applies"],
                       "fp32x2_applies": info_m["fp32x2_applies"],
                       "sweeps": info_m["sweeps"], "rel_residual": info_m["rel_residual"],
                       "accuracy_ok": err_mixed <= ACCURACY}, **mixed_block),
        "speedup_mixed_vs_fp64_plain": round(sum(ms_fp64) / sum(ms_mixed), 3),
        "stage_ms_per_solve_host_driven": {k: round(v[0] / K, 4) for k, v in stages_mixed.items()},
        "stage_launches_per_solve": {k: round(v[1] / K, 2) for k, v in stages_mixed.items()},
        "apply_kernel_us": {**{k: round(v[0] / v[1] * 1e3, 2) for k, v in st32.items()},
                            **{k: round(v[0] / v[1] * 1e3, 2) for k, v in st64.items()}},
        "roofline": roof,
        "clocks": clocks.summary(),
        "e2e": {"value": round(e2e_value, 3), "unit": "solves/s", "h2d_bytes_per_step": nd * 8,
                "d2h_bytes_per_step": nd * 8, "error_vs_fp64_plain": err_e2e},
        "gpu_launches": launches,
        "workloads": extras,
        "cufft_transforms_only": cufft,
        "wall_s_timed_region": round(t_wall, 3),
        "gmres_driver": "host (one launch per kernel)" if args.host_driven else "CUDA graph per cycle",
        "launch_plan": {prec: geom.launch_plan(prec) for prec in ("fp32", "fp32x2", "fp64")},
        "cpu_baseline": cpu,
    }
    geom.close()
    return out


# ------------------------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle
# ------------------------------------------------------------------------------------------

def run_reference(args, rank: int):
    if rank != 0:
        return None
    o = run_oracle(budget_s=1e9, max_solves=args.warmup + args.steps)
    times = o["times"][args.warmup:]
    K = len(times)
    value = K / sum(times)
    return {
        "metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": args.gpus, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(sum(times) / K * 1e3, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": _reference_config(),
        "impl": "reference",
        "cpu_baseline": {"value": round(value, 4), "unit": "solves/s", "kind": "oracle", "cores": 1,
                         "sample": f"{K} FP64 numpy oracle solves of the 512² Stokes star, single thread"},
        "e2e": {"value": round(value, 4), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other workload shapes")
    ap.add_argument("--no-oracle-errors", action="store_true",
                    help="skip the oracle solutions the workloads' errors are measured against")
    ap.add_argument("--host-driven", action="store_true",
                    help="drive GMRES from the host with one launch per kernel (for profilers that do not "
                         "see kernels inside CUDA-graph conditional bodies); slower")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)  # at least three untimed warm-up steps
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist

            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        out = run_ours(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
