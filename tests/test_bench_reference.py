"""bench.py's reference arm on the CPU: the oracle's FP64 solve of the 512² Stokes star timed on a
host core, printed as one JSON line with the bench contract's keys; ranks other than 0 print
nothing and exit 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(rank: str):
    env = dict(os.environ, RANK=rank, WORLD_SIZE="2" if rank != "0" else "1")
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "3"], capture_output=True, text=True, env=env, timeout=600)


def test_reference_arm_json_line():
    r = _run("0")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference"
    assert out["unit"] == "solves/s" and out["higher_is_better"] is True
    assert out["steps"] == 1 and out["warmup"] == 3
    assert out["value"] > 0 and out["ms_per_step"] > 0
    assert out["config"]["workload"] == "stokes_star_512"
    assert out["config"]["precision"].startswith("fp64") and "mixed" not in out["config"]["precision"]
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["value"] == out["value"]
    assert out["e2e"] == {"value": out["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    r = _run("1")
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_oracle_on_all_host_cores():
    """The all-core oracle baseline: single-threaded processes from a common start time; every
    process completes at least one solve and the throughput counts them all."""
    sys.path.insert(0, ROOT)
    import bench

    r = bench.run_oracle_all_cores(budget_s=0.5, procs=2)
    assert r["procs"] == 2 and r["solves"] >= 2
    assert r["value"] > 0 and r["seconds"] > 0
    assert bench.host_cores() >= 1
