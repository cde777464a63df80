"""In-tree build of libibdl.so for GB300 (sm_103a) with nvcc.

Every translation unit of csrc/ is compiled in parallel with one ``-gencode`` and linked into
``paper_2210_07403_gb300/libibdl.so`` (static CUDA runtime, no PyTorch dependency). Objects go to
``paper_2210_07403_gb300/_build/``. The build is skipped when the library is newer than every
source and header.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libibdl.so")
# every translation unit in csrc/: the host and driver units plus the per-size kernel units
# (apply2d_n*.cu: one per 2-D grid size and precision, or both precisions for the small sizes;
# apply3d_n*.cu: one per 3-D grid size), compiled in parallel
SOURCES = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libibdl.so")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return files + [os.path.abspath(__file__)]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile and link libibdl.so if any input changed; return its path."""
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    # the slowest units first, so that they do not start last: the per-size kernel units by
    # decreasing grid size, then the other kernel units, then the host units
    def cost(f):
        m = re.match(r"apply[23]d_n(\d+)", f)
        return (not f.startswith("apply"), -(int(m.group(1)) ** (2 if f.startswith("apply2d") else 1.5)) if m else 0, f)

    order = sorted(SOURCES, key=cost)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(SOURCES), os.cpu_count() or 1))) as ex:
        results = list(ex.map(compile_one, order))
    if verbose:
        for obj, log in results:
            sys.stderr.write(f"--- {os.path.basename(obj)}\n{log}")
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
