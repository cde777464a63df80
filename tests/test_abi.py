"""The C-ABI library builds, loads and exports every entry point of include/ibdl.h, the ctypes
mirrors of its structs have the C layout, and the host-side argument checks answer without a GPU."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ibdl.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2210_07403_gb300 import build as b
    from paper_2210_07403_gb300 import ibdl

    b.build()
    return ibdl.load()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ibdl_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2210_07403_gb300 import ibdl

    names = _declared_functions()
    assert len(names) >= 9
    for name in names:
        assert hasattr(lib, name), f"{name} not exported"
        assert name in ibdl.SIGNATURES, f"{name} has no binding"


def test_struct_layouts_match_c():
    from paper_2210_07403_gb300 import ibdl

    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "ibdl.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(ibdl_geometry_desc), offsetof(ibdl_geometry_desc, n_points),
         offsetof(ibdl_geometry_desc, lambda), offsetof(ibdl_geometry_desc, inputs_on_device),
         offsetof(ibdl_geometry_desc, weights));
  printf("%zu %zu %zu %zu\n", sizeof(ibdl_solve_opts), offsetof(ibdl_solve_opts, inner_rtol), offsetof(ibdl_solve_opts, io_on_host),
         offsetof(ibdl_solve_opts, residual));
  printf("%zu %zu %zu\n", sizeof(ibdl_solve_info), offsetof(ibdl_solve_info, seconds), offsetof(ibdl_solve_info, fp32x2_applies));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    D, O, S = ibdl.ibdl_geometry_desc, ibdl.ibdl_solve_opts, ibdl.ibdl_solve_info
    assert list(map(int, out[0].split())) == [ctypes.sizeof(D), D.n_points.offset, D.lambda_.offset,
                                             D.inputs_on_device.offset, D.weights.offset]
    assert list(map(int, out[1].split())) == [ctypes.sizeof(O), O.inner_rtol.offset, O.io_on_host.offset,
                                             O.residual.offset]
    assert list(map(int, out[2].split())) == [ctypes.sizeof(S), S.seconds.offset, S.fp32x2_applies.offset]


def test_host_side_argument_checks(lib):
    """Calls that fail validation before touching the device return their status without a GPU."""
    from paper_2210_07403_gb300 import ibdl

    o = ibdl.ibdl_default_solve_opts()
    assert (o.rtol, o.restart, o.maxit, o.precision) == (1e-8, 50, 200, ibdl.IBDL_FP64)
    assert o.residual == ibdl.IBDL_FP32X2
    assert lib.ibdl_create_geometry(None, None, ctypes.byref(ctypes.c_void_p())) == ibdl.IBDL_ERR_INVALID_ARG
    assert "null" in ibdl.ibdl_last_error().lower()
    assert lib.ibdl_apply(None, 0, None, None, None) == ibdl.IBDL_ERR_INVALID_ARG
    assert lib.ibdl_adjoint(None, 0, None, None, None) == ibdl.IBDL_ERR_INVALID_ARG
    assert lib.ibdl_evaluate_field(None, None, None, None) == ibdl.IBDL_ERR_INVALID_ARG
    assert lib.ibdl_indicator(None, None, None, None) == ibdl.IBDL_ERR_INVALID_ARG
    assert lib.ibdl_near_boundary(None, None, None, None, 6.0, 8.0, None, None) == ibdl.IBDL_ERR_INVALID_ARG
    info = ibdl.ibdl_solve_info()
    assert lib.ibdl_solve(None, None, None, ctypes.byref(o), ctypes.byref(info), None) == ibdl.IBDL_ERR_INVALID_ARG
    assert lib.ibdl_destroy_geometry(None) == ibdl.IBDL_OK
    d = ibdl.ibdl_geometry_desc()
    d.dim, d.n, d.box, d.n_points = 4, 64, 1.0, 10
    out = ctypes.c_void_p()
    assert lib.ibdl_create_geometry(ctypes.byref(d), None, ctypes.byref(out)) == ibdl.IBDL_ERR_INVALID_ARG
    d.dim, d.n = 2, 100  # not a power of two
    assert lib.ibdl_create_geometry(ctypes.byref(d), None, ctypes.byref(out)) == ibdl.IBDL_ERR_INVALID_ARG
    assert "power of two" in ibdl.ibdl_last_error()
    d.n, d.dim = 64, 3
    d.X, d.normals, d.weights = 1, None, None  # 3-D needs normals and weights (rejected before any copy)
    assert lib.ibdl_create_geometry(ctypes.byref(d), None, ctypes.byref(out)) == ibdl.IBDL_ERR_INVALID_ARG
    assert "required" in ibdl.ibdl_last_error()
    d.n, d.pde, d.dim = 64, ibdl.IBDL_PDE_STOKES, 3
    d.X = d.normals = d.weights = 1  # never dereferenced: the combination is rejected first
    d.mu = 1.0
    assert lib.ibdl_create_geometry(ctypes.byref(d), None, ctypes.byref(out)) == ibdl.IBDL_ERR_UNSUPPORTED


def test_missing_library_fails_loudly(tmp_path):
    from paper_2210_07403_gb300 import ibdl

    saved = ibdl._lib
    try:
        ibdl._lib = None
        with pytest.raises(RuntimeError, match="not found"):
            ibdl.load(str(tmp_path / "libibdl.so"))
    finally:
        ibdl._lib = saved
