"""Python binding of the IBDL C ABI (``include/ibdl.h``).

The functions ``ibdl_*`` below have the names, arguments and return values of the C entry
points and only marshal arguments through ctypes; every step of the operator and the solve runs
in the CUDA library ``libibdl.so``. ``Geometry`` is a small convenience wrapper that takes
numpy arrays or CUDA ``torch`` tensors (PyTorch supplies device memory and streams).

Loading fails loudly: if ``libibdl.so`` is missing (not built) or cannot be loaded, every call
raises ``RuntimeError``; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_char_p, c_double, c_int, c_int64, c_void_p

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libibdl.so")

# status codes (ibdl_status)
IBDL_OK = 0
IBDL_ERR_INVALID_ARG = 1
IBDL_ERR_CUDA = 2
IBDL_ERR_NO_MEMORY = 3
IBDL_ERR_NOT_CONVERGED = 4
IBDL_ERR_NONFINITE = 5
IBDL_ERR_TIMEOUT = 6
IBDL_ERR_UNSUPPORTED = 7
STATUS_NAMES = {0: "IBDL_OK", 1: "IBDL_ERR_INVALID_ARG", 2: "IBDL_ERR_CUDA", 3: "IBDL_ERR_NO_MEMORY",
                4: "IBDL_ERR_NOT_CONVERGED", 5: "IBDL_ERR_NONFINITE", 6: "IBDL_ERR_TIMEOUT",
                7: "IBDL_ERR_UNSUPPORTED"}

IBDL_PDE_SCALAR, IBDL_PDE_STOKES = 0, 1
IBDL_DELTA_COS, IBDL_DELTA_SQRT = 0, 1
IBDL_DIPOLE_ANALYTIC, IBDL_DIPOLE_SPECTRAL_DIV = 0, 1
IBDL_SYMBOL_SPECTRAL, IBDL_SYMBOL_FD2 = 0, 1
IBDL_FP64, IBDL_FP32, IBDL_MIXED, IBDL_FP32X2 = 0, 1, 2, 3

_PDE = {"scalar": IBDL_PDE_SCALAR, "stokes": IBDL_PDE_STOKES}
_DELTA = {"cos": IBDL_DELTA_COS, "sqrt": IBDL_DELTA_SQRT}
_DIPOLE = {"analytic": IBDL_DIPOLE_ANALYTIC, "spectral_div": IBDL_DIPOLE_SPECTRAL_DIV}
_SYMBOL = {"spectral": IBDL_SYMBOL_SPECTRAL, "fd2": IBDL_SYMBOL_FD2}
_PREC = {"fp64": IBDL_FP64, "fp32": IBDL_FP32, "mixed": IBDL_MIXED, "fp32x2": IBDL_FP32X2}
IBDL_BC_DIRICHLET, IBDL_BC_NEUMANN = 0, 1
_BC = {"dirichlet": IBDL_BC_DIRICHLET, "neumann": IBDL_BC_NEUMANN}


class ibdl_geometry_desc(ctypes.Structure):
    _fields_ = [("dim", c_int), ("n", c_int), ("box", c_double), ("origin", c_double * 3),
                ("n_points", c_int64), ("X", c_void_p), ("normals", c_void_p), ("weights", c_void_p),
                ("pde", c_int), ("lambda_", c_double), ("mu", c_double), ("delta", c_int),
                ("dipole", c_int), ("symbol", c_int), ("inputs_on_device", c_int), ("bc", c_int),
                ("eta", c_double)]


class ibdl_solve_opts(ctypes.Structure):
    _fields_ = [("rtol", c_double), ("restart", c_int), ("maxit", c_int), ("precision", c_int),
                ("inner_rtol", c_double), ("max_refine", c_int), ("io_on_host", c_int), ("residual", c_int)]


class ibdl_solve_info(ctypes.Structure):
    _fields_ = [("iterations", c_int), ("fp64_applies", c_int), ("fp32_applies", c_int),
                ("sweeps", c_int), ("rel_residual", c_double), ("seconds", c_double),
                ("kernel_launches", c_int64), ("fp32x2_applies", c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# exported symbols and their ctypes signatures
SIGNATURES = {
    "ibdl_create_geometry": (c_int, [POINTER(ibdl_geometry_desc), c_void_p, POINTER(c_void_p)]),
    "ibdl_destroy_geometry": (c_int, [c_void_p]),
    "ibdl_apply": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "ibdl_adjoint": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "ibdl_solve": (c_int, [c_void_p, c_void_p, c_void_p, POINTER(ibdl_solve_opts),
                           POINTER(ibdl_solve_info), c_void_p]),
    "ibdl_evaluate_field": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "ibdl_solve_forced": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, POINTER(ibdl_solve_opts),
                                  POINTER(ibdl_solve_info), c_void_p]),
    "ibdl_evaluate_field_forced": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ibdl_default_solve_opts": (None, [POINTER(ibdl_solve_opts)]),
    "ibdl_geometry_sizes": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int64)]),
    "ibdl_launch_plan": (c_int, [c_void_p, c_int, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int),
                                 POINTER(c_int)]),
    "ibdl_apply_noalloc": (c_int, [POINTER(ibdl_geometry_desc), c_int, c_void_p, c_void_p, c_void_p]),
    "ibdl_create_batch": (c_int, [POINTER(ibdl_geometry_desc), c_int, c_void_p, POINTER(c_void_p)]),
    "ibdl_destroy_batch": (c_int, [c_void_p]),
    "ibdl_batch_sizes": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int64), POINTER(c_int64)]),
    "ibdl_batch_apply": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "ibdl_batch_solve": (c_int, [c_void_p, c_void_p, c_void_p, POINTER(ibdl_solve_opts),
                                 POINTER(ibdl_solve_info), c_void_p]),
    "ibdl_autotune": (c_int, [c_void_p, c_int, c_void_p]),
    "ibdl_batch_autotune": (c_int, [c_void_p, c_int, c_void_p]),
    "ibdl_set_stage_timing": (c_int, [c_void_p, c_int]),
    "ibdl_get_stage_times": (c_int, [c_void_p, POINTER(c_double), POINTER(c_int64)]),
    "ibdl_apply_transpose": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "ibdl_solve_transpose": (c_int, [c_void_p, c_void_p, c_void_p, POINTER(ibdl_solve_opts),
                                     POINTER(ibdl_solve_info), c_void_p]),
    "ibdl_solve_vjp": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ibdl_single_layer": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "ibdl_probe_evaluate": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "ibdl_probe_vjp": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                               c_void_p, c_void_p]),
    "ibdl_indicator": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "ibdl_near_boundary": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_double, c_void_p, c_void_p]),
    "ibdl_last_error": (c_char_p, []),
}

IBDL_STAGE_COUNT = 8
STAGE_NAMES = ["spread_rowfft_fp64", "column_fp64", "rowifft_gather_fp64", "spread_rowfft_fp32",
               "column_fp32", "rowifft_gather_fp32", "arnoldi", "other"]

_lib = None
_load_error = None


def load(path: str = LIB_PATH):
    """Load libibdl.so (once) and attach the ctypes signatures. Raises RuntimeError on failure."""
    global _lib, _load_error
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        _load_error = f"{path} not found: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
        raise RuntimeError(_load_error)
    try:
        lib = ctypes.CDLL(path)
    except OSError as e:  # pragma: no cover - depends on the machine
        _load_error = f"cannot load {path}: {e}"
        raise RuntimeError(_load_error) from e
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class IbdlError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _check(status: int):
    if status != IBDL_OK:
        raise IbdlError(status, ibdl_last_error())
    return status


# ---- the C entry points, one to one --------------------------------------------------------


def ibdl_create_geometry(desc: ibdl_geometry_desc, stream: int = 0) -> c_void_p:
    out = c_void_p()
    _check(load().ibdl_create_geometry(byref(desc), c_void_p(stream), byref(out)))
    return out


def ibdl_destroy_geometry(geom) -> int:
    return _check(load().ibdl_destroy_geometry(geom))


def ibdl_apply(geom, precision: int, Q: int, Y: int, stream: int = 0) -> int:
    return _check(load().ibdl_apply(geom, precision, c_void_p(Q), c_void_p(Y), c_void_p(stream)))


def ibdl_adjoint(geom, precision: int, W: int, Z: int, stream: int = 0) -> int:
    return _check(load().ibdl_adjoint(geom, precision, c_void_p(W), c_void_p(Z), c_void_p(stream)))


def ibdl_solve(geom, Ub: int, Q: int, opts: ibdl_solve_opts, info: ibdl_solve_info, stream: int = 0,
               check: bool = True) -> int:
    st = load().ibdl_solve(geom, c_void_p(Ub), c_void_p(Q), byref(opts), byref(info), c_void_p(stream))
    return _check(st) if check else st


def ibdl_solve_forced(geom, Ub: int, g_grid: int, Q: int, opts: ibdl_solve_opts, info: ibdl_solve_info,
                      stream: int = 0, check: bool = True) -> int:
    st = load().ibdl_solve_forced(geom, c_void_p(Ub), c_void_p(g_grid or None), c_void_p(Q), byref(opts),
                                  byref(info), c_void_p(stream))
    return _check(st) if check else st


def ibdl_evaluate_field_forced(geom, Q: int, g_grid: int, u_grid: int, stream: int = 0) -> int:
    return _check(load().ibdl_evaluate_field_forced(geom, c_void_p(Q), c_void_p(g_grid or None), c_void_p(u_grid),
                                                    c_void_p(stream)))


def ibdl_apply_transpose(geom, precision: int, G: int, Z: int, stream: int = 0) -> int:
    return _check(load().ibdl_apply_transpose(geom, precision, c_void_p(G), c_void_p(Z), c_void_p(stream)))


def ibdl_solve_transpose(geom, G: int, lam: int, opts: ibdl_solve_opts, info: ibdl_solve_info, stream: int = 0,
                         check: bool = True) -> int:
    st = load().ibdl_solve_transpose(geom, c_void_p(G), c_void_p(lam), byref(opts), byref(info), c_void_p(stream))
    return _check(st) if check else st


def ibdl_solve_vjp(geom, Q: int, lam: int, dX: int, dn: int, dw: int, stream: int = 0) -> int:
    """Pointers may be 0 (NULL) for outputs that are not wanted."""
    return _check(load().ibdl_solve_vjp(geom, c_void_p(Q), c_void_p(lam), c_void_p(dX or None),
                                        c_void_p(dn or None), c_void_p(dw or None), c_void_p(stream)))


def ibdl_single_layer(geom, precision: int, V: int, Z: int, stream: int = 0) -> int:
    return _check(load().ibdl_single_layer(geom, precision, c_void_p(V), c_void_p(Z), c_void_p(stream)))


def ibdl_probe_evaluate(geom, P: int, n_probes: int, Q: int, U: int, stream: int = 0) -> int:
    return _check(load().ibdl_probe_evaluate(geom, c_void_p(P), n_probes, c_void_p(Q), c_void_p(U),
                                             c_void_p(stream)))


def ibdl_probe_vjp(geom, P: int, n_probes: int, Q: int, nu: int, dQ: int, dX: int, dn: int, dw: int,
                   stream: int = 0) -> int:
    """Pointers may be 0 (NULL) for outputs that are not wanted."""
    return _check(load().ibdl_probe_vjp(geom, c_void_p(P), n_probes, c_void_p(Q), c_void_p(nu), c_void_p(dQ or None),
                                        c_void_p(dX or None), c_void_p(dn or None), c_void_p(dw or None),
                                        c_void_p(stream)))


def ibdl_indicator(geom, chi: int, flags: int, stream: int = 0) -> int:
    return _check(load().ibdl_indicator(geom, c_void_p(chi), c_void_p(flags), c_void_p(stream)))


def ibdl_near_boundary(geom, Ub: int, u: int, omega: int, m1: float, m2: float, out: int, stream: int = 0) -> int:
    return _check(load().ibdl_near_boundary(geom, c_void_p(Ub), c_void_p(u), c_void_p(omega), c_double(m1),
                                            c_double(m2), c_void_p(out), c_void_p(stream)))


def ibdl_evaluate_field(geom, Q: int, u_grid: int, stream: int = 0) -> int:
    return _check(load().ibdl_evaluate_field(geom, c_void_p(Q), c_void_p(u_grid), c_void_p(stream)))


def ibdl_default_solve_opts() -> ibdl_solve_opts:
    o = ibdl_solve_opts()
    load().ibdl_default_solve_opts(byref(o))
    return o


def ibdl_launch_plan(geom, precision: int):
    v = [c_int() for _ in range(5)]
    _check(load().ibdl_launch_plan(geom, precision, *[byref(x) for x in v]))
    return dict(zip(("rows", "cols", "threads", "staged", "split"), (x.value for x in v)))


def ibdl_geometry_sizes(geom):
    c, m = c_int(), c_int64()
    _check(load().ibdl_geometry_sizes(geom, byref(c), byref(m)))
    return c.value, m.value


def ibdl_create_batch(descs, stream: int = 0) -> c_void_p:
    arr = (ibdl_geometry_desc * len(descs))(*descs)
    out = c_void_p()
    _check(load().ibdl_create_batch(arr, len(descs), c_void_p(stream), byref(out)))
    return out


def ibdl_destroy_batch(batch) -> int:
    return _check(load().ibdl_destroy_batch(batch))


def ibdl_batch_sizes(batch):
    cnt, tot = c_int(), c_int64()
    _check(load().ibdl_batch_sizes(batch, byref(cnt), None, byref(tot)))
    offs = (c_int64 * (cnt.value + 1))()
    _check(load().ibdl_batch_sizes(batch, None, offs, None))
    return cnt.value, list(offs), tot.value


def ibdl_batch_apply(batch, precision: int, Q: int, Y: int, stream: int = 0) -> int:
    return _check(load().ibdl_batch_apply(batch, precision, c_void_p(Q), c_void_p(Y), c_void_p(stream)))


def ibdl_batch_solve(batch, Ub: int, Q: int, opts: ibdl_solve_opts, infos, stream: int = 0,
                     check: bool = True) -> int:
    st = load().ibdl_batch_solve(batch, c_void_p(Ub), c_void_p(Q), byref(opts), infos, c_void_p(stream))
    return _check(st) if check else st


def ibdl_autotune(geom, precision_mask: int = 7, stream: int = 0) -> int:
    return _check(load().ibdl_autotune(geom, int(precision_mask), c_void_p(stream)))


def ibdl_batch_autotune(batch, precision_mask: int = 7, stream: int = 0) -> int:
    return _check(load().ibdl_batch_autotune(batch, int(precision_mask), c_void_p(stream)))


def ibdl_set_stage_timing(geom, enable: int) -> int:
    return _check(load().ibdl_set_stage_timing(geom, int(enable)))


def ibdl_get_stage_times(geom):
    ms = (c_double * IBDL_STAGE_COUNT)()
    n = (c_int64 * IBDL_STAGE_COUNT)()
    _check(load().ibdl_get_stage_times(geom, ms, n))
    return list(ms), list(n)


def ibdl_last_error() -> str:
    return load().ibdl_last_error().decode()


# ---- convenience wrapper ------------------------------------------------------------------


def _host(a):
    """FP64 numpy view of a host array or a torch tensor (copied to the host if on a device)."""
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.asarray(a, dtype=np.float64)


def _stream_handle(stream) -> int:
    import torch

    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _desc(X, normals, weights, n, box, origin, pde, lam, mu, delta, dipole, symbol, bc="dirichlet"):
    """Descriptor over host arrays (returned arrays must stay alive while it is used)."""
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    nrm = np.ascontiguousarray(np.asarray(normals, dtype=np.float64))
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    d = ibdl_geometry_desc()
    d.dim, d.n, d.box = X.shape[0], int(n), float(box)
    for j in range(3):
        d.origin[j] = float(origin[j]) if j < len(origin) else 0.0
    d.n_points = X.shape[1]
    d.X, d.normals, d.weights = X.ctypes.data, nrm.ctypes.data, w.ctypes.data
    d.pde, d.lambda_, d.mu = _PDE[pde], float(lam), float(mu)
    d.delta, d.dipole, d.symbol = _DELTA[delta], _DIPOLE[dipole], _SYMBOL[symbol]
    d.inputs_on_device = 0
    d.bc = _BC[bc]
    return d, (X, nrm, w)


class Batch:
    """A batch of independent 2-D problems (``ibdl_inputs.Problem`` objects); boundary vectors
    are concatenated in problem order."""

    def __init__(self, problems, stream=None):
        import torch

        self._torch = torch
        descs, keep = [], []
        for p in problems:
            d, k = _desc(p.bd.X, p.bd.n, p.bd.w, p.N, p.box, p.origin, p.pde, p.lam, p.mu, p.delta,
                         p.dipole, p.symbol, getattr(p, "bc", "dirichlet"))
            descs.append(d)
            keep.append(k)
        self._h = ibdl_create_batch(descs, _stream_handle(stream))
        self.count, self.offsets, self.total = ibdl_batch_sizes(self._h)

    def autotune(self, precision_mask: int = 7, stream=None):
        """precision_mask bits: 1 FP64, 2 FP32, 4 float-float."""
        ibdl_batch_autotune(self._h, precision_mask, _stream_handle(stream))

    def split(self, v):
        return [v[self.offsets[b]:self.offsets[b + 1]] for b in range(self.count)]

    def apply(self, Q, Y=None, precision: str = "fp64", stream=None):
        if Y is None:
            Y = self._torch.empty_like(Q)
        ibdl_batch_apply(self._h, _PREC[precision], Q.data_ptr(), Y.data_ptr(), _stream_handle(stream))
        return Y

    def solve(self, Ub, rtol: float = 1e-8, precision: str = "fp64", restart: int = 50, maxit: int = 200,
              inner_rtol: float = 1e-4, max_refine: int = 6, Q=None, stream=None, check: bool = True,
              residual: str = "fp32x2"):
        """residual: arithmetic of the mixed-precision refinement residual's application ("fp32x2"
        float-float, or "fp64")."""
        t = self._torch
        o = ibdl_default_solve_opts()
        o.rtol, o.restart, o.maxit, o.precision = rtol, restart, maxit, _PREC[precision]
        o.inner_rtol, o.max_refine, o.residual = inner_rtol, max_refine, _PREC[residual]
        if not Ub.is_cuda:
            o.io_on_host = 1
        if Q is None:
            Q = t.empty_like(Ub)
        infos = (ibdl_solve_info * self.count)()
        st = ibdl_batch_solve(self._h, Ub.data_ptr(), Q.data_ptr(), o, infos, _stream_handle(stream), check=check)
        return Q, [i.as_dict() for i in infos], st

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            ibdl_destroy_batch(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Geometry:
    """An IBDL geometry on the current CUDA device (arguments mirror ``ibdl_geometry_desc``)."""

    def __init__(self, X, normals, weights, n: int, box: float = 1.0, origin=(0.0, 0.0, 0.0),
                 pde: str = "scalar", lam: float = 0.0, mu: float = 1.0, delta: str = "cos",
                 dipole: str = "analytic", symbol: str = "spectral", stream=None, bc: str = "dirichlet",
                 eta: float = 0.0):
        import torch

        self._torch = torch
        # normals or weights None (2-D): the library estimates them from the ordered points
        given = [a for a in (X, normals, weights) if a is not None]
        on_device = all(isinstance(a, torch.Tensor) and a.is_cuda for a in given)
        if on_device:  # CUDA tensors: the library reads the boundary from device memory
            X, nrm, w = (None if a is None else a.detach().to(torch.float64).contiguous() for a in (X, normals, weights))
            ptrs = tuple(0 if a is None else a.data_ptr() for a in (X, nrm, w))
        else:
            X, nrm, w = (None if a is None else np.ascontiguousarray(_host(a)) for a in (X, normals, weights))
            ptrs = tuple(0 if a is None else a.ctypes.data for a in (X, nrm, w))
        self._keep = (X, nrm, w)
        dim, M = X.shape
        d = ibdl_geometry_desc()
        d.dim, d.n, d.box = dim, int(n), float(box)
        for j in range(3):
            d.origin[j] = float(origin[j]) if j < len(origin) else 0.0
        d.n_points = M
        d.X, d.normals, d.weights = (p or None for p in ptrs)
        d.pde, d.lambda_, d.mu = _PDE[pde], float(lam), float(mu)
        d.delta, d.dipole, d.symbol = _DELTA[delta], _DIPOLE[dipole], _SYMBOL[symbol]
        d.inputs_on_device = int(on_device)
        d.bc = _BC[bc]
        d.eta = float(eta)
        self.dim, self.n, self.M, self.pde = dim, int(n), M, pde
        self.ncomp = dim if pde == "stokes" else 1
        # completed method: ū (one mean per component) follows the density in every vector
        self.naug = self.ncomp if eta > 0 else 0
        self.nd = self.ncomp * M + self.naug
        self._h = ibdl_create_geometry(d, _stream_handle(stream))

    @classmethod
    def from_problem(cls, p, **overrides):
        kw = dict(n=p.N, box=p.box, origin=p.origin, pde=p.pde, lam=p.lam, mu=p.mu, delta=p.delta,
                  bc=getattr(p, "bc", "dirichlet"), eta=getattr(p, "eta", 0.0),
                  dipole=p.dipole, symbol=p.symbol)
        kw.update(overrides)
        return cls(p.bd.X, p.bd.n, p.bd.w, **kw)

    @property
    def handle(self):
        return self._h

    def _vec(self, v):
        t = self._torch
        if isinstance(v, np.ndarray):
            v = t.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).cuda()
        assert v.is_cuda and v.dtype == t.float64 and v.is_contiguous()
        assert v.numel() == self.nd
        return v

    def apply(self, Q, Y=None, precision: str = "fp64", stream=None):
        Q = self._vec(Q)
        if Y is None:
            Y = self._torch.empty_like(Q)
        ibdl_apply(self._h, _PREC[precision], Q.data_ptr(), Y.data_ptr(), _stream_handle(stream))
        return Y

    def single_layer(self, V, Z=None, precision: str = "fp64", stream=None):
        """Z = S*(−L⁻¹)(S V) (scalar); −Z(V_b) is the Neumann right-hand side."""
        V = self._vec(V)
        if Z is None:
            Z = self._torch.empty_like(V)
        ibdl_single_layer(self._h, _PREC[precision], V.data_ptr(), Z.data_ptr(), _stream_handle(stream))
        return Z

    def adjoint(self, W, Z=None, precision: str = "fp64", stream=None):
        W = self._vec(W)
        if Z is None:
            Z = self._torch.empty_like(W)
        ibdl_adjoint(self._h, _PREC[precision], W.data_ptr(), Z.data_ptr(), _stream_handle(stream))
        return Z

    def _source(self, g):
        """The source term g̃ as a contiguous CUDA float64 tensor of the field's shape."""
        t = self._torch
        if not isinstance(g, t.Tensor):
            g = t.from_numpy(np.ascontiguousarray(np.asarray(g, dtype=np.float64)))
        g = g.detach().to(device="cuda", dtype=t.float64).contiguous()
        assert g.numel() == self.ncomp * self.n ** self.dim
        return g

    def evaluate_field(self, Q, stream=None, g=None):
        """The grid solution of Q (scalar u or Stokes velocity); with a source g̃ ([c][n][n]) the
        response u_g to it is added (Sec. 5.1.2)."""
        Q = self._vec(Q)
        shape = (self.n,) * self.dim
        if self.pde == "stokes":
            shape = (self.dim,) + shape
        u = self._torch.empty(shape, dtype=self._torch.float64, device=Q.device)
        if g is None:
            ibdl_evaluate_field(self._h, Q.data_ptr(), u.data_ptr(), _stream_handle(stream))
        else:
            g = self._source(g)
            ibdl_evaluate_field_forced(self._h, Q.data_ptr(), g.data_ptr(), u.data_ptr(), _stream_handle(stream))
        return u

    def solve(self, Ub, rtol: float = 1e-8, precision: str = "fp64", restart: int = 50, maxit: int = 200,
              inner_rtol: float = 1e-4, max_refine: int = 6, Q=None, stream=None, check: bool = True, g=None,
              residual: str = "fp32x2"):
        """Solve A Q = U_b (with a source g̃, [c][n][n]: A Q = U_b − S*u_g). U_b on the device (torch
        float64) or a host numpy array / CPU tensor (then the copies happen inside the call,
        io_on_host); g̃ on the device. residual: arithmetic of the mixed-precision refinement
        residual's application ("fp32x2" float-float, or "fp64"). Returns (Q, info dict, status)."""
        if g is None:
            entry = ibdl_solve
        else:
            gs = self._source(g)

            def entry(h, ub, q, o, info, stream, check=True):
                return ibdl_solve_forced(h, ub, gs.data_ptr(), q, o, info, stream, check=check)
        return self._solve(entry, Ub, rtol, precision, restart, maxit, inner_rtol, max_refine, Q, stream, check,
                           residual)

    def solve_transpose(self, G, rtol: float = 1e-8, precision: str = "fp64", restart: int = 50,
                        maxit: int = 200, inner_rtol: float = 1e-4, max_refine: int = 6, lam=None, stream=None,
                        check: bool = True, residual: str = "fp32x2"):
        """Solve Aᵀ λ = G (scalar PDE), same options as ``solve``. Returns (λ, info dict, status)."""
        return self._solve(ibdl_solve_transpose, G, rtol, precision, restart, maxit, inner_rtol, max_refine, lam,
                           stream, check, residual)

    def apply_transpose(self, G, Z=None, precision: str = "fp64", stream=None):
        G = self._vec(G)
        if Z is None:
            Z = self._torch.empty_like(G)
        ibdl_apply_transpose(self._h, _PREC[precision], G.data_ptr(), Z.data_ptr(), _stream_handle(stream))
        return Z

    def solve_vjp(self, Q, lam, stream=None, want=(True, True, True)):
        """∂J/∂X, ∂J/∂n ([dim][M]) and ∂J/∂Δs ([M]) from the solution Q and the adjoint state
        λ = A⁻ᵀ ∂J/∂Q; an entry of ``want`` that is False gives None for that output."""
        t = self._torch
        Q, lam = self._vec(Q), self._vec(lam)
        outs = [t.empty((self.dim, self.M), dtype=t.float64, device=Q.device) if want[0] else None,
                t.empty((self.dim, self.M), dtype=t.float64, device=Q.device) if want[1] else None,
                t.empty((self.M,), dtype=t.float64, device=Q.device) if want[2] else None]
        ptrs = [o.data_ptr() if o is not None else 0 for o in outs]
        ibdl_solve_vjp(self._h, Q.data_ptr(), lam.data_ptr(), *ptrs, _stream_handle(stream))
        return tuple(outs)

    def _probes(self, P):
        t = self._torch
        if not isinstance(P, t.Tensor):
            P = t.from_numpy(np.ascontiguousarray(np.asarray(P, dtype=np.float64)))
        P = P.detach().to(device="cuda", dtype=t.float64).contiguous()
        assert P.dim() == 2 and P.shape[0] == 2
        return P

    def probe_evaluate(self, P, Q, stream=None):
        """Values of the grid solution of Q at the probes P [2][n_p]: shape [c][n_p]."""
        t = self._torch
        P, Q = self._probes(P), self._vec(Q)
        U = t.empty((self.ncomp, P.shape[1]), dtype=t.float64, device=Q.device)
        ibdl_probe_evaluate(self._h, P.data_ptr(), P.shape[1], Q.data_ptr(), U.data_ptr(), _stream_handle(stream))
        return U

    def probe_vjp(self, P, Q, nu, stream=None, want=(True, True, True, True)):
        """(Eᵀν [c·M], ∂(νᵀEQ)/∂X [dim][M], ∂/∂n [dim][M], ∂/∂Δs [M]); False in ``want`` gives None."""
        t = self._torch
        P, Q = self._probes(P), self._vec(Q)
        nu = nu.detach().to(dtype=t.float64).contiguous()
        assert nu.numel() == self.ncomp * P.shape[1]
        shapes = [(self.ncomp * self.M,), (self.dim, self.M), (self.dim, self.M), (self.M,)]
        outs = [t.empty(sh, dtype=t.float64, device=Q.device) if w else None for sh, w in zip(shapes, want)]
        ptrs = [o.data_ptr() if o is not None else 0 for o in outs]
        ibdl_probe_vjp(self._h, P.data_ptr(), P.shape[1], Q.data_ptr(), nu.data_ptr(), *ptrs, _stream_handle(stream))
        return tuple(outs)

    def indicator(self, stream=None):
        """(χ shifted to 0 at the box corner [n]*dim float64, flags |χ| > ½ [n]*dim uint8): the nodes
        enclosed by the boundary (Sec. 5.3.5)."""
        t = self._torch
        shape = (self.n,) * self.dim
        chi = t.empty(shape, dtype=t.float64, device="cuda")
        flags = t.empty(shape, dtype=t.uint8, device="cuda")
        ibdl_indicator(self._h, chi.data_ptr(), flags.data_ptr(), _stream_handle(stream))
        return chi, flags

    def near_boundary(self, Ub, u, omega, m1: float, m2: float, out=None, stream=None):
        """Grid solution u with the values of Ω within m1·h of Γ replaced by the linear interpolation
        of Sec. 5.3.4 between U_b on Γ and u at m2·h (2-D). ``omega`` is a uint8 (or bool) mask of Ω."""
        t = self._torch
        Ub = t.as_tensor(Ub, dtype=t.float64).to("cuda").contiguous()
        u = u.to(dtype=t.float64).contiguous()
        omega = omega.to(device="cuda", dtype=t.uint8).contiguous()
        assert Ub.numel() >= self.ncomp * self.M and u.numel() == self.ncomp * self.n ** 2
        assert omega.numel() == self.n ** 2
        if out is None:
            out = t.empty_like(u)
        ibdl_near_boundary(self._h, Ub.data_ptr(), u.data_ptr(), omega.data_ptr(), m1, m2, out.data_ptr(),
                           _stream_handle(stream))
        return out

    def _solve(self, entry, Ub, rtol, precision, restart, maxit, inner_rtol, max_refine, Q, stream, check,
               residual="fp32x2"):
        t = self._torch
        o = ibdl_default_solve_opts()
        o.rtol, o.restart, o.maxit, o.precision = rtol, restart, maxit, _PREC[precision]
        o.inner_rtol, o.max_refine, o.residual = inner_rtol, max_refine, _PREC[residual]
        host = isinstance(Ub, np.ndarray) or (hasattr(Ub, "is_cuda") and not Ub.is_cuda)
        if host:
            Ub = t.as_tensor(np.ascontiguousarray(np.asarray(Ub, dtype=np.float64)).reshape(-1)) \
                if isinstance(Ub, np.ndarray) else Ub.contiguous()
            o.io_on_host = 1
            if Q is None:
                Q = t.empty_like(Ub)
        else:
            Ub = self._vec(Ub)
            if Q is None:
                Q = t.empty_like(Ub)
        info = ibdl_solve_info()
        st = entry(self._h, Ub.data_ptr(), Q.data_ptr(), o, info, _stream_handle(stream), check=check)
        return Q, info.as_dict(), st

    def autotune(self, precision_mask: int = 7, stream=None):
        """precision_mask bits: 1 FP64, 2 FP32, 4 float-float (2-D)."""
        ibdl_autotune(self._h, precision_mask, _stream_handle(stream))

    def set_stage_timing(self, enable: bool = True):
        ibdl_set_stage_timing(self._h, int(enable))

    def launch_plan(self, precision: str = "fp32"):
        """The 2-D launch plan of one grid arithmetic: rows, cols, threads, staged, split."""
        return ibdl_launch_plan(self._h, _PREC[precision])

    def stage_times(self):
        """{stage name: (total device ms, launches)} since the previous call."""
        ms, n = ibdl_get_stage_times(self._h)
        return {STAGE_NAMES[i]: (ms[i], n[i]) for i in range(IBDL_STAGE_COUNT) if n[i]}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            ibdl_destroy_geometry(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
