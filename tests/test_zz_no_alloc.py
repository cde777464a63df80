"""ibdl_apply_noalloc, the operator application that allocates nothing (for callers that cannot
call cudaMalloc, such as a latency-bound loop that must not take the allocator's locks or a plug-in
whose host application owns all device memory), against the regular ibdl_apply through the C ABI
and against the FP64 oracle.

Collected last on purpose: if it fails, a run that stops at the first failure has already run
every other test. It also passes on its own in a fresh process (the fixture builds and loads the
library itself)."""
import ctypes

import numpy as np
import pytest

import ibdl_inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ibdl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_07403_gb300 import build as b
    from paper_2210_07403_gb300 import ibdl as m

    b.build()
    m.load()
    return m


def _desc(m, p, dev):
    """Descriptor with device copies of the boundary arrays (kept alive by the returned list)."""
    X = torch.from_numpy(np.ascontiguousarray(p.bd.X)).to(dev)
    nrm = torch.from_numpy(np.ascontiguousarray(p.bd.n)).to(dev)
    w = torch.from_numpy(np.ascontiguousarray(p.bd.w)).to(dev)
    d = m.ibdl_geometry_desc()
    d.dim, d.n, d.box = 2, p.N, p.box
    d.origin[0], d.origin[1] = p.origin[0], p.origin[1]
    d.n_points = p.bd.M
    d.X, d.normals, d.weights = X.data_ptr(), nrm.data_ptr(), w.data_ptr()
    d.pde = m._PDE[p.pde]
    d.lambda_, d.mu = p.lam, p.mu
    d.delta, d.dipole, d.symbol = m._DELTA[p.delta], m._DIPOLE[p.dipole], m._SYMBOL[p.symbol]
    d.inputs_on_device = 1
    return d, [X, nrm, w]


CASES = [
    ("circle_laplace", lambda: I.circle_laplace(64, 100)),
    ("star_stokes_256", lambda: I.star_stokes(256, 400)),
    ("circle_spectral_div_fd2", lambda: I.circle_laplace(128, 201, delta="sqrt", dipole="spectral_div", symbol="fd2", lam=4.0)),
    # the largest documented case: three FP64 half spectra of 512² (6 MiB) and the tables of 800
    # points, close to the array's 8 MiB
    ("star_stokes_512", lambda: I.star_stokes(512, 800)),
]


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_noalloc_matches_apply(ibdl, name, make, precision, tol):
    from paper_2210_07403_gb300 import Geometry

    dev = torch.device("cuda", 0)
    p = make()
    from oracle import ibdl_oracle as O

    geom = Geometry.from_problem(p)
    og = O.geometry_from_problem(p)
    d, keep = _desc(ibdl, p, dev)
    prec = ibdl._PREC[precision]
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(len(name))
    for _ in range(2):  # two calls in a row: the shared array keeps the previous call's contents
        qh = rng.standard_normal(p.ncomp * p.bd.M)
        q = torch.from_numpy(qh).to(dev)
        y_ref = geom.apply(q, precision=precision)
        y = torch.full_like(q, float("nan"))
        st = ibdl.load().ibdl_apply_noalloc(ctypes.byref(d), prec, ctypes.c_void_p(q.data_ptr()),
                                            ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(stream))
        assert st == ibdl.IBDL_OK, ibdl.ibdl_last_error()
        torch.cuda.synchronize()
        rel = float(torch.linalg.norm(y - y_ref) / torch.linalg.norm(y_ref))
        assert rel < tol, (name, precision, rel)
        # and against the oracle, in the relative 2-norm and element by element
        yh, yo = y.cpu().numpy(), O.apply(og, qh)
        assert np.linalg.norm(yh - yo) / np.linalg.norm(yo) < tol, (name, precision)
        assert np.abs(yh - yo).max() < tol * np.abs(yo).max(), (name, precision)
    geom.close()
    del keep


def test_noalloc_rejects_oversized_problem(ibdl):
    dev = torch.device("cuda", 0)
    p = I.star_stokes(1024, 1600)  # 3 FP64 half spectra of 1024² need 24 MiB > 8 MiB
    d, keep = _desc(ibdl, p, dev)
    q = torch.zeros(2 * p.bd.M, dtype=torch.float64, device=dev)
    y = torch.zeros_like(q)
    st = ibdl.load().ibdl_apply_noalloc(ctypes.byref(d), ibdl.IBDL_FP32, ctypes.c_void_p(q.data_ptr()),
                                        ctypes.c_void_p(y.data_ptr()), None)
    assert st == ibdl.IBDL_ERR_INVALID_ARG
    assert "8 MiB" in ibdl.ibdl_last_error()
    d.inputs_on_device = 0
    st = ibdl.load().ibdl_apply_noalloc(ctypes.byref(d), ibdl.IBDL_FP32, ctypes.c_void_p(q.data_ptr()),
                                        ctypes.c_void_p(y.data_ptr()), None)
    assert st == ibdl.IBDL_ERR_INVALID_ARG
    del keep


def test_noalloc_in_cuda_graph(ibdl):
    """The call captured into a CUDA graph (its use case: a caller whose loop is one captured
    graph), then replayed with new densities written into the same input buffer. Each replay
    rebuilds the point tables and applies the operator; its result is compared with the regular
    application and the FP64 oracle. Neither torch's allocator nor the driver's free-memory count
    may change over the replays."""
    from oracle import ibdl_oracle as O
    from paper_2210_07403_gb300 import Geometry

    dev = torch.device("cuda", 0)
    p = I.star_stokes(256, 400)
    geom = Geometry.from_problem(p)
    og = O.geometry_from_problem(p)
    d, keep = _desc(ibdl, p, dev)
    lib = ibdl.load()
    nd = p.ncomp * p.bd.M
    q = torch.zeros(nd, dtype=torch.float64, device=dev)
    y = torch.zeros_like(q)
    s = torch.cuda.Stream()

    def call(stream_handle):
        return lib.ibdl_apply_noalloc(ctypes.byref(d), ibdl.IBDL_FP32, ctypes.c_void_p(q.data_ptr()),
                                      ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(stream_handle))

    # the first call outside any capture (its one-time set-up makes no stream call)
    assert call(s.cuda_stream) == ibdl.IBDL_OK, ibdl.ibdl_last_error()
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s, capture_error_mode="thread_local"):
        st = call(s.cuda_stream)
    assert st == ibdl.IBDL_OK, ibdl.ibdl_last_error()

    rng = np.random.default_rng(7)
    qs = [rng.standard_normal(nd) for _ in range(4)]
    refs = [geom.apply(torch.from_numpy(qh).to(dev), precision="fp32").cpu().numpy() for qh in qs]
    torch.cuda.synchronize()

    def replay(qh):
        q.copy_(torch.from_numpy(qh))
        graph.replay()
        return y.cpu().numpy()

    replay(qs[0])  # the first replay uploads the graph
    torch.cuda.synchronize()
    alloc0, free0 = torch.cuda.memory_allocated(dev), torch.cuda.mem_get_info(dev)[0]
    outs = [replay(qh) for qh in qs[1:]]
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated(dev) == alloc0
    assert torch.cuda.mem_get_info(dev)[0] == free0
    for qh, yr, yg in zip(qs[1:], refs[1:], outs):
        assert np.linalg.norm(yg - yr) / np.linalg.norm(yr) < 2e-5
        yo = O.apply(og, qh)
        assert np.abs(yg - yo).max() < 2e-5 * np.abs(yo).max()
    del graph
    geom.close()
    del keep
