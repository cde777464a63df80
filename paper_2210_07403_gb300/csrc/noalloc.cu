// ibdl_apply_noalloc: the 2-D operator application A Q with no memory allocation at all.
//
// Who needs it: code that runs where allocating device memory is not allowed or not possible, for
// example a real-time or latency-bound loop that must not take the allocator's locks or wait on
// it, a plug-in whose host application owns all device memory through its own allocator, or a
// process that has already given the GPU's memory away and must not fail for want of more. Such
// a caller cannot create an ibdl_geometry (creating one allocates its tables and work buffers), so
// this entry point takes the geometry description directly and keeps everything it needs in one
// fixed array that is part of the library image.
//
// The array: g_noalloc_scratch below, kNoAllocScratchBytes (8 MiB) per GPU, created when the
// library is loaded and held by every GPU that loads it until the process exits. Each call carves
// it into the sorted point tables, kernel weights, FFT twiddles, Fourier symbols and grid spectra
// of the problem, rebuilds all of them (the per-cell counters are cleared first; every other part
// is fully overwritten before it is read), then runs the same three kernels as ibdl_apply.
//
// Sharing: all calls on one GPU use the same array and it keeps the last call's contents. Two calls
// whose work overlaps on the GPU (different streams, or different host threads) race on it and
// give wrong results; serialise them on one stream.
#include <cmath>
#include <cstring>
#include <mutex>

#include "ibdl_internal.cuh"

namespace ibdl {
ibdl_status fill_geometry_tables(Geometry* g, const double* dX, const double* dN, const double* dW, int* key,
                                 int* count, int* cursor, cudaStream_t s);
}

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Host code may not use g_noalloc_scratch as a pointer: in host code that name is a stand-in, not
// the device address. The address is looked up once per device, with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices];

ibdl_status scratch_address(void** out) {
  int dev = -1;
  IBDL_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return ibdl::fail(IBDL_ERR_UNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return ibdl::cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return IBDL_OK;
}

// bump allocation inside the static array, 256-byte aligned pieces
struct Carve {
  unsigned char* base;
  size_t used;
  template <typename T>
  T* take(size_t count) {
    used = (used + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + used);
    used += count * sizeof(T);
    return p;
  }
};

ibdl_status device_ptr(const void* p, const char* name) {
  if (!p) return ibdl::fail(IBDL_ERR_INVALID_ARG, std::string(name) + " is NULL");
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return ibdl::fail(IBDL_ERR_INVALID_ARG, std::string(name) + " is not a CUDA device pointer");
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return ibdl::fail(IBDL_ERR_INVALID_ARG, std::string(name) + " is not a CUDA device pointer");
  return IBDL_OK;
}

}  // namespace

using namespace ibdl;

extern "C" ibdl_status ibdl_apply_noalloc(const ibdl_geometry_desc* d, int precision, const double* Q, double* Y,
                                          void* stream) {
  set_error("");
  if (!d) return fail(IBDL_ERR_INVALID_ARG, "descriptor is NULL");
  if (d->dim != 2) return fail(IBDL_ERR_UNSUPPORTED, "ibdl_apply_noalloc handles 2-D problems only");
  if (d->n < 16 || d->n > 8192 || (d->n & (d->n - 1))) return fail(IBDL_ERR_INVALID_ARG, "n must be a power of two in [16, 8192]");
  if (!(d->box > 0) || !std::isfinite(d->box)) return fail(IBDL_ERR_INVALID_ARG, "box must be positive and finite");
  if (!std::isfinite(d->origin[0]) || !std::isfinite(d->origin[1])) return fail(IBDL_ERR_INVALID_ARG, "origin must be finite");
  if (d->n_points < 1 || d->n_points > (int64_t)1 << 28) return fail(IBDL_ERR_INVALID_ARG, "n_points must be in [1, 2^28]");
  if (!d->inputs_on_device) return fail(IBDL_ERR_INVALID_ARG, "X, normals and weights must be device pointers (inputs_on_device = 1)");
  if (d->pde != IBDL_PDE_SCALAR && d->pde != IBDL_PDE_STOKES) return fail(IBDL_ERR_INVALID_ARG, "unknown pde");
  if (!(d->lambda >= 0) || !std::isfinite(d->lambda)) return fail(IBDL_ERR_INVALID_ARG, "lambda must be finite and >= 0");
  if (d->bc != IBDL_BC_DIRICHLET && d->bc != IBDL_BC_NEUMANN) return fail(IBDL_ERR_INVALID_ARG, "unknown boundary condition");
  if (d->eta != 0) return fail(IBDL_ERR_UNSUPPORTED, "ibdl_apply_noalloc: the completed method (eta > 0) is not supported");
  if (d->bc == IBDL_BC_NEUMANN && d->pde != IBDL_PDE_SCALAR)
    return fail(IBDL_ERR_UNSUPPORTED, "Neumann conditions are implemented for the scalar PDE");
  if (d->pde == IBDL_PDE_STOKES && (!(d->mu > 0) || !std::isfinite(d->mu)))
    return fail(IBDL_ERR_INVALID_ARG, "mu must be finite and > 0");
  if (d->delta != IBDL_DELTA_COS && d->delta != IBDL_DELTA_SQRT) return fail(IBDL_ERR_INVALID_ARG, "unknown delta");
  if (d->dipole != IBDL_DIPOLE_ANALYTIC && d->dipole != IBDL_DIPOLE_SPECTRAL_DIV) return fail(IBDL_ERR_INVALID_ARG, "unknown dipole");
  if (d->symbol != IBDL_SYMBOL_SPECTRAL && d->symbol != IBDL_SYMBOL_FD2) return fail(IBDL_ERR_INVALID_ARG, "unknown symbol");
  if (precision != IBDL_FP64 && precision != IBDL_FP32) return fail(IBDL_ERR_INVALID_ARG, "precision must be IBDL_FP64 or IBDL_FP32");
  IBDL_TRY(device_ptr(d->X, "X"));
  IBDL_TRY(device_ptr(d->normals, "normals"));
  IBDL_TRY(device_ptr(d->weights, "weights"));
  IBDL_TRY(device_ptr(Q, "Q"));
  IBDL_TRY(device_ptr(Y, "Y"));

  // a geometry view on the stack whose buffers all live in the static array
  Geometry g;
  std::memset(&g, 0, sizeof(g));
  g.dim = 2;
  g.n = d->n;
  g.pde = d->pde;
  g.delta = d->delta;
  g.dipole = d->dipole;
  g.symbol = d->symbol;
  g.box = d->box;
  g.h = d->box / d->n;
  g.lambda = d->lambda;
  g.mu = d->mu;
  g.bc = d->bc;
  g.origin[0] = d->origin[0];
  g.origin[1] = d->origin[1];
  g.M = d->n_points;
  g.ncomp = d->pde == IBDL_PDE_STOKES ? 2 : 1;
  const bool sd = d->dipole == IBDL_DIPOLE_SPECTRAL_DIV;
  g.nf_in = d->pde == IBDL_PDE_STOKES ? (sd ? 4 : 3) : (sd ? 2 : 1);
  g.nf_out = d->pde == IBDL_PDE_STOKES ? 2 : (sd ? 2 : 1);
  g.ncell = g.n;
  const size_t M = (size_t)g.M, n = (size_t)g.n;
  if (Q + g.ncomp * M > Y && Y + g.ncomp * M > Q) return fail(IBDL_ERR_INVALID_ARG, "Q and Y overlap");

  void* base = nullptr;
  IBDL_TRY(scratch_address(&base));
  Carve c{static_cast<unsigned char*>(base), 0};
  int* key = c.take<int>(M);
  int* count = c.take<int>(n);
  int* cursor = c.take<int>(n + 1);
  g.perm = c.take<int>(M);
  g.base = c.take<int>(2 * M);
  g.cell_start = c.take<int>(n + 1);
  g.t64.phi = c.take<double>(8 * M);
  g.t64.dphi = c.take<double>(8 * M);
  g.t64.wscale = c.take<double>(M);
  g.t64.nrm = c.take<double>(2 * M);
  g.t32.phi = c.take<float>(8 * M);
  g.t32.dphi = c.take<float>(8 * M);
  g.t32.wscale = c.take<float>(M);
  g.t32.nrm = c.take<float>(2 * M);
  const int nf = g.nf_in > g.nf_out ? g.nf_in : g.nf_out;
  g.spec_bytes = (size_t)nf * n * (n / 2) * sizeof(double2);
  g.spec = c.take<unsigned char>(g.spec_bytes);
  g.tw64 = c.take<double2>(n);
  g.tw32 = c.take<float2>(n);
  g.lap64 = c.take<double>(n);
  g.der64 = c.take<double>(n);
  g.lap32 = c.take<float>(n);
  g.der32 = c.take<float>(n);
  if (c.used > kNoAllocScratchBytes)
    return fail(IBDL_ERR_INVALID_ARG, "problem needs " + std::to_string(c.used) + " bytes of scratch; ibdl_apply_noalloc holds " +
                                          std::to_string(kNoAllocScratchBytes) + " (8 MiB): use a smaller grid or fewer points, or ibdl_apply");

  IBDL_TRY(plan_2d(&g));
  g.col_stage = 0;  // the view has no error flag for the staged column pass: the direct pass runs
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  IBDL_TRY(fill_geometry_tables(&g, d->X, d->normals, d->weights, key, count, cursor, s));
  return apply_2d(&g, precision, Q, Y, s, nullptr);
}
