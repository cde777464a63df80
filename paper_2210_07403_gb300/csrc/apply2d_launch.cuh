// Host-side launch helpers of the 2-D kernels, and the launch of one application for a
// compile-time grid size. Included by apply2d.cu and by the per-size translation units
// apply2d_n*.cu, each of which instantiates the kernels of one size (so the sizes compile in
// parallel).
#pragma once

#include <atomic>
#include <cstdlib>
#include <type_traits>
#include <utility>

#include "apply2d_kernels.cuh"

namespace ibdl {

// Dynamic shared memory per CTA: the 227 KiB a block may hold (the 2-D kernels have no static
// shared memory).
constexpr size_t kSmemLimit2d = 227 * 1024;

// Programmatic dependent launch: the kernel may start while the previous kernel on the stream
// drains; it runs its prologue and then waits in cudaGridDependencySynchronize(). IBDL_NO_PDL=1
// turns it off.
inline bool use_pdl() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("IBDL_NO_PDL");
    v = (e && atoi(e) != 0) ? 0 : 1;
  }
  return v == 1;
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s, bool pdl,
                            Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &at;
  cfg.numAttrs = pdl && use_pdl() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Opt a kernel in to the full dynamic shared memory once per device: the attribute belongs to the
// function on the current device, so a per-device bit records it (setting it twice is harmless,
// so two threads racing on a first call need no lock).
template <typename K>
inline cudaError_t opt_in_smem(K kernel, std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit2d);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

template <typename T, int OP, int L>
ibdl_status set_attrs_2d() {
  static std::atomic<unsigned long long> d1{0}, d2{0}, d3{0}, d4{0};
  IBDL_CUDA(opt_in_smem(k_spread_rowfft<T, OP, L>, d1));
  IBDL_CUDA(opt_in_smem(k_colpass<T, OP, L>, d2));
  IBDL_CUDA(opt_in_smem(k_rowifft_gather<T, OP, G_INTERP, L>, d3));
  IBDL_CUDA(opt_in_smem(k_rowifft_gather<T, OP, G_GRID, L>, d4));
  return IBDL_OK;
}

template <typename T, int OP, int L>
ibdl_status launch_apply_2d(Geometry* g, const RowParams<T>& rp, const ColParams<T>& cp, const Launch2D& lc,
                            cudaStream_t s) {
  constexpr int pi = std::is_same<T, float>::value ? 1 : 0;
  constexpr int n = 1 << L;
  IBDL_TRY((set_attrs_2d<T, OP, L>()));
  const int st0 = pi ? IBDL_STAGE_SPREAD_ROWFFT_FP32 : IBDL_STAGE_SPREAD_ROWFFT_FP64;
  if (g->timing) timing_mark(g, s, -1);
  IBDL_CUDA(launch_k(k_spread_rowfft<T, OP, L>, n / lc.R, lc.threads_row, lc.smem_row, s, lc.pdl, rp));
  if (g->timing) timing_mark(g, s, st0);
  IBDL_CUDA(launch_k(k_colpass<T, OP, L>, (n / 2) / lc.C, lc.threads_col, lc.smem_col, s, lc.pdl, cp));
  if (g->timing) timing_mark(g, s, st0 + 1);
  if (lc.grid_mode == G_GRID)
    IBDL_CUDA(launch_k(k_rowifft_gather<T, OP, G_GRID, L>, n / lc.R, lc.threads_gather, lc.smem_gather, s, lc.pdl,
                       rp));
  else
    IBDL_CUDA(launch_k(k_rowifft_gather<T, OP, G_INTERP, L>, n / lc.R, lc.threads_gather, lc.smem_gather, s, lc.pdl,
                       rp));
  if (g->timing) timing_mark(g, s, st0 + 2);
  g->launches += 3;
  IBDL_CUDA(cudaGetLastError());
  return IBDL_OK;
}

// every operator and both precisions at one size
#define IBDL_INSTANTIATE_2D_OP(T, OP, L)                                                                  \
  template ibdl_status launch_apply_2d<T, OP, L>(Geometry*, const RowParams<T>&, const ColParams<T>&,    \
                                                 const Launch2D&, cudaStream_t);
#define IBDL_INSTANTIATE_2D_T(T, L)          \
  IBDL_INSTANTIATE_2D_OP(T, OP_SCALAR_AN, L) \
  IBDL_INSTANTIATE_2D_OP(T, OP_SCALAR_SD, L) \
  IBDL_INSTANTIATE_2D_OP(T, OP_STOKES_AN, L) \
  IBDL_INSTANTIATE_2D_OP(T, OP_STOKES_SD, L) \
  IBDL_INSTANTIATE_2D_OP(T, OP_ADJ_AN, L)    \
  IBDL_INSTANTIATE_2D_OP(T, OP_ADJ_SD, L)    \
  IBDL_INSTANTIATE_2D_OP(T, OP_STOKES_T, L)  \
  IBDL_INSTANTIATE_2D_OP(T, OP_SL, L)
#define IBDL_INSTANTIATE_2D(L)   \
  IBDL_INSTANTIATE_2D_T(float, L) \
  IBDL_INSTANTIATE_2D_T(double, L)

// declarations for the users of the per-size units
#define IBDL_DECLARE_2D_OP(T, OP, L)                                                                           \
  extern template ibdl_status launch_apply_2d<T, OP, L>(Geometry*, const RowParams<T>&, const ColParams<T>&, \
                                                        const Launch2D&, cudaStream_t);
#define IBDL_DECLARE_2D_T(T, L)          \
  IBDL_DECLARE_2D_OP(T, OP_SCALAR_AN, L) \
  IBDL_DECLARE_2D_OP(T, OP_SCALAR_SD, L) \
  IBDL_DECLARE_2D_OP(T, OP_STOKES_AN, L) \
  IBDL_DECLARE_2D_OP(T, OP_STOKES_SD, L) \
  IBDL_DECLARE_2D_OP(T, OP_ADJ_AN, L)    \
  IBDL_DECLARE_2D_OP(T, OP_ADJ_SD, L)    \
  IBDL_DECLARE_2D_OP(T, OP_STOKES_T, L)  \
  IBDL_DECLARE_2D_OP(T, OP_SL, L)
#define IBDL_DECLARE_2D(L)   \
  IBDL_DECLARE_2D_T(float, L) \
  IBDL_DECLARE_2D_T(double, L)

// Batched launches of one operator and precision: one launch per stage over the (problem, unit)
// tables; each CTA reads its problem's parameter block and runs the body of that problem's size.
// mode 0: the caller's vectors; mode 1: the batched GMRES Krylov basis. Instantiated in
// apply2d_batch_*.cu.
template <typename T, int OP, int LMAX>
ibdl_status batch_launch_range(Batch* B, int mode, const double* in_base, double* out_base, cudaStream_t s) {
  constexpr int pi = std::is_same<T, float>::value ? 1 : 0;
  static std::atomic<unsigned long long> d1{0}, d2{0}, d3{0};
  IBDL_CUDA(opt_in_smem(kb_spread_rowfft<T, OP, LMAX>, d1));
  IBDL_CUDA(opt_in_smem(kb_colpass<T, OP, LMAX>, d2));
  IBDL_CUDA(opt_in_smem(kb_rowifft_gather<T, OP, LMAX>, d3));
  const RowParams<T>* rp = static_cast<const RowParams<T>*>(B->rowp[pi][mode]);
  const ColParams<T>* cp = static_cast<const ColParams<T>*>(B->colp[pi]);
  IBDL_CUDA(launch_k(kb_spread_rowfft<T, OP, LMAX>, B->nrow_units[pi], B->threads_row[pi], B->smem_row[pi], s, false,
                     rp, (const int2*)B->row_units[pi], in_base, out_base));
  IBDL_CUDA(launch_k(kb_colpass<T, OP, LMAX>, B->ncol_units[pi], B->threads_col[pi], B->smem_col[pi], s, true, cp,
                     (const int2*)B->col_units[pi]));
  IBDL_CUDA(launch_k(kb_rowifft_gather<T, OP, LMAX>, B->nrow_units[pi], B->threads_gather[pi], B->smem_gather[pi], s,
                     true, rp, (const int2*)B->row_units[pi], in_base, out_base));
  B->launches += 3;
  IBDL_CUDA(cudaGetLastError());
  return IBDL_OK;
}

// Batched launches of one operator and precision: one launch per stage over the (problem, unit)
// tables; each CTA reads its problem's parameter block and runs the body of that problem's size.
// mode 0: the caller's vectors; mode 1: the batched GMRES Krylov basis. Instantiated in
// apply2d_batch_*.cu.
template <typename T, int OP>
ibdl_status batch_launch_2d(Batch* B, int mode, const double* in_base, double* out_base, cudaStream_t s) {
  return B->max_log2n <= kBatchSmallL2d ? batch_launch_range<T, OP, kBatchSmallL2d>(B, mode, in_base, out_base, s)
                                        : batch_launch_range<T, OP, kMaxL2d>(B, mode, in_base, out_base, s);
}

}  // namespace ibdl
