// Host-side launch helpers of the 2-D kernels, and the launch of one application for a
// compile-time grid size. Included by apply2d.cu and by the per-size translation units
// apply2d_n*.cu, each of which instantiates the kernels of one size (so the sizes compile in
// parallel).
#pragma once

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <mutex>
#include <type_traits>
#include <utility>
#include <vector>

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

// Persistent launches: as many CTAs of `kernel` as fit on the device at once (at most `units`),
// from an occupancy query cached per kernel, device, thread count and shared memory size.
template <typename K>
inline int persistent_grid(K kernel, int threads, size_t smem, int units) {
  struct Entry {
    int dev, threads;
    size_t smem;
    int blocks;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  int blocks = -1;
  {
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry& e : cache)
      if (e.dev == dev && e.threads == threads && e.smem == smem) blocks = e.blocks;
  }
  if (blocks < 0) {
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess) per_sm = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 1;
    blocks = std::max(per_sm, 1) * std::max(sms, 1);
    std::lock_guard<std::mutex> lock(mu);
    cache.push_back({dev, threads, smem, blocks});
  }
  return std::max(1, std::min(units, blocks));
}

// Shared memory of the staged column pass: 128 bytes of alignment slack, 128 bytes of barriers,
// NS stages of one unit (NIN fields of C columns, then the two symbol tables; a multiple of 128
// bytes) and the exchange buffers (NMAX fields of C skewed columns). Up to `want` stages (at
// least 2); false if two do not fit or the box would be wider than 256 floats.
struct ColStageShape {
  int stages, stage_bytes;
  size_t smem;
};
inline bool col_stage_shape(int nin, int nmax, int C, int R, int L, int want, ColStageShape* sh) {
  const size_t n = size_t(1) << L;
  // the box's inner extent 2·C·R floats is at most 256 elements
  if (C < 1 || (C & (C - 1)) || R < 2 || 2 * C * R > 256) return false;
  size_t sb = (size_t)nin * C * n * sizeof(float2) + 2 * n * sizeof(float);
  sb = (sb + 127) & ~size_t(127);
  const size_t xb = (size_t)nmax * C * col_stride_2d(L, C, (int)sizeof(float2)) * sizeof(float2);
  for (int ns = std::max(2, std::min(want, 4)); ns >= 2; --ns) {
    const size_t tot = 256 + ns * sb + xb;
    if (tot <= kSmemLimit2d) {
      sh->stages = ns;
      sh->stage_bytes = (int)sb;
      sh->smem = tot;
      return true;
    }
  }
  return false;
}
// IBDL_COL_STAGES: stages of the staged column pass (2 … 4, default 3)
inline int col_stages_env() {
  static int v = 0;
  if (v == 0) {
    const char* e = getenv("IBDL_COL_STAGES");
    int k = e ? atoi(e) : 3;
    v = k < 2 ? 2 : (k > 4 ? 4 : k);
  }
  return v;
}

// The staged FP32 column pass of one application: persistent CTAs over the (n/2)/C units.
template <int OP, int L>
ibdl_status launch_col_staged(Geometry* g, const ColParams<float>& cp, cudaStream_t s, bool pdl) {
  constexpr int NIN = Traits<OP>::NIN, NOUT = Traits<OP>::NOUT, NMAX = NIN > NOUT ? NIN : NOUT;
  constexpr int n = 1 << L;
  const CUtensorMap* map = nullptr;
  IBDL_TRY(col_stage_map(g, cp.R, cp.C, &map));
  ColStageShape sh;
  if (!col_stage_shape(NIN, NMAX, cp.C, cp.R, L, col_stages_env(), &sh))
    return fail(IBDL_ERR_UNSUPPORTED, "staged column pass: the column group does not fit shared memory");
  static std::atomic<unsigned long long> d{0};
  IBDL_CUDA(opt_in_smem(kt_colpass<OP, L>, d));
  const int threads = field_groups_2d(NMAX, L, true) * cp.C * threads_per_seq_2d(L, true);
  const int units = (n / 2) / cp.C;
  const int grid = persistent_grid(kt_colpass<OP, L>, threads, sh.smem, units);
  ColStageArgs a;
  a.P = nullptr;
  a.maps = nullptr;
  a.units = nullptr;
  a.nunits = units;
  a.stages = sh.stages;
  a.stage_bytes = sh.stage_bytes;
  a.err = cp.err;
  IBDL_CUDA(launch_k(kt_colpass<OP, L>, grid, threads, sh.smem, s, pdl, cp, *map, a));
  return IBDL_OK;
}

// whether a geometry's FP32 column pass runs staged: its mode is on and the unit fits
inline bool col_staged_for(const Geometry* g, const ColParams<float>& cp, int nin, int nmax, int L) {
  if (g->col_stage != 1) return false;
  ColStageShape sh;
  return col_stage_shape(nin, nmax, cp.C, cp.R, L, 2, &sh);
}

template <typename T, int OP, int L>
ibdl_status set_attrs_2d() {
  static std::atomic<unsigned long long> d1{0}, d2{0}, d3{0}, d4{0};
  IBDL_CUDA(opt_in_smem(k_spread_rowfft<T, OP, L>, d1));
  IBDL_CUDA(opt_in_smem(k_colpass<T, OP, L>, d2));
  IBDL_CUDA(opt_in_smem(k_rowifft_gather<T, OP, G_INTERP, L>, d3));
  if constexpr (!std::is_same<T, ff>::value) IBDL_CUDA(opt_in_smem(k_rowifft_gather<T, OP, G_GRID, L>, d4));
  return IBDL_OK;
}

// One application one field per launch (grids whose fields do not fit shared memory together):
// a spread + row FFT launch per input field, the forward column transform of each input field,
// one symbol launch over the spectrum, the inverse column transform of each output field, and an
// inverse row FFT + interpolation launch per output field (which add into Y). 2·NIN + 2·NOUT + 1
// launches, chained by programmatic launch.
template <typename T, int OP, int L>
ibdl_status launch_apply_split_2d(Geometry* g, const RowParams<T>& rp, const ColParams<T>& cp, const Launch2D& lc,
                                  cudaStream_t s) {
  constexpr int NIN = Traits<OP>::NIN, NOUT = Traits<OP>::NOUT;
  constexpr int n = 1 << L;
  static std::atomic<unsigned long long> d1{0}, d2{0}, d3{0}, d4{0}, d5{0};
  const int st0 = std::is_same<T, float>::value ? IBDL_STAGE_SPREAD_ROWFFT_FP32 : IBDL_STAGE_SPREAD_ROWFFT_FP64;
  if (g->timing) timing_mark(g, s, -1);
  RowParams<T> r = rp;
  if constexpr (NIN > 1) {
    IBDL_CUDA(opt_in_smem(k_spread_rowfft1<T, OP, L>, d1));
    for (int f = 0; f < NIN; ++f) {
      r.fsel = f;
      IBDL_CUDA(launch_k(k_spread_rowfft1<T, OP, L>, n / lc.R, lc.threads_row, lc.smem_row, s, lc.pdl, r));
    }
  } else {
    IBDL_CUDA(launch_k(k_spread_rowfft<T, OP, L>, n / lc.R, lc.threads_row, lc.smem_row, s, lc.pdl, rp));
  }
  if (g->timing) timing_mark(g, s, st0);
  IBDL_CUDA(opt_in_smem(k_colfft<T, L, false>, d2));
  IBDL_CUDA(opt_in_smem(k_colfft<T, L, true>, d3));
  for (int f = 0; f < NIN; ++f)
    IBDL_CUDA(launch_k(k_colfft<T, L, false>, (n / 2) / lc.C, lc.threads_col, lc.smem_col, s, lc.pdl, cp, f));
  const int sgrid = (int)std::min<long>((long)n * (n / 2) / 256, 152L * 16);
  IBDL_CUDA(launch_k(k_symbol2d<T, OP, L>, sgrid > 0 ? sgrid : 1, 256, 0, s, lc.pdl, cp));
  for (int f = 0; f < NOUT; ++f)
    IBDL_CUDA(launch_k(k_colfft<T, L, true>, (n / 2) / lc.C, lc.threads_col, lc.smem_col, s, lc.pdl, cp, f));
  if (g->timing) timing_mark(g, s, st0 + 1);
  if constexpr (NOUT > 1) {
    if (lc.grid_mode == G_GRID) {
      if constexpr (!std::is_same<T, ff>::value) {
        IBDL_CUDA(opt_in_smem(k_rowifft_gather1<T, OP, G_GRID, L>, d4));
        for (int f = 0; f < NOUT; ++f) {
          r.fsel = f;
          IBDL_CUDA(launch_k(k_rowifft_gather1<T, OP, G_GRID, L>, n / lc.R, lc.threads_gather, lc.smem_gather, s,
                             lc.pdl, r));
        }
      } else {
        return fail(IBDL_ERR_UNSUPPORTED, "float-float grid output");
      }
    } else {
      IBDL_CUDA(opt_in_smem(k_rowifft_gather1<T, OP, G_INTERP, L>, d5));
      for (int f = 0; f < NOUT; ++f) {
        r.fsel = f;
        IBDL_CUDA(launch_k(k_rowifft_gather1<T, OP, G_INTERP, L>, n / lc.R, lc.threads_gather, lc.smem_gather, s,
                           lc.pdl, r));
      }
    }
  } else {
    if constexpr (std::is_same<T, ff>::value) {
      if (lc.grid_mode == G_GRID) return fail(IBDL_ERR_UNSUPPORTED, "float-float grid output");
      IBDL_CUDA(launch_k(k_rowifft_gather<T, OP, G_INTERP, L>, n / lc.R, lc.threads_gather, lc.smem_gather, s, lc.pdl,
                         rp));
    } else if (lc.grid_mode == G_GRID) {
      IBDL_CUDA(launch_k(k_rowifft_gather<T, OP, G_GRID, L>, n / lc.R, lc.threads_gather, lc.smem_gather, s, lc.pdl,
                         rp));
    } else {
      IBDL_CUDA(launch_k(k_rowifft_gather<T, OP, G_INTERP, L>, n / lc.R, lc.threads_gather, lc.smem_gather, s, lc.pdl,
                         rp));
    }
  }
  if (g->timing) timing_mark(g, s, st0 + 2);
  g->launches += (NIN > 1 ? NIN : 1) + NIN + 1 + NOUT + (NOUT > 1 ? NOUT : 1);
  IBDL_CUDA(cudaGetLastError());
  return IBDL_OK;
}

template <typename T, int OP, int L>
ibdl_status launch_apply_2d(Geometry* g, const RowParams<T>& rp, const ColParams<T>& cp, const Launch2D& lc,
                            cudaStream_t s) {
  constexpr int pi = std::is_same<T, float>::value ? 1 : 0;
  constexpr int n = 1 << L;
  IBDL_TRY((set_attrs_2d<T, OP, L>()));
  if constexpr (Traits<OP>::NIN > 1 || Traits<OP>::NOUT > 1) {
    if (lc.split) return launch_apply_split_2d<T, OP, L>(g, rp, cp, lc, s);
  }
  const int st0 = pi ? IBDL_STAGE_SPREAD_ROWFFT_FP32 : IBDL_STAGE_SPREAD_ROWFFT_FP64;
  if (g->timing) timing_mark(g, s, -1);
  IBDL_CUDA(launch_k(k_spread_rowfft<T, OP, L>, n / lc.R, lc.threads_row, lc.smem_row, s, lc.pdl, rp));
  if (g->timing) timing_mark(g, s, st0);
  bool staged = false;
  if constexpr (std::is_same<T, float>::value) {
    constexpr int NIN = Traits<OP>::NIN, NOUT = Traits<OP>::NOUT;
    staged = col_staged_for(g, cp, NIN, NIN > NOUT ? NIN : NOUT, L);
    if (staged) IBDL_TRY((launch_col_staged<OP, L>(g, cp, s, lc.pdl)));
  }
  if (!staged) IBDL_CUDA(launch_k(k_colpass<T, OP, L>, (n / 2) / lc.C, lc.threads_col, lc.smem_col, s, lc.pdl, cp));
  if (g->timing) timing_mark(g, s, st0 + 1);
  if constexpr (std::is_same<T, ff>::value) {
    // float-float serves boundary applications only (the refinement residual)
    if (lc.grid_mode == G_GRID) return fail(IBDL_ERR_UNSUPPORTED, "float-float grid output");
    IBDL_CUDA(launch_k(k_rowifft_gather<T, OP, G_INTERP, L>, n / lc.R, lc.threads_gather, lc.smem_gather, s, lc.pdl,
                       rp));
  } else if (lc.grid_mode == G_GRID) {
    IBDL_CUDA(launch_k(k_rowifft_gather<T, OP, G_GRID, L>, n / lc.R, lc.threads_gather, lc.smem_gather, s, lc.pdl,
                       rp));
  } else {
    IBDL_CUDA(launch_k(k_rowifft_gather<T, OP, G_INTERP, L>, n / lc.R, lc.threads_gather, lc.smem_gather, s, lc.pdl,
                       rp));
  }
  if (g->timing) timing_mark(g, s, st0 + 2);
  g->launches += 3;
  IBDL_CUDA(cudaGetLastError());
  return IBDL_OK;
}

// One batched stage (0 spread + row FFT, 1 column pass, 2 inverse row FFT + gather) for the
// problems of grid size 2^L: a launch over their (problem, unit) range of the batch's tables.
template <typename T, int OP, int L>
ibdl_status batch_stage_2d(Batch* B, int stage, int mode, const double* in_base, double* out_base, cudaStream_t s,
                           bool pdl) {
  constexpr int pi = std::is_same<T, float>::value ? 1 : (std::is_same<T, ff>::value ? 2 : 0);
  const BatchSize& z = B->lv[pi][L];
  const RowParams<T>* rp = static_cast<const RowParams<T>*>(B->rowp[pi][mode]);
  const ColParams<T>* cp = static_cast<const ColParams<T>*>(B->colp[pi]);
  if (stage == 0) {
    static std::atomic<unsigned long long> d{0};
    IBDL_CUDA(opt_in_smem(kb_spread_rowfft<T, OP, L>, d));
    IBDL_CUDA(launch_k(kb_spread_rowfft<T, OP, L>, z.row_count, z.threads_row, z.smem_row, s, pdl, rp,
                       (const int2*)B->row_units[pi] + z.row_start, in_base, out_base));
  } else if (stage == 1) {
    if constexpr (Traits<OP>::NIN == 1 && Traits<OP>::NOUT == 1) {
      if (B->persistent) {
        // persistent CTAs (as many as fit on the GPU at once) walk the size's units
        static std::atomic<unsigned long long> d{0};
        IBDL_CUDA(opt_in_smem(kbp_colpass<T, OP, L>, d));
        int per_sm = 0, dev = 0, sms = 0;
        IBDL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kbp_colpass<T, OP, L>, z.threads_col,
                                                                z.smem_col));
        IBDL_CUDA(cudaGetDevice(&dev));
        IBDL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int grid = std::max(1, std::min(z.col_count, std::max(per_sm, 1) * sms));
        IBDL_CUDA(launch_k(kbp_colpass<T, OP, L>, grid, z.threads_col, z.smem_col, s, pdl, cp,
                           (const int2*)B->col_units[pi] + z.col_start, z.col_count));
        B->launches += 1;
        return IBDL_OK;
      }
    }
    if constexpr (std::is_same<T, float>::value) {
      if (z.col_staged) {
        // the staged pass: persistent CTAs over the size's units, each problem's tensor map
        static std::atomic<unsigned long long> d{0};
        IBDL_CUDA(opt_in_smem(kt_colpass<OP, L>, d));
        ColStageArgs a;
        a.P = cp;
        a.maps = B->tmaps;
        a.units = (const int2*)B->col_units[pi] + z.col_start;
        a.nunits = z.col_count;
        a.stages = z.stages;
        a.stage_bytes = z.stage_bytes;
        a.err = B->geoms[0]->err_dev;
        ColParams<float> none = {};
        CUtensorMap nomap = {};
        const int grid = persistent_grid(kt_colpass<OP, L>, z.threads_col, z.smem_staged, z.col_count);
        IBDL_CUDA(launch_k(kt_colpass<OP, L>, grid, z.threads_col, z.smem_staged, s, pdl, none, nomap, a));
        B->launches += 1;
        return IBDL_OK;
      }
    }
    static std::atomic<unsigned long long> d{0};
    IBDL_CUDA(opt_in_smem(kb_colpass<T, OP, L>, d));
    IBDL_CUDA(launch_k(kb_colpass<T, OP, L>, z.col_count, z.threads_col, z.smem_col, s, pdl, cp,
                       (const int2*)B->col_units[pi] + z.col_start));
  } else {
    static std::atomic<unsigned long long> d{0};
    IBDL_CUDA(opt_in_smem(kb_rowifft_gather<T, OP, L>, d));
    IBDL_CUDA(launch_k(kb_rowifft_gather<T, OP, L>, z.row_count, z.threads_gather, z.smem_gather, s, pdl, rp,
                       (const int2*)B->row_units[pi] + z.row_start, in_base, out_base));
  }
  B->launches += 1;
  return IBDL_OK;
}

// every operator at one size: FP32 and FP64 (with grid output), float-float (boundary output
// only, and not the single layer), and the batched stages of the four forward operators
#define IBDL_INSTANTIATE_2D_OP(T, OP, L)                                                                  \
  template ibdl_status launch_apply_2d<T, OP, L>(Geometry*, const RowParams<T>&, const ColParams<T>&,    \
                                                 const Launch2D&, cudaStream_t);
#define IBDL_INSTANTIATE_2D_B(T, OP, L) \
  template ibdl_status batch_stage_2d<T, OP, L>(Batch*, int, int, const double*, double*, cudaStream_t, bool);
#define IBDL_INSTANTIATE_2D_FWD(T, L)         \
  IBDL_INSTANTIATE_2D_OP(T, OP_SCALAR_AN, L) \
  IBDL_INSTANTIATE_2D_OP(T, OP_SCALAR_SD, L) \
  IBDL_INSTANTIATE_2D_OP(T, OP_STOKES_AN, L) \
  IBDL_INSTANTIATE_2D_OP(T, OP_STOKES_SD, L) \
  IBDL_INSTANTIATE_2D_B(T, OP_SCALAR_AN, L)  \
  IBDL_INSTANTIATE_2D_B(T, OP_SCALAR_SD, L)  \
  IBDL_INSTANTIATE_2D_B(T, OP_STOKES_AN, L)  \
  IBDL_INSTANTIATE_2D_B(T, OP_STOKES_SD, L)
#define IBDL_INSTANTIATE_2D_TRANS(T, L)   \
  IBDL_INSTANTIATE_2D_OP(T, OP_ADJ_AN, L) \
  IBDL_INSTANTIATE_2D_OP(T, OP_ADJ_SD, L) \
  IBDL_INSTANTIATE_2D_OP(T, OP_STOKES_T, L)
#define IBDL_INSTANTIATE_2D_T(T, L) \
  IBDL_INSTANTIATE_2D_FWD(T, L)     \
  IBDL_INSTANTIATE_2D_TRANS(T, L)   \
  IBDL_INSTANTIATE_2D_OP(T, OP_SL, L)
#define IBDL_INSTANTIATE_2D(L)   \
  IBDL_INSTANTIATE_2D_T(float, L) \
  IBDL_INSTANTIATE_2D_T(double, L)

// declarations for the users of the per-size units
#define IBDL_DECLARE_2D_OP(T, OP, L)                                                                           \
  extern template ibdl_status launch_apply_2d<T, OP, L>(Geometry*, const RowParams<T>&, const ColParams<T>&, \
                                                        const Launch2D&, cudaStream_t);
#define IBDL_DECLARE_2D_B(T, OP, L) \
  extern template ibdl_status batch_stage_2d<T, OP, L>(Batch*, int, int, const double*, double*, cudaStream_t, bool);
#define IBDL_DECLARE_2D_FWD(T, L)         \
  IBDL_DECLARE_2D_OP(T, OP_SCALAR_AN, L) \
  IBDL_DECLARE_2D_OP(T, OP_SCALAR_SD, L) \
  IBDL_DECLARE_2D_OP(T, OP_STOKES_AN, L) \
  IBDL_DECLARE_2D_OP(T, OP_STOKES_SD, L) \
  IBDL_DECLARE_2D_B(T, OP_SCALAR_AN, L)  \
  IBDL_DECLARE_2D_B(T, OP_SCALAR_SD, L)  \
  IBDL_DECLARE_2D_B(T, OP_STOKES_AN, L)  \
  IBDL_DECLARE_2D_B(T, OP_STOKES_SD, L)
#define IBDL_DECLARE_2D_TRANS(T, L)   \
  IBDL_DECLARE_2D_OP(T, OP_ADJ_AN, L) \
  IBDL_DECLARE_2D_OP(T, OP_ADJ_SD, L) \
  IBDL_DECLARE_2D_OP(T, OP_STOKES_T, L)
#define IBDL_DECLARE_2D_T(T, L) \
  IBDL_DECLARE_2D_FWD(T, L)     \
  IBDL_DECLARE_2D_TRANS(T, L)   \
  IBDL_DECLARE_2D_OP(T, OP_SL, L)
#define IBDL_DECLARE_2D(L)   \
  IBDL_DECLARE_2D_T(float, L) \
  IBDL_DECLARE_2D_T(double, L)

// float-float is compiled for grids up to 4096²
constexpr int kMaxLff = 12;

}  // namespace ibdl
