// Two-dimensional IBDL operator, host side: launch shapes, the application of each operator and
// precision, batched launch tables, the autotuner and the source-term helpers. The kernels are in
// apply2d_kernels.cuh; each grid size n = 2^L is compiled in its own unit (apply2d_n*.cu) and
// reached through launch_apply_2d<T, OP, L>.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "apply2d_launch.cuh"

namespace ibdl {

IBDL_DECLARE_2D(4)
IBDL_DECLARE_2D(5)
IBDL_DECLARE_2D(6)
IBDL_DECLARE_2D(7)
IBDL_DECLARE_2D(8)
IBDL_DECLARE_2D(9)
IBDL_DECLARE_2D(10)
IBDL_DECLARE_2D(11)
IBDL_DECLARE_2D(12)
IBDL_DECLARE_2D(13)
#define IBDL_DECLARE_2D_FF(L) IBDL_DECLARE_2D_FWD(ff, L) IBDL_DECLARE_2D_TRANS(ff, L)
IBDL_DECLARE_2D_FF(4)
IBDL_DECLARE_2D_FF(5)
IBDL_DECLARE_2D_FF(6)
IBDL_DECLARE_2D_FF(7)
IBDL_DECLARE_2D_FF(8)
IBDL_DECLARE_2D_FF(9)
IBDL_DECLARE_2D_FF(10)
IBDL_DECLARE_2D_FF(11)
IBDL_DECLARE_2D_FF(12)

// precision slot and tables of a grid arithmetic type
template <typename T>
struct Slot2;
template <>
struct Slot2<double> {
  static constexpr int pi = 0;
  static const PointTable<double>& points(const Geometry* g) { return g->t64; }
  static const void* tw(const Geometry* g) { return g->tw64; }
  static const void* lap(const Geometry* g) { return g->lap64; }
  static const void* der(const Geometry* g) { return g->der64; }
};
template <>
struct Slot2<float> {
  static constexpr int pi = 1;
  static const PointTable<float>& points(const Geometry* g) { return g->t32; }
  static const void* tw(const Geometry* g) { return g->tw32; }
  static const void* lap(const Geometry* g) { return g->lap32; }
  static const void* der(const Geometry* g) { return g->der32; }
};
template <>
struct Slot2<ff> {
  static constexpr int pi = 2;
  static const PointTable<double>& points(const Geometry* g) { return g->t64; }
  static const void* tw(const Geometry* g) { return g->twff; }
  static const void* lap(const Geometry* g) { return g->lapff; }
  static const void* der(const Geometry* g) { return g->derff; }
};

static int log2i(int n) { return __builtin_ctz(n); }

template <typename T>
static RowParams<T> row_params(Geometry* g, const double* in, double* out, const int* stop, double* grid) {
  using PT = typename Prec2<T>::PT;
  const int pi = Slot2<T>::pi;
  RowParams<T> rp;
  rp.n = g->n;
  rp.log2n = log2i(g->n);
  rp.R = g->rows_per_cta[pi];
  rp.M = (int)g->M;
  rp.cell_start = g->cell_start;
  rp.base = g->base;
  rp.perm = g->perm;
  const PointTable<PT>& tb = Slot2<T>::points(g);
  rp.phi = tb.phi;
  rp.dphi = tb.dphi;
  rp.wscale = tb.wscale;
  rp.nrm = tb.nrm;
  rp.in = in;
  rp.out = out;
  rp.spec = reinterpret_cast<cplx<T>*>(g->spec);
  rp.tw = static_cast<const cplx<T>*>(Slot2<T>::tw(g));
  rp.stop = stop;
  rp.grid = grid;
  rp.idx = nullptr;
  rp.vstride = 0;
  rp.io_off = 0;
  rp.trans = 0;
  rp.fsel = 0;
  rp.grid_in = nullptr;
  rp.jump = g->bc == IBDL_BC_NEUMANN ? -0.5 : 0.5;
  rp.aug = g->naug > 0;
  rp.eta = g->eta;
  rp.hd = g->h * g->h;
  rp.eta_src = PT(g->naug ? (g->pde == IBDL_PDE_STOKES ? g->eta / g->mu : g->eta) : 0.0);
  return rp;
}

template <typename T>
static ColParams<T> col_params(Geometry* g, const int* stop) {
  const int pi = Slot2<T>::pi;
  ColParams<T> cp;
  cp.n = g->n;
  cp.log2n = log2i(g->n);
  cp.C = g->cols_per_cta[pi];
  cp.R = g->rows_per_cta[pi];
  cp.lam = T(g->lambda);
  cp.mu = T(g->mu);
  cp.scale = T(1.0 / ((double)g->n * (double)g->n));
  cp.lap1 = static_cast<const T*>(Slot2<T>::lap(g));
  cp.der1 = static_cast<const T*>(Slot2<T>::der(g));
  cp.spec = reinterpret_cast<cplx<T>*>(g->spec);
  cp.tw = static_cast<const cplx<T>*>(Slot2<T>::tw(g));
  cp.stop = stop;
  cp.err = g->err_dev;
  return cp;
}

// Launch shape of one operator at one precision: threads and shared memory of the three kernels
// for band height R, column group C and the row kernels' least thread count `floor`, or an error
// if they do not fit.
static int row_threads(int nf, int R, int L, bool f32, int floor) {
  const int need = field_groups_2d(nf, L, f32) * (R / 2) * threads_per_seq_2d(L, f32);
  return need > floor ? need : (floor < kMaxThreads2d ? floor : kMaxThreads2d);
}
static int col_threads(int nf, int C, int L, bool f32) {
  return field_groups_2d(nf, L, f32) * C * threads_per_seq_2d(L, f32);
}

template <typename T, int OP>
static ibdl_status launch_shape(const Geometry* g, int R, int C, int floor, Launch2D* lc) {
  // one field per launch: every kernel holds one field
  const bool split = g->split[Slot2<T>::pi] != 0;
  const int NIN = split ? 1 : Traits<OP>::NIN, NOUT = split ? 1 : Traits<OP>::NOUT;
  const int NMAX = NIN > NOUT ? NIN : NOUT;
  const int L = log2i(g->n);
  lc->split = split;
  if (R < 2 || C < 1)
    return fail(IBDL_ERR_UNSUPPORTED, "grid too large for the shared-memory FFT at this precision");
  lc->R = R;
  lc->C = C;
  lc->smem_row = smem_rows_2d<T>(NIN, R, L);
  lc->smem_gather = smem_rows_2d<T>(NOUT, R, L);
  lc->smem_col = smem_cols_2d<T>(NMAX, C, L);
  constexpr bool f32 = sizeof(T) == 4;
  lc->threads_row = row_threads(NIN, R, L, f32, floor);
  lc->threads_gather = row_threads(NOUT, R, L, f32, floor);
  lc->threads_col = col_threads(NMAX, C, L, f32);
  if (lc->smem_row > kSmemLimit2d || lc->smem_gather > kSmemLimit2d || lc->smem_col > kSmemLimit2d)
    return fail(IBDL_ERR_UNSUPPORTED, "grid too large for the shared-memory FFT at this precision");
  if (lc->threads_row > kMaxThreads2d || lc->threads_gather > kMaxThreads2d || lc->threads_col > kMaxThreads2d)
    return fail(IBDL_ERR_UNSUPPORTED, "launch shape exceeds the thread limit");
  return IBDL_OK;
}

// the per-size launch for n = 2^L; float-float exists to 4096² and not for the single layer
template <typename T, int OP, int L>
static ibdl_status launch_for_size(int lg, Geometry* g, const RowParams<T>& rp, const ColParams<T>& cp,
                                   const Launch2D& lc, cudaStream_t s) {
  constexpr bool is_ff = std::is_same<T, ff>::value;
  if constexpr (L > kMaxL2d) {
    return fail(IBDL_ERR_UNSUPPORTED, "2-D grid size outside 16 … 8192");
  } else if constexpr (is_ff && (L > kMaxLff || OP == OP_SL)) {
    return fail(IBDL_ERR_UNSUPPORTED, "float-float applications: grids to 4096², not the single layer");
  } else {
    if (lg == L) return launch_apply_2d<T, OP, L>(g, rp, cp, lc, s);
    return launch_for_size<T, OP, L + 1>(lg, g, rp, cp, lc, s);
  }
}

// run_op mode bits: RUN_LAPLACE solves the plain Laplace problem (λ → 0) without the completed
// method's terms; RUN_NO_AUG only drops those terms
enum { RUN_LAPLACE = 1, RUN_NO_AUG = 2 };

template <typename T, int OP>
static ibdl_status run_op(Geometry* g, const double* in, double* out, cudaStream_t s, const int* stop,
                          double* grid, const int* idx = nullptr, int vstride = 0, int trans = 0,
                          const double* grid_in = nullptr, int mode = 0) {
  const int pi = Slot2<T>::pi;
  if (pi == 2 && !g->twff) return fail(IBDL_ERR_UNSUPPORTED, "this geometry has no float-float tables");
  Launch2D lc;
  IBDL_TRY((launch_shape<T, OP>(g, g->rows_per_cta[pi], g->cols_per_cta[pi], g->threads[pi], &lc)));
  lc.pdl = !g->timing;
  lc.grid_mode = grid ? G_GRID : G_INTERP;
  RowParams<T> rp = row_params<T>(g, in, out, stop, grid);
  rp.idx = idx;
  rp.vstride = vstride;
  rp.trans = trans;
  rp.grid_in = grid_in;
  if (OP == OP_SL) rp.jump = 0.0;
  if (OP != OP_SCALAR_AN && OP != OP_STOKES_AN) {  // the completed method exists for these two only
    rp.aug = 0;
    rp.eta_src = 0;
  }
  ColParams<T> cp = col_params<T>(g, stop);
  if (mode & RUN_LAPLACE) cp.lam = T(0);  // the plain Laplace problem (indicator)
  if (mode & (RUN_LAPLACE | RUN_NO_AUG)) {  // no completed-method terms
    rp.aug = 0;
    rp.eta_src = 0;
  }
  return launch_for_size<T, OP, kMinL2d>(log2i(g->n), g, rp, cp, lc, s);
}

template <typename T>
static ibdl_status apply_t(Geometry* g, const double* Q, double* Y, cudaStream_t s, const int* stop, double* grid,
                           const int* idx = nullptr, int vstride = 0, int op = OPK_A) {
  if (op == OPK_AT) {
    if (g->pde == IBDL_PDE_STOKES) {
      if (g->dipole != IBDL_DIPOLE_ANALYTIC)
        return fail(IBDL_ERR_UNSUPPORTED, "Stokes transpose: analytic dipole only");
      return run_op<T, OP_STOKES_T>(g, Q, Y, s, stop, grid, idx, vstride);
    }
    return g->dipole == IBDL_DIPOLE_ANALYTIC ? run_op<T, OP_ADJ_AN>(g, Q, Y, s, stop, grid, idx, vstride, 1)
                                             : run_op<T, OP_ADJ_SD>(g, Q, Y, s, stop, grid, idx, vstride, 1);
  }
  if (g->pde == IBDL_PDE_STOKES)
    return g->dipole == IBDL_DIPOLE_ANALYTIC ? run_op<T, OP_STOKES_AN>(g, Q, Y, s, stop, grid, idx, vstride)
                                             : run_op<T, OP_STOKES_SD>(g, Q, Y, s, stop, grid, idx, vstride);
  return g->dipole == IBDL_DIPOLE_ANALYTIC ? run_op<T, OP_SCALAR_AN>(g, Q, Y, s, stop, grid, idx, vstride)
                                           : run_op<T, OP_SCALAR_SD>(g, Q, Y, s, stop, grid, idx, vstride);
}

// Y = A Q with Q = V + (*idx)·nd and Y = V + (*idx + 1)·nd read on the device (Krylov basis)
ibdl_status apply_2d_indexed(Geometry* g, int precision, double* V, const int* idx, int nd, cudaStream_t s,
                             const int* stop, int op) {
  if (precision == IBDL_FP32X2) return apply_t<ff>(g, V, V, s, stop, nullptr, idx, nd, op);
  return precision == IBDL_FP32 ? apply_t<float>(g, V, V, s, stop, nullptr, idx, nd, op)
                                : apply_t<double>(g, V, V, s, stop, nullptr, idx, nd, op);
}

ibdl_status apply_2d(Geometry* g, int precision, const double* Q, double* Y, cudaStream_t s, const int* stop,
                     int op) {
  IBDL_TRY(take_device_error(g));  // a failure of an earlier, completed application
  if (precision == IBDL_FP32X2) return apply_t<ff>(g, Q, Y, s, stop, nullptr, nullptr, 0, op);
  return precision == IBDL_FP32 ? apply_t<float>(g, Q, Y, s, stop, nullptr, nullptr, 0, op)
                                : apply_t<double>(g, Q, Y, s, stop, nullptr, nullptr, 0, op);
}

// u = K[sources(Q)] (the forward op's grid field: c fields) and v = Kᵀψ, ψ_l = Σ_j λ_{l,j} Φ(x − X_j)
// (the transpose op's grid field: 1 field scalar, v_s and v_g Stokes), FP64 on [·][n][n]
ibdl_status field_pair_2d(Geometry* g, const double* Q, const double* lam, double* u, double* v, cudaStream_t s) {
  IBDL_TRY(apply_t<double>(g, Q, g->tmp_m, s, nullptr, u));
  return apply_t<double>(g, lam, g->tmp_m, s, nullptr, v, nullptr, 0, OPK_AT);
}

// Z = S*(−L⁻¹)(S V) (scalar PDE)
ibdl_status single_layer_2d(Geometry* g, int precision, const double* V, double* Z, cudaStream_t s) {
  if (g->pde != IBDL_PDE_SCALAR) return fail(IBDL_ERR_UNSUPPORTED, "single layer: scalar PDE only");
  if (precision == IBDL_FP32X2) return fail(IBDL_ERR_UNSUPPORTED, "single layer: FP64 or FP32");
  return precision == IBDL_FP32 ? run_op<float, OP_SL>(g, V, Z, s, nullptr, nullptr)
                                : run_op<double, OP_SL>(g, V, Z, s, nullptr, nullptr);
}

// v = Kᵀψ for a grid field ψ ([c][n][n]): the transpose op's Fourier stage with its row bands read
// from ψ instead of spread from the boundary
ibdl_status transform_T_2d(Geometry* g, const double* psi, double* v, cudaStream_t s) {
  if (g->dipole != IBDL_DIPOLE_ANALYTIC) return fail(IBDL_ERR_UNSUPPORTED, "analytic dipole only");
  if (g->pde == IBDL_PDE_STOKES)
    return run_op<double, OP_STOKES_T>(g, nullptr, nullptr, s, nullptr, v, nullptr, 0, 0, psi);
  return run_op<double, OP_ADJ_AN>(g, nullptr, nullptr, s, nullptr, v, nullptr, 0, 1, psi);
}

// u = −Δ₀⁻¹S̃Q (mean-zero) with the geometry's δ_h, dipole spread and symbol, whatever its PDE
ibdl_status laplace_field_2d(Geometry* g, const double* Q, double* u, cudaStream_t s) {
  return g->dipole == IBDL_DIPOLE_ANALYTIC
             ? run_op<double, OP_SCALAR_AN>(g, Q, g->tmp_m, s, nullptr, u, nullptr, 0, 0, nullptr, RUN_LAPLACE)
             : run_op<double, OP_SCALAR_SD>(g, Q, g->tmp_m, s, nullptr, u, nullptr, 0, 0, nullptr, RUN_LAPLACE);
}

// grid-input fields of the source term for the forward op's Fourier stage: scalar −g̃ (the op's
// symbol is that of −L⁻¹); Stokes (s, f_x, f_y) = (0, −g̃_x/μ, −g̃_y/μ) in the slots of the dipole
// source ∇·(SA), whose velocity P̂f̂/|k|² (Brinkman μP̂f̂/(μ|k|² + λ)) is then −P̂ĝ/(μ|k|² + λ)
__global__ void k_source_fields(const double* __restrict__ gsrc, int stokes, double inv_mu, int64_t cells,
                                double* __restrict__ f) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cells; i += (int64_t)gridDim.x * blockDim.x) {
    if (stokes) {
      f[i] = 0.0;
      f[cells + i] = -gsrc[i] * inv_mu;
      f[2 * cells + i] = -gsrc[cells + i] * inv_mu;
    } else {
      f[i] = -gsrc[i];
    }
  }
}

// rows[i] −= w[i] over the c·M boundary rows; with sums (completed method) rows[c·M + l] = hd·sums[l]
__global__ void k_source_rows(double* __restrict__ rows, const double* __restrict__ w, int cm, int naug,
                              const double* __restrict__ sums, double hd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cm) rows[i] -= w[i];
  if (sums && i < naug) rows[cm + i] = hd * sums[i];
}

// sums[l] = Σ_g g̃_l, one block per component (fixed order, deterministic)
__global__ void __launch_bounds__(1024) k_grid_sums(const double* __restrict__ gsrc, int64_t cells, double* sums) {
  __shared__ double red[32];
  const double* f = gsrc + (int64_t)blockIdx.x * cells;
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < cells; i += blockDim.x) a += f[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) sums[blockIdx.x] = t;
  }
}

__global__ void k_add(double* __restrict__ y, const double* __restrict__ x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}

ibdl_status source_terms_2d(Geometry* g, const double* gsrc, double* rhs, double* grid, cudaStream_t s) {
  const bool stokes = g->pde == IBDL_PDE_STOKES;
  const int nf = stokes ? 3 : 1, c = g->ncomp;
  const int64_t cells = (int64_t)g->n * g->n;
  const int cm = c * (int)g->M;
  // fields [nf][n][n] | u_g [c][n][n] | S*u_g [c·M] | sums [c]
  if (!g->src_buf)
    IBDL_CUDA(cudaMalloc((void**)&g->src_buf, sizeof(double) * ((nf + c) * cells + cm + c)));
  double* f = g->src_buf;
  double* ug = f + nf * cells;
  double* w = ug + c * cells;
  double* sums = w + cm;
  const int blocks = (int)std::min<int64_t>((cells + 255) / 256, 152 * 8);
  k_source_fields<<<blocks, 256, 0, s>>>(gsrc, stokes ? 1 : 0, 1.0 / g->mu, cells, f);
  IBDL_CUDA(cudaGetLastError());
  g->launches += 1;
  if (rhs) {
    IBDL_CUDA(cudaMemsetAsync(w, 0, sizeof(double) * cm, s));
    IBDL_TRY((stokes ? run_op<double, OP_STOKES_AN>(g, nullptr, w, s, nullptr, nullptr, nullptr, 0, 0, f, RUN_NO_AUG)
                     : run_op<double, OP_SCALAR_AN>(g, nullptr, w, s, nullptr, nullptr, nullptr, 0, 0, f, RUN_NO_AUG)));
    if (g->naug) {
      k_grid_sums<<<c, 1024, 0, s>>>(gsrc, cells, sums);
      g->launches += 1;
    }
    k_source_rows<<<(cm + 255) / 256, 256, 0, s>>>(rhs, w, cm, g->naug, g->naug ? sums : nullptr, g->h * g->h);
    IBDL_CUDA(cudaGetLastError());
    g->launches += 1;
  }
  if (grid) {
    IBDL_TRY((stokes ? run_op<double, OP_STOKES_AN>(g, nullptr, w, s, nullptr, ug, nullptr, 0, 0, f, RUN_NO_AUG)
                     : run_op<double, OP_SCALAR_AN>(g, nullptr, w, s, nullptr, ug, nullptr, 0, 0, f, RUN_NO_AUG)));
    k_add<<<blocks, 256, 0, s>>>(grid, ug, c * cells);
    IBDL_CUDA(cudaGetLastError());
    g->launches += 1;
  }
  return IBDL_OK;
}

ibdl_status field_2d(Geometry* g, const double* Q, double* u, cudaStream_t s) {
  return apply_t<double>(g, Q, g->tmp_m, s, nullptr, u);
}

ibdl_status adjoint_2d(Geometry* g, int precision, const double* W, double* Z, cudaStream_t s) {
  if (g->pde != IBDL_PDE_SCALAR) return fail(IBDL_ERR_UNSUPPORTED, "adjoint: scalar PDE only");
  if (precision == IBDL_FP32)
    return g->dipole == IBDL_DIPOLE_ANALYTIC ? run_op<float, OP_ADJ_AN>(g, W, Z, s, nullptr, nullptr)
                                             : run_op<float, OP_ADJ_SD>(g, W, Z, s, nullptr, nullptr);
  return g->dipole == IBDL_DIPOLE_ANALYTIC ? run_op<double, OP_ADJ_AN>(g, W, Z, s, nullptr, nullptr)
                                           : run_op<double, OP_ADJ_SD>(g, W, Z, s, nullptr, nullptr);
}

// ------------------------------------------------------------------------------------------
// batched launches: one grid per stage covers every problem of a batch (kernels and launches in
// apply2d_batch_*.cu); here the per-problem parameter blocks and (problem, unit) tables
// ------------------------------------------------------------------------------------------
// a batched stage for the problems of size 2^L (those that exist for this type)
template <typename T, int OP, int L>
static ibdl_status batch_stage_for_size(int lg, Batch* B, int stage, int mode, const double* in_base, double* out_base,
                                        cudaStream_t s, bool pdl) {
  constexpr bool is_ff = std::is_same<T, ff>::value;
  if constexpr (L > (is_ff ? kMaxLff : kMaxL2d)) {
    return fail(IBDL_ERR_UNSUPPORTED, "batched float-float applications: grids to 4096²");
  } else {
    if (lg == L) return batch_stage_2d<T, OP, L>(B, stage, mode, in_base, out_base, s, pdl);
    return batch_stage_for_size<T, OP, L + 1>(lg, B, stage, mode, in_base, out_base, s, pdl);
  }
}

// One batched application: for each grid size present, its three stages, one launch each (a
// launch waits, by programmatic launch, for the launch before it; only the first launch of the
// application is an ordinary stream-ordered launch). The sizes are independent, so they run one
// after another: a size's spectra are then read back by its column pass and gather while they
// are still in L2, instead of after every other size's spread has written its own.
template <typename T, int OP>
static ibdl_status batch_launch_2d(Batch* B, int mode, const double* in_base, double* out_base, cudaStream_t s) {
  const int pi = Slot2<T>::pi;
  bool first = true;
  for (int L = kMinL2d; L <= kMaxL2d; ++L)
    for (int stage = 0; stage < 3; ++stage) {
      if (B->lv[pi][L].row_count == 0) continue;
      IBDL_TRY((batch_stage_for_size<T, OP, kMinL2d>(L, B, stage, mode, in_base, out_base, s, !first)));
      first = false;
    }
  IBDL_CUDA(cudaGetLastError());
  return IBDL_OK;
}

template <typename T>
static ibdl_status batch_apply_t(Batch* B, int mode, const double* in_base, double* out_base, cudaStream_t s) {
  if (B->pde == IBDL_PDE_STOKES)
    return B->dipole == IBDL_DIPOLE_ANALYTIC ? batch_launch_2d<T, OP_STOKES_AN>(B, mode, in_base, out_base, s)
                                             : batch_launch_2d<T, OP_STOKES_SD>(B, mode, in_base, out_base, s);
  return B->dipole == IBDL_DIPOLE_ANALYTIC ? batch_launch_2d<T, OP_SCALAR_AN>(B, mode, in_base, out_base, s)
                                           : batch_launch_2d<T, OP_SCALAR_SD>(B, mode, in_base, out_base, s);
}

ibdl_status batch_apply_2d(Batch* B, int precision, int mode, const double* in_base, double* out_base, cudaStream_t s) {
  if (precision == IBDL_FP32X2) {
    if (B->max_log2n > kMaxLff) return fail(IBDL_ERR_UNSUPPORTED, "batched float-float applications: grids to 4096²");
    return batch_apply_t<ff>(B, mode, in_base, out_base, s);
  }
  return precision == IBDL_FP32 ? batch_apply_t<float>(B, mode, in_base, out_base, s)
                                : batch_apply_t<double>(B, mode, in_base, out_base, s);
}

template <typename T, int OP>
static ibdl_status batch_shape(Batch* B, Geometry* g, int pi) {
  if (g->split[pi]) return fail(IBDL_ERR_UNSUPPORTED, "batched launches hold every field of a band at once");
  Launch2D lc;
  IBDL_TRY((launch_shape<T, OP>(g, g->rows_per_cta[pi], g->cols_per_cta[pi], g->threads[pi], &lc)));
  BatchSize& z = B->lv[pi][log2i(g->n)];
  z.smem_row = std::max(z.smem_row, lc.smem_row);
  z.smem_col = std::max(z.smem_col, lc.smem_col);
  z.smem_gather = std::max(z.smem_gather, lc.smem_gather);
  z.threads_row = std::max(z.threads_row, lc.threads_row);
  z.threads_col = std::max(z.threads_col, lc.threads_col);
  z.threads_gather = std::max(z.threads_gather, lc.threads_gather);
  return IBDL_OK;
}

template <typename T>
static ibdl_status batch_shape_any(Batch* B, Geometry* g, int pi) {
  if (B->pde == IBDL_PDE_STOKES)
    return B->dipole == IBDL_DIPOLE_ANALYTIC ? batch_shape<T, OP_STOKES_AN>(B, g, pi) : batch_shape<T, OP_STOKES_SD>(B, g, pi);
  return B->dipole == IBDL_DIPOLE_ANALYTIC ? batch_shape<T, OP_SCALAR_AN>(B, g, pi) : batch_shape<T, OP_SCALAR_SD>(B, g, pi);
}

// The staged FP32 column pass of a batch: per grid size whose problems share one column group
// (the kernel keeps a lane's twiddles across its units), the stage shape; per problem its tensor
// map. Sizes with mixed column groups, or whose group does not fit, keep the direct pass.
template <int OP>
static void batch_staged_shapes(Batch* B) {
  constexpr int NIN = Traits<OP>::NIN, NOUT = Traits<OP>::NOUT, NMAX = NIN > NOUT ? NIN : NOUT;
  for (int L = kMinL2d; L <= kMaxL2d; ++L) {
    BatchSize& z = B->lv[1][L];
    z.col_staged = 0;
    if (!B->col_stage || z.col_count == 0) continue;
    int C = -1, R = 0;
    bool same = true;
    for (int b = 0; b < B->count; ++b) {
      const Geometry* g = B->geoms[b];
      if (log2i(g->n) != L) continue;
      if (C < 0) C = g->cols_per_cta[1];
      same = same && g->cols_per_cta[1] == C;
      R = std::max(R, g->rows_per_cta[1]);
    }
    ColStageShape sh;
    // (every R of the size must fit the box: the largest one decides)
    if (!same || !col_stage_shape(NIN, NMAX, C, R, L, col_stages_env(), &sh)) continue;
    z.col_staged = 1;
    z.stages = sh.stages;
    z.stage_bytes = sh.stage_bytes;
    z.smem_staged = sh.smem;
  }
}

static ibdl_status batch_prepare_staged(Batch* B) {
  if (B->tmaps) cudaFree(B->tmaps);
  B->tmaps = nullptr;
  if (B->pde == IBDL_PDE_STOKES)
    B->dipole == IBDL_DIPOLE_ANALYTIC ? batch_staged_shapes<OP_STOKES_AN>(B) : batch_staged_shapes<OP_STOKES_SD>(B);
  else
    B->dipole == IBDL_DIPOLE_ANALYTIC ? batch_staged_shapes<OP_SCALAR_AN>(B) : batch_staged_shapes<OP_SCALAR_SD>(B);
  bool any = false;
  for (int L = kMinL2d; L <= kMaxL2d; ++L) any = any || B->lv[1][L].col_staged;
  if (!any) return IBDL_OK;
  std::vector<CUtensorMap> maps(B->count);
  std::memset(maps.data(), 0, sizeof(CUtensorMap) * maps.size());
  for (int b = 0; b < B->count; ++b) {
    Geometry* g = B->geoms[b];
    if (!B->lv[1][log2i(g->n)].col_staged) continue;
    IBDL_TRY(encode_col_map(g->spec, g->n, g->rows_per_cta[1], g->cols_per_cta[1], spec_fields_fp32(g), &maps[b]));
  }
  IBDL_CUDA(cudaMalloc((void**)&B->tmaps, sizeof(CUtensorMap) * B->count));
  IBDL_CUDA(cudaMemcpy(B->tmaps, maps.data(), sizeof(CUtensorMap) * B->count, cudaMemcpyHostToDevice));
  return IBDL_OK;
}

template <typename T>
static ibdl_status batch_prepare_t(Batch* B, const int* kptr /* device &st[b].k, stride in bytes */, size_t kstride) {
  const int pi = Slot2<T>::pi;
  std::vector<RowParams<T>> user(B->count), kry(B->count);
  std::vector<ColParams<T>> col(B->count);
  std::vector<int2> ru, cu;
  for (int L = 0; L < 14; ++L) B->lv[pi][L] = BatchSize{};
  // float-float batches exist to 4096²: larger ones keep empty tables (their residuals use FP64)
  if (std::is_same<T, ff>::value && B->max_log2n > kMaxLff) {
    B->nrow_units[pi] = B->ncol_units[pi] = 0;
    return IBDL_OK;
  }
  for (int b = 0; b < B->count; ++b) {
    Geometry* g = B->geoms[b];
    if (batch_shape_any<T>(B, g, pi) != IBDL_OK)
      return fail(IBDL_ERR_UNSUPPORTED, "problem " + std::to_string(b) + ": its grid is too large for a batched launch");
    user[b] = row_params<T>(g, nullptr, nullptr, nullptr, nullptr);
    user[b].io_off = B->off[b];
    kry[b] = user[b];
    col[b] = col_params<T>(g, nullptr);
    if (kptr) {
      const int* kb = reinterpret_cast<const int*>(reinterpret_cast<const char*>(kptr) + kstride * b);
      kry[b].idx = kb;                               // &st[b].k
      kry[b].stop = kb - 2;                          // &st[b].stop (two ints before k)
      kry[b].vstride = (int)(g->ncomp * g->M);
      kry[b].io_off = B->voff[b];
    }
  }
  // unit tables grouped by grid size (one launch per size and stage)
  for (int L = kMinL2d; L <= kMaxL2d; ++L) {
    BatchSize& z = B->lv[pi][L];
    z.row_start = (int)ru.size();
    z.col_start = (int)cu.size();
    for (int b = 0; b < B->count; ++b) {
      Geometry* g = B->geoms[b];
      if (log2i(g->n) != L) continue;
      for (int u = 0; u < g->n / g->rows_per_cta[pi]; ++u) ru.push_back(make_int2(b, u));
      for (int u = 0; u < (g->n / 2) / g->cols_per_cta[pi]; ++u) cu.push_back(make_int2(b, u));
    }
    z.row_count = (int)ru.size() - z.row_start;
    z.col_count = (int)cu.size() - z.col_start;
  }
  auto upload = [&](void** dst, const void* src, size_t bytes) -> ibdl_status {
    if (*dst) cudaFree(*dst);
    *dst = nullptr;
    IBDL_CUDA(cudaMalloc(dst, bytes));
    IBDL_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    return IBDL_OK;
  };
  IBDL_TRY(upload(&B->rowp[pi][0], user.data(), sizeof(RowParams<T>) * B->count));
  IBDL_TRY(upload(&B->rowp[pi][1], kry.data(), sizeof(RowParams<T>) * B->count));
  IBDL_TRY(upload(&B->colp[pi], col.data(), sizeof(ColParams<T>) * B->count));
  IBDL_TRY(upload(reinterpret_cast<void**>(&B->row_units[pi]), ru.data(), sizeof(int2) * ru.size()));
  IBDL_TRY(upload(reinterpret_cast<void**>(&B->col_units[pi]), cu.data(), sizeof(int2) * cu.size()));
  B->nrow_units[pi] = (int)ru.size();
  B->ncol_units[pi] = (int)cu.size();
  if constexpr (std::is_same<T, float>::value) IBDL_TRY(batch_prepare_staged(B));
  return IBDL_OK;
}

// Parameter blocks and unit tables of both precisions; the Krylov-basis mode points at the
// batched GMRES state when it exists (B->st), else mirrors the user mode.
ibdl_status batch_prepare_2d(Batch* B) {
  const int* kptr = nullptr;
  size_t kstride = 0;
  if (B->st) {
    kptr = reinterpret_cast<const int*>(static_cast<const char*>(B->st) + 2 * sizeof(int));
    kstride = batch_state_bytes();
  }
  IBDL_TRY(batch_prepare_t<double>(B, kptr, kstride));
  IBDL_TRY(batch_prepare_t<float>(B, kptr, kstride));
  IBDL_TRY(batch_prepare_t<ff>(B, kptr, kstride));
  return IBDL_OK;
}

// ------------------------------------------------------------------------------------------
// launch shapes. A row kernel's CTA has (R/2)·QT threads and a column kernel's C·QT, with
// QT = n/8 threads per transform (n/16 at n = 8192); both hold one padded sequence of n + n/8
// complex values per field and row pair (column) in shared memory.
// ------------------------------------------------------------------------------------------
static int nf_row_max(const Geometry* g) { return g->nf_in > g->nf_out ? g->nf_in : g->nf_out; }

// largest power of two in [lo, hi] not above v (lo if none)
static int pow2_in(int v, int lo, int hi) {
  int r = lo;
  while (r * 2 <= hi && r * 2 <= v) r *= 2;
  return r;
}

// fields a row band or column group holds at once
static int nf_held(const Geometry* g, int pi) { return g->split[pi] ? 1 : nf_row_max(g); }

static bool row_fits(const Geometry* g, int pi, int R) {
  const int L = log2i(g->n), nf = nf_held(g, pi);
  const size_t bytes = pi == 1 ? smem_rows_2d<float>(nf, R, L) : smem_rows_2d<double>(nf, R, L);
  // R ≤ n/8 (the column pass's lanes then address their rows with one stride per band)
  return R >= 2 && R <= std::max(2, g->n / 8) && bytes <= kSmemLimit2d &&
         row_threads(nf, R, L, pi == 1, 0) <= kMaxThreads2d;
}
static bool col_fits(const Geometry* g, int pi, int C) {
  const int L = log2i(g->n), nf = nf_held(g, pi);
  const size_t bytes = pi == 1 ? smem_cols_2d<float>(nf, C, L) : smem_cols_2d<double>(nf, C, L);
  return C >= 1 && C <= g->n / 2 && bytes <= kSmemLimit2d && col_threads(nf, C, L, pi == 1) <= kMaxThreads2d;
}

// ------------------------------------------------------------------------------------------
// autotuner: time candidate launch shapes of the 2-D application on a geometry's own data and
// keep the fastest; results are cached per (n, fields in, fields out, pde, dipole, precision)
// so geometries created later with the same key start from the tuned shape
// ------------------------------------------------------------------------------------------
struct TuneKey {
  int n, nf_in, nf_out, pde, dipole, pi, split;
  bool operator==(const TuneKey& o) const {
    return n == o.n && nf_in == o.nf_in && nf_out == o.nf_out && pde == o.pde && dipole == o.dipole && pi == o.pi &&
           split == o.split;
  }
};
struct TuneVal {
  int R, C, floor;
  int staged;  // FP32: the staged column pass (1) or the direct one (0)
};
static std::vector<std::pair<TuneKey, TuneVal>> g_tuned;
static std::mutex g_tune_mu;

static bool tuned_lookup(const TuneKey& k, TuneVal* v) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (auto& e : g_tuned)
    if (e.first == k) {
      *v = e.second;
      return true;
    }
  return false;
}

static void tuned_store(const TuneKey& k, const TuneVal& v) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (auto& e : g_tuned)
    if (e.first == k) {
      e.second = v;
      return;
    }
  g_tuned.push_back({k, v});
}

static TuneKey tune_key(const Geometry* g, int pi) {
  return {g->n, g->nf_in, g->nf_out, g->pde, g->dipole, pi, g->split[pi]};
}

// The row kernels' shape (band height R ∈ {2 … 64} and least thread count ∈ {0, 256, 512}) is
// tuned first with the column group fixed, then the column group C ∈ {1 … 32}: the kernels are
// independent, so the two sweeps find the best pair. Candidates must fit shared memory and 512
// threads per CTA; each is timed on back-to-back applications (below) after one warm-up.
ibdl_status autotune_2d(Geometry* g, int pi, bool /*fixed_threads*/, cudaStream_t s, const double* Q, double* Y) {
  const int saved_timing = g->timing;
  g->timing = 0;
  cudaEvent_t e0, e1;
  IBDL_CUDA(cudaEventCreate(&e0));
  IBDL_CUDA(cudaEventCreate(&e1));
  ibdl_status err = IBDL_OK;
  auto time_shape = [&](int R, int C, int floor, float* med) -> ibdl_status {
    g->rows_per_cta[pi] = R;
    g->cols_per_cta[pi] = C;
    g->threads[pi] = floor;
    // applications back to back, as a solve runs them (each launch overlapping its predecessor's
    // tail by programmatic launch): chains of about 1 ms (1 … 8 applications, the length from one
    // timed application), the median of 5 chains per application
    float ms[5], one = 0.f;
    IBDL_TRY(apply_2d(g, slot_precision(pi), Q, Y, s, nullptr));
    cudaEventRecord(e0, s);
    IBDL_TRY(apply_2d(g, slot_precision(pi), Q, Y, s, nullptr));
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return fail(IBDL_ERR_CUDA, "autotune: event synchronize");
    cudaEventElapsedTime(&one, e0, e1);
    const int chain = one > 0.f ? std::max(1, std::min(8, (int)(1.0f / one))) : 8;
    for (int k = 0; k < 5; ++k) {
      cudaEventRecord(e0, s);
      for (int c = 0; c < chain; ++c) IBDL_TRY(apply_2d(g, slot_precision(pi), Q, Y, s, nullptr));
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) return fail(IBDL_ERR_CUDA, "autotune: event synchronize");
      cudaEventElapsedTime(&ms[k], e0, e1);
      ms[k] /= chain;
    }
    std::sort(ms, ms + 5);
    *med = ms[2];
    return IBDL_OK;
  };
  TuneVal best{g->rows_per_cta[pi], g->cols_per_cta[pi], g->threads[pi], g->col_stage};
  float best_ms = 1e30f;
  const int floors[3] = {0, 256, 512};
  for (int R = 2; R <= 64 && err == IBDL_OK; R *= 2) {
    if (!row_fits(g, pi, R)) continue;
    for (int fi = 0; fi < 3 && err == IBDL_OK; ++fi) {
      float ms = 0;
      err = time_shape(R, best.C, floors[fi], &ms);
      if (err == IBDL_OK && ms < best_ms) {
        best_ms = ms;
        best.R = R;
        best.floor = floors[fi];
      }
    }
  }
  // the column group, and for FP32 (unless IBDL_COL_STAGED fixes it) the column pass's form:
  // direct loads or the staged pass
  const int saved_stage = g->col_stage;
  for (int staged = 0; staged < 2 && err == IBDL_OK; ++staged) {
    if (staged && (pi != 1 || g->col_stage_forced)) break;
    if (pi == 1 && !g->col_stage_forced) g->col_stage = staged;
    for (int C = 1; C <= 32 && err == IBDL_OK; C *= 2) {
      if (!col_fits(g, pi, C)) continue;
      float ms = 0;
      err = time_shape(best.R, C, best.floor, &ms);
      if (err == IBDL_OK && ms < best_ms) {
        best_ms = ms;
        best.C = C;
        best.staged = g->col_stage;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g->timing = saved_timing;
  g->rows_per_cta[pi] = best.R;
  g->cols_per_cta[pi] = best.C;
  g->threads[pi] = best.floor;
  g->col_stage = pi == 1 ? best.staged : saved_stage;
  if (err == IBDL_OK) tuned_store(tune_key(g, pi), best);
  return err;
}

// Shapes from the volume rule: about `target` complex elements of FFT per CTA (so about
// target/8 lane-threads), R ≤ n/8, within shared memory and the thread limit; `floor` is the row
// kernels' least thread count.
void shape_for_target_2d(Geometry* g, int pi, int row_target, int col_target, int floor) {
  const int n = g->n;
  int R = 2 * pow2_in(row_target / (n * g->nf_in), 1, n / 4 > 1 ? n / 4 : 1);
  while (R > 2 && !row_fits(g, pi, R)) R /= 2;
  int C = pow2_in(col_target / (n * nf_row_max(g)), 1, n / 2);
  while (C > 1 && !col_fits(g, pi, C)) C /= 2;
  if (row_fits(g, pi, R) && col_fits(g, pi, C)) {
    g->rows_per_cta[pi] = R;
    g->cols_per_cta[pi] = C;
    g->threads[pi] = floor;
  }
}

// Default shapes: about 256 FFT lanes per CTA, but at least 2·152 CTAs per kernel where the grid
// allows (one GB300 has 152 SMs), and at least 256 threads in the row kernels; the autotuner
// refines them. IBDL_PLAN_R and IBDL_PLAN_C override (for tuning experiments).
ibdl_status plan_2d(Geometry* g) {
  const int n = g->n, L = log2i(n);
  const int min_ctas = 2 * 152;
  int tuned_stage = 0;
  const char* se = getenv("IBDL_SPLIT_FIELDS");
  const bool force_split = se && atoi(se) != 0 && nf_row_max(g) > 1;
  for (int pi = 0; pi < 3; ++pi) {
    const int qt = threads_per_seq_2d(L, pi == 1);
    int R = 0, C = 0;
    // all fields of a band or column group at once where they fit shared memory, else one field
    // per launch (multi-field operators only)
    for (int split = force_split ? 1 : 0; split < 2; ++split) {
      if (split && nf_row_max(g) == 1) break;
      g->split[pi] = split;
      R = 2 * pow2_in(256 / qt, 1, n / 4 > 1 ? n / 4 : 1);
      while (R > 2 && (n / R < std::min(min_ctas, n / 2) || !row_fits(g, pi, R))) R /= 2;
      if (!row_fits(g, pi, R)) R = 0;
      C = pow2_in(256 / qt, 1, n / 2);
      while (C > 1 && ((n / 2) / C < std::min(min_ctas, n / 4) || !col_fits(g, pi, C))) C /= 2;
      if (!col_fits(g, pi, C)) C = 0;
      if (R && C) break;
    }
    if (const char* e = getenv("IBDL_PLAN_R")) {
      const int v = atoi(e);
      if ((v & (v - 1)) == 0 && row_fits(g, pi, v)) R = v;
    }
    if (const char* e = getenv("IBDL_PLAN_C")) {
      const int v = atoi(e);
      if (v >= 1 && (v & (v - 1)) == 0 && col_fits(g, pi, v)) C = v;
    }
    if (R == 0 || C == 0) R = C = 0;
    g->rows_per_cta[pi] = R;
    g->cols_per_cta[pi] = C;
    g->threads[pi] = 256;  // the row kernels' loops (clearing, spreading, unpacking) get 256 threads
    TuneVal tv;
    if (R && tuned_lookup(tune_key(g, pi), &tv) && row_fits(g, pi, tv.R) && col_fits(g, pi, tv.C)) {
      g->rows_per_cta[pi] = tv.R;
      g->cols_per_cta[pi] = tv.C;
      g->threads[pi] = tv.floor;
      if (pi == 1) tuned_stage = tv.staged;
    }
  }
  if (const char* e = getenv("IBDL_THREADS")) {
    const int v = atoi(e);
    if (v >= 0 && v <= kMaxThreads2d && v % 32 == 0) g->threads[0] = g->threads[1] = g->threads[2] = v;
  }
  if (g->rows_per_cta[0] == 0 && g->rows_per_cta[1] == 0)
    return fail(IBDL_ERR_UNSUPPORTED, "grid too large for the shared-memory FFT");
  // the FP32 column pass: IBDL_COL_STAGED if set, else the tuned form of this key (direct untuned)
  const int env = col_stage_env();
  g->col_stage_forced = env >= 0;
  g->col_stage = env >= 0 ? env : tuned_stage;
  return IBDL_OK;
}

// ------------------------------------------------------------------------------------------
// tensor maps of the staged column pass
// ------------------------------------------------------------------------------------------
int col_stage_env() {
  const char* e = getenv("IBDL_COL_STAGED");
  if (!e || !*e) return -1;
  return atoi(e) != 0 ? 1 : 0;
}

int spec_fields_fp32(const Geometry* g) {
  return (int)(g->spec_bytes / ((size_t)g->n * (g->n / 2) * sizeof(float2)));
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (the library links no
// driver library)
static PFN_cuTensorMapEncodeTiled_v12000 encode_tiled_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

ibdl_status encode_col_map(void* spec, int n, int R, int C, int nf, CUtensorMap* out) {
  const int nb = n / R;
  if (R < 2 || n % R || C < 1 || 2 * C * R > 256 || nf < 1 || (reinterpret_cast<uintptr_t>(spec) & 15))
    return fail(IBDL_ERR_UNSUPPORTED, "staged column pass: unsupported band height or column group");
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled_fn();
  if (!fn) return fail(IBDL_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const cuuint64_t dims[3] = {(cuuint64_t)R * n, (cuuint64_t)nb, (cuuint64_t)nf};
  const cuuint64_t strides[2] = {(cuuint64_t)R * n * sizeof(float), (cuuint64_t)n * (n / 2) * sizeof(float2)};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * C * R), (cuuint32_t)(nb < 256 ? nb : 256), 1};
  const cuuint32_t estride[3] = {1, 1, 1};
  const CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, spec, dims, strides, box, estride,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(IBDL_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return IBDL_OK;
}

ibdl_status col_stage_map(Geometry* g, int R, int C, const CUtensorMap** out) {
  if (g->tmap_R != R || g->tmap_C != C) {
    IBDL_TRY(encode_col_map(g->spec, g->n, R, C, spec_fields_fp32(g), &g->tmap_col));
    g->tmap_R = R;
    g->tmap_C = C;
  }
  *out = &g->tmap_col;
  return IBDL_OK;
}

}  // namespace ibdl
