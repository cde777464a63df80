// Internal declarations of the IBDL CUDA library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ibdl.h"

namespace ibdl {

// ------------------------------------------------------------------------------------------
// error handling: every failure becomes an ibdl_status plus a thread-local message
// ------------------------------------------------------------------------------------------
void set_error(const std::string& msg);
ibdl_status fail(ibdl_status st, const std::string& msg);
ibdl_status cuda_fail(cudaError_t e, const char* what);

#define IBDL_CUDA(call)                                         \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return ::ibdl::cuda_fail(e_, #call); \
  } while (0)

#define IBDL_TRY(call)                    \
  do {                                    \
    ibdl_status s_ = (call);              \
    if (s_ != IBDL_OK) return s_;         \
  } while (0)

// ------------------------------------------------------------------------------------------
// complex arithmetic
// ------------------------------------------------------------------------------------------
// aligned to its own size, so that a complex FP32 value moves as one 64-bit access and a complex
// FP64 or float-float value as one 128-bit access (every array of them starts on such a boundary)
template <typename T>
struct alignas(2 * sizeof(T)) cplx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cplx<T> mk(T a, T b) {
  cplx<T> c;
  c.x = a;
  c.y = b;
  return c;
}
template <typename T>
__device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ cplx<T> cconj(cplx<T> a) { return mk(a.x, -a.y); }
template <typename T>
__device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) { return mk(a.x * s, a.y * s); }
// multiply by i
template <typename T>
__device__ __forceinline__ cplx<T> cmuli(cplx<T> a) { return mk(-a.y, a.x); }

// ------------------------------------------------------------------------------------------
// geometry: everything an operator application needs, resident on the device
// ------------------------------------------------------------------------------------------
enum { MAX_FIELDS_IN = 4, MAX_FIELDS_OUT = 3 };

// Per-point stencil table in sorted (cell) order, one copy per precision. For axis j the
// four nodes are base[j] + a (mod n), a = 0..3, with kernel weights phi[j][a] = φ(r) and
// dphi[j][a] = φ'(r)/h where r = (x_node − X)/h.
template <typename T>
struct PointTable {
  T* phi;      // [dim][4][M]
  T* dphi;     // [dim][4][M]
  T* wscale;   // [M] Δs_i / h^dim
  T* nrm;      // [dim][M] unit normals
};

struct Geometry {
  // description
  int dim, n, pde, delta, dipole, symbol;
  int bc;          // IBDL_BC_*: the jump term is +½Q (Dirichlet) or −½Q (Neumann)
  double box, h, lambda, mu;
  double eta;      // completed method (> 0): ηSQ joins the sources, and the unknowns gain
  int naug;        // ... naug = ncomp means ū after the density (0 otherwise)
  double origin[3];
  int64_t M;
  int ncomp;       // c: 1 scalar, dim Stokes
  int nf_in;       // grid fields spread per application
  int nf_out;      // grid fields interpolated per application

  // sorted points
  int* perm;       // [M] sorted position -> original index
  int* base;       // [dim][M] base node per axis (sorted order), already wrapped to [0, n)
  int* cell_start; // [ncell + 1], cells = n^(dim-1) rows of constant (y, z) base
  int ncell;
  PointTable<double> t64;
  PointTable<float> t32;
  double* ddphi64; // [dim][4][M] φ''(r)/h² in sorted order (boundary derivatives); may be NULL
  double* X64;     // [dim][M] the caller's coordinates, original order (post-processing)
  void* pp_buf;    // post-processing scratch, allocated on first use
  size_t pp_bytes;

  // workspace: half spectra, packed format (see apply kernels): [nf][rows][n/2] complex
  void* spec;      // sized for nf_in fields in FP64
  size_t spec_bytes;
  double2* tw64;   // [n] e^{-2πi j/n}
  float2* tw32;
  // per-axis Fourier symbols indexed by FFT index j (wavenumber 2π m/box, m = j or j − n):
  // lap = symbol of −∂² along one axis, der = k̃ with ∂ ↦ i k̃ (0 at Nyquist)
  double *lap64, *der64;
  float *lap32, *der32;
  // float-float copies of the twiddles and symbols (2-D): [n] complex pairs and [n] pairs
  void* twff;
  void* lapff;
  void* derff;
  double* ubuf;    // evaluate_field / adjoint helpers: [c][n^dim] FP64
  double* tmp_m;   // [c*M] scratch boundary vector
  double* vjp_buf; // boundary derivatives: grid fields u and v, allocated on first use
  double* src_buf; // source term g̃: grid-input fields, u_g and S*u_g, allocated on first use

  // launch plan (2-D and 3-D)
  // per precision slot (0 = fp64, 1 = fp32, 2 = float-float, 2-D only)
  int rows_per_cta[3];   // band height R for the row kernels
  int cols_per_cta[3];   // kx columns per CTA in the column kernels (3-D: the y passes)
  int zcols_per_cta[3];  // 3-D: kx columns per CTA in the z pass
  size_t smem_row[2], smem_col[2], smem_row_inv[2];
  int threads[3];        // 2-D: least threads per CTA of the row kernels (0: none)
  int split[3];          // 2-D: one field per launch (the fields' row bands or columns do not fit
                         // shared memory together, or IBDL_SPLIT_FIELDS=1)

  // GMRES workspace (allocated lazily, sized for `krylov_m`)
  int krylov_m;
  double* V;       // [(m+1)][c*M]
  double* gm;      // small device state (Hessenberg, Givens, g, status)
  double* vec;     // [4][c*M] work vectors (b, x, r, d)
  void* host_status;   // pinned
  cudaEvent_t ev;

  // captured GMRES cycles (CUDA graph with a device-side while loop), per operator (A, Aᵀ)
  // and precision: index 2·op + (0 fp64, 1 fp32)
  cudaGraphExec_t cycle_exec[4];
  int cycle_m[4];

  // staged column pass of FP32 applications (2-D): on (1) or off (0), whether IBDL_COL_STAGED
  // fixed it (else the autotuner chooses), the tensor map of the FP32 half spectra for the
  // column group it was encoded for, and the flag its bounded waits set (pinned host memory
  // mapped into the device, so the host reads it without a copy)
  int col_stage, col_stage_forced;
  int tmap_R, tmap_C;
  CUtensorMap tmap_col;
  int* err_host;
  int* err_dev;

  // counters and optional stage timing (events around every kernel)
  int64_t launches;
  int timing;
  cudaEvent_t* ev_pool;
  int* ev_stage;   // stage id of the interval that ends at event i (−1: a start marker)
  int ev_cap, ev_used;
};

// Launch shapes of one grid size's batched kernels, and that size's range of the unit tables.
struct BatchSize {
  int row_start, row_count, col_start, col_count;
  int threads_row, threads_col, threads_gather;
  size_t smem_row, smem_col, smem_gather;
  // FP32: the staged column pass (its units all have one column group), stages and stage bytes
  int col_staged, stages, stage_bytes;
  size_t smem_staged;
};

// A batch of independent 2-D problems (same PDE and dipole form; any grid size, point count,
// λ, delta and symbol per problem). Boundary vectors of all problems are concatenated: problem b
// owns [off[b], off[b] + c·M_b).
struct Batch {
  int count;
  int pde, dipole, ncomp;
  Geometry** geoms;      // host array of per-problem geometries (tables, spectra, symbols)
  int64_t* off;          // host [count + 1]
  int64_t total;
  // batched-launch data per precision slot p (0 fp64, 1 fp32, 2 float-float) and mode (0 user
  // buffers, 1 Krylov basis)
  void* rowp[3][2];      // device RowParams<T>[count]
  void* colp[3];         // device ColParams<T>[count]
  int2* row_units[3];    // device (problem, unit) tables
  int2* col_units[3];
  int nrow_units[3], ncol_units[3];
  // per precision slot and grid size 2^L: the problems' unit ranges in the tables (sorted by size)
  // and the launch shapes of that size's batched kernels
  BatchSize lv[3][14];
  int max_log2n;         // log2 of the largest grid size in the batch
  int persistent;        // 1: persistent column-pass CTAs for one-field operators (IBDL_BATCH_PERSISTENT=1)
  int col_stage;         // FP32 column pass: 1 staged (tensor-memory-accelerator copies), 0 direct loads
  int col_stage_forced;  // IBDL_COL_STAGED fixed it (else the batch autotuner chooses)
  CUtensorMap* tmaps;    // device [count]: each problem's FP32 half-spectrum tensor map (staged pass)
  // batched GMRES
  int m;                 // restart length the workspace was sized for (0: none yet)
  int64_t* voff;         // host [count]: offset of problem b's basis in V
  double* V;
  void* st;              // device GmresState[count]
  void* ctl;             // device control block of the batched while loop
  void* host_st;         // pinned copy of the states' status headers (HostStatus per problem)
  double* vec;           // [5][total]: b, x, r, d, scratch
  double* target;        // device [count]
  int* active;           // device [count]
  cudaGraphExec_t exec[2];
  int exec_m[2];
  int64_t launches;
  int cl;                // Arnoldi cluster size
  int64_t* d_off;        // device copies of the per-problem offsets, sizes and slices
  int64_t* d_voff;
  int* d_nd;
  int* d_slice;
};

ibdl_status batch_prepare_2d(Batch* B);
// tensor map of FP32 half spectra [nf][n][n/2] in band-major order for the staged column pass:
// dimensions (R·n floats of a band, n/R bands, nf fields), box (2·C·R, min(n/R, 256), 1)
ibdl_status encode_col_map(void* spec, int n, int R, int C, int nf, CUtensorMap* out);
// the geometry's map for (R, C), re-encoded when either changed
ibdl_status col_stage_map(Geometry* g, int R, int C, const CUtensorMap** out);
// fields of FP32 half spectra a geometry's workspace holds
int spec_fields_fp32(const Geometry* g);
// IBDL_COL_STAGED: unset −1 (not fixed), "0" off, otherwise on
int col_stage_env();
ibdl_status autotune_2d(Geometry* g, int pi, bool fixed_threads, cudaStream_t s, const double* Q, double* Y);
// launch shape from FFT volumes per CTA: rows per band from row_target, kx columns from col_target;
// floor: the row kernels' least thread count
void shape_for_target_2d(Geometry* g, int pi, int row_target, int col_target, int floor);
size_t batch_state_bytes();  // sizeof the per-problem GMRES state (stop, status, k are its first ints)
ibdl_status batch_apply_2d(Batch* B, int precision, int mode, const double* in_base, double* out_base,
                           cudaStream_t s);
ibdl_status batch_solve_impl(Batch* B, const double* Ub, double* Q, const ibdl_solve_opts* o,
                             ibdl_solve_info* infos, cudaStream_t s);

// record an event on `s` closing an interval of `stage` (−1 opens a new interval)
void timing_mark(Geometry* g, cudaStream_t s, int stage);
ibdl_status set_stage_timing(Geometry* g, int enable);
ibdl_status get_stage_times(Geometry* g, double* ms, int64_t* launches);

// precision slot of the per-precision launch plans: 0 FP64, 1 FP32, 2 float-float
inline int prec_slot(int precision) { return precision == IBDL_FP32 ? 1 : (precision == IBDL_FP32X2 ? 2 : 0); }
inline int slot_precision(int slot) { return slot == 1 ? IBDL_FP32 : (slot == 2 ? IBDL_FP32X2 : IBDL_FP64); }

// ------------------------------------------------------------------------------------------
// launchers implemented in the .cu files
// ------------------------------------------------------------------------------------------
// operator selector: A, or its Euclidean transpose Aᵀ = W A* W⁻¹ (W = diag Δs; scalar PDE)
enum { OPK_A = 0, OPK_AT = 1 };

ibdl_status apply_2d(Geometry* g, int precision, const double* Q, double* Y, cudaStream_t s,
                     const int* stop_flag, int op = OPK_A);
ibdl_status apply_3d(Geometry* g, int precision, const double* Q, double* Y, cudaStream_t s,
                     const int* stop_flag, int op = OPK_A);
ibdl_status field_2d(Geometry* g, const double* Q, double* u, cudaStream_t s);
ibdl_status field_3d(Geometry* g, const double* Q, double* u, cudaStream_t s);
ibdl_status adjoint_2d(Geometry* g, int precision, const double* W, double* Z, cudaStream_t s);
ibdl_status adjoint_3d(Geometry* g, int precision, const double* W, double* Z, cudaStream_t s);
ibdl_status plan_2d(Geometry* g);
ibdl_status plan_3d(Geometry* g);
ibdl_status solve_impl(Geometry* g, const double* Ub, double* Q, const ibdl_solve_opts* o,
                       ibdl_solve_info* info, cudaStream_t s, int op = OPK_A, const double* gsrc = nullptr);
// grid fields u = K[sources(Q)] and v = Kᵀ(Σ_j λ_j Φ(x − X_j)) (K = −L⁻¹ scalar, the Stokes
// multiplier otherwise), then the boundary derivatives; Kᵀ of a given grid field (2-D)
ibdl_status transform_T_2d(Geometry* g, const double* psi, double* v, cudaStream_t s);
ibdl_status single_layer_2d(Geometry* g, int precision, const double* V, double* Z, cudaStream_t s);
ibdl_status field_pair_2d(Geometry* g, const double* Q, const double* lam, double* u, double* v, cudaStream_t s);
// the source term g̃ (2-D): rhs[0..c·M) −= S*u_g and, for the completed method, rhs[c·M + l] =
// h^d Σ g̃_l (rhs may be NULL); grid[c][n][n] += u_g (grid may be NULL)
ibdl_status source_terms_2d(Geometry* g, const double* gsrc, double* rhs, double* grid, cudaStream_t s);
ibdl_status source_terms_3d(Geometry* g, const double* gsrc, double* rhs, double* grid, cudaStream_t s);
inline ibdl_status source_terms(Geometry* g, const double* gsrc, double* rhs, double* grid, cudaStream_t s) {
  return g->dim == 2 ? source_terms_2d(g, gsrc, rhs, grid, s) : source_terms_3d(g, gsrc, rhs, grid, s);
}
ibdl_status laplace_field_2d(Geometry* g, const double* Q, double* u, cudaStream_t s);
ibdl_status laplace_field_3d(Geometry* g, const double* Q, double* u, cudaStream_t s);
ibdl_status indicator_impl(Geometry* g, double* chi, uint8_t* flags, cudaStream_t s);
ibdl_status near_boundary_impl(Geometry* g, const double* Ub, const double* u, const uint8_t* omega, double m1,
                               double m2, double* out, cudaStream_t s);
ibdl_status field_pair_3d(Geometry* g, const double* Q, const double* lam, double* u, double* v, cudaStream_t s);
ibdl_status solve_vjp_impl(Geometry* g, const double* Q, const double* lam, double* dX, double* dn, double* dw,
                           cudaStream_t s);
ibdl_status probe_evaluate_impl(Geometry* g, const double* P, int np, const double* Q, double* U, cudaStream_t s);
ibdl_status probe_vjp_impl(Geometry* g, const double* P, int np, const double* Q, const double* nu, double* dQ,
                           double* dX, double* dn, double* dw, cudaStream_t s);

ibdl_status apply_2d_indexed(Geometry* g, int precision, double* V, const int* idx, int nd, cudaStream_t s,
                             const int* stop, int op = OPK_A);
ibdl_status apply_3d_indexed(Geometry* g, int precision, double* V, const int* idx, int nd, cudaStream_t s,
                             const int* stop, int op = OPK_A);

// IBDL_ERR_TIMEOUT (and the flag cleared) if a staged column pass of this geometry gave up waiting
// for its copies since the last check; the flag lives in mapped host memory, so no copy is needed
inline ibdl_status take_device_error(Geometry* g) {
  if (g->err_host && *reinterpret_cast<volatile int*>(g->err_host)) {
    *reinterpret_cast<volatile int*>(g->err_host) = 0;
    return fail(IBDL_ERR_TIMEOUT, "a staged column pass gave up waiting for its shared-memory copies");
  }
  return IBDL_OK;
}

// length of a boundary vector of the (possibly augmented) system: c·M density values, then ū
inline int geom_nd(const Geometry* g) { return (int)(g->ncomp * g->M) + g->naug; }

inline ibdl_status apply_any(Geometry* g, int precision, const double* Q, double* Y,
                             cudaStream_t s, const int* stop_flag, int op = OPK_A) {
  return g->dim == 2 ? apply_2d(g, precision, Q, Y, s, stop_flag, op)
                     : apply_3d(g, precision, Q, Y, s, stop_flag, op);
}

}  // namespace ibdl
