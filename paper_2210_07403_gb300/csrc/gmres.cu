// GMRES for A Q = U_b (Sec. 5.3.2: the Schur operator is not symmetric) on the device.
//
// Arnoldi runs on one 16-CTA cluster per iteration (8 where 16 is unavailable; arnoldi.cuh):
// classical Gram–Schmidt against the basis in FP64 with one cluster reduction per step (the
// second projection of CGS2 is taken from the basis' Gram matrix, h = (2I − G)t), the new
// Hessenberg column is reduced by the stored Givens rotations, and the residual estimate |g_{k}|
// is compared with the target on the device. When the target is met (or the cycle is full, or a non-finite
// value appears) the step raises a stop flag that every kernel of the following iterations reads
// first.
//
// A restart cycle is one CUDA graph: a conditional while node whose body is one operator
// application and one Arnoldi step; the Arnoldi step sets the loop condition, so the host waits
// once per cycle. With stage timing on, the cycle is instead driven from the host (one launch
// per kernel, the host queuing iteration j+1 before it reads iteration j's status).
//
// Mixed precision: iterative refinement. Each sweep solves A₃₂ d = r with FP32 grid arithmetic
// and the same FP64 Arnoldi/Hessenberg, then forms the residual r = U_b − A Q with an application
// in float-float (default) or FP64 arithmetic and the subtraction and norm in FP64.
#include <cooperative_groups.h>

#include <chrono>
#include <cstddef>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <algorithm>
#include <vector>

#include "arnoldi.cuh"
#include "ibdl_internal.cuh"

namespace ibdl {

// block-wide sum; every thread gets the result
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = threadIdx.x < (unsigned)nw ? red[threadIdx.x] : 0.0;
  if (warp == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  const double r = red[0];
  __syncthreads();
  return r;
}

// y = R⁻¹ g for the k × k upper-triangular R of the rotated Hessenberg matrix (k ≤ 64), by one
// warp: the reciprocals of the diagonal in parallel, then the column sweep y_i = r_i / R_ii,
// r_l −= R_li y_i (l < i), whose per-row chain is one multiply, one shuffle and one FMA (FP64
// division and long dependent sums are slow on this GPU). Rc holds R by columns (stride KMAX).
__device__ void upper_solve_warp(const double* Rc, const double* g, int k, double* y) {
  const int lane = threadIdx.x & 31;
  double r0 = lane < k ? g[lane] : 0.0, r1 = lane + 32 < k ? g[lane + 32] : 0.0;
  const double d0 = lane < k ? Rc[lane * KMAX + lane] : 1.0;
  const double d1 = lane + 32 < k ? Rc[(lane + 32) * KMAX + lane + 32] : 1.0;
  const double q0 = d0 != 0.0 ? 1.0 / d0 : 0.0, q1 = d1 != 0.0 ? 1.0 / d1 : 0.0;
  for (int i = k - 1; i >= 0; --i) {
    const int src = i & 31;
    const double mine = i < 32 ? r0 * q0 : r1 * q1;
    const double yi = __shfl_sync(0xffffffffu, mine, src);
    if (lane == src) y[i] = yi;
    if (lane < i) r0 = fma(-Rc[i * KMAX + lane], yi, r0);
    if (lane + 32 < i) r1 = fma(-Rc[i * KMAX + lane + 32], yi, r1);
  }
}

// stage the k × k upper triangle of the rotated Hessenberg matrix by columns, and g
__device__ void stage_upper(const GmresState* s, int k, int m, double* Rc, double* g) {
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    const int col = t / k, row = t - col * k;
    Rc[col * KMAX + row] = row <= col ? s->H[(size_t)col * (m + 1) + row] : 0.0;
  }
  for (int t = threadIdx.x; t < k; t += blockDim.x) g[t] = s->g[t];
}

// start a cycle: V_0 = r/‖r‖, g = ‖r‖ e_1. With rel > 0 the absolute target is formed here as
// max(rel·‖r‖, floor_rel·‖U_b‖), ‖U_b‖ being ‖r‖ itself in the first cycle (first = 1, which records
// it) and the recorded value afterwards: the refinement sweeps set their inner targets without a
// host round trip.
__global__ void __launch_bounds__(1024) k_gmres_start(GmresState* st, const double* __restrict__ r, double* V, int nd,
                                                      double target, int kmax, double rel = 0.0,
                                                      double floor_rel = 0.0, int first = 0,
                                                      double* zero_x = nullptr) {
  __shared__ double red[32];
  if (zero_x)  // the cycle's correction starts at zero (a refinement sweep)
    for (int i = threadIdx.x; i < nd; i += blockDim.x) zero_x[i] = 0.0;
  double s = 0;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) s += r[i] * r[i];
  const double beta = sqrt(block_sum(s, red));
  const bool bad = !isfinite(beta);
  const double inv = (beta > 0 && !bad) ? 1.0 / beta : 0.0;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) V[i] = r[i] * inv;
  if (threadIdx.x == 0) {
    if (rel > 0.0) {
      const double bn = first ? beta : st->bnorm;
      if (first) st->bnorm = beta;
      target = fmax(rel * beta, floor_rel * bn);
    }
    st->beta = beta;
    st->target = target;
    st->res = beta;
    st->k = 0;
    st->kmax = kmax;
    st->body_iters = 0;
    st->g[0] = beta;
    if (bad) {
      st->status = ST_NONFINITE;
      st->stop = 1;
    } else if (beta <= target) {
      st->status = ST_CONVERGED;
      st->stop = 1;
    } else {
      st->status = ST_RUNNING;
      st->stop = 0;
    }
  }
}

// One problem. In a captured cycle (cond != 0) the step sets the while-loop condition on every
// path: 0 once the cycle has stopped, or after more loop bodies than the cycle allows (a guard
// on the device-side loop), else 1.
template <bool STAGED, int CL>
__global__ void __launch_bounds__(ATH)
    k_arnoldi_cluster(GmresState* st, double* V, int j, int nd, int m, int slice, cudaGraphConditionalHandle cond) {
  const int r = arnoldi_body<STAGED, CL>(st, V, j, nd, m, slice);
  if (cond && cg::this_cluster().block_rank() == 0 && threadIdx.x == ALEAD) {
    if (r < 0) {
      st->stop = 1;
      cudaGraphSetConditional(cond, 0);
    } else {
      st->body_iters += 1;
      if (st->body_iters > st->kmax + 2) st->stop = 1;
      cudaGraphSetConditional(cond, st->stop ? 0u : 1u);
    }
  }
}

// ------------------------------------------------------------------------------------------
// batched GMRES: one Arnoldi cluster per problem in one launch; the while loop of the captured
// cycle ends when no problem is running. Exactly one thread sets the loop condition (the
// cond_set flag), either the problem whose step brings the running count to zero, or problem
// 0's first thread when it sees no problem running or the loop-body guard exceeded.
// ------------------------------------------------------------------------------------------
struct BatchCtl {
  int running;
  int cond_set;
  int body_iters;
  int max_bodies;
};

size_t batch_state_bytes() { return sizeof(GmresState); }

__device__ __forceinline__ void batch_end_loop(BatchCtl* ctl, cudaGraphConditionalHandle cond) {
  if (atomicExch(&ctl->cond_set, 1) == 0) cudaGraphSetConditional(cond, 0);
}

template <bool STAGED, int CL>
__global__ void __launch_bounds__(ATH)
    kb_arnoldi(GmresState* st, double* V, const int64_t* __restrict__ voff, const int* __restrict__ nd_arr,
               const int* __restrict__ slice_arr, int m, BatchCtl* ctl, cudaGraphConditionalHandle cond) {
  const int b = blockIdx.x / CL;
  const bool lead = cg::this_cluster().block_rank() == 0 && threadIdx.x == 0;
  if (b == 0 && lead) {
    const int it = atomicAdd(&ctl->body_iters, 1) + 1;
    if (it > ctl->max_bodies || atomicAdd(&ctl->running, 0) <= 0) batch_end_loop(ctl, cond);
  }
  const int r = arnoldi_body<STAGED, CL>(st + b, V + voff[b], -1, nd_arr[b], m, slice_arr[b]);
  if (cg::this_cluster().block_rank() == 0 && threadIdx.x == ALEAD && r == 1) {
    if (atomicSub(&ctl->running, 1) == 1) batch_end_loop(ctl, cond);
  }
}

__global__ void kb_ctl_reset(BatchCtl* ctl, int max_bodies) {
  ctl->running = 0;
  ctl->cond_set = 0;
  ctl->body_iters = 0;
  ctl->max_bodies = max_bodies;
}

// start a cycle for every problem: V_b,0 = r_b/‖r_b‖; inactive or already converged problems stop
__global__ void __launch_bounds__(256)
    kb_gmres_start(GmresState* st, const double* __restrict__ rhs, const int64_t* __restrict__ off, double* V,
                   const int64_t* __restrict__ voff, const int* __restrict__ nd_arr, const double* __restrict__ target,
                   const int* __restrict__ active, int kmax, BatchCtl* ctl) {
  __shared__ double red[32];
  const int b = blockIdx.x, nd = nd_arr[b];
  const double* r = rhs + off[b];
  double* Vb = V + voff[b];
  double sacc = 0;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) sacc += r[i] * r[i];
  const double beta = sqrt(block_sum(sacc, red));
  const bool bad = !isfinite(beta);
  const double inv = (beta > 0 && !bad) ? 1.0 / beta : 0.0;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) Vb[i] = r[i] * inv;
  if (threadIdx.x == 0) {
    GmresState* s = st + b;
    s->beta = beta;
    s->target = target[b];
    s->res = beta;
    s->k = 0;
    s->kmax = kmax;
    s->body_iters = 0;
    s->g[0] = beta;
    if (bad) {
      s->status = ST_NONFINITE;
      s->stop = 1;
    } else if (!active[b] || beta <= target[b]) {
      s->status = ST_CONVERGED;
      s->stop = 1;
    } else {
      s->status = ST_RUNNING;
      s->stop = 0;
      atomicAdd(&ctl->running, 1);
    }
  }
}

// x_b += V_b y_b for every problem (one CTA per problem)
__global__ void __launch_bounds__(256)
    kb_gmres_update(GmresState* st, const double* __restrict__ V, const int64_t* __restrict__ voff, double* x,
                    const int64_t* __restrict__ off, const int* __restrict__ nd_arr, int m) {
  __shared__ double Rc[KMAX * KMAX];
  __shared__ double gs[KMAX], y[KMAX];
  const int b = blockIdx.x, nd = nd_arr[b];
  const GmresState* s = st + b;
  const int k = s->k;
  stage_upper(s, k, m, Rc, gs);
  __syncthreads();
  if (threadIdx.x < 32) upper_solve_warp(Rc, gs, k, y);
  __syncthreads();
  const double* Vb = V + voff[b];
  double* xb = x + off[b];
  for (int idx = threadIdx.x; idx < nd; idx += blockDim.x) {
    double acc = xb[idx];
    for (int i = 0; i < k; ++i) acc += y[i] * Vb[(size_t)i * nd + idx];
    xb[idx] = acc;
  }
}

// r_b = b_b − (Ax)_b and st[b].rnorm = ‖r_b‖ for every problem (Ax = NULL: ‖b_b‖)
__global__ void __launch_bounds__(256)
    kb_residual(GmresState* st, const double* __restrict__ bv, const double* __restrict__ Ax, double* r,
                const int64_t* __restrict__ off, const int* __restrict__ nd_arr) {
  __shared__ double red[32];
  const int b = blockIdx.x, nd = nd_arr[b];
  const size_t o = off[b];
  double sacc = 0;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) {
    const double v = bv[o + i] - (Ax ? Ax[o + i] : 0.0);
    if (r) r[o + i] = v;
    sacc += v * v;
  }
  const double nrm = sqrt(block_sum(sacc, red));
  if (threadIdx.x == 0) st[b].rnorm = nrm;
}

__global__ void kb_axpy(double* x, const double* __restrict__ d, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] += d[i];
}

// x += V_{0..k-1} y with R y = g, many CTAs; each CTA solves the small triangular system in
// shared memory and updates its own elements of x
__global__ void __launch_bounds__(256) k_gmres_update_par(GmresState* st, const double* __restrict__ V, double* x,
                                                          int nd, int m) {
  __shared__ double Rc[KMAX * KMAX];
  __shared__ double gs[KMAX], y[KMAX];
  const int k = st->k;
  stage_upper(st, k, m, Rc, gs);
  __syncthreads();
  if (threadIdx.x < 32) upper_solve_warp(Rc, gs, k, y);
  __syncthreads();
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < nd) {
    double acc = x[idx];
    for (int i = 0; i < k; ++i) acc += y[i] * V[(size_t)i * nd + idx];
    x[idx] = acc;
  }
}

// r = b − Ax, st->rnorm = ‖r‖
__global__ void __launch_bounds__(1024) k_residual(GmresState* st, const double* __restrict__ b,
                                                   const double* __restrict__ Ax, double* r, int nd) {
  __shared__ double red[32];
  double s = 0;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) {
    const double v = b[i] - Ax[i];
    r[i] = v;
    s += v * v;
  }
  const double nrm = sqrt(block_sum(s, red));
  if (threadIdx.x == 0) st->rnorm = nrm;
}

__global__ void k_axpy(double* x, const double* __restrict__ d, int nd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nd) x[i] += d[i];
}

// ------------------------------------------------------------------------------------------
// host driver
// ------------------------------------------------------------------------------------------
static ibdl_status ensure_workspace(Geometry* g, int m) {
  if (g->V && g->krylov_m >= m) return IBDL_OK;
  if (g->V) cudaFree(g->V);
  g->V = nullptr;
  const size_t nd = (size_t)geom_nd(g);
  IBDL_CUDA(cudaMalloc((void**)&g->V, sizeof(double) * nd * (m + 1)));
  if (!g->gm) IBDL_CUDA(cudaMalloc((void**)&g->gm, sizeof(GmresState)));
  if (!g->vec) IBDL_CUDA(cudaMalloc((void**)&g->vec, sizeof(double) * nd * 5));
  if (!g->host_status) IBDL_CUDA(cudaMallocHost(&g->host_status, 2 * sizeof(HostStatus)));
  g->krylov_m = m;
  return IBDL_OK;
}

struct CycleResult {
  int its;
  int status;
  double res;
  double beta;          // ‖r0‖ of the cycle
  bool copied = false;  // the OutCopy ran after the cycle's update (so the caller's copy is current)
};

// A device copy enqueued after a cycle's update and before its status read, so that a solve whose
// last cycle this is needs no further copy and synchronisation (the solution into the caller's
// device buffer).
struct OutCopy {
  void* dst;
  const void* src;
  size_t bytes;
};

static ibdl_status build_cycle_graph(Geometry* g, int prec, int m, int op, cudaGraphExec_t* out);

// Iterations (application + Arnoldi step) per body of the captured while loop. Inside a body the
// kernels follow each other with programmatic launch; between bodies the graph waits for the
// body to finish and re-evaluates the loop condition (about 6 µs at 512²), and the slots of the
// last body after the stop still launch their kernels, which return at once (about 12 µs per
// slot). 8 was the fastest of 1–16 on the 512² Stokes star (about 13 iterations per refinement
// sweep, 22 per plain solve) and on the 64² circle (6). IBDL_UNROLL=u (1..16) overrides.
static int cycle_unroll() {
  static int v = 0;
  if (!v) {
    const char* e = getenv("IBDL_UNROLL");
    const int u = e ? atoi(e) : 0;
    v = (u >= 1 && u <= 16) ? u : 8;
  }
  return v;
}

// kernels a graph-driven cycle launched: start, update, and 4 per iteration of each loop body run
static int64_t cycle_launches(const HostStatus& fin) {
  const int U = cycle_unroll();
  const int bodies = fin.body_iters > 0 ? (fin.body_iters + U - 1) / U : 1;
  return 2 + 4 * (int64_t)U * bodies;
}

// Relative inner target of a refinement sweep (rel > 0; see k_gmres_start), or none (rel = 0: the
// absolute target is used).
struct RelTarget {
  double rel = 0.0, floor_rel = 0.0;
  int first = 0;
};

// Launch the cycle's start kernel, graph and correction update. With sync the status is read back
// and cr filled; without, the caller reads the state later (cycle_launches counts the kernels).
static ibdl_status gmres_cycle_graph(Geometry* g, int prec, int op, const double* r0, double* x, double target,
                                     int m, int budget, cudaStream_t s, CycleResult* cr, const RelTarget& rt,
                                     bool sync, bool zero_x, const OutCopy* oc) {
  const int pi = 2 * op + (prec == IBDL_FP32 ? 1 : 0);
  if (!g->cycle_exec[pi] || g->cycle_m[pi] != m) {
    if (g->cycle_exec[pi]) cudaGraphExecDestroy(g->cycle_exec[pi]);
    g->cycle_exec[pi] = nullptr;
    IBDL_TRY(build_cycle_graph(g, prec, m, op, &g->cycle_exec[pi]));
    g->cycle_m[pi] = m;
  }
  GmresState* st = reinterpret_cast<GmresState*>(g->gm);
  HostStatus* hs = reinterpret_cast<HostStatus*>(g->host_status);
  const int nd = geom_nd(g);
  const int steps = m < budget ? m : budget;
  k_gmres_start<<<1, 1024, 0, s>>>(st, r0, g->V, nd, target, steps, rt.rel, rt.floor_rel, rt.first,
                                   zero_x ? x : nullptr);
  IBDL_CUDA(cudaGetLastError());
  IBDL_CUDA(cudaGraphLaunch(g->cycle_exec[pi], s));
  k_gmres_update_par<<<(nd + 255) / 256, 256, 0, s>>>(st, g->V, x, nd, m);
  IBDL_CUDA(cudaGetLastError());
  if (!sync) return IBDL_OK;
  if (oc) {
    IBDL_CUDA(cudaMemcpyAsync(oc->dst, oc->src, oc->bytes, cudaMemcpyDeviceToDevice, s));
    cr->copied = true;
  }
  IBDL_CUDA(cudaMemcpyAsync(&hs[0], st, sizeof(HostStatus), cudaMemcpyDeviceToHost, s));
  IBDL_CUDA(cudaStreamSynchronize(s));
  const HostStatus fin = hs[0];
  g->launches += cycle_launches(fin);
  cr->its = fin.k;
  cr->status = fin.status;
  cr->res = fin.res;
  cr->beta = fin.beta;
  return IBDL_OK;
}

// programmatic dependent launch of the Arnoldi step after the application (IBDL_NO_PDL=1: off)
static bool pdl_allowed() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("IBDL_NO_PDL");
    v = (e && atoi(e) != 0) ? 0 : 1;
  }
  return v == 1;
}

struct ArnoldiCfg {
  int cl;  // CTAs per cluster (16 or 8)
  int slice;
  bool staged;
  size_t dyn;
};

template <bool STAGED, int CL>
static cudaError_t arnoldi_attrs() {
  cudaError_t e = cudaFuncSetAttribute(k_arnoldi_cluster<STAGED, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess && CL > 8)
    e = cudaFuncSetAttribute(k_arnoldi_cluster<STAGED, CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

// Cluster size: 16 when a 16-CTA cluster of this kernel fits on the device, else 8
// (IBDL_ARNOLDI_CLUSTER=8 selects 8 on any device). The basis slices are staged in shared memory
// when w's slice and m + 1 basis rows fit.
static ibdl_status arnoldi_cfg(Geometry* g, int m, ArnoldiCfg* c) {
  static int cl_choice = 0;
  if (!cl_choice) {
    IBDL_CUDA((arnoldi_attrs<true, 8>()));
    IBDL_CUDA((arnoldi_attrs<false, 8>()));
    cl_choice = 8;
    const char* force = getenv("IBDL_ARNOLDI_CLUSTER");
    const bool force8 = force && atoi(force) == 8;
    if (!force8 && arnoldi_attrs<true, 16>() == cudaSuccess && arnoldi_attrs<false, 16>() == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(16);
      cfg.blockDim = dim3(ATH);
      cfg.dynamicSmemBytes = 200 * 1024;
      cudaLaunchAttribute at;
      at.id = cudaLaunchAttributeClusterDimension;
      at.val.clusterDim.x = 16;
      at.val.clusterDim.y = 1;
      at.val.clusterDim.z = 1;
      cfg.attrs = &at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, (void*)k_arnoldi_cluster<true, 16>, &cfg) == cudaSuccess &&
          nclusters >= 1)
        cl_choice = 16;
    }
    cudaGetLastError();
  }
  const int nd = geom_nd(g);
  c->cl = cl_choice;
  c->slice = (nd + c->cl - 1) / c->cl;
  const size_t staged_bytes = arnoldi_dyn_doubles(m, c->slice, true) * sizeof(double);
  c->staged = staged_bytes <= 200 * 1024;
  c->dyn = c->staged ? staged_bytes : arnoldi_dyn_doubles(m, c->slice, false) * sizeof(double);
  if (c->dyn > 200 * 1024) return fail(IBDL_ERR_UNSUPPORTED, "too many boundary unknowns for the Arnoldi kernel");
  return IBDL_OK;
}

template <bool STAGED, int CL>
static cudaError_t launch_arnoldi_t(const ArnoldiCfg& c, GmresState* st, double* V, int j, int nd, int m,
                                    cudaGraphConditionalHandle cond, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(ATH);
  cfg.dynamicSmemBytes = c.dyn;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_allowed() ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, k_arnoldi_cluster<STAGED, CL>, st, V, j, nd, m, c.slice, cond);
}

static cudaError_t launch_arnoldi(const ArnoldiCfg& c, GmresState* st, double* V, int j, int nd, int m,
                                  cudaGraphConditionalHandle cond, cudaStream_t s) {
  if (c.cl == 16)
    return c.staged ? launch_arnoldi_t<true, 16>(c, st, V, j, nd, m, cond, s)
                    : launch_arnoldi_t<false, 16>(c, st, V, j, nd, m, cond, s);
  return c.staged ? launch_arnoldi_t<true, 8>(c, st, V, j, nd, m, cond, s)
                  : launch_arnoldi_t<false, 8>(c, st, V, j, nd, m, cond, s);
}

// A GMRES cycle as a CUDA graph: one conditional while node whose body is cycle_unroll() pairs of
// the operator application on V_k (k read on the device) and the Arnoldi step; every Arnoldi step
// sets the loop condition (a step after the stop only returns). Built once per geometry, operator
// (A or Aᵀ), precision and restart length.
static ibdl_status build_cycle_graph(Geometry* g, int prec, int m, int op, cudaGraphExec_t* out) {
  *out = nullptr;
  const int nd = geom_nd(g);
  GmresState* st = reinterpret_cast<GmresState*>(g->gm);
  ArnoldiCfg c;
  IBDL_TRY(arnoldi_cfg(g, m, &c));
  cudaGraph_t graph = nullptr;
  cudaStream_t cs = nullptr;
  IBDL_CUDA(cudaGraphCreate(&graph, 0));
  ibdl_status ret = IBDL_OK;
  bool capturing = false;
  do {
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { ret = cuda_fail(e, "cudaGraphConditionalHandleCreate"); break; }
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) { ret = cuda_fail(e, "cudaGraphAddNode(conditional)"); break; }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) { ret = cuda_fail(e, "cudaStreamCreate"); break; }
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { ret = cuda_fail(e, "cudaStreamBeginCaptureToGraph"); break; }
    capturing = true;
    const int saved_timing = g->timing;
    g->timing = 0;
    for (int u = 0; u < cycle_unroll() && ret == IBDL_OK; ++u) {
      ret = g->dim == 2 ? apply_2d_indexed(g, prec, g->V, &st->k, nd, cs, &st->stop, op)
                        : apply_3d_indexed(g, prec, g->V, &st->k, nd, cs, &st->stop, op);
      if (ret == IBDL_OK) {
        const cudaError_t le = launch_arnoldi(c, st, g->V, -1, nd, m, h, cs);
        if (le != cudaSuccess) ret = cuda_fail(le, "Arnoldi launch");
      }
    }
    g->timing = saved_timing;
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(cs, &captured);
    capturing = false;
    if (ret != IBDL_OK) break;
    if (e != cudaSuccess) { ret = cuda_fail(e, "cudaStreamEndCapture"); break; }
    e = cudaGraphInstantiate(out, graph, 0);
    if (e != cudaSuccess) { ret = cuda_fail(e, "cudaGraphInstantiate"); *out = nullptr; break; }
  } while (false);
  if (capturing) {
    cudaGraph_t captured = nullptr;
    cudaStreamEndCapture(cs, &captured);
  }
  if (cs) cudaStreamDestroy(cs);
  cudaGraphDestroy(graph);
  cudaGetLastError();
  return ret;
}

// One GMRES(m) cycle on right-hand side r0 from a zero correction, accumulating into x.
static ibdl_status gmres_cycle(Geometry* g, int prec, int op, const double* r0, double* x, double target, int m,
                               int budget, cudaStream_t s, CycleResult* cr, const RelTarget& rt = RelTarget(),
                               bool sync = true, bool zero_x = false, const OutCopy* oc = nullptr) {
  GmresState* st = reinterpret_cast<GmresState*>(g->gm);
  HostStatus* hs = reinterpret_cast<HostStatus*>(g->host_status);
  const int nd = geom_nd(g);
  double* V = g->V;
  if (!g->timing) return gmres_cycle_graph(g, prec, op, r0, x, target, m, budget, s, cr, rt, sync, zero_x, oc);
  // host-driven loop (used while stage timing records an event around every kernel)
  const int steps = m < budget ? m : budget;
  ArnoldiCfg acfg;
  IBDL_TRY(arnoldi_cfg(g, m, &acfg));
  k_gmres_start<<<1, 1024, 0, s>>>(st, r0, V, nd, target, steps, rt.rel, rt.floor_rel, rt.first,
                                   zero_x ? x : nullptr);
  g->launches += 1;
  IBDL_CUDA(cudaGetLastError());
  cudaEvent_t evs[2] = {g->ev, g->ev};
  // the geometry owns one event; a second one is created per call for the double buffer
  cudaEvent_t ev2;
  IBDL_CUDA(cudaEventCreateWithFlags(&ev2, cudaEventDisableTiming));
  evs[1] = ev2;
  IBDL_CUDA(cudaMemcpyAsync(&hs[1], st, sizeof(HostStatus), cudaMemcpyDeviceToHost, s));
  IBDL_CUDA(cudaEventRecord(evs[1], s));
  ibdl_status err = IBDL_OK;
  for (int j = 0; j < steps; ++j) {
    err = apply_any(g, prec, V + (size_t)j * nd, V + (size_t)(j + 1) * nd, s, &st->stop, op);
    if (err != IBDL_OK) break;
    if (g->timing) timing_mark(g, s, -1);
    if (launch_arnoldi(acfg, st, V, j, nd, m, 0, s) != cudaSuccess) {
      err = fail(IBDL_ERR_CUDA, "Arnoldi launch failed");
      break;
    }
    if (g->timing) timing_mark(g, s, IBDL_STAGE_ARNOLDI);
    g->launches += 1;
    if (cudaGetLastError() != cudaSuccess) {
      err = fail(IBDL_ERR_CUDA, "k_arnoldi launch failed");
      break;
    }
    // wait for the previous step's status while this step runs
    const int prev = (j + 1) & 1;
    if (cudaEventSynchronize(evs[prev]) != cudaSuccess) {
      err = fail(IBDL_ERR_CUDA, "event synchronize failed");
      break;
    }
    const bool stopped = hs[prev].stop != 0;
    if (cudaMemcpyAsync(&hs[j & 1], st, sizeof(HostStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaEventRecord(evs[j & 1], s) != cudaSuccess) {
      err = fail(IBDL_ERR_CUDA, "status copy failed");
      break;
    }
    if (stopped) break;
  }
  cudaStreamSynchronize(s);
  cudaEventDestroy(ev2);
  if (err != IBDL_OK) return err;
  HostStatus fin;
  IBDL_CUDA(cudaMemcpy(&fin, st, sizeof(HostStatus), cudaMemcpyDeviceToHost));
  k_gmres_update_par<<<(nd + 255) / 256, 256, 0, s>>>(st, V, x, nd, m);
  g->launches += 1;
  IBDL_CUDA(cudaGetLastError());
  cr->its = fin.k;
  cr->status = fin.status;
  cr->res = fin.res;
  cr->beta = fin.beta;
  return IBDL_OK;
}

// r = b − A₆₄ x (or b − Aᵀ₆₄ x), returns ‖r‖ (synchronous)
static ibdl_status true_residual(Geometry* g, int op, const double* b, const double* x, double* r, double* Ax,
                                 cudaStream_t s, double* rnorm) {
  GmresState* st = reinterpret_cast<GmresState*>(g->gm);
  const int nd = geom_nd(g);
  IBDL_TRY(apply_any(g, IBDL_FP64, x, Ax, s, nullptr, op));
  k_residual<<<1, 1024, 0, s>>>(st, b, Ax, r, nd);
  g->launches += 1;
  IBDL_CUDA(cudaGetLastError());
  HostStatus fin;
  IBDL_CUDA(cudaMemcpyAsync(&fin, st, sizeof(HostStatus), cudaMemcpyDeviceToHost, s));
  IBDL_CUDA(cudaStreamSynchronize(s));
  *rnorm = fin.rnorm;
  return IBDL_OK;
}


ibdl_status solve_impl(Geometry* g, const double* Ub, double* Q, const ibdl_solve_opts* o, ibdl_solve_info* info,
                       cudaStream_t s, int op, const double* gsrc) {
  const auto t0 = std::chrono::steady_clock::now();
  const int m = o->restart;
  IBDL_TRY(ensure_workspace(g, m));
  const int nd = geom_nd(g);
  double* b = g->vec;
  double* x = g->vec + (size_t)nd;
  double* r = g->vec + 2 * (size_t)nd;
  double* d = g->vec + 3 * (size_t)nd;
  IBDL_CUDA(cudaMemcpyAsync(b, Ub, sizeof(double) * nd, o->io_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  IBDL_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * nd, s));
  // a source term: b = U_b − S*u_g (and the completed method's constraint rows from g̃)
  if (gsrc) IBDL_TRY(source_terms(g, gsrc, b, nullptr, s));
  // ‖U_b‖ comes from the first cycle (its ‖r0‖), which also forms its own target rtol·‖U_b‖
  const bool mixed = o->precision == IBDL_MIXED;
  ibdl_solve_info inf = {};
  ibdl_status ret = IBDL_OK;
  // a device Q is copied before each cycle's (sweep's) status read, so the last one leaves it current
  const OutCopy qcopy = {Q, x, sizeof(double) * nd};
  const OutCopy* oc = o->io_on_host ? nullptr : &qcopy;
  bool q_current = false;
  if (!mixed) {
    // plain restarted GMRES(m) with FP64 (or FP32) applies
    int used = 0;
    bool done = false;
    const double* rhs = b;
    double bnorm = 0.0, target = 0.0;
    for (int cycle = 0; !done; ++cycle) {
      CycleResult cr;
      RelTarget rt;
      if (cycle == 0) {
        rt.rel = o->rtol;
        rt.first = 1;
      }
      IBDL_TRY(gmres_cycle(g, o->precision, op, rhs, x, target, m, o->maxit - used, s, &cr, rt, true, false, oc));
      q_current = cr.copied;  // the restart's residual below leaves x as it is
      if (cycle == 0) {
        bnorm = cr.beta;
        target = o->rtol * bnorm;
        if (!std::isfinite(bnorm)) return fail(IBDL_ERR_NONFINITE, "U_b contains NaN or Inf");
        if (bnorm == 0.0) {
          inf.rel_residual = 0.0;
          break;
        }
      }
      used += cr.its;
      inf.sweeps += 1;
      if (o->precision == IBDL_FP32)
        inf.fp32_applies += cr.its;
      else
        inf.fp64_applies += cr.its;
      inf.rel_residual = cr.res / bnorm;
      if (cr.status == ST_NONFINITE) {
        ret = fail(IBDL_ERR_NONFINITE, "non-finite value in the GMRES iteration");
        break;
      }
      if (cr.status == ST_CONVERGED || cr.status == ST_BREAKDOWN) break;
      if (used >= o->maxit) {
        ret = fail(IBDL_ERR_NOT_CONVERGED, "GMRES reached maxit");
        break;
      }
      // restart from the true residual
      double rn = 0;
      IBDL_TRY(true_residual(g, op, b, x, r, d, s, &rn));
      inf.fp64_applies += 1;
      inf.rel_residual = rn / bnorm;
      if (rn <= target) break;
      rhs = r;
    }
    inf.iterations = used;
  } else {
    // iterative refinement. A sweep runs one inner GMRES cycle (at most m iterations) with FP32
    // applications on the current FP64 residual from a zero correction d, to the inner target
    // max(inner_rtol·‖r‖, ½·rtol·‖U_b‖) formed on the device; then x += d and r = b − A x in FP64.
    // The host reads the cycle's status and ‖r‖ once per sweep; ‖U_b‖ comes from the first cycle.
    // A cycle that ends at its restart length is followed by an FP64 residual like any sweep and
    // does not count against max_refine (which bounds the sweeps whose inner solve converged).
    GmresState* st = reinterpret_cast<GmresState*>(g->gm);
    HostStatus* hs = reinterpret_cast<HostStatus*>(g->host_status);
    // the residual's application: float-float (2-D) or FP64; its subtraction and norm are FP64
    // (float-float grids are built to 4096² in 2-D and for every 3-D size)
    const int res_prec = o->residual == IBDL_FP32X2 && (g->dim == 3 || g->n <= 4096) ? IBDL_FP32X2 : IBDL_FP64;
    int used = 0, refined = 0;
    const double* rhs = b;
    double bn = 0.0;
    bool done = false;
    for (int sweep = 0; !done; ++sweep) {
      RelTarget rt;
      rt.rel = o->inner_rtol;
      rt.floor_rel = 0.5 * o->rtol;
      rt.first = sweep == 0;
      CycleResult cr = {};
      IBDL_TRY(gmres_cycle(g, IBDL_FP32, op, rhs, d, 0.0, m, o->maxit - used, s, &cr, rt, false, true));
      k_axpy<<<(nd + 255) / 256, 256, 0, s>>>(x, d, nd);
      g->launches += 1;
      IBDL_CUDA(cudaGetLastError());
      IBDL_TRY(apply_any(g, res_prec, x, d, s, nullptr, op));
      k_residual<<<1, 1024, 0, s>>>(st, b, d, r, nd);
      g->launches += 1;
      IBDL_CUDA(cudaGetLastError());
      if (oc) IBDL_CUDA(cudaMemcpyAsync(oc->dst, oc->src, oc->bytes, cudaMemcpyDeviceToDevice, s));
      q_current = oc != nullptr;
      IBDL_CUDA(cudaMemcpyAsync(&hs[0], st, sizeof(HostStatus), cudaMemcpyDeviceToHost, s));
      IBDL_CUDA(cudaStreamSynchronize(s));
      const HostStatus fin = hs[0];
      if (!g->timing) g->launches += cycle_launches(fin);
      if (sweep == 0) bn = fin.beta;
      used += fin.k;
      inf.fp32_applies += fin.k;
      (res_prec == IBDL_FP32X2 ? inf.fp32x2_applies : inf.fp64_applies) += 1;
      inf.sweeps += 1;
      if (fin.status == ST_NONFINITE || !std::isfinite(fin.rnorm))
        return fail(IBDL_ERR_NONFINITE, sweep == 0 && !std::isfinite(bn) ? "U_b contains NaN or Inf"
                                                                          : "non-finite value in the GMRES iteration");
      const double rn = fin.rnorm;
      if (bn == 0.0) {
        inf.rel_residual = 0.0;
        break;
      }
      inf.rel_residual = rn / bn;
      if (fin.status != ST_RUNNING) ++refined;
      done = rn <= o->rtol * bn || used >= o->maxit || refined >= o->max_refine;
      rhs = r;
    }
    inf.iterations = used;
    if (inf.rel_residual > o->rtol && ret == IBDL_OK)
      ret = fail(IBDL_ERR_NOT_CONVERGED, "mixed-precision refinement did not reach rtol");
  }
  if (!q_current) {
    IBDL_CUDA(cudaMemcpyAsync(Q, x, sizeof(double) * nd, o->io_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    IBDL_CUDA(cudaStreamSynchronize(s));
  }
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  const ibdl_status dev = take_device_error(g);
  return dev != IBDL_OK ? dev : ret;
}

}  // namespace ibdl

namespace ibdl {

// ------------------------------------------------------------------------------------------
// batched solve driver
// ------------------------------------------------------------------------------------------
// Workspace for restart length m: per-problem Krylov bases (offsets voff), states, control
// block, work vectors, targets, activity flags, and the parameter blocks of the batched apply
// in Krylov-basis mode (which point at the states).
static ibdl_status batch_workspace(Batch* B, int m, const ArnoldiCfg& c) {
  if (B->m == m && B->V) return IBDL_OK;
  if (B->V) cudaFree(B->V);
  B->V = nullptr;
  std::vector<int64_t> voff(B->count);
  std::vector<int> nd(B->count), slice(B->count);
  int64_t vtot = 0;
  for (int b = 0; b < B->count; ++b) {
    nd[b] = (int)(B->off[b + 1] - B->off[b]);
    voff[b] = vtot;
    vtot += (int64_t)(m + 1) * nd[b];
    slice[b] = (nd[b] + c.cl - 1) / c.cl;
  }
  for (int b = 0; b < B->count; ++b) B->voff[b] = voff[b];
  IBDL_CUDA(cudaMalloc((void**)&B->V, sizeof(double) * vtot));
  if (!B->st) IBDL_CUDA(cudaMalloc(&B->st, sizeof(GmresState) * B->count));
  if (!B->ctl) IBDL_CUDA(cudaMalloc(&B->ctl, sizeof(BatchCtl)));
  if (!B->host_st) IBDL_CUDA(cudaMallocHost(&B->host_st, sizeof(HostStatus) * B->count));
  if (!B->vec) IBDL_CUDA(cudaMalloc((void**)&B->vec, sizeof(double) * 5 * B->total));
  if (!B->target) IBDL_CUDA(cudaMalloc((void**)&B->target, sizeof(double) * B->count));
  if (!B->active) IBDL_CUDA(cudaMalloc((void**)&B->active, sizeof(int) * B->count));
  auto up = [&](void** dst, const void* src, size_t bytes) -> ibdl_status {
    if (*dst) cudaFree(*dst);
    *dst = nullptr;
    IBDL_CUDA(cudaMalloc(dst, bytes));
    IBDL_CUDA(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    return IBDL_OK;
  };
  std::vector<int64_t> off(B->off, B->off + B->count);
  IBDL_TRY(up(reinterpret_cast<void**>(&B->d_off), off.data(), sizeof(int64_t) * B->count));
  IBDL_TRY(up(reinterpret_cast<void**>(&B->d_voff), voff.data(), sizeof(int64_t) * B->count));
  IBDL_TRY(up(reinterpret_cast<void**>(&B->d_nd), nd.data(), sizeof(int) * B->count));
  IBDL_TRY(up(reinterpret_cast<void**>(&B->d_slice), slice.data(), sizeof(int) * B->count));
  B->m = m;
  B->cl = c.cl;
  for (int i = 0; i < 2; ++i) {
    if (B->exec[i]) cudaGraphExecDestroy(B->exec[i]);
    B->exec[i] = nullptr;
  }
  return batch_prepare_2d(B);  // Krylov-basis mode now points at the states
}

template <bool STAGED, int CL>
static cudaError_t launch_kb_arnoldi(Batch* B, size_t dyn, cudaGraphConditionalHandle cond, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(B->count * CL);
  cfg.blockDim = dim3(ATH);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_allowed() ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, kb_arnoldi<STAGED, CL>, static_cast<GmresState*>(B->st), B->V,
                            (const int64_t*)B->d_voff, (const int*)B->d_nd, (const int*)B->d_slice, B->m,
                            static_cast<BatchCtl*>(B->ctl), cond);
}

template <bool STAGED, int CL>
static cudaError_t kb_arnoldi_attrs() {
  cudaError_t e = cudaFuncSetAttribute(kb_arnoldi<STAGED, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess && CL > 8)
    e = cudaFuncSetAttribute(kb_arnoldi<STAGED, CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

// the batched cycle graph: while (any problem running) { batched apply on V_b,k ; batched Arnoldi }
static ibdl_status build_batch_graph(Batch* B, int prec, cudaGraphExec_t* out) {
  *out = nullptr;
  int maxslice = 0;
  for (int b = 0; b < B->count; ++b) {
    const int nd = (int)(B->off[b + 1] - B->off[b]);
    maxslice = std::max(maxslice, (nd + B->cl - 1) / B->cl);
  }
  const size_t staged_bytes = arnoldi_dyn_doubles(B->m, maxslice, true) * sizeof(double);
  const bool staged = staged_bytes <= 200 * 1024;
  const size_t dyn = staged ? staged_bytes : arnoldi_dyn_doubles(B->m, maxslice, false) * sizeof(double);
  if (dyn > 200 * 1024) return fail(IBDL_ERR_UNSUPPORTED, "too many boundary unknowns for the Arnoldi kernel");
  static bool attrs = false;
  if (!attrs) {
    IBDL_CUDA((kb_arnoldi_attrs<true, 8>()));
    IBDL_CUDA((kb_arnoldi_attrs<false, 8>()));
    if (B->cl == 16) {
      IBDL_CUDA((kb_arnoldi_attrs<true, 16>()));
      IBDL_CUDA((kb_arnoldi_attrs<false, 16>()));
    }
    attrs = true;
  }
  cudaGraph_t graph = nullptr;
  cudaStream_t cs = nullptr;
  IBDL_CUDA(cudaGraphCreate(&graph, 0));
  ibdl_status ret = IBDL_OK;
  bool capturing = false;
  do {
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { ret = cuda_fail(e, "cudaGraphConditionalHandleCreate"); break; }
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) { ret = cuda_fail(e, "cudaGraphAddNode(conditional)"); break; }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) { ret = cuda_fail(e, "cudaStreamCreate"); break; }
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { ret = cuda_fail(e, "cudaStreamBeginCaptureToGraph"); break; }
    capturing = true;
    ret = batch_apply_2d(B, prec, 1, B->V, B->V, cs);
    if (ret == IBDL_OK) {
      cudaError_t le;
      if (B->cl == 16)
        le = staged ? launch_kb_arnoldi<true, 16>(B, dyn, h, cs) : launch_kb_arnoldi<false, 16>(B, dyn, h, cs);
      else
        le = staged ? launch_kb_arnoldi<true, 8>(B, dyn, h, cs) : launch_kb_arnoldi<false, 8>(B, dyn, h, cs);
      if (le != cudaSuccess) ret = cuda_fail(le, "batched Arnoldi launch");
    }
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(cs, &captured);
    capturing = false;
    if (ret != IBDL_OK) break;
    if (e != cudaSuccess) { ret = cuda_fail(e, "cudaStreamEndCapture"); break; }
    e = cudaGraphInstantiate(out, graph, 0);
    if (e != cudaSuccess) { ret = cuda_fail(e, "cudaGraphInstantiate"); *out = nullptr; break; }
  } while (false);
  if (capturing) {
    cudaGraph_t captured = nullptr;
    cudaStreamEndCapture(cs, &captured);
  }
  if (cs) cudaStreamDestroy(cs);
  cudaGraphDestroy(graph);
  cudaGetLastError();
  return ret;
}

// the status header (HostStatus, the leading fields of GmresState) of every problem into
// B->host_st: one strided copy of count × 48 bytes instead of the whole states
static_assert(offsetof(GmresState, rnorm) == offsetof(HostStatus, rnorm) && sizeof(HostStatus) <= sizeof(GmresState),
              "HostStatus mirrors the head of GmresState");
static ibdl_status batch_status_to_host(Batch* B, cudaStream_t s) {
  IBDL_CUDA(cudaMemcpy2DAsync(B->host_st, sizeof(HostStatus), B->st, sizeof(GmresState), sizeof(HostStatus),
                              (size_t)B->count, cudaMemcpyDeviceToHost, s));
  return IBDL_OK;
}

// one batched GMRES cycle on right-hand sides rhs (concatenated) from zero corrections, added
// into x; per-problem targets in B->target, activity in B->active; returns the states on the host
static ibdl_status batch_cycle(Batch* B, int prec, const double* rhs, double* x, int kmax, cudaStream_t s) {
  const int pi = prec == IBDL_FP32 ? 1 : 0;
  if (!B->exec[pi]) IBDL_TRY(build_batch_graph(B, prec, &B->exec[pi]));
  GmresState* st = static_cast<GmresState*>(B->st);
  BatchCtl* ctl = static_cast<BatchCtl*>(B->ctl);
  kb_ctl_reset<<<1, 1, 0, s>>>(ctl, kmax + 2);
  kb_gmres_start<<<B->count, 256, 0, s>>>(st, rhs, B->d_off, B->V, B->d_voff, B->d_nd, B->target, B->active, kmax, ctl);
  IBDL_CUDA(cudaGetLastError());
  IBDL_CUDA(cudaGraphLaunch(B->exec[pi], s));
  kb_gmres_update<<<B->count, 256, 0, s>>>(st, B->V, B->d_voff, x, B->d_off, B->d_nd, B->m);
  IBDL_CUDA(cudaGetLastError());
  IBDL_TRY(batch_status_to_host(B, s));
  IBDL_CUDA(cudaStreamSynchronize(s));
  BatchCtl hc;
  IBDL_CUDA(cudaMemcpy(&hc, ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost));
  B->launches += 4 + 4 * (int64_t)(hc.body_iters > 0 ? hc.body_iters : 1);
  return IBDL_OK;
}

// r = b − A x for every problem (r may be NULL), the application in FP64 or float-float
// (`precision`), the subtraction and norms in FP64, norms into the host states (synchronous)
static ibdl_status batch_residual(Batch* B, const double* bvec, const double* x, double* r, double* Ax,
                                  std::vector<double>& rn, cudaStream_t s, int precision = IBDL_FP64) {
  GmresState* st = static_cast<GmresState*>(B->st);
  if (x) IBDL_TRY(batch_apply_2d(B, precision, 0, x, Ax, s));
  kb_residual<<<B->count, 256, 0, s>>>(st, bvec, x ? Ax : nullptr, r, B->d_off, B->d_nd);
  B->launches += 1;
  IBDL_CUDA(cudaGetLastError());
  IBDL_TRY(batch_status_to_host(B, s));
  IBDL_CUDA(cudaStreamSynchronize(s));
  const HostStatus* hs = static_cast<const HostStatus*>(B->host_st);
  rn.resize(B->count);
  for (int b = 0; b < B->count; ++b) rn[b] = hs[b].rnorm;
  return IBDL_OK;
}

ibdl_status batch_solve_impl(Batch* B, const double* Ub, double* Q, const ibdl_solve_opts* o, ibdl_solve_info* infos,
                             cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  const int m = o->restart;
  // the Arnoldi cluster choice of the single-problem path (needs a geometry to size against)
  ArnoldiCfg c;
  IBDL_TRY(arnoldi_cfg(B->geoms[0], m, &c));
  IBDL_TRY(batch_workspace(B, m, c));
  const int64_t T = B->total;
  double* bvec = B->vec;
  double* x = B->vec + T;
  double* r = B->vec + 2 * T;
  double* d = B->vec + 3 * T;
  double* tmp = B->vec + 4 * T;
  IBDL_CUDA(cudaMemcpyAsync(bvec, Ub, sizeof(double) * T, o->io_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  IBDL_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * T, s));
  std::vector<double> bn, rn;
  IBDL_TRY(batch_residual(B, bvec, nullptr, nullptr, nullptr, bn, s));
  const int C = B->count;
  std::vector<ibdl_solve_info> inf(C);
  std::memset(inf.data(), 0, sizeof(ibdl_solve_info) * C);
  std::vector<int> active(C), status(C, ST_RUNNING);
  std::vector<double> target(C);
  ibdl_status ret = IBDL_OK;
  for (int b = 0; b < C; ++b) {
    if (!std::isfinite(bn[b])) return fail(IBDL_ERR_NONFINITE, "U_b of problem " + std::to_string(b) + " contains NaN or Inf");
    active[b] = bn[b] > 0.0;
  }
  auto upload = [&]() -> ibdl_status {
    IBDL_CUDA(cudaMemcpyAsync(B->active, active.data(), sizeof(int) * C, cudaMemcpyHostToDevice, s));
    IBDL_CUDA(cudaMemcpyAsync(B->target, target.data(), sizeof(double) * C, cudaMemcpyHostToDevice, s));
    return IBDL_OK;
  };
  auto any_active = [&]() {
    for (int b = 0; b < C; ++b)
      if (active[b]) return true;
    return false;
  };
  const HostStatus* hs = static_cast<const HostStatus*>(B->host_st);
  int used = 0;  // loop bodies (the longest problem's iterations), counted against maxit
  if (o->precision != IBDL_MIXED) {
    // restarted GMRES(m) on every problem at once
    const double* rhs = bvec;
    for (int b = 0; b < C; ++b) target[b] = o->rtol * bn[b];
    while (any_active() && used < o->maxit) {
      IBDL_TRY(upload());
      const int kmax = std::min(m, o->maxit - used);
      IBDL_TRY(batch_cycle(B, o->precision, rhs, x, kmax, s));
      int longest = 0;
      for (int b = 0; b < C; ++b) {
        if (!active[b]) continue;
        longest = std::max(longest, hs[b].k);
        inf[b].iterations += hs[b].k;
        (o->precision == IBDL_FP32 ? inf[b].fp32_applies : inf[b].fp64_applies) += hs[b].k;
        inf[b].sweeps += 1;
        inf[b].rel_residual = hs[b].res / bn[b];
        status[b] = hs[b].status;
        if (hs[b].status != ST_RUNNING) active[b] = 0;
      }
      used += std::max(longest, 1);
      if (!any_active()) break;
      // restart the unconverged problems from their true residuals
      IBDL_TRY(batch_residual(B, bvec, x, r, tmp, rn, s));
      for (int b = 0; b < C; ++b)
        if (active[b]) {
          inf[b].fp64_applies += 1;
          inf[b].rel_residual = rn[b] / bn[b];
          if (rn[b] <= target[b]) {
            active[b] = 0;
            status[b] = ST_CONVERGED;
          }
        }
      rhs = r;
    }
  } else {
    // iterative refinement: inner FP32-apply GMRES cycles on the residuals (applications in
    // float-float or FP64, subtraction and norms in FP64)
    const int res_prec = o->residual == IBDL_FP32X2 && B->max_log2n <= 12 ? IBDL_FP32X2 : IBDL_FP64;
    const double* rhs = bvec;
    rn = bn;
    for (int sweep = 0; sweep < o->max_refine && any_active() && used < o->maxit; ++sweep) {
      for (int b = 0; b < C; ++b) target[b] = std::max(o->inner_rtol * rn[b], 0.5 * o->rtol * bn[b]);
      IBDL_TRY(upload());
      IBDL_CUDA(cudaMemsetAsync(d, 0, sizeof(double) * T, s));
      const int kmax = std::min(m, o->maxit - used);
      IBDL_TRY(batch_cycle(B, IBDL_FP32, rhs, d, kmax, s));
      int longest = 0;
      for (int b = 0; b < C; ++b) {
        if (!active[b]) continue;
        longest = std::max(longest, hs[b].k);
        inf[b].iterations += hs[b].k;
        inf[b].fp32_applies += hs[b].k;
        inf[b].sweeps += 1;
        if (hs[b].status == ST_NONFINITE) {
          status[b] = ST_NONFINITE;
          active[b] = 0;
        }
      }
      used += std::max(longest, 1);
      kb_axpy<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(x, d, T);
      B->launches += 1;
      IBDL_CUDA(cudaGetLastError());
      IBDL_TRY(batch_residual(B, bvec, x, r, tmp, rn, s, res_prec));
      for (int b = 0; b < C; ++b) {
        if (!active[b]) continue;
        (res_prec == IBDL_FP32X2 ? inf[b].fp32x2_applies : inf[b].fp64_applies) += 1;
        inf[b].rel_residual = rn[b] / bn[b];
        if (rn[b] <= o->rtol * bn[b]) {
          active[b] = 0;
          status[b] = ST_CONVERGED;
        }
      }
      rhs = r;
    }
  }
  for (int b = 0; b < C; ++b) {
    if (status[b] == ST_NONFINITE && ret == IBDL_OK) ret = fail(IBDL_ERR_NONFINITE, "non-finite value in problem " + std::to_string(b));
    if (bn[b] > 0 && status[b] != ST_CONVERGED && status[b] != ST_BREAKDOWN && ret == IBDL_OK)
      ret = fail(IBDL_ERR_NOT_CONVERGED, "problem " + std::to_string(b) + " did not reach rtol");
  }
  IBDL_CUDA(cudaMemcpyAsync(Q, x, sizeof(double) * T, o->io_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
  IBDL_CUDA(cudaStreamSynchronize(s));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (infos)
    for (int b = 0; b < C; ++b) {
      inf[b].seconds = secs;
      infos[b] = inf[b];
    }
  const ibdl_status dev = take_device_error(B->geoms[0]);  // the batch's staged passes report here
  return dev != IBDL_OK ? dev : ret;
}

}  // namespace ibdl
