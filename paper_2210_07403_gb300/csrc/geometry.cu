// Geometry set-up (once per boundary): validation, stencil cells, counting sort of the points
// by cell, per-point kernel tables in FP64 and FP32, FFT twiddles and per-axis Fourier symbols.
#include <cmath>
#include <cstring>
#include <vector>

#include "ff.cuh"
#include "fft.cuh"

namespace ibdl {

// Base node of the 4-point stencil along one axis: floor((X − origin)/h) − 1, so the nodes
// base..base+3 straddle X (Sec. 2.2.2: at most 4 nonzero weights per axis).
__device__ __forceinline__ long long stencil_base(double xi) { return (long long)floor(xi) - 1; }

__device__ __forceinline__ int wrap(long long b, int n) {
  long long r = b % n;
  return (int)(r < 0 ? r + n : r);
}

// cell key of each point: the wrapped base row (2-D: y) or (z, y) pair (3-D)
__global__ void k_point_keys(int dim, int n, int M, const double* __restrict__ X, double ox, double oy,
                             double oz, double h, int* __restrict__ key, int* __restrict__ count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const int by = wrap(stencil_base((X[M + i] - oy) / h), n);
  int k = by;
  if (dim == 3) k = wrap(stencil_base((X[2 * M + i] - oz) / h), n) * n + by;
  key[i] = k;
  atomicAdd(count + k, 1);
}

// exclusive prefix sum of count[0..ncell) into start[0..ncell], one block
__global__ void k_scan(int ncell, const int* __restrict__ count, int* __restrict__ start) {
  __shared__ int part[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < ncell; base += blockDim.x) {
    const int i = base + threadIdx.x;
    part[threadIdx.x] = i < ncell ? count[i] : 0;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
      const int v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
      __syncthreads();
      part[threadIdx.x] += v;
      __syncthreads();
    }
    if (i < ncell) start[i] = carry + part[threadIdx.x] - (i < ncell ? count[i] : 0);
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += part[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) start[ncell] = carry;
}

__global__ void k_scatter(int M, const int* __restrict__ key, int* __restrict__ cursor, int* __restrict__ perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  perm[atomicAdd(cursor + key[i], 1)] = i;
}

// order each cell's points by original index, so the sorted order is deterministic
__global__ void k_sort_cells(int ncell, const int* __restrict__ start, int* __restrict__ perm) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int a = start[c], b = start[c + 1];
  for (int i = a + 1; i < b; ++i) {
    const int v = perm[i];
    int j = i - 1;
    while (j >= a && perm[j] > v) {
      perm[j + 1] = perm[j];
      --j;
    }
    perm[j + 1] = v;
  }
}

// kernel weights per sorted point: φ(r) and φ'(r)/h at r = (x_node − X)/h for the four
// nodes of each axis; Δs/h^d; normals. FP64 values, and FP32 copies rounded from them. When
// dd is not NULL also φ''(r)/h² in FP64 (the boundary derivatives need it).
__global__ void k_tables(int dim, int n, int M, int delta, const double* __restrict__ X,
                         const double* __restrict__ nrm, const double* __restrict__ w, double ox, double oy,
                         double oz, double h, const int* __restrict__ perm, int* __restrict__ base,
                         PointTable<double> t64, PointTable<float> t32, double* __restrict__ dd) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  const int i = perm[s];
  const double org[3] = {ox, oy, oz};
  for (int j = 0; j < dim; ++j) {
    const double xi = (X[j * M + i] - org[j]) / h;
    const long long b = stencil_base(xi);
    base[j * M + s] = wrap(b, n);
    for (int a = 0; a < 4; ++a) {
      const double r = (double)(b + a) - xi;
      const double ph = delta == IBDL_DELTA_SQRT ? phi_sqrt(r) : phi_cos(r);
      const double dp = (delta == IBDL_DELTA_SQRT ? dphi_sqrt(r) : dphi_cos(r)) / h;
      t64.phi[(j * 4 + a) * M + s] = ph;
      t64.dphi[(j * 4 + a) * M + s] = dp;
      t32.phi[(j * 4 + a) * M + s] = (float)ph;
      t32.dphi[(j * 4 + a) * M + s] = (float)dp;
      if (dd) dd[(j * 4 + a) * M + s] = (delta == IBDL_DELTA_SQRT ? ddphi_sqrt(r) : ddphi_cos(r)) / (h * h);
    }
    t64.nrm[j * M + s] = nrm[j * M + i];
    t32.nrm[j * M + s] = (float)nrm[j * M + i];
  }
  double hd = h * h;
  if (dim == 3) hd *= h;
  t64.wscale[s] = w[i] / hd;
  t32.wscale[s] = (float)(w[i] / hd);
}

// tw[j] = e^{−2πi j/n}
__global__ void k_twiddles(int n, double2* tw64, float2* tw32) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s, c;
  sincospi(-2.0 * (double)j / (double)n, &s, &c);
  tw64[j] = make_double2(c, s);
  tw32[j] = make_float2((float)c, (float)s);
}

// float-float copies of the FP64 twiddles and symbols (hi = fl32(x), lo = fl32(x − hi))
__global__ void k_ff_tables(int n, const double2* tw64, const double* lap64, const double* der64, ff* twff, ff* lapff,
                            ff* derff) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  twff[2 * j] = ff(tw64[j].x);
  twff[2 * j + 1] = ff(tw64[j].y);
  lapff[j] = ff(lap64[j]);
  derff[j] = ff(der64[j]);
}

// per-axis symbols at FFT index j, m = j (j < n/2) or j − n, k = 2π m/box:
//   spectral: lap = k², der = k (0 at the Nyquist index j = n/2)
//   fd2:      lap = (4/h²) sin²(k h/2) = (4/h²) sin²(π m/n), der = sin(k h)/h = sin(2π m/n)/h
__global__ void k_symbols(int n, double box, int symbol, double* lap64, double* der64, float* lap32, float* der32) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int m = j < n / 2 ? j : j - n;
  const double h = box / n;
  double lap, der;
  if (symbol == IBDL_SYMBOL_FD2) {
    const double sh = sinpi((double)m / n);
    lap = 4.0 / (h * h) * sh * sh;
    der = j == n / 2 ? 0.0 : sinpi(2.0 * m / n) / h;
  } else {
    const double k = 2.0 * 3.14159265358979323846 * m / box;
    lap = k * k;
    der = j == n / 2 ? 0.0 : k;
  }
  lap64[j] = lap;
  der64[j] = der;
  lap32[j] = (float)lap;
  der32[j] = (float)der;
}

// Runs the set-up kernels of a geometry into buffers the caller already holds (g's table,
// spectrum and symbol pointers, plus key/count/cursor work arrays); allocates nothing.
ibdl_status fill_geometry_tables(Geometry* g, const double* dX, const double* dN, const double* dW, int* key,
                                 int* count, int* cursor, cudaStream_t s) {
  const int M = (int)g->M, n = g->n, dim = g->dim, tb = 256;
  IBDL_CUDA(cudaMemsetAsync(count, 0, sizeof(int) * g->ncell, s));
  k_point_keys<<<(M + tb - 1) / tb, tb, 0, s>>>(dim, n, M, dX, g->origin[0], g->origin[1], g->origin[2], g->h, key, count);
  k_scan<<<1, 1024, 0, s>>>(g->ncell, count, g->cell_start);
  IBDL_CUDA(cudaMemcpyAsync(cursor, g->cell_start, sizeof(int) * (g->ncell + 1), cudaMemcpyDeviceToDevice, s));
  k_scatter<<<(M + tb - 1) / tb, tb, 0, s>>>(M, key, cursor, g->perm);
  k_sort_cells<<<(g->ncell + tb - 1) / tb, tb, 0, s>>>(g->ncell, g->cell_start, g->perm);
  k_tables<<<(M + tb - 1) / tb, tb, 0, s>>>(dim, n, M, g->delta, dX, dN, dW, g->origin[0], g->origin[1], g->origin[2],
                                             g->h, g->perm, g->base, g->t64, g->t32, g->ddphi64);
  k_twiddles<<<(n + tb - 1) / tb, tb, 0, s>>>(n, g->tw64, g->tw32);
  k_symbols<<<(n + tb - 1) / tb, tb, 0, s>>>(n, g->box, g->symbol, g->lap64, g->der64, g->lap32, g->der32);
  if (g->twff)
    k_ff_tables<<<(n + tb - 1) / tb, tb, 0, s>>>(n, g->tw64, g->lap64, g->der64, static_cast<ff*>(g->twff),
                                                  static_cast<ff*>(g->lapff), static_cast<ff*>(g->derff));
  IBDL_CUDA(cudaGetLastError());
  return IBDL_OK;
}

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// minimum-image difference on a periodic box of side L
static double min_image(double d, double L) { return d - L * std::nearbyint(d / L); }

// Normals and weights of one closed 2-D curve from its ordered points (Sec. 5.3.1, Eq. "normal
// vector approximations"): n_i = (Y_{i+1} − Y_{i−1}, −(X_{i+1} − X_{i−1}))/‖X_{i+1} − X_{i−1}‖, pointing to
// the right of the direction of travel (outward for a counter-clockwise curve), and
// Δs_i = ‖X_{i+1} − X_i‖; X is [2][M], differences by minimum image. A degenerate chord leaves a
// non-unit normal or a zero weight, which the validation that follows rejects.
static void estimate_normals(const double* X, int M, double L, double* n) {
  for (int i = 0; i < M; ++i) {
    const int a = i + 1 == M ? 0 : i + 1, b = i == 0 ? M - 1 : i - 1;
    const double dx = min_image(X[a] - X[b], L), dy = min_image(X[M + a] - X[M + b], L);
    const double len = std::hypot(dx, dy);
    n[i] = dy / len;
    n[M + i] = -dx / len;
  }
}
static void estimate_weights(const double* X, int M, double L, double* w) {
  for (int i = 0; i < M; ++i) {
    const int a = i + 1 == M ? 0 : i + 1;
    w[i] = std::hypot(min_image(X[a] - X[i], L), min_image(X[M + a] - X[M + i], L));
  }
}

template <typename P>
static ibdl_status dalloc(P** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  IBDL_CUDA(cudaMalloc((void**)p, bytes));
  return IBDL_OK;
}

static void free_geometry(Geometry* g) {
  if (!g) return;
  void* ptrs[] = {g->perm, g->base, g->cell_start, g->t64.phi, g->t64.dphi, g->t64.wscale, g->t64.nrm,
                  g->t32.phi, g->t32.dphi, g->t32.wscale, g->t32.nrm, g->spec, g->tw64, g->tw32,
                  g->lap64, g->der64, g->lap32, g->der32, g->ubuf, g->tmp_m, g->V, g->gm, g->vec,
                  g->ddphi64, g->vjp_buf, g->X64, g->pp_buf, g->src_buf, g->twff, g->lapff, g->derff};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int i = 0; i < 4; ++i)
    if (g->cycle_exec[i]) cudaGraphExecDestroy(g->cycle_exec[i]);
  if (g->host_status) cudaFreeHost(g->host_status);
  if (g->err_host) cudaFreeHost(g->err_host);
  if (g->ev) cudaEventDestroy(g->ev);
  if (g->ev_pool) {
    for (int i = 0; i < g->ev_cap; ++i) cudaEventDestroy(g->ev_pool[i]);
    delete[] g->ev_pool;
    delete[] g->ev_stage;
  }
  delete g;
}

void timing_mark(Geometry* g, cudaStream_t s, int stage) {
  if (!g->ev_pool || g->ev_used >= g->ev_cap) return;
  // an interval needs its opening marker; drop a closing mark whose opener was not recorded
  if (stage >= 0 && g->ev_used == 0) return;
  cudaEventRecord(g->ev_pool[g->ev_used], s);
  g->ev_stage[g->ev_used] = stage;
  ++g->ev_used;
}

ibdl_status set_stage_timing(Geometry* g, int enable) {
  if (enable && !g->ev_pool) {
    const int cap = 16384;
    g->ev_pool = new cudaEvent_t[cap];
    g->ev_stage = new int[cap];
    for (int i = 0; i < cap; ++i) {
      cudaError_t e = cudaEventCreate(&g->ev_pool[i]);
      if (e != cudaSuccess) {
        for (int j = 0; j < i; ++j) cudaEventDestroy(g->ev_pool[j]);
        delete[] g->ev_pool;
        delete[] g->ev_stage;
        g->ev_pool = nullptr;
        g->ev_stage = nullptr;
        return cuda_fail(e, "cudaEventCreate");
      }
    }
    g->ev_cap = cap;
  }
  g->ev_used = 0;
  g->timing = enable ? 1 : 0;
  return IBDL_OK;
}

ibdl_status get_stage_times(Geometry* g, double* ms, int64_t* launches) {
  for (int k = 0; k < IBDL_STAGE_COUNT; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  if (!g->ev_pool || g->ev_used == 0) return IBDL_OK;
  IBDL_CUDA(cudaEventSynchronize(g->ev_pool[g->ev_used - 1]));
  for (int i = 1; i < g->ev_used; ++i) {
    const int st = g->ev_stage[i];
    if (st < 0 || st >= IBDL_STAGE_COUNT) continue;
    float t = 0.f;
    IBDL_CUDA(cudaEventElapsedTime(&t, g->ev_pool[i - 1], g->ev_pool[i]));
    ms[st] += t;
    launches[st] += 1;
  }
  g->ev_used = 0;
  return IBDL_OK;
}

ibdl_status destroy_geometry(Geometry* g) {
  if (!g) return IBDL_OK;
  cudaDeviceSynchronize();
  free_geometry(g);
  return IBDL_OK;
}

ibdl_status create_geometry(const ibdl_geometry_desc* d, cudaStream_t s, Geometry** out) {
  if (!d || !out) return fail(IBDL_ERR_INVALID_ARG, "create_geometry: null descriptor or output");
  *out = nullptr;
  if (d->dim != 2 && d->dim != 3) return fail(IBDL_ERR_INVALID_ARG, "dim must be 2 or 3");
  const int nmax = d->dim == 2 ? 8192 : 256;
  if (!is_pow2(d->n) || d->n < 16 || d->n > nmax)
    return fail(IBDL_ERR_INVALID_ARG, "n must be a power of two in [16, " + std::to_string(nmax) + "]");
  if (!(d->box > 0) || !std::isfinite(d->box)) return fail(IBDL_ERR_INVALID_ARG, "box must be positive and finite");
  for (int j = 0; j < d->dim; ++j)
    if (!std::isfinite(d->origin[j])) return fail(IBDL_ERR_INVALID_ARG, "origin must be finite");
  if (d->n_points < 1 || d->n_points > (int64_t)1 << 28) return fail(IBDL_ERR_INVALID_ARG, "n_points must be in [1, 2^28]");
  if (!d->X) return fail(IBDL_ERR_INVALID_ARG, "X is required");
  if ((!d->normals || !d->weights) && (d->dim != 2 || d->n_points < 3))
    return fail(IBDL_ERR_INVALID_ARG, "normals and weights are required in 3-D and for fewer than three points");
  if (d->pde != IBDL_PDE_SCALAR && d->pde != IBDL_PDE_STOKES) return fail(IBDL_ERR_INVALID_ARG, "unknown pde");
  if (d->pde == IBDL_PDE_STOKES && d->dim != 2) return fail(IBDL_ERR_UNSUPPORTED, "Stokes is implemented in 2-D only");
  if (!(d->lambda >= 0) || !std::isfinite(d->lambda)) return fail(IBDL_ERR_INVALID_ARG, "lambda must be finite and >= 0");
  if (d->bc != IBDL_BC_DIRICHLET && d->bc != IBDL_BC_NEUMANN) return fail(IBDL_ERR_INVALID_ARG, "unknown boundary condition");
  if (d->bc == IBDL_BC_NEUMANN && d->pde != IBDL_PDE_SCALAR)
    return fail(IBDL_ERR_UNSUPPORTED, "Neumann conditions are implemented for the scalar PDE");
  if (!(d->eta >= 0) || !std::isfinite(d->eta)) return fail(IBDL_ERR_INVALID_ARG, "eta must be finite and >= 0");
  if (d->eta > 0 && (d->dim != 2 || d->lambda != 0 || d->dipole != IBDL_DIPOLE_ANALYTIC || d->bc != IBDL_BC_DIRICHLET))
    return fail(IBDL_ERR_UNSUPPORTED, "the completed method needs dim 2, lambda 0, the analytic dipole and Dirichlet data");
  if (d->pde == IBDL_PDE_STOKES && (!(d->mu > 0) || !std::isfinite(d->mu)))
    return fail(IBDL_ERR_INVALID_ARG, "mu must be finite and > 0");
  if (d->delta != IBDL_DELTA_COS && d->delta != IBDL_DELTA_SQRT) return fail(IBDL_ERR_INVALID_ARG, "unknown delta");
  if (d->dipole != IBDL_DIPOLE_ANALYTIC && d->dipole != IBDL_DIPOLE_SPECTRAL_DIV)
    return fail(IBDL_ERR_INVALID_ARG, "unknown dipole discretisation");
  if (d->symbol != IBDL_SYMBOL_SPECTRAL && d->symbol != IBDL_SYMBOL_FD2) return fail(IBDL_ERR_INVALID_ARG, "unknown symbol");

  const int dim = d->dim;
  const int M = (int)d->n_points;
  const double h = d->box / d->n;
  // host copies for validation (finite coordinates, unit normals, positive weights)
  std::vector<double> hX((size_t)dim * M), hN((size_t)dim * M), hW(M);
  const cudaMemcpyKind kind = d->inputs_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
  IBDL_CUDA(cudaMemcpy(hX.data(), d->X, hX.size() * sizeof(double), kind));
  if (d->normals)
    IBDL_CUDA(cudaMemcpy(hN.data(), d->normals, hN.size() * sizeof(double), kind));
  else
    estimate_normals(hX.data(), M, d->box, hN.data());
  if (d->weights)
    IBDL_CUDA(cudaMemcpy(hW.data(), d->weights, hW.size() * sizeof(double), kind));
  else
    estimate_weights(hX.data(), M, d->box, hW.data());
  for (int i = 0; i < M; ++i) {
    double nn = 0;
    for (int j = 0; j < dim; ++j) {
      const double x = hX[(size_t)j * M + i];
      if (!std::isfinite(x)) return fail(IBDL_ERR_NONFINITE, "non-finite boundary coordinate at point " + std::to_string(i));
      if (std::fabs((x - d->origin[j]) / h) > 1e9) return fail(IBDL_ERR_INVALID_ARG, "boundary point too far from the box");
      nn += hN[(size_t)j * M + i] * hN[(size_t)j * M + i];
    }
    if (!(std::fabs(nn - 1.0) < 1e-6)) return fail(IBDL_ERR_INVALID_ARG, "normal " + std::to_string(i) + " is not a unit vector");
    if (!(hW[i] > 0) || !std::isfinite(hW[i])) return fail(IBDL_ERR_INVALID_ARG, "weights must be positive and finite");
  }

  Geometry* g = new Geometry();
  std::memset(g, 0, sizeof(Geometry));
  g->dim = dim;
  g->n = d->n;
  g->pde = d->pde;
  g->delta = d->delta;
  g->dipole = d->dipole;
  g->symbol = d->symbol;
  g->box = d->box;
  g->h = h;
  g->lambda = d->lambda;
  g->mu = d->mu;
  g->bc = d->bc;
  g->eta = d->eta;
  for (int j = 0; j < 3; ++j) g->origin[j] = j < dim ? d->origin[j] : 0.0;
  g->M = M;
  g->ncomp = d->pde == IBDL_PDE_STOKES ? dim : 1;
  g->naug = d->eta > 0 ? g->ncomp : 0;
  const bool sd = d->dipole == IBDL_DIPOLE_SPECTRAL_DIV;
  if (d->pde == IBDL_PDE_STOKES) {
    g->nf_in = sd ? 4 : 3;
    g->nf_out = 2;
  } else {
    g->nf_in = sd ? dim : 1;
    g->nf_out = sd ? dim : 1;  // the adjoint of the spectral divergence interpolates dim fields
  }
  const int n = g->n;
  g->ncell = dim == 2 ? n : n * n;
  size_t rows = (size_t)n;
  if (dim == 3) rows *= n;

  ibdl_status st = IBDL_OK;
  double *dX = nullptr, *dN = nullptr, *dW = nullptr;
  int *key = nullptr, *count = nullptr, *cursor = nullptr;
#define GTRY(call)                 \
  do {                             \
    st = (call);                   \
    if (st != IBDL_OK) goto fail_; \
  } while (0)
#define GCUDA(call)                                 \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) {                        \
      st = cuda_fail(e_, #call);                    \
      goto fail_;                                   \
    }                                               \
  } while (0)
  {
    GTRY(dalloc(&dX, sizeof(double) * dim * M));
    GTRY(dalloc(&dN, sizeof(double) * dim * M));
    GTRY(dalloc(&dW, sizeof(double) * M));
    GCUDA(cudaMemcpyAsync(dX, hX.data(), sizeof(double) * dim * M, cudaMemcpyHostToDevice, s));
    GCUDA(cudaMemcpyAsync(dN, hN.data(), sizeof(double) * dim * M, cudaMemcpyHostToDevice, s));
    GCUDA(cudaMemcpyAsync(dW, hW.data(), sizeof(double) * M, cudaMemcpyHostToDevice, s));
    GTRY(dalloc(&key, sizeof(int) * M));
    GTRY(dalloc(&count, sizeof(int) * g->ncell));
    GTRY(dalloc(&cursor, sizeof(int) * (g->ncell + 1)));
    GTRY(dalloc(&g->perm, sizeof(int) * M));
    GTRY(dalloc(&g->base, sizeof(int) * dim * M));
    GTRY(dalloc(&g->cell_start, sizeof(int) * (g->ncell + 1)));
    GTRY(dalloc(&g->t64.phi, sizeof(double) * dim * 4 * M));
    GTRY(dalloc(&g->t64.dphi, sizeof(double) * dim * 4 * M));
    GTRY(dalloc(&g->t64.wscale, sizeof(double) * M));
    GTRY(dalloc(&g->t64.nrm, sizeof(double) * dim * M));
    GTRY(dalloc(&g->ddphi64, sizeof(double) * dim * 4 * M));
    GTRY(dalloc(&g->t32.phi, sizeof(float) * dim * 4 * M));
    GTRY(dalloc(&g->t32.dphi, sizeof(float) * dim * 4 * M));
    GTRY(dalloc(&g->t32.wscale, sizeof(float) * M));
    GTRY(dalloc(&g->t32.nrm, sizeof(float) * dim * M));
    const int nf = g->nf_in > g->nf_out ? g->nf_in : g->nf_out;
    g->spec_bytes = (size_t)nf * rows * (n / 2) * sizeof(double2);
    GTRY(dalloc(&g->spec, g->spec_bytes));
    GTRY(dalloc(&g->tw64, sizeof(double2) * n));
    GTRY(dalloc(&g->tw32, sizeof(float2) * n));
    GTRY(dalloc(&g->lap64, sizeof(double) * n));
    GTRY(dalloc(&g->der64, sizeof(double) * n));
    GTRY(dalloc(&g->lap32, sizeof(float) * n));
    GTRY(dalloc(&g->der32, sizeof(float) * n));
    // float-float twiddles and symbols (2-D and 3-D)
    GTRY(dalloc(&g->twff, 2 * sizeof(ff) * n));
    GTRY(dalloc(&g->lapff, sizeof(ff) * n));
    GTRY(dalloc(&g->derff, sizeof(ff) * n));
    GTRY(dalloc(&g->tmp_m, sizeof(double) * (g->ncomp * M + g->ncomp)));  // room for ū / constraint rows

    const int tb = 256;
    GCUDA(cudaMemsetAsync(count, 0, sizeof(int) * g->ncell, s));
    k_point_keys<<<(M + tb - 1) / tb, tb, 0, s>>>(dim, n, M, dX, g->origin[0], g->origin[1], g->origin[2], h, key, count);
    k_scan<<<1, 1024, 0, s>>>(g->ncell, count, g->cell_start);
    GCUDA(cudaMemcpyAsync(cursor, g->cell_start, sizeof(int) * (g->ncell + 1), cudaMemcpyDeviceToDevice, s));
    k_scatter<<<(M + tb - 1) / tb, tb, 0, s>>>(M, key, cursor, g->perm);
    k_sort_cells<<<(g->ncell + tb - 1) / tb, tb, 0, s>>>(g->ncell, g->cell_start, g->perm);
    k_tables<<<(M + tb - 1) / tb, tb, 0, s>>>(dim, n, M, g->delta, dX, dN, dW, g->origin[0], g->origin[1],
                                               g->origin[2], h, g->perm, g->base, g->t64, g->t32, g->ddphi64);
    k_twiddles<<<(n + tb - 1) / tb, tb, 0, s>>>(n, g->tw64, g->tw32);
    k_symbols<<<(n + tb - 1) / tb, tb, 0, s>>>(n, g->box, g->symbol, g->lap64, g->der64, g->lap32, g->der32);
    if (g->twff)
      k_ff_tables<<<(n + tb - 1) / tb, tb, 0, s>>>(n, g->tw64, g->lap64, g->der64, static_cast<ff*>(g->twff),
                                                    static_cast<ff*>(g->lapff), static_cast<ff*>(g->derff));
    GCUDA(cudaGetLastError());
    GCUDA(cudaStreamSynchronize(s));
    GCUDA(cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming));
    // the flag of the staged column pass's bounded waits, written by the device only on failure
    GCUDA(cudaHostAlloc((void**)&g->err_host, sizeof(int), cudaHostAllocMapped));
    *g->err_host = 0;
    GCUDA(cudaHostGetDevicePointer((void**)&g->err_dev, g->err_host, 0));
    GTRY(dim == 2 ? plan_2d(g) : plan_3d(g));
  }
  g->X64 = dX;  // kept: the near-boundary interpolation decides on the caller's coordinates
  cudaFree(dN);
  cudaFree(dW);
  cudaFree(key);
  cudaFree(count);
  cudaFree(cursor);
  *out = g;
  return IBDL_OK;
fail_:
  cudaStreamSynchronize(s);
  if (dX) cudaFree(dX);
  if (dN) cudaFree(dN);
  if (dW) cudaFree(dW);
  if (key) cudaFree(key);
  if (count) cudaFree(count);
  if (cursor) cudaFree(cursor);
  free_geometry(g);
  return st;
#undef GTRY
#undef GCUDA
}

}  // namespace ibdl
