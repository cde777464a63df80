// Solution post-processing: flagging the region enclosed by the immersed boundary (Sec. 5.3.5)
// and the linear interpolation that replaces grid values near Γ (Sec. 5.3.4).
//
// Indicator. χ solves Δχ = −S̃1: the IBDL grid field of the unit density for the plain Laplace
// problem (mean-zero inverse), with the geometry's δ_h, dipole spread and symbol. In the
// continuum χ = 1_enclosed − |enclosed|/|C|; subtracting the value at the box corner leaves ≈ 1
// inside the curves and ≈ 0 outside (≈ −1 inside for inward normals), and the flags are |χ| > ½.
//
// Near-boundary interpolation (2-D). A node x_p of the caller's mask Ω whose nearest boundary
// point lies closer than m1·h takes
//     u(x_p) = u_A |x_B − x_p|/|x_B − x_A| + u_B |x_A − x_p|/|x_B − x_A|,
// with x_A the point of the chord of its two nearest boundary points closest to x_p (if that
// projection leaves the chord: the chord of the two of the three nearest points that lie
// farthest apart, the projection clamped to it), u_A the linear interpolation of U_b along the
// chord, x_B = x_A + m2·h (x_p − x_A)/|x_p − x_A| and u_B the bilinear interpolation of the grid
// values around x_B. Which nodes are replaced and which boundary points are nearest are integer
// decisions: they are taken on FP64 squared minimum-image distances dx·dx + dy·dy, each
// operation rounded on its own (no contraction), equal distances ordered by point index.
//
// Kernels (the interpolation): k_mark flags the nodes within ceil(m1) + 2 cells of some point
// (a superset of the nodes to replace), k_compact lists the flagged nodes of Ω, and k_near
// gives each listed node one warp. The warp scans the points whose cell row lies within K rows
// of the node (rows of the geometry's cell-sorted order), keeps the three nearest per lane,
// merges them across the warp, and rescans all M points when the row slab cannot guarantee the
// result (the third distance not below (K − 1)·h).
#include <math_constants.h>

#include <climits>
#include <cmath>

#include "fft.cuh"

namespace ibdl {

namespace {

constexpr int kPPThreads = 256;

__global__ void k_fill(double* __restrict__ p, int64_t n, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void k_indicator_shift(const double* __restrict__ raw, int64_t cells, double* __restrict__ chi,
                                  uint8_t* __restrict__ flags) {
  const double corner = raw[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cells; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = raw[i] - corner;
    chi[i] = v;
    flags[i] = fabs(v) > 0.5 ? 1 : 0;
  }
}

__device__ __forceinline__ int wrapn(long long v, int n) {
  long long r = v % n;
  return (int)(r < 0 ? r + n : r);
}

// flag every node within k1 cells (per axis) of a point's first stencil node + 1
__global__ void k_mark(int n, int M, int k1, const int* __restrict__ base, uint8_t* __restrict__ marks) {
  const int w = 2 * k1 + 1;
  const int64_t items = (int64_t)M * w * w;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < items; t += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(t / (w * w));
    const int o = (int)(t - (int64_t)s * w * w);
    const int ix = wrapn((long long)base[s] + 1 - k1 + o % w, n);
    const int iy = wrapn((long long)base[M + s] + 1 - k1 + o / w, n);
    marks[(size_t)iy * n + ix] = 1;
  }
}

// list the marked nodes of Ω (warp-aggregated append; the list order is irrelevant)
__global__ void k_compact(int64_t cells, const uint8_t* __restrict__ marks, const uint8_t* __restrict__ omega,
                          int* __restrict__ list, int* __restrict__ count) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) - lane; b < cells; b += stride) {
    const int64_t i = b + lane;
    const bool take = i < cells && marks[i] && omega[i];
    const unsigned m = __ballot_sync(0xffffffffu, take);
    if (!m) continue;
    int at = 0;
    if (lane == 0) at = atomicAdd(count, __popc(m));
    at = __shfl_sync(0xffffffffu, at, 0);
    if (take) list[at + __popc(m & ((1u << lane) - 1u))] = (int)i;
  }
}

struct NearParams {
  int n, M, c, K;
  double h, L, o0, o1;
  double r1sq;    // (m1·h)²
  double slabsq;  // ((K − 1)·h)²: a slab result is exact when its third distance is below this
  double m2h;     // m2·h
  const double* X;         // [2][M] original order
  const int* perm;         // sorted position → original index
  const int* cell_start;   // [n + 1] rows of constant base y
  const double* Ub;        // [c][M]
  const double* u;         // [c][n][n]
  double* out;             // [c][n][n]
  const int* list;
  const int* count;
};

// minimum-image offset d − L·rint(d/L), each operation rounded on its own
__device__ __forceinline__ double mimg(double d, double L) {
  return __dsub_rn(d, __dmul_rn(L, rint(__ddiv_rn(d, L))));
}

__device__ __forceinline__ bool lex_less(double da, int ia, double db, int ib) {
  return da < db || (da == db && ia < ib);
}

struct Top3 {
  double d[3];
  int i[3];
  __device__ void init() {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      d[k] = CUDART_INF;
      i[k] = INT_MAX;
    }
  }
  __device__ void insert(double dd, int ii) {
    if (!lex_less(dd, ii, d[2], i[2])) return;
    if (lex_less(dd, ii, d[1], i[1])) {
      d[2] = d[1];
      i[2] = i[1];
      if (lex_less(dd, ii, d[0], i[0])) {
        d[1] = d[0];
        i[1] = i[0];
        d[0] = dd;
        i[0] = ii;
      } else {
        d[1] = dd;
        i[1] = ii;
      }
    } else {
      d[2] = dd;
      i[2] = ii;
    }
  }
};

__device__ __forceinline__ void offset(const NearParams& p, int i, double px, double py, double& dx, double& dy) {
  dx = mimg(__dsub_rn(p.X[i], px), p.L);
  dy = mimg(__dsub_rn(p.X[p.M + i], py), p.L);
}

__device__ __forceinline__ double sqdist(double dx, double dy) { return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)); }

// lanes scan sorted positions [a, b) into their own three nearest
__device__ __forceinline__ void scan_range(const NearParams& p, int a, int b, int lane, double px, double py, Top3& t) {
  for (int s = a + lane; s < b; s += 32) {
    const int i = p.perm[s];
    double dx, dy;
    offset(p, i, px, py, dx, dy);
    t.insert(sqdist(dx, dy), i);
  }
}

// the warp's three nearest (d², index), in every lane
__device__ __forceinline__ void warp_top3(const Top3& t, int lane, double* d, int* idx) {
  int ptr = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double bd = ptr < 3 ? t.d[ptr] : CUDART_INF;
    int bi = ptr < 3 ? t.i[ptr] : INT_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double od = __shfl_xor_sync(0xffffffffu, bd, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (lex_less(od, oi, bd, bi)) {
        bd = od;
        bi = oi;
      }
    }
    d[k] = bd;
    idx[k] = bi;
    if (ptr < 3 && t.i[ptr] == bi && bi != INT_MAX) ++ptr;
  }
}

__device__ __forceinline__ double dot2(double ax, double ay, double bx, double by) {
  return __dadd_rn(__dmul_rn(ax, bx), __dmul_rn(ay, by));
}

__global__ void __launch_bounds__(kPPThreads) k_near(NearParams p) {
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  const int count = *p.count;
  const int n = p.n;
  for (int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < count; w += warps) {
    const int node = p.list[w];
    const int ix = node % n, iy = node / n;
    const double px = __dadd_rn(p.o0, __dmul_rn(p.h, (double)ix));
    const double py = __dadd_rn(p.o1, __dmul_rn(p.h, (double)iy));
    Top3 t;
    t.init();
    const bool whole = 2 * p.K + 3 >= n;
    if (whole) {
      scan_range(p, 0, p.M, lane, px, py, t);
    } else {
      const int lo = iy - p.K - 2, hi = iy + p.K + 1;  // cell rows [lo, hi), wrapped
      if (lo < 0) {
        scan_range(p, p.cell_start[lo + n], p.cell_start[n], lane, px, py, t);
        scan_range(p, p.cell_start[0], p.cell_start[hi], lane, px, py, t);
      } else if (hi > n) {
        scan_range(p, p.cell_start[lo], p.cell_start[n], lane, px, py, t);
        scan_range(p, p.cell_start[0], p.cell_start[hi - n], lane, px, py, t);
      } else {
        scan_range(p, p.cell_start[lo], p.cell_start[hi], lane, px, py, t);
      }
    }
    double d3[3];
    int i3[3];
    warp_top3(t, lane, d3, i3);
    if (!(d3[0] < p.r1sq)) continue;  // not within m1·h of Γ (a point beyond the slab is farther still)
    if (!whole && !(d3[2] < p.slabsq)) {
      t.init();
      scan_range(p, 0, p.M, lane, px, py, t);
      warp_top3(t, lane, d3, i3);
    }
    if (lane != 0) continue;
    // offsets of the three nearest from x_p (x_p at the origin)
    double dx[3], dy[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) offset(p, i3[k], px, py, dx[k], dy[k]);
    int a = 0, b = 1;
    double sx = __dsub_rn(dx[a], dx[b]), sy = __dsub_rn(dy[a], dy[b]);
    double tt = -__ddiv_rn(dot2(dx[b], dy[b], sx, sy), dot2(sx, sy, sx, sy));
    if (tt < 0.0 || tt > 1.0) {
      // the pair of the three nearest that lies farthest apart
      const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
      double best = -1.0;
      for (int q = 0; q < 3; ++q) {
        const double ex = __dsub_rn(dx[pa[q]], dx[pb[q]]), ey = __dsub_rn(dy[pa[q]], dy[pb[q]]);
        const double sep = sqdist(ex, ey);
        if (sep > best) {
          best = sep;
          a = pa[q];
          b = pb[q];
        }
      }
      sx = __dsub_rn(dx[a], dx[b]);
      sy = __dsub_rn(dy[a], dy[b]);
      tt = -__ddiv_rn(dot2(dx[b], dy[b], sx, sy), dot2(sx, sy, sx, sy));
      tt = fmin(1.0, fmax(0.0, tt));
    }
    const double ax_ = dx[b] + tt * sx, ay_ = dy[b] + tt * sy;  // x_A − x_p
    const double lseg = hypot(sx, sy);
    const double wa1 = hypot(ax_ - dx[b], ay_ - dy[b]) / lseg;  // weight of U_b(x_1)
    const double wa2 = hypot(ax_ - dx[a], ay_ - dy[a]) / lseg;  // weight of U_b(x_2)
    const double rA = hypot(ax_, ay_);
    const int i1 = i3[a], i2 = i3[b];
    const size_t cells = (size_t)n * n;
    if (rA == 0.0) {
      for (int c = 0; c < p.c; ++c)
        p.out[c * cells + node] = p.Ub[(size_t)c * p.M + i1] * wa1 + p.Ub[(size_t)c * p.M + i2] * wa2;
      continue;
    }
    const double bx = ax_ - ax_ / rA * p.m2h, by = ay_ - ay_ / rA * p.m2h;  // x_B − x_p
    const double gx = (px + bx - p.o0) / p.h, gy = (py + by - p.o1) / p.h;
    const double fx = floor(gx), fy = floor(gy);
    const double wx = gx - fx, wy = gy - fy;
    const int jx0 = wrapn((long long)fx, n), jy0 = wrapn((long long)fy, n);
    const int jx1 = jx0 + 1 == n ? 0 : jx0 + 1, jy1 = jy0 + 1 == n ? 0 : jy0 + 1;
    const double rB = hypot(bx, by);
    for (int c = 0; c < p.c; ++c) {
      const double* F = p.u + c * cells;
      const double uA = p.Ub[(size_t)c * p.M + i1] * wa1 + p.Ub[(size_t)c * p.M + i2] * wa2;
      const double uB = (1 - wx) * (1 - wy) * F[(size_t)jy0 * n + jx0] + wx * (1 - wy) * F[(size_t)jy0 * n + jx1] +
                        (1 - wx) * wy * F[(size_t)jy1 * n + jx0] + wx * wy * F[(size_t)jy1 * n + jx1];
      p.out[c * cells + node] = (uA * rB + uB * rA) / p.m2h;
    }
  }
}

int pp_blocks(int64_t items) {
  const int64_t b = (items + kPPThreads - 1) / kPPThreads;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// scratch: ones [M] | raw field [n^d] | marks [n²] bytes | list [n²] | count
ibdl_status pp_workspace(Geometry* g, double** ones, double** raw, uint8_t** marks, int** list, int** count) {
  size_t cells = (size_t)g->n * g->n;
  if (g->dim == 3) cells *= g->n;
  const size_t b_ones = align256(sizeof(double) * g->M), b_raw = align256(sizeof(double) * cells);
  const size_t b_marks = g->dim == 2 ? align256(cells) : 0, b_list = g->dim == 2 ? align256(sizeof(int) * cells) : 0;
  const size_t need = b_ones + b_raw + b_marks + b_list + 256;
  if (!g->pp_buf) {
    IBDL_CUDA(cudaMalloc(&g->pp_buf, need));
    g->pp_bytes = need;
  }
  char* p = static_cast<char*>(g->pp_buf);
  *ones = reinterpret_cast<double*>(p);
  *raw = reinterpret_cast<double*>(p + b_ones);
  *marks = reinterpret_cast<uint8_t*>(p + b_ones + b_raw);
  *list = reinterpret_cast<int*>(p + b_ones + b_raw + b_marks);
  *count = reinterpret_cast<int*>(p + b_ones + b_raw + b_marks + b_list);
  return IBDL_OK;
}

}  // namespace

ibdl_status indicator_impl(Geometry* g, double* chi, uint8_t* flags, cudaStream_t s) {
  double *ones, *raw;
  uint8_t* marks;
  int *list, *count;
  IBDL_TRY(pp_workspace(g, &ones, &raw, &marks, &list, &count));
  int64_t cells = (int64_t)g->n * g->n;
  if (g->dim == 3) cells *= g->n;
  k_fill<<<pp_blocks(g->M), kPPThreads, 0, s>>>(ones, g->M, 1.0);
  IBDL_CUDA(cudaGetLastError());
  IBDL_TRY(g->dim == 2 ? laplace_field_2d(g, ones, raw, s) : laplace_field_3d(g, ones, raw, s));
  k_indicator_shift<<<pp_blocks(cells), kPPThreads, 0, s>>>(raw, cells, chi, flags);
  g->launches += 2;
  IBDL_CUDA(cudaGetLastError());
  return IBDL_OK;
}

ibdl_status near_boundary_impl(Geometry* g, const double* Ub, const double* u, const uint8_t* omega, double m1,
                               double m2, double* out, cudaStream_t s) {
  double *ones, *raw;
  uint8_t* marks;
  int *list, *count;
  IBDL_TRY(pp_workspace(g, &ones, &raw, &marks, &list, &count));
  const int n = g->n;
  const int64_t cells = (int64_t)n * n;
  IBDL_CUDA(cudaMemcpyAsync(out, u, sizeof(double) * g->ncomp * cells, cudaMemcpyDeviceToDevice, s));
  IBDL_CUDA(cudaMemsetAsync(marks, 0, cells, s));
  IBDL_CUDA(cudaMemsetAsync(count, 0, sizeof(int), s));
  const int k1 = (int)std::ceil(m1) + 2;
  k_mark<<<pp_blocks((int64_t)g->M * (2 * k1 + 1) * (2 * k1 + 1)), kPPThreads, 0, s>>>(n, (int)g->M, k1, g->base,
                                                                                        marks);
  k_compact<<<pp_blocks(cells), kPPThreads, 0, s>>>(cells, marks, omega, list, count);
  NearParams p;
  p.n = n;
  p.M = (int)g->M;
  p.c = g->ncomp;
  p.K = (int)std::ceil(m1) + 4;
  p.h = g->h;
  p.L = g->box;
  p.o0 = g->origin[0];
  p.o1 = g->origin[1];
  const double r1 = m1 * g->h;
  p.r1sq = r1 * r1;
  const double slab = (p.K - 1) * g->h;
  p.slabsq = slab * slab;
  p.m2h = m2 * g->h;
  p.X = g->X64;
  p.perm = g->perm;
  p.cell_start = g->cell_start;
  p.Ub = Ub;
  p.u = u;
  p.out = out;
  p.list = list;
  p.count = count;
  k_near<<<152 * 4, kPPThreads, 0, s>>>(p);
  g->launches += 3;
  IBDL_CUDA(cudaGetLastError());
  return IBDL_OK;
}

}  // namespace ibdl
