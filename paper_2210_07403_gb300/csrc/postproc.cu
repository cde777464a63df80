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
// takes the listed nodes in batches of kNearBatch per warp. For each node in turn the warp scans
// the points whose cell row lies within K rows of the node (rows of the geometry's cell-sorted
// order), keeps the three nearest per lane, merges them across the warp, and rescans all M
// points when the row slab cannot guarantee the result (the third distance not below
// W = (K − 1)·h); lane k keeps node k's result and finally interpolates it. Within the slab a point
// whose |dx| is not below W is dropped after one FP64 subtraction and an integer comparison; the
// distance comparisons run on the integer pipe (non-negative doubles order as their bits), so the
// FP64 unit only forms the distances.
#include <climits>
#include <cmath>
#include <cstring>

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
  unsigned long long r1key;    // bits of (m1·h)²
  unsigned long long slabkey;  // bits of W², W = (K − 1)·h: a slab result is exact when its third
                               // distance is below W
  unsigned long long slabbits, halfbits;  // bits of W and of L/2
  double halfL;
  double m2h;                  // m2·h
  const double* X;             // [2][M] original order
  const int* perm;             // sorted position → original index
  const int* cell_start;       // [n + 1] rows of constant base y
  const double* Ub;            // [c][M]
  const double* u;             // [c][n][n]
  double* out;                 // [c][n][n]
  const int* list;
  const int* count;
};

// Non-negative doubles order as their bit patterns (as unsigned integers), so distances are
// compared on the integer pipe: the FP64 unit, the bound of this kernel, only forms them.
__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ __forceinline__ unsigned long long absbits(double v) { return dbits(v) & 0x7fffffffffffffffull; }

// minimum-image offset d − L·rint(d/L), each operation rounded on its own
__device__ __forceinline__ double mimg(double d, double L) {
  return __dsub_rn(d, __dmul_rn(L, rint(__ddiv_rn(d, L))));
}

// the same for |d| < L/2 without the division: d/L then rounds to a value of magnitude ≤ ½,
// which rounds to zero (ties to even), and the formula returns d
__device__ __forceinline__ double mimg_fast(double d, const NearParams& p) {
  return absbits(d) < p.halfbits ? d : mimg(d, p.L);
}

__device__ __forceinline__ double sqdist(double dx, double dy) { return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)); }

__device__ __forceinline__ bool key_less(unsigned long long ka, int ia, unsigned long long kb, int ib) {
  return ka < kb || (ka == kb && ia < ib);
}

constexpr unsigned long long kInfKey = 0x7ff0000000000000ull;  // +∞

// a lane's three nearest, (squared-distance bits, index) ascending
struct Top3 {
  unsigned long long k0, k1, k2;
  int i0, i1, i2;
  __device__ void init() {
    k0 = k1 = k2 = kInfKey;
    i0 = i1 = i2 = INT_MAX;
  }
  __device__ void insert(unsigned long long k, int i) {
    if (!key_less(k, i, k2, i2)) return;
    if (key_less(k, i, k1, i1)) {
      k2 = k1;
      i2 = i1;
      if (key_less(k, i, k0, i0)) {
        k1 = k0;
        i1 = i0;
        k0 = k;
        i0 = i;
      } else {
        k1 = k;
        i1 = i;
      }
    } else {
      k2 = k;
      i2 = i;
    }
  }
};

// lanes scan sorted positions [a, b) into their own three nearest. With WINDOW a point whose |dx| is
// not below W is skipped: it is no nearer than W, and a slab result is kept only when its third
// distance is below W (otherwise every point is rescanned without the window)
template <bool WINDOW>
__device__ __forceinline__ void scan_range(const NearParams& p, int a, int b, int lane, double px, double py, Top3& t) {
  for (int s = a + lane; s < b; s += 32) {
    const int i = p.perm[s];
    const double dx = mimg_fast(__dsub_rn(p.X[i], px), p);
    if (WINDOW && absbits(dx) >= p.slabbits) continue;
    const double dy = mimg_fast(__dsub_rn(p.X[p.M + i], py), p);
    t.insert(dbits(sqdist(dx, dy)), i);
  }
}

// the warp's three nearest, in every lane: three rounds of a butterfly minimum over the lanes'
// heads; the lane whose head wins pops it
__device__ __forceinline__ void warp_top3(Top3 t, unsigned long long* key, int* idx) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    unsigned long long bk = t.k0;
    int bi = t.i0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (key_less(ok, oi, bk, bi)) {
        bk = ok;
        bi = oi;
      }
    }
    key[r] = bk;
    idx[r] = bi;
    if (t.i0 == bi && bi != INT_MAX) {
      t.k0 = t.k1;
      t.i0 = t.i1;
      t.k1 = t.k2;
      t.i1 = t.i2;
      t.k2 = kInfKey;
      t.i2 = INT_MAX;
    }
  }
}

__device__ __forceinline__ double dot2(double ax, double ay, double bx, double by) {
  return __dadd_rn(__dmul_rn(ax, bx), __dmul_rn(ay, by));
}

__device__ __forceinline__ double node_x(const NearParams& p, int i) { return __dadd_rn(p.o0, __dmul_rn(p.h, (double)i)); }
__device__ __forceinline__ double node_y(const NearParams& p, int i) { return __dadd_rn(p.o1, __dmul_rn(p.h, (double)i)); }

// the interpolated value(s) of one node from its three nearest boundary points (original indices)
__device__ void near_tail(const NearParams& p, int node, const int* i3) {
  const int n = p.n;
  const int ix = node % n, iy = node / n;
  const double px = node_x(p, ix), py = node_y(p, iy);
  double dx[3], dy[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dx[k] = mimg_fast(__dsub_rn(p.X[i3[k]], px), p);
    dy[k] = mimg_fast(__dsub_rn(p.X[p.M + i3[k]], py), p);
  }
  int a = 0, b = 1;
  double sx = __dsub_rn(dx[0], dx[1]), sy = __dsub_rn(dy[0], dy[1]);
  double tt = -__ddiv_rn(dot2(dx[1], dy[1], sx, sy), dot2(sx, sy, sx, sy));
  if (tt < 0.0 || tt > 1.0) {
    // the pair of the three nearest that lies farthest apart (the first of equal ones)
    const double s01 = sqdist(__dsub_rn(dx[0], dx[1]), __dsub_rn(dy[0], dy[1]));
    const double s02 = sqdist(__dsub_rn(dx[0], dx[2]), __dsub_rn(dy[0], dy[2]));
    const double s12 = sqdist(__dsub_rn(dx[1], dx[2]), __dsub_rn(dy[1], dy[2]));
    if (s02 > s01 && s02 >= s12) {
      b = 2;
    } else if (s12 > s01 && s12 > s02) {
      a = 1;
      b = 2;
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
    return;
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

// Each warp takes kNearBatch listed nodes at a time: for each in turn all lanes scan its candidate
// points and merge; lane k keeps node k's three nearest. Then lanes 0..kNearBatch−1 each finish
// their own node, so the FP64 arithmetic of the interpolation runs on many lanes instead of one.
// The warp's nodes are scanned one after another (a latency-bound chain), so the batch trades the
// chain's length against the lanes the interpolation keeps busy; adjacent batches stay in one block
// (they share slab points in L1).
constexpr int kNearBatch = 16;
__global__ void __launch_bounds__(kPPThreads, 2) k_near(NearParams p) {
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int warps = gridDim.x * (blockDim.x >> 5);
  const int count = *p.count;
  const int n = p.n;
  const bool whole = 2 * p.K + 3 >= n;
  for (int base = gw * kNearBatch; base < count; base += warps * kNearBatch) {
    const int nb = min(kNearBatch, count - base);
    int mine[3] = {-1, -1, -1};
    for (int k = 0; k < nb; ++k) {
      const int node = p.list[base + k];
      const int ix = node % n, iy = node / n;
      const double px = node_x(p, ix), py = node_y(p, iy);
      Top3 t;
      t.init();
      if (whole) {
        scan_range<false>(p, 0, p.M, lane, px, py, t);
      } else {
        const int lo = iy - p.K - 2, hi = iy + p.K + 1;  // cell rows [lo, hi), wrapped
        if (lo < 0) {
          scan_range<true>(p, p.cell_start[lo + n], p.cell_start[n], lane, px, py, t);
          scan_range<true>(p, p.cell_start[0], p.cell_start[hi], lane, px, py, t);
        } else if (hi > n) {
          scan_range<true>(p, p.cell_start[lo], p.cell_start[n], lane, px, py, t);
          scan_range<true>(p, p.cell_start[0], p.cell_start[hi - n], lane, px, py, t);
        } else {
          scan_range<true>(p, p.cell_start[lo], p.cell_start[hi], lane, px, py, t);
        }
      }
      unsigned long long key[3];
      int idx[3];
      warp_top3(t, key, idx);
      // not within m1·h of Γ (a point beyond the slab or the window is farther still)
      if (!(key[0] < p.r1key)) continue;
      if (!whole && !(key[2] < p.slabkey)) {
        t.init();
        scan_range<false>(p, 0, p.M, lane, px, py, t);
        warp_top3(t, key, idx);
      }
      if (lane == k) {
        mine[0] = idx[0];
        mine[1] = idx[1];
        mine[2] = idx[2];
      }
    }
    if (mine[0] >= 0) near_tail(p, p.list[base + lane], mine);
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
  const double r1sq = r1 * r1;
  const double slab = (p.K - 1) * g->h;
  const double slabsq = slab * slab;
  p.halfL = 0.5 * g->box;
  std::memcpy(&p.r1key, &r1sq, 8);
  std::memcpy(&p.slabkey, &slabsq, 8);
  std::memcpy(&p.slabbits, &slab, 8);
  std::memcpy(&p.halfbits, &p.halfL, 8);
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
