// Device side of the three-dimensional IBDL operator (scalar PDE): A Q = S* u + ½Q,
// u = −L⁻¹ S̃ Q (Sec. 5.3.2; the method's formulation needs no change in 3-D, Sec. 1 and Sec. 7:
// area weights replace arclength weights and δ_h is the tensor product of three 4-point kernels),
// specialised on the grid size n = 2^L at compile time (one translation unit per size,
// apply3d_n*.cu).
//
// Five kernels per application, each owning a disjoint part of the grid:
//   k3_spread_rowfft   band of R y-rows at one z: spread (shared-memory atomics), FFT along x of
//                      row pairs packed as a + ib, packed half spectrum (slot 0 = (A_0, A_{n/2}))
//   k3_ypass<fwd>      C kx columns at one z: FFT along y, no symbol
//   k3_zpass           C kx columns at the y-frequencies ky and −ky: FFT along z, Fourier symbol,
//                      inverse FFT along z. The packed kx = 0 | kx = n/2 column holds P = Â + iB̂
//                      where Â, B̂ are Hermitian in (ky, kz); separating them needs P(−ky, −kz),
//                      which is why a CTA owns both ky and −ky.
//   k3_ypass<inv>      inverse FFT along y
//   k3_rowifft_gather  band of R y-rows: inverse FFT along x, interpolation into Y (set to ½Q by
//                      the first kernel), or the grid itself.
// Layout: spec[f][z][y][kx], kx ∈ [0, n/2), rows z·n + y. The transforms are the register FFT of
// fft8.cuh (the 2-D kernels' transform): a thread holds eight elements of one lane of a sequence,
// kThreads3/QT sequences per pass, each sequence in its padded shared-memory buffer (sequence b at
// b·(n + n/8), the layout the spread's accumulation and the gather's sums index with pidx).
#pragma once

#include <cstdlib>
#include <type_traits>

#include <algorithm>
#include <atomic>
#include <utility>

#include "ff.cuh"
#include "fft.cuh"
#include "fft8.cuh"
#include "ibdl_internal.cuh"

namespace ibdl {

enum { OP3_SCALAR_AN = 0, OP3_SCALAR_SD = 1, OP3_ADJ_AN = 2, OP3_ADJ_SD = 3 };

template <int OP>
struct Traits3;
template <>
struct Traits3<OP3_SCALAR_AN> { static constexpr int NIN = 1, NOUT = 1; };  // f = S̃Q
template <>
struct Traits3<OP3_SCALAR_SD> { static constexpr int NIN = 3, NOUT = 1; };  // S(Q n_m), m = x, y, z
template <>
struct Traits3<OP3_ADJ_AN> { static constexpr int NIN = 1, NOUT = 1; };     // S W
template <>
struct Traits3<OP3_ADJ_SD> { static constexpr int NIN = 1, NOUT = 3; };     // S W → ∂_m v

enum { G3_INTERP = 0, G3_GRID = 1 };

// Point type of a grid arithmetic: the point tables, the spread's accumulation and the gather's
// sums. Float-float grids keep FP64 points (the spread accumulates in FP64 and converts each
// value once before the FFT; the gather sums in FP64), as in 2-D.
template <typename T>
struct Prec3 {
  using PT = T;
  static __device__ __forceinline__ PT to_pt(T v) { return v; }
};
template <>
struct Prec3<ff> {
  using PT = double;
  static __device__ __forceinline__ double to_pt(ff v) { return double(v); }
};
constexpr int kThreads3 = 256;

// element accessors of fft3_run: shared memory (the sequence's own padded buffer) or global
// memory through a column or row accessor with load(b, m) / store(b, m, v)
template <typename T>
struct SmemLd3 {
  __device__ __forceinline__ cplx<T> operator()(int, const cplx<T>* sb, int, int pos) const { return sb[pos]; }
};
template <typename T>
struct SmemSt3 {
  __device__ __forceinline__ void operator()(int, cplx<T>* sb, int, int pos, cplx<T> v) const { sb[pos] = v; }
};
template <class IO>
struct GlobLd3 {
  IO io;
  template <typename C>
  __device__ __forceinline__ C operator()(int b, const C*, int m, int) const { return io.load(b, m); }
};
template <class IO>
struct GlobSt3 {
  IO io;
  template <typename C>
  __device__ __forceinline__ void operator()(int b, C*, int m, int, C v) const { io.store(b, m, v); }
};

// The register FFT (fft8.cuh) of `nseq` sequences of length 2^L, sequence b exchanging through
// buf + b·(n + n/8): lane j of a sequence reads its elements j + s·Q through `ld` before the
// transform and writes their transforms through `st` after it. kThreads3/QT sequences per pass;
// every thread of the block calls it (the passes have the same count on every thread).
// Register FFT configuration of the 3-D transforms (n ≤ 256: one lane per thread); twiddles in
// registers when they fit the budget of the 2-D kernels (42 FP32, 56 FP64, 28 float-float
// registers), else read from the table at each use.
template <typename T, int L>
struct Cfg3 {
  static constexpr int V = 1;
  static constexpr int QT = (1 << L) / 8;
  static constexpr int NTW = F8<L, 1>::NTW;
  static constexpr bool TWR =
      sizeof(T) == 4 ? NTW <= 21 : (std::is_same<T, ff>::value ? NTW <= 7 : NTW <= 14);
  using TW = std::conditional_t<TWR, TwRegs<T, L>, TwTable<T, L>>;
};

// Stride (elements) between the exchange buffers of sequences interleaved across threads: the
// padded sequence rounded up to ≡ max(1, w/W) (mod w), w = 16 for 8-byte and 8 for 16-byte
// elements, W = min(32, the sequences of a pass) interleaved in a warp: the rule of the 2-D column
// groups, which puts the warp's sequences in different shared-memory banks.
__host__ __device__ constexpr int seq_stride3(int L, int esize) {
  const int pn = (1 << L) + (1 << L) / 8;
  const int sp = kThreads3 / ((1 << L) / 8);
  const int W = sp < 32 ? sp : 32;
  const int w = esize == 8 ? 16 : 8;
  const int t = (w / W > 1 ? w / W : 1) % w;
  return pn + (((t - pn) % w) + w) % w;
}

// IL: the sequences of a pass interleaved across threads (sequence = thread mod SP, lane = thread /
// SP), each exchanging through buf + b·seq_stride3: consecutive threads then touch the same
// element of consecutive sequences, which the column passes' global accesses want (adjacent kx
// columns are adjacent in memory). Otherwise sequence b is thread / QT, at buf + b·(n + n/8).
template <typename T, bool INV, int L, bool IL = false, class LD, class ST>
__device__ __forceinline__ void fft3_run(cplx<T>* buf, int nseq, const cplx<T>* __restrict__ twg, const LD& ld,
                                         const ST& st) {
  using CF = Cfg3<T, L>;
  using F = F8<L, CF::V>;
  constexpr int V = CF::V, QT = CF::QT, Q = F::Q, SP = kThreads3 / QT;
  static_assert(kThreads3 % QT == 0, "whole sequences per pass");
  constexpr int PS = IL ? seq_stride3(L, (int)sizeof(cplx<T>)) : F::PN;
  const int sl = IL ? (int)threadIdx.x % SP : (int)threadIdx.x / QT;
  const int j0 = IL ? (int)threadIdx.x / SP : (int)threadIdx.x - sl * QT;
  typename CF::TW tw[V];
#pragma unroll
  for (int v = 0; v < V; ++v) tw[v].load(twg, j0 + v * QT);
  for (int b0 = 0; b0 < nseq; b0 += SP) {
    const int b = b0 + sl;
    const bool act = b < nseq;
    cplx<T>* sb = buf + (size_t)(act ? b : 0) * PS;
    cplx<T> x[1][V][8];
    if (act) {
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int s = 0; s < 8; ++s)
          x[0][v][s] = ld(b, sb, j0 + v * QT + s * Q, ppos_strided<Q>(j0 + v * QT, s));
    }
    f8_fft<T, INV, L, V, 1>(x, sb, 0, j0, tw, act);
    if (act) {
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int s = 0; s < 8; ++s) st(b, sb, j0 + v * QT + s * Q, ppos_strided<Q>(j0 + v * QT, s), x[0][v][s]);
    }
  }
}

struct Row3Params {
  int n, log2n, R;
  int M;
  const int* cell_start;  // [n·n + 1], cell = base_z·n + base_y
  const int* base;        // [3][M]
  const int* perm;
  const void* phi;        // T [3][4][M]
  const void* dphi;
  const void* wscale;
  const void* nrm;        // T [3][M]
  const double* in;
  double* out;
  void* spec;
  const void* tw;
  const int* stop;
  double* grid;
  const int* idx;
  int vstride;
  // adjoint ops only: 1 = the Euclidean transpose Aᵀ = W A* W⁻¹ (λ spread with weight 1, gathered
  // values multiplied by Δs/h³ in place of the spread's Δs/h³ · W⁻¹)
  int trans;
  double jump;  // jump term coefficient: ½ (Dirichlet) or −½ (Neumann)
  const double* grid_in;  // optional [NIN][n][n][n]: the row bands are read from it instead of spread
};

struct Col3Params {
  int n, log2n, C, lc;
  int nf;        // fields transformed (y passes)
  double lam, scale;
  const void* lap1;
  const void* der1;
  void* spec;
  const void* tw;
  const int* stop;
};

__device__ __forceinline__ void resolve_io3(const Row3Params& p, const double*& in, double*& out) {
  in = p.in;
  out = p.out;
  if (p.idx) {
    const int k = *p.idx;
    in += (size_t)k * p.vstride;
    out += (size_t)(k + 1) * p.vstride;
  }
}

// Sorted points whose stencil meets the band of y-rows [y0, y0 + R) at plane z: cells (cz, cy)
// with cz ∈ {z−3, …, z} and cy ∈ [y0 − 3, y0 + R) (mod n): at most 8 contiguous ranges.
struct Ranges3 {
  int start[8], count[8];
  int nr, total;
  __device__ int at(int t) const {
    int r = 0;
    while (t >= count[r]) {
      t -= count[r];
      ++r;
    }
    return start[r] + t;
  }
};

__device__ __forceinline__ Ranges3 band_points3(const int* cell_start, int n, int z, int y0, int R) {
  Ranges3 rg;
  rg.nr = 0;
  rg.total = 0;
  for (int dz = -3; dz <= 0; ++dz) {
    const int cz = (z + dz + n) & (n - 1);
    const int lo = y0 - 3, hi = y0 + R;
    const int base = cz * n;
    if (lo >= 0) {
      const int a = cell_start[base + lo], b = cell_start[base + hi];
      rg.start[rg.nr] = a;
      rg.count[rg.nr] = b - a;
      rg.total += b - a;
      ++rg.nr;
    } else {
      const int a = cell_start[base + lo + n], b = cell_start[base + n];
      rg.start[rg.nr] = a;
      rg.count[rg.nr] = b - a;
      rg.total += b - a;
      ++rg.nr;
      const int c = cell_start[base], d = cell_start[base + hi];
      rg.start[rg.nr] = c;
      rg.count[rg.nr] = d - c;
      rg.total += d - c;
      ++rg.nr;
    }
  }
  for (int r = rg.nr; r < 8; ++r) rg.count[r] = 1 << 30;
  return rg;
}

// ------------------------------------------------------------------------------------------
// kernel 1: spread + FFT along x
// ------------------------------------------------------------------------------------------
template <typename T, int OP, int L>
__global__ void __launch_bounds__(kThreads3) k3_spread_rowfft(Row3Params p) {
  // programmatic launch: wait for the previous kernel, then let the next one launch; a GMRES
  // cycle's stop flag is read after the wait (the step just before may have written it)
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
  if (p.stop && *p.stop) return;
  constexpr int NIN = Traits3<OP>::NIN;
  constexpr int n = 1 << L;
  using PT = typename Prec3<T>::PT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int R = p.R, half = R >> 1, M = p.M;
  const int seqs = NIN * half;
  const PT* phi = static_cast<const PT*>(p.phi);
  const PT* dphi = static_cast<const PT*>(p.dphi);
  const PT* wsc = static_cast<const PT*>(p.wscale);
  const PT* nrm = static_cast<const PT*>(p.nrm);
  cplx<T>* spec = static_cast<cplx<T>*>(p.spec);
  cplx<T>* bufA = reinterpret_cast<cplx<T>*>(smem_raw);  // the padded sequences (field, row pair)
  PT* acc = reinterpret_cast<PT*>(bufA);  // (the same bytes per complex element as cplx<T>)
  const int bands = n / R;
  const int z = blockIdx.x / bands, y0 = (blockIdx.x - z * bands) * R;
  const double* pin;
  double* pout;
  resolve_io3(p, pin, pout);
  if (!p.grid_in)  // jump term: out = ±½·in (the gather adds S*u afterwards); none for grid input
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) pout[i] = p.jump * pin[i];
  for (int i = threadIdx.x; i < (int)padded((size_t)seqs * n) * 2; i += blockDim.x) acc[i] = PT(0);
  __syncthreads();

  if (p.grid_in) {  // rows of a grid field ([NIN][z][y][x]) in place of the spread
    for (int t = threadIdx.x; t < NIN * R * n; t += blockDim.x) {
      const int f = t / (R * n);
      const int rem = t - f * R * n;
      const int lr = rem / n, x = rem - lr * n;
      acc[2 * pidx((f * half + (lr >> 1)) * n + x) + (lr & 1)] =
          PT(p.grid_in[(((size_t)f * n + z) * n + y0 + lr) * n + x]);
    }
  }
  const Ranges3 rg = band_points3(p.cell_start, n, z, y0, R);
  // one thread per (point, stencil row ay): the point's plane and row weights and its density are
  // read once, then the four nodes along x of that row are added
  for (int t = threadIdx.x; t < (p.grid_in ? 0 : rg.total * 4); t += blockDim.x) {
    const int s = rg.at(t >> 2);
    const int ay = t & 3;
    const int az = (z - p.base[2 * M + s]) & (n - 1);  // the one stencil plane at z (0..3)
    const int row = (p.base[M + s] + ay) & (n - 1);
    const int lr = (row - y0) & (n - 1);
    if (lr >= R || az > 3) continue;
    const int i = p.perm[s];
    const int bx = p.base[s];
    const PT py = phi[(1 * 4 + ay) * M + s], pz = phi[(2 * 4 + az) * M + s];
    const PT ws = wsc[s];
    const int eb = (lr >> 1) * n;
    const int odd = lr & 1;
    const PT qv = PT(pin[i]);
    PT c0 = 0, cy = 0, cz = 0, n0 = 0, n1 = 0, n2 = 0;
    if (OP == OP3_SCALAR_AN) {
      // n·∇δ_h = n_x φ'(x)φ(y)φ(z) + n_y φ(x)φ'(y)φ(z) + n_z φ(x)φ(y)φ'(z): per node along x,
      // c0·φ'(x) + (cy + cz)·φ(x)
      n0 = nrm[s];
      n1 = nrm[M + s];
      n2 = nrm[2 * M + s];
      c0 = qv * ws * n0 * py * pz;
      cy = qv * ws * n1 * dphi[(1 * 4 + ay) * M + s] * pz;
      cz = qv * ws * n2 * py * dphi[(2 * 4 + az) * M + s];
    } else if (OP == OP3_SCALAR_SD) {
      n0 = nrm[s];
      n1 = nrm[M + s];
      n2 = nrm[2 * M + s];
      c0 = qv * ws * py * pz;
    } else {
      c0 = qv * (p.trans ? PT(1) : ws) * py * pz;  // A*: W with weight Δs/h³; Aᵀ: λ with weight 1
    }
#pragma unroll
    for (int ax = 0; ax < 4; ++ax) {
      const int e = eb + ((bx + ax) & (n - 1));
      const PT px = phi[(0 * 4 + ax) * M + s];
      if (OP == OP3_SCALAR_AN) {
        atomicAdd(acc + 2 * pidx(e) + odd, c0 * dphi[(0 * 4 + ax) * M + s] + (cy + cz) * px);
      } else if (OP == OP3_SCALAR_SD) {
        const PT q = c0 * px;
        atomicAdd(acc + 2 * pidx(e) + odd, q * n0);
        atomicAdd(acc + 2 * pidx(e + half * n) + odd, q * n1);
        atomicAdd(acc + 2 * pidx(e + 2 * half * n) + odd, q * n2);
      } else {
        atomicAdd(acc + 2 * pidx(e) + odd, c0 * px);
      }
    }
  }
  __syncthreads();
  if constexpr (!std::is_same<T, PT>::value) {
    // float-float: each FP64 accumulated value becomes the nearest float-float, in place
    for (int i = threadIdx.x; i < (int)padded((size_t)seqs * n); i += blockDim.x) {
      const double2 d = reinterpret_cast<const double2*>(bufA)[i];
      bufA[i] = mk(ff_from_double(d.x), ff_from_double(d.y));
    }
    __syncthreads();
  }
  fft3_run<T, false, L>(bufA, seqs, static_cast<const cplx<T>*>(p.tw), SmemLd3<T>(), SmemSt3<T>());
  __syncthreads();
  const cplx<T>* res = bufA;
  constexpr int nh = n >> 1, lnh = L - 1;
  for (int t = threadIdx.x; t < seqs * nh; t += blockDim.x) {
    const int sq = t >> lnh, k = t & (nh - 1);
    const int f = sq / half, j = sq - f * half;
    const int zb = sq * n;
    cplx<T> A, B;
    if (k == 0) {
      const cplx<T> z0 = res[pidx(zb)], zh = res[pidx(zb + nh)];
      A = mk(z0.x, zh.x);
      B = mk(z0.y, zh.y);
    } else {
      const cplx<T> zk = res[pidx(zb + k)], zc = res[pidx(zb + n - k)];
      A = mk(T(0.5) * (zk.x + zc.x), T(0.5) * (zk.y - zc.y));
      B = mk(T(0.5) * (zk.y + zc.y), T(0.5) * (zc.x - zk.x));
    }
    const size_t row = (size_t)z * n + y0 + 2 * j;
    spec[((size_t)f * n * n + row) * nh + k] = A;
    spec[((size_t)f * n * n + row + 1) * nh + k] = B;
  }
}

// ------------------------------------------------------------------------------------------
// kernel 2/4: FFT along y of C kx columns at one z, for nf fields (first and last stages read
// and write the half spectra directly)
// ------------------------------------------------------------------------------------------
template <typename T>
struct YColumnIO {
  cplx<T>* spec;
  int n, nh, z, k0, lc, C;
  __device__ __forceinline__ size_t at(int bi, int m) const {
    return (((size_t)(bi >> lc) * n + z) * n + m) * nh + k0 + (bi & (C - 1));
  }
  __device__ __forceinline__ cplx<T> load(int bi, int m) const { return spec[at(bi, m)]; }
  __device__ __forceinline__ void store(int bi, int m, cplx<T> v) const { spec[at(bi, m)] = v; }
};

template <typename T, bool INV, int L>
__global__ void __launch_bounds__(kThreads3) k3_ypass(Col3Params p) {
  // programmatic launch: wait for the previous kernel, then let the next one launch; a GMRES
  // cycle's stop flag is read after the wait (the step just before may have written it)
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
  if (p.stop && *p.stop) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int n = 1 << L, nh = n >> 1;
  const int C = p.C;
  const int groups = nh / C;
  const int z = blockIdx.x / groups, k0 = (blockIdx.x - z * groups) * C;
  cplx<T>* bufA = reinterpret_cast<cplx<T>*>(smem_raw);
  const YColumnIO<T> io{static_cast<cplx<T>*>(p.spec), n, nh, z, k0, p.lc, C};
  fft3_run<T, INV, L, true>(bufA, p.nf * C, static_cast<const cplx<T>*>(p.tw), GlobLd3<YColumnIO<T>>{io},
                            GlobSt3<YColumnIO<T>>{io});
}

// ------------------------------------------------------------------------------------------
// kernel 3: FFT along z, symbol, inverse FFT along z at (ky, −ky) × C kx columns
// ------------------------------------------------------------------------------------------
// sequence bi = (f·2 + q)·C + c: field f, y-frequency slot q (0: ky1, 1: ky2), column c
template <typename T>
struct ZColumnIO {
  cplx<T>* spec;
  int n, nh, ky1, ky2, k0, lc, C;
  __device__ __forceinline__ size_t at(int bi, int m) const {
    const int c = bi & (C - 1), fq = bi >> lc;
    const int f = fq >> 1, ky = (fq & 1) ? ky2 : ky1;
    return (((size_t)f * n + m) * n + ky) * nh + k0 + c;
  }
  __device__ __forceinline__ cplx<T> load(int bi, int m) const { return spec[at(bi, m)]; }
  // with ky1 = ky2 the q = 1 slots alias the q = 0 column and carry no symbol: never stored
  __device__ __forceinline__ void store(int bi, int m, cplx<T> v) const {
    if (ky1 == ky2 && ((bi >> lc) & 1)) return;
    spec[at(bi, m)] = v;
  }
};

template <typename T, int OP>
__device__ __forceinline__ void symbol3(const T* lap1, const T* der1, T lam, T scale, int kx, int ky, int kz,
                                        const cplx<T>* in, cplx<T>* out) {
  const T lap = lap1[kx] + lap1[ky] + lap1[kz];
  const T den = lap + lam;
  const T sig = den != T(0) ? scale / den : T(0);
  if (OP == OP3_SCALAR_AN || OP == OP3_ADJ_AN) {
    out[0] = cscale(in[0], sig);
  } else if (OP == OP3_SCALAR_SD) {
    const cplx<T> d = cadd(cadd(cscale(in[0], der1[kx]), cscale(in[1], der1[ky])), cscale(in[2], der1[kz]));
    out[0] = cscale(cmuli(d), sig);
  } else {
    const cplx<T> v = cmuli(cscale(in[0], sig));
    out[0] = cscale(v, der1[kx]);
    out[1] = cscale(v, der1[ky]);
    out[2] = cscale(v, der1[kz]);
  }
}

template <typename T, int OP, int L>
__global__ void __launch_bounds__(kThreads3) k3_zpass(Col3Params p) {
  // programmatic launch: wait for the previous kernel, then let the next one launch; a GMRES
  // cycle's stop flag is read after the wait (the step just before may have written it)
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
  if (p.stop && *p.stop) return;
  constexpr int NIN = Traits3<OP>::NIN;
  constexpr int NOUT = Traits3<OP>::NOUT;
  constexpr int NMAX = NIN > NOUT ? NIN : NOUT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int n = 1 << L, nh = n >> 1;
  const int C = p.C, lc = p.lc;
  const int groups = nh / C;
  const int pair = blockIdx.x / groups, k0 = (blockIdx.x - pair * groups) * C;
  const int ky1 = pair, ky2 = (n - pair) & (n - 1);
  const int nq = ky1 == ky2 ? 1 : 2;  // y-frequency columns in this CTA
  cplx<T>* bufA = reinterpret_cast<cplx<T>*>(smem_raw);
  constexpr int PS = seq_stride3(L, (int)sizeof(cplx<T>));  // sequences interleaved (fft3_run)
  T* lap1 = reinterpret_cast<T*>(bufA + (size_t)NMAX * 2 * C * PS);
  T* der1 = lap1 + n;
  const cplx<T>* twg = static_cast<const cplx<T>*>(p.tw);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    lap1[i] = static_cast<const T*>(p.lap1)[i];
    der1[i] = static_cast<const T*>(p.der1)[i];
  }
  __syncthreads();
  const ZColumnIO<T> io{static_cast<cplx<T>*>(p.spec), n, nh, ky1, ky2, k0, lc, C};
  // with one column (ky = −ky) only the q = 0 sequences exist: sequence index bi maps to
  // (f·2 + 0)·C + c, so transform all 2·C slots per field and ignore q = 1 (it aliases q = 0)
  fft3_run<T, false, L, true>(bufA, NIN * 2 * C, twg, GlobLd3<ZColumnIO<T>>{io}, SmemSt3<T>());
  __syncthreads();
  cplx<T>* res = bufA;
  const T lam = T(p.lam), scale = T(p.scale);
  auto at = [&](int f, int q, int c, int kz) { return (((f * 2 + q) << lc) + c) * PS + ppos(kz); };
  for (int t = threadIdx.x; t < nq * C * n; t += blockDim.x) {
    const int kz = t & (n - 1);
    const int qc = t >> L;
    const int c = qc & (C - 1), q = qc >> lc;
    const int kx = k0 + c;
    const int ky = q ? ky2 : ky1;
    cplx<T> in[NIN], out[NOUT];
    if (kx != 0) {
#pragma unroll
      for (int f = 0; f < NIN; ++f) in[f] = res[at(f, q, c, kz)];
      symbol3<T, OP>(lap1, der1, lam, scale, kx, ky, kz, in, out);
#pragma unroll
      for (int f = 0; f < NOUT; ++f) res[at(f, q, c, kz)] = out[f];
      continue;
    }
    // packed column: element (ky, kz) pairs with (−ky, −kz); one thread per unordered pair
    const int kzp = (n - kz) & (n - 1);
    int qp;
    if (nq == 2) {
      if (q == 1) continue;  // the q = 0 thread of the pair handles it
      qp = 1;
    } else {
      if (kz > kzp) continue;
      qp = 0;
    }
    const int kyp = qp ? ky2 : ky1;
    cplx<T> Aa[NIN], Ba[NIN], Ab[NIN], Bb[NIN];
#pragma unroll
    for (int f = 0; f < NIN; ++f) {
      const cplx<T> P = res[at(f, q, c, kz)];
      const cplx<T> Pp = res[at(f, qp, c, kzp)];
      Aa[f] = mk(T(0.5) * (P.x + Pp.x), T(0.5) * (P.y - Pp.y));
      Ba[f] = mk(T(0.5) * (P.y + Pp.y), T(0.5) * (Pp.x - P.x));
      Ab[f] = mk(T(0.5) * (Pp.x + P.x), T(0.5) * (Pp.y - P.y));
      Bb[f] = mk(T(0.5) * (Pp.y + P.y), T(0.5) * (P.x - Pp.x));
    }
    cplx<T> oA[NOUT], oB[NOUT], oAp[NOUT], oBp[NOUT];
    symbol3<T, OP>(lap1, der1, lam, scale, 0, ky, kz, Aa, oA);
    symbol3<T, OP>(lap1, der1, lam, scale, nh, ky, kz, Ba, oB);
    symbol3<T, OP>(lap1, der1, lam, scale, 0, kyp, kzp, Ab, oAp);
    symbol3<T, OP>(lap1, der1, lam, scale, nh, kyp, kzp, Bb, oBp);
    const bool self = (qp == q) && (kzp == kz);
#pragma unroll
    for (int f = 0; f < NOUT; ++f) {
      res[at(f, q, c, kz)] = cadd(oA[f], cmuli(oB[f]));
      if (!self) res[at(f, qp, c, kzp)] = cadd(oAp[f], cmuli(oBp[f]));
    }
  }
  __syncthreads();
  fft3_run<T, true, L, true>(bufA, NOUT * 2 * C, twg, SmemLd3<T>(), GlobSt3<ZColumnIO<T>>{io});
}

// ------------------------------------------------------------------------------------------
// kernel 5: inverse FFT along x, interpolation (or the grid)
// ------------------------------------------------------------------------------------------
template <typename T>
struct RowZLoad3 {
  const cplx<T>* spec;
  int n, nh, row0, half, nrows;  // row0 = z·n + y0; field stride nrows rows
  __device__ __forceinline__ cplx<T> load(int sq, int m) const {
    const int f = sq / half, j = sq - f * half;
    const size_t ra = ((size_t)f * nrows + row0 + 2 * j) * nh;
    const size_t rb = ra + nh;
    if (m == 0 || m == nh) {
      const cplx<T> A = spec[ra], B = spec[rb];
      return m == 0 ? mk(A.x, B.x) : mk(A.y, B.y);
    }
    if (m < nh) {
      const cplx<T> A = spec[ra + m], B = spec[rb + m];
      return mk(A.x - B.y, A.y + B.x);
    }
    const cplx<T> A = spec[ra + (n - m)], B = spec[rb + (n - m)];
    return mk(A.x + B.y, B.x - A.y);
  }
};

template <typename T, int OP, int GMODE, int L>
__global__ void __launch_bounds__(kThreads3) k3_rowifft_gather(Row3Params p) {
  // programmatic launch: wait for the previous kernel, then let the next one launch; a GMRES
  // cycle's stop flag is read after the wait (the step just before may have written it)
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
  if (p.stop && *p.stop) return;
  constexpr int NOUT = Traits3<OP>::NOUT;
  using PT = typename Prec3<T>::PT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int n = 1 << L, nh = n >> 1;
  const int R = p.R, half = R >> 1, M = p.M;
  const int seqs = NOUT * half;
  const PT* phi = static_cast<const PT*>(p.phi);
  const PT* dphi = static_cast<const PT*>(p.dphi);
  const PT* nrm = static_cast<const PT*>(p.nrm);
  cplx<T>* bufA = reinterpret_cast<cplx<T>*>(smem_raw);
  const int bands = n / R;
  const int z = blockIdx.x / bands, y0 = (blockIdx.x - z * bands) * R;
  const RowZLoad3<T> zl{static_cast<const cplx<T>*>(p.spec), n, nh, z * n + y0, half, n * n};
  fft3_run<T, true, L>(bufA, seqs, static_cast<const cplx<T>*>(p.tw), GlobLd3<RowZLoad3<T>>{zl}, SmemSt3<T>());
  __syncthreads();
  const T* u = reinterpret_cast<const T*>(bufA);
  if (GMODE == G3_GRID) {
    for (int t = threadIdx.x; t < NOUT * R * n; t += blockDim.x) {
      const int f = t / (R * n);
      const int rem = t - f * R * n;
      const int lr = rem / n, x = rem - lr * n;
      p.grid[(((size_t)f * n + z) * n + y0 + lr) * n + x] =
          double(Prec3<T>::to_pt(u[2 * pidx((f * half + (lr >> 1)) * n + x) + (lr & 1)]));
    }
    return;
  }
  const double* pin;
  double* pout;
  resolve_io3(p, pin, pout);
  const Ranges3 rg = band_points3(p.cell_start, n, z, y0, R);
  for (int t = threadIdx.x; t < rg.total * 4; t += blockDim.x) {
    const int s = rg.at(t >> 2);
    const int ay = t & 3;
    const int az = (z - p.base[2 * M + s]) & (n - 1);
    const int row = (p.base[M + s] + ay) & (n - 1);
    const int lr = (row - y0) & (n - 1);
    if (lr >= R || az > 3) continue;
    const int i = p.perm[s];
    const int bx = p.base[s];
    const PT py = phi[(1 * 4 + ay) * M + s], pz = phi[(2 * 4 + az) * M + s];
    const int eb = (lr >> 1) * n, odd = lr & 1;
    auto uval = [&](int e) { return Prec3<T>::to_pt(u[2 * pidx(e) + odd]); };
    PT a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
    for (int ax = 0; ax < 4; ++ax) {
      const int col = (bx + ax) & (n - 1);
      const PT px = phi[(0 * 4 + ax) * M + s];
      const PT v0 = uval(eb + col);
      if (OP == OP3_ADJ_AN) {
        a0 += v0 * dphi[(0 * 4 + ax) * M + s] * py * pz;
        a1 += v0 * px * dphi[(1 * 4 + ay) * M + s] * pz;
        a2 += v0 * px * py * dphi[(2 * 4 + az) * M + s];
      } else {
        const PT w3 = px * py * pz;
        a0 += v0 * w3;
        if (NOUT == 3) {
          a1 += uval(eb + half * n + col) * w3;
          a2 += uval(eb + 2 * half * n + col) * w3;
        }
      }
    }
    if (OP == OP3_ADJ_AN || OP == OP3_ADJ_SD) {
      double val = double(nrm[s]) * double(a0) + double(nrm[M + s]) * double(a1) + double(nrm[2 * M + s]) * double(a2);
      if (OP == OP3_ADJ_SD) val = -val;
      if (p.trans) val *= double(static_cast<const PT*>(p.wscale)[s]);
      atomicAdd(pout + i, val);
    } else {
      atomicAdd(pout + i, double(a0));
    }
  }
}

// ------------------------------------------------------------------------------------------
// shared memory per CTA and the launch of one application for a compile-time size
// ------------------------------------------------------------------------------------------
constexpr size_t kSmemLimit3 = 227 * 1024;

template <typename T>
__host__ __device__ constexpr size_t smem_rows3(int n, int nf, int R) {
  return padded((size_t)nf * (R / 2) * n) * sizeof(cplx<T>);
}
template <typename T>
constexpr size_t smem_y3(int n, int nf, int C) {  // host side (launch shapes)
  return (size_t)nf * C * seq_stride3(__builtin_ctz(n), (int)sizeof(cplx<T>)) * sizeof(cplx<T>);
}
template <typename T>
constexpr size_t smem_z3(int n, int nf, int C) {  // host side (launch shapes)
  return (size_t)nf * 2 * C * seq_stride3(__builtin_ctz(n), (int)sizeof(cplx<T>)) * sizeof(cplx<T>) +
         2 * n * sizeof(T);
}

// Opt a kernel in to the full dynamic shared memory once per device (a per-device bit records it;
// setting it twice is harmless, so threads racing on a first call need no lock).
template <typename K>
inline cudaError_t opt_in_smem3(K kernel, std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit3);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// The five kernels of one application at n = 2^L: rows R per band, C kx columns per y pass, Cz per
// z pass; `grid` selects the grid output of the last kernel.
// Programmatic dependent launch of an application's kernels (IBDL_NO_PDL=1 turns it off): a kernel
// may launch once every CTA of the previous one has passed its wait, and it waits in turn before
// it reads anything; the launch latency is taken while the previous kernel drains.
inline bool use_pdl3() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("IBDL_NO_PDL");
    v = (e && atoi(e) != 0) ? 0 : 1;
  }
  return v == 1;
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch3(void (*kernel)(KArgs...), int grid, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads3);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &at;
  cfg.numAttrs = use_pdl3() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <typename T, int OP, int L>
ibdl_status launch_apply_3d(Geometry* g, const Row3Params& rp, const Col3Params& cp, int R, int C, int Cz,
                            bool grid, cudaStream_t s) {
  constexpr int NIN = Traits3<OP>::NIN, NOUT = Traits3<OP>::NOUT, NMAX = NIN > NOUT ? NIN : NOUT;
  constexpr int n = 1 << L;
  constexpr bool f32 = std::is_same<T, float>::value;
  static std::atomic<unsigned long long> d[6];
  IBDL_CUDA(opt_in_smem3(k3_spread_rowfft<T, OP, L>, d[0]));
  IBDL_CUDA(opt_in_smem3(k3_ypass<T, false, L>, d[1]));
  IBDL_CUDA(opt_in_smem3(k3_zpass<T, OP, L>, d[2]));
  IBDL_CUDA(opt_in_smem3(k3_ypass<T, true, L>, d[3]));
  IBDL_CUDA(opt_in_smem3(k3_rowifft_gather<T, OP, G3_GRID, L>, d[4]));
  IBDL_CUDA(opt_in_smem3(k3_rowifft_gather<T, OP, G3_INTERP, L>, d[5]));
  const int rows_grid = n * (n / R), col_grid = n * ((n / 2) / C), z_grid = (n / 2 + 1) * ((n / 2) / Cz);
  const int st0 = f32 ? IBDL_STAGE_SPREAD_ROWFFT_FP32 : IBDL_STAGE_SPREAD_ROWFFT_FP64;
  if (g->timing) timing_mark(g, s, -1);
  IBDL_CUDA(launch3(k3_spread_rowfft<T, OP, L>, rows_grid, smem_rows3<T>(n, NIN, R), s, rp));
  if (g->timing) timing_mark(g, s, st0);
  Col3Params yp = cp;
  yp.nf = NIN;
  IBDL_CUDA(launch3(k3_ypass<T, false, L>, col_grid, smem_y3<T>(n, NIN, C), s, yp));
  Col3Params zp = cp;
  zp.C = Cz;
  zp.lc = __builtin_ctz(Cz);
  IBDL_CUDA(launch3(k3_zpass<T, OP, L>, z_grid, smem_z3<T>(n, NMAX, Cz), s, zp));
  yp.nf = NOUT;
  IBDL_CUDA(launch3(k3_ypass<T, true, L>, col_grid, smem_y3<T>(n, NOUT, C), s, yp));
  if (g->timing) timing_mark(g, s, st0 + 1);
  if (grid)
    IBDL_CUDA(launch3(k3_rowifft_gather<T, OP, G3_GRID, L>, rows_grid, smem_rows3<T>(n, NOUT, R), s, rp));
  else
    IBDL_CUDA(launch3(k3_rowifft_gather<T, OP, G3_INTERP, L>, rows_grid, smem_rows3<T>(n, NOUT, R), s, rp));
  if (g->timing) timing_mark(g, s, st0 + 2);
  g->launches += 5;
  IBDL_CUDA(cudaGetLastError());
  return IBDL_OK;
}

// every operator and grid arithmetic at one size (instantiated by apply3d_n<n>.cu)
#define IBDL_3D_OPS(X, T, L) X(T, OP3_SCALAR_AN, L) X(T, OP3_SCALAR_SD, L) X(T, OP3_ADJ_AN, L) X(T, OP3_ADJ_SD, L)
#define IBDL_3D_INST1(T, OP, L)                                                                          \
  template ibdl_status launch_apply_3d<T, OP, L>(Geometry*, const Row3Params&, const Col3Params&, int, int, int, \
                                                 bool, cudaStream_t);
#define IBDL_3D_DECL1(T, OP, L)                                                                                 \
  extern template ibdl_status launch_apply_3d<T, OP, L>(Geometry*, const Row3Params&, const Col3Params&, int, int, \
                                                        int, bool, cudaStream_t);
#define IBDL_INSTANTIATE_3D(L) IBDL_3D_OPS(IBDL_3D_INST1, double, L) IBDL_3D_OPS(IBDL_3D_INST1, float, L) IBDL_3D_OPS(IBDL_3D_INST1, ff, L)
#define IBDL_DECLARE_3D(L) IBDL_3D_OPS(IBDL_3D_DECL1, double, L) IBDL_3D_OPS(IBDL_3D_DECL1, float, L) IBDL_3D_OPS(IBDL_3D_DECL1, ff, L)

}  // namespace ibdl
