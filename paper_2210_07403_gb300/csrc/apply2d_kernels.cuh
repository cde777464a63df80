// Device side of the two-dimensional IBDL operator: spread → FFT → Fourier symbol → inverse FFT →
// interpolate, specialised on the grid size n = 2^L at compile time.
//
// One application A Q = S* u + ½Q, u = −L⁻¹ S̃ Q (Sec. 5.3.2) or the Stokes velocity (Sec. 6.3.3),
// runs as three kernels, each owning a disjoint piece of the grid (no global atomics on the grid
// and no grid memset):
//
//   k_spread_rowfft   band of R rows: accumulate the dipole sources of every point whose 4×4
//                     stencil meets the band (shared-memory atomics), FFT along x with two real
//                     rows packed as one complex row, unpack to the packed half spectrum.
//   k_colpass         group of C kx columns: FFT along y, Fourier symbol, inverse FFT along y.
//   k_rowifft_gather  band of R rows: inverse FFT along x, then interpolate (S*) the band's part
//                     of every point's stencil and add it to Y (which the first kernel set to ½Q).
//
// The transforms are the register FFT of fft8.cuh: a thread holds eight elements (per lane) of
// a sequence; a CTA has (R/2)·QT threads in the row kernels and C·QT in the column pass (QT
// threads per sequence), and one padded shared-memory buffer per sequence, used for the spread's
// accumulation, the exchanges between FFT stages and the final layout.
//
// Packed half spectrum: for a real row a, A_k (k = 0..n/2) is stored in n/2 slots with slot 0
// holding (A_0, A_{n/2}), both real. Along y, the kx = 0 and kx = n/2 columns are therefore one
// complex column a + i b with a, b real columns; the column pass separates them by Hermitian
// symmetry before the symbol and repacks after it.
//
// Band-major storage: the n rows of a field form bands of R rows (the row kernels' work unit),
// and element (row, k) of field f sits at (f·n + band·R)·(n/2) + k·R + (row mod R). A row band is
// one contiguous block, and a column reads R contiguous values per band.
#pragma once

#include <type_traits>
#include <utility>

#include "ff.cuh"
#include "fft8.cuh"
#include "tma.cuh"

namespace ibdl {

// Grid arithmetic type T and its point type PT: the point tables, the spread's shared-memory
// accumulation and the gather's partial sums use PT (FP32 for FP32, FP64 for FP64 and for
// float-float, whose point work is O(M) and whose accuracy the FP64 tables carry).
template <typename T>
struct Prec2 {
  using PT = T;
  static __device__ __forceinline__ cplx<T> acc_load(const cplx<T>* b, int i) { return b[i]; }
  static __device__ __forceinline__ PT to_pt(T v) { return v; }
};
template <>
struct Prec2<ff> {
  using PT = double;
  static __device__ __forceinline__ cplx<ff> acc_load(const cplx<ff>* b, int i) {
    const cplx<double> d = reinterpret_cast<const cplx<double>*>(b)[i];
    return mk(ff_from_double(d.x), ff_from_double(d.y));
  }
  static __device__ __forceinline__ double to_pt(ff v) { return double(v); }
};

enum { OP_SCALAR_AN = 0, OP_SCALAR_SD = 1, OP_STOKES_AN = 2, OP_STOKES_SD = 3, OP_ADJ_AN = 4,
       OP_ADJ_SD = 5, OP_STOKES_T = 6, OP_SL = 7 };

// grid fields entering / leaving the Fourier stage, and boundary components in / out
template <int OP>
struct Traits;
template <>
struct Traits<OP_SCALAR_AN> { static constexpr int NIN = 1, NOUT = 1, C = 1; };  // f = S̃Q
template <>
struct Traits<OP_SCALAR_SD> { static constexpr int NIN = 2, NOUT = 1, C = 1; };  // S(Qn_x), S(Qn_y)
template <>
struct Traits<OP_STOKES_AN> { static constexpr int NIN = 3, NOUT = 2, C = 2; };  // s, g_x, g_y
template <>
struct Traits<OP_STOKES_SD> { static constexpr int NIN = 4, NOUT = 2, C = 2; };  // s, A11, A22, A12
template <>
struct Traits<OP_ADJ_AN> { static constexpr int NIN = 1, NOUT = 1, C = 1; };     // S W
template <>
struct Traits<OP_ADJ_SD> { static constexpr int NIN = 1, NOUT = 2, C = 1; };     // S W → ∂_x v, ∂_y v
// Stokes transpose (analytic dipole): ψ_x, ψ_y → v_s, v_gx, v_gy
template <>
struct Traits<OP_STOKES_T> { static constexpr int NIN = 2, NOUT = 3, C = 2; };
// single layer S*(−L⁻¹)(S V): plain spread, −L⁻¹, plain interpolation, no jump term
template <>
struct Traits<OP_SL> { static constexpr int NIN = 1, NOUT = 1, C = 1; };

enum { G_INTERP = 0, G_GRID = 1 };

// At most 512 threads per CTA in every 2-D kernel (at least 128 registers per thread).
constexpr int kMaxThreads2d = 512;
constexpr int kMinL2d = 4, kMaxL2d = 13;

// Lanes per thread and threads per sequence of the n = 2^L transforms. Large grids give a thread
// several lanes, so that a CTA of at most 512 threads can hold more than one column or row pair:
// the band-major spectra then move in pieces of R·C elements per band (at least one 32-byte
// sector). FP32 (8-byte elements): 2 lanes from 2048², 4 at 8192²; FP64 and float-float
// (16-byte elements): 2 lanes at 8192².
__host__ __device__ constexpr int lanes_per_thread_2d(int L, bool f32) {
  return f32 ? (L >= 13 ? 4 : (L >= 11 ? 2 : 1)) : (L >= 13 ? 2 : 1);
}
__host__ __device__ constexpr int threads_per_seq_2d(int L, bool f32) { return (1 << L) / 8 / lanes_per_thread_2d(L, f32); }

// Thread groups across the NF fields of a kernel: one group per field when NF·QT threads fit in a
// CTA (each thread transforms one field), else a single group that transforms the fields one
// after another.
__host__ __device__ constexpr int field_groups_2d(int nf, int L, bool f32) {
  return nf * threads_per_seq_2d(L, f32) <= kMaxThreads2d ? nf : 1;
}

// Per-precision register policy: twiddles in registers when they fit the budget, else read from
// the table at each use.
template <typename T, int L, int NF>
struct Cfg2 {
  static constexpr bool F32 = sizeof(T) == 4;
  static constexpr int V = lanes_per_thread_2d(L, F32);
  static constexpr int QT = threads_per_seq_2d(L, F32);
  static constexpr int NGRP = field_groups_2d(NF, L, F32);
  static constexpr int NTW = F8<L, V>::NTW;
  // register budget for twiddles: 42 FP32 registers; 56 in FP64; 28 in float-float, whose
  // arithmetic needs the most temporaries
  static constexpr bool TWR =
      F32 ? (NTW * V <= 21) : (std::is_same<T, ff>::value ? (NTW * V <= 7) : (NTW * V <= 14));
  using TW = std::conditional_t<TWR, TwRegs<T, L>, TwTable<T, L>>;
};

// Column kernels (and the row kernels, with the row pairs of a band in place of the columns):
// the C columns of a thread group are interleaved across consecutive threads
// (column c = t mod C, lane j0 = t / C for thread t of the group), so a warp holds 32/C lanes of
// each of C adjacent columns (one lane of each of 32 columns when C ≥ 32): its accesses to the
// band-major spectra cover whole 32-byte sectors (C·R adjacent values per band). Each column's
// exchange buffer holds the padded sequence and is rounded up to a stride ≡ max(1, w/C) (mod w)
// elements, w = 16 for 8-byte and 8 for 16-byte elements, which puts the C columns of a warp in
// different shared-memory banks: every exchange then takes the least number of wavefronts the
// warp's bytes need (checked by counting banks per warp for every size, C ≤ 32 and R ≤ 8 on the
// CPU, against a search over all strides).
__host__ __device__ constexpr int col_stride_2d(int L, int C, int esize) {
  const int pn = (1 << L) + (1 << L) / 8;
  const int w = esize == 8 ? 16 : 8;
  const int t = (w / C > 1 ? w / C : 1) % w;
  return C < 2 ? pn : pn + (((t - pn) % w) + w) % w;
}
template <int QT>
__device__ __forceinline__ void col_lane_2d(int C, int& g, int& c, int& j0) {
  const int per = C * QT;
  g = (int)threadIdx.x / per;
  const int t = (int)threadIdx.x - g * per;
  c = t & (C - 1);
  j0 = t >> (__ffs(C) - 1);
}

// Row kernels interleave their row pairs like the column groups, except where a thread holds four
// lanes (FP32 at 8192²): measured slower there (848 against 903 µs per application), they keep one
// row pair per run of consecutive threads and the plain padded stride.
__host__ __device__ constexpr bool row_interleave_2d(int L, bool f32) { return lanes_per_thread_2d(L, f32) < 4; }
__host__ __device__ constexpr int row_stride_2d(int L, int half, int esize) {
  return row_interleave_2d(L, esize == 8) ? col_stride_2d(L, half, esize) : (1 << L) + (1 << L) / 8;
}
template <int QT, bool IL>
__device__ __forceinline__ void row_lane_2d(int half, int& g, int& rp, int& j0) {
  if constexpr (IL) {
    col_lane_2d<QT>(half, g, rp, j0);
  } else {
    const int q = (int)threadIdx.x / QT;
    j0 = (int)threadIdx.x - q * QT;
    g = q / half;
    rp = q - g * half;
  }
}

template <typename T>
struct RowParams {
  using PT = typename Prec2<T>::PT;
  int n, log2n, R;
  int M;
  const int* cell_start;
  const int* base;
  const int* perm;
  const PT* phi;
  const PT* dphi;
  const PT* wscale;
  const PT* nrm;
  const double* in;   // [c][M] density
  double* out;        // [c][M] result (first kernel stores ½·in, last kernel adds S*u)
  cplx<T>* spec;      // [nf][n][n/2]
  const cplx<T>* tw;  // [n] e^{−2πi j/n}
  const int* stop;    // optional: skip all work when *stop != 0
  double* grid;       // G_GRID: [nf][n][n]
  const int* idx;     // optional: in += (*idx)·vstride, out += (*idx + 1)·vstride (Krylov basis)
  int vstride;
  int64_t io_off;     // batched launches: in = in_base + io_off, out = out_base + io_off
  // scalar adjoint ops only: 1 = the Euclidean transpose Aᵀ = W A* W⁻¹ (W⁻¹λ spread with weight
  // Δs/h^d is λ spread with weight h^−d = 1 · h^−d: the spread weight is 1 and the gathered values
  // carry Δs/h^d instead of 1)
  int trans;
  const double* grid_in;  // optional [NIN][n][n]: the band rows are read from it instead of spread
  double jump;            // jump term coefficient: ½ (Dirichlet), −½ (Neumann), 0 (single layer)
  // completed method (Sec. 5.3.3, Sec. 6.3.3): the vectors hold ū after the c·M density values
  int aug;                // 1: add ū_l to the boundary rows, write the rows η Σ_i Δs_i Q_{l,i}
  double eta;             // η
  double hd;              // h^d
  PT eta_src;             // weight of the ηSQ source: η (scalar) or η/μ (Stokes, projected part)
  int fsel;               // one-field launches: the field this launch spreads or interpolates
};

template <typename T>
__device__ __forceinline__ void resolve_io(const RowParams<T>& p, const double*& in, double*& out) {
  in = p.in;
  out = p.out;
  if (p.idx) {
    const int k = *p.idx;
    in += (size_t)k * p.vstride;
    out += (size_t)(k + 1) * p.vstride;
  }
}

template <typename T>
struct ColParams {
  int n, log2n, C;
  int R;  // rows per band of the band-major spectrum
  T lam, scale;
  T mu;   // viscosity (Brinkman: L = μΔ − λ)
  const T* lap1;
  const T* der1;
  cplx<T>* spec;
  const cplx<T>* tw;
  const int* stop;
  int* err;  // the staged column pass sets it to 1 when a bounded wait runs out
};

// Sorted points whose base row lies in the cell rows [r0 − 3, r0 + R) (mod n): at most two
// contiguous ranges of the cell-sorted order.
struct PointRanges {
  int s0, cnt1, s2, cnt;
  __device__ int at(int t) const { return t < cnt1 ? s0 + t : s2 + (t - cnt1); }
};
__device__ __forceinline__ PointRanges band_points(const int* cell_start, int n, int r0, int R) {
  PointRanges pr;
  const int lo = r0 - 3, hi = r0 + R;
  if (lo >= 0) {
    pr.s0 = cell_start[lo];
    pr.cnt1 = cell_start[hi] - pr.s0;
    pr.s2 = 0;
    pr.cnt = pr.cnt1;
  } else {
    pr.s0 = cell_start[lo + n];
    pr.cnt1 = cell_start[n] - pr.s0;
    pr.s2 = cell_start[0];
    pr.cnt = pr.cnt1 + (cell_start[hi] - pr.s2);
  }
  return pr;
}

// Two adjacent complex values of a band-major spectrum (A_k and B_k of a row pair, at an even
// element offset): one 16-byte access in FP32, two otherwise.
__device__ __forceinline__ void store_pair(cplx<float>* p, cplx<float> a, cplx<float> b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
template <typename T>
__device__ __forceinline__ void store_pair(cplx<T>* p, cplx<T> a, cplx<T> b) {
  p[0] = a;
  p[1] = b;
}
__device__ __forceinline__ void load_pair(const cplx<float>* p, cplx<float>& a, cplx<float>& b) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = mk(v.x, v.y);
  b = mk(v.z, v.w);
}
template <typename T>
__device__ __forceinline__ void load_pair(const cplx<T>* p, cplx<T>& a, cplx<T>& b) {
  a = p[0];
  b = p[1];
}

// ------------------------------------------------------------------------------------------
// kernel 1: spread + forward FFT along x
// ------------------------------------------------------------------------------------------
// Bodies take the work unit (row band / column group) and the problem's number of units, so
// the same code serves one problem (unit = blockIdx.x) and a batch of problems (unit from a
// (problem, unit) table).
// One spread work item (point, stencil node): everything but the density, read from the geometry's
// point tables, which no kernel writes (so a kernel may load them before its dependency wait).
template <typename T>
struct SpreadItem {
  int lr, i, col;
  T px, py, dpx, dpy, ws, nx, ny;
};
template <typename T>
__device__ __forceinline__ SpreadItem<typename Prec2<T>::PT> spread_item(const RowParams<T>& p, const PointRanges& pr,
                                                                         int t, int r0) {
  const int n = p.n, M = p.M;
  const int s = pr.at(t >> 4);
  const int ay = (t >> 2) & 3, ax = t & 3;
  SpreadItem<typename Prec2<T>::PT> it;
  it.lr = (((p.base[M + s] + ay) & (n - 1)) - r0) & (n - 1);
  it.i = p.perm[s];
  it.col = (p.base[s] + ax) & (n - 1);
  it.px = p.phi[(0 * 4 + ax) * M + s];
  it.py = p.phi[(1 * 4 + ay) * M + s];
  it.dpx = p.dphi[(0 * 4 + ax) * M + s];
  it.dpy = p.dphi[(1 * 4 + ay) * M + s];
  it.ws = p.wscale[s];
  it.nx = p.nrm[s];
  it.ny = p.nrm[M + s];
  return it;
}

// PF: load the FFT twiddles (and, in the column pass, the symbol rows) before the dependency
// wait, for latency (single problems); batched launches load them where they are used, which
// keeps registers down and occupancy up.
// SPLIT: one input field (p.fsel) per launch, for grids whose row bands of every field do not
// fit shared memory together: the band holds that field only, and the first launch (field 0)
// also writes the jump term and the completed method's rows.
template <typename T, int OP, int L, bool PF = true, bool SPLIT = false>
__device__ __forceinline__ void spread_rowfft_body(const RowParams<T>& p, int unit, int nunits,
                                                   unsigned char* smem_raw) {
  constexpr int NIN = Traits<OP>::NIN;
  constexpr int NB = SPLIT ? 1 : NIN;  // fields held in shared memory
  constexpr int NC = Traits<OP>::C;
  using CF = Cfg2<T, L, NB>;
  using F = F8<L, CF::V>;
  using PT = typename Prec2<T>::PT;
  constexpr int n = F::N, V = CF::V, QT = CF::QT, NGRP = CF::NGRP;
  const int R = p.R, half = R >> 1, M = p.M;
  // sequence (field f, row pair rp) at buf + (f·half + rp)·PN (the padded sequence rounded up as
  // for the column groups, with the row pairs of a group interleaved across threads like the
  // columns); accumulation view (point type PT, the same bytes per element): field f, local row
  // lr, column x → real part (even lr) or imaginary part (odd lr) of element ppos(x) of sequence
  // f·half + lr/2
  const int PN = row_stride_2d(L, half, (int)sizeof(cplx<T>));
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  PT* acc = reinterpret_cast<PT*>(buf);
  auto aidx = [&](int seq, int x) { return 2 * (seq * PN + ppos(x)); };
  const int r0 = unit * R;
  // FFT lanes: thread (group g, row pair rp, lane j0); threads past NGRP·half·QT only help with
  // the loops (clearing, spreading, unpacking)
  int g, rp, j0;
  row_lane_2d<QT, row_interleave_2d(L, sizeof(T) == 4)>(half, g, rp, j0);
  const bool active = g < NGRP;
  // prologue independent of the previous kernel, then wait for it (programmatic launch)
  {
    // clear the accumulation buffer (NIN·half padded sequences, a multiple of 16 bytes) with
    // 16-byte stores
    uint4* z = reinterpret_cast<uint4*>(buf);
    const int nz = (int)((size_t)NB * half * PN * sizeof(cplx<T>) / 16);
    for (int i = threadIdx.x; i < nz; i += blockDim.x) z[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  typename CF::TW tw[V];
  if constexpr (PF) {
#pragma unroll
    for (int v = 0; v < V; ++v) tw[v].load(p.tw, j0 + v * QT);
  }
  // the points whose stencil meets the band, and this thread's first work item (16 per point)
  const PointRanges pr = band_points(p.cell_start, n, r0, R);
  const int nitems = p.grid_in ? 0 : pr.cnt * 16;
  SpreadItem<PT> it0 = {};
  if ((int)threadIdx.x < nitems) it0 = spread_item(p, pr, threadIdx.x, r0);
  cudaGridDependencySynchronize();
  // Let the next kernel launch and run its prologue. Triggered only after this kernel's own
  // wait, so every kernel before the previous one has completed by then: a prologue overlaps
  // its direct predecessor only (its wait still covers this grid's completion and writes).
  cudaTriggerProgrammaticLaunchCompletion();
  // In a GMRES cycle the step just before this kernel writes the stop flag and the Krylov index:
  // both loads go out together, then the branch
  const int stopped = p.stop ? *p.stop : 0;
  const double* pin;
  double* pout;
  resolve_io(p, pin, pout);
  if (stopped) return;

  const bool first = !SPLIT || p.fsel == 0;
  // jump term: out = ±½·in (the gather kernel adds S*u afterwards); none for grid input
  if (!p.grid_in && first)
    for (int i = unit * blockDim.x + threadIdx.x; i < NC * M; i += nunits * blockDim.x)
      pout[i] = p.jump * pin[i] + (p.aug ? pin[NC * M + i / M] : 0.0);
  __syncthreads();  // the accumulation buffer is cleared
  if (p.aug && unit == 0 && first) {
    // constraint rows of the completed method: η Σ_i Δs_i Q_{l,i} (Δs = wscale·h^d); the block
    // size is a power of two (a partial warp below 32 threads), the partial sums go to the
    // reduction slots after the sequence buffers
    double* red = reinterpret_cast<double*>(buf + (size_t)NB * half * PN);
    const int wl = blockDim.x < 32 ? blockDim.x : 32;
    const unsigned wmask = wl == 32 ? 0xffffffffu : ((1u << wl) - 1u);
    for (int l = 0; l < NC; ++l) {
      double v = 0.0;
      for (int s = threadIdx.x; s < M; s += blockDim.x) v += double(p.wscale[s]) * pin[(size_t)l * M + p.perm[s]];
      for (int o = wl >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(wmask, v, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
      __syncthreads();
      if (threadIdx.x < wl) {
        const int nw = (blockDim.x + 31) >> 5;
        double t = (int)threadIdx.x < nw ? red[threadIdx.x] : 0.0;
        for (int o = wl >> 1; o > 0; o >>= 1) t += __shfl_xor_sync(wmask, t, o);
        if (threadIdx.x == 0) pout[NC * M + l] = p.eta * p.hd * t;
      }
      __syncthreads();
    }
  }

  if (p.grid_in) {
    for (int t = threadIdx.x; t < NB * R * n; t += blockDim.x) {
      const int f = t / (R * n);
      const int rem = t - f * R * n;
      const int lr = rem / n, x = rem - lr * n;
      const int fi = SPLIT ? p.fsel : f;  // the input field
      acc[aidx(f * half + (lr >> 1), x) + (lr & 1)] = PT(p.grid_in[((size_t)fi * n + r0 + lr) * n + x]);
    }
  }

  // one thread per (point, stencil node): 16 work items per point whose stencil meets the band
  // (the next item's table values are loaded before this item's additions, so a band with more
  // items than threads waits for the tables once, not once per round)
  SpreadItem<PT> cur = it0;
  for (int t = threadIdx.x; t < nitems; t += blockDim.x) {
    SpreadItem<PT> nxt = {};
    if (t + (int)blockDim.x < nitems) nxt = spread_item(p, pr, t + blockDim.x, r0);
    const SpreadItem<PT> it = cur;
    cur = nxt;
    const int lr = it.lr;
    if (lr >= R) continue;
    const int i = it.i;
    const PT px = it.px, py = it.py, ws = it.ws, nx = it.nx, ny = it.ny;
    const int e0 = aidx(lr >> 1, it.col) + (lr & 1);  // field 0; field f adds 2·f·half·PN
    const PT pp = px * py;
    // add v to field f's band (SPLIT: only field p.fsel, held in the first slot)
    auto add = [&](int f, PT v) {
      if (SPLIT) {
        if (f == p.fsel) atomicAdd(acc + e0, v);
      } else {
        atomicAdd(acc + e0 + 2 * f * half * PN, v);
      }
    };
    if (OP == OP_SCALAR_AN) {
      const PT q = PT(pin[i]) * ws;
      const PT ddx = it.dpx * py, ddy = px * it.dpy;
      // dipole source n·∇δ_h, plus ηδ_h for the completed method
      add(0, q * (nx * ddx + ny * ddy + p.eta_src * pp));
    } else if (OP == OP_SCALAR_SD) {
      const PT q = PT(pin[i]) * ws * pp;
      add(0, q * nx);
      add(1, q * ny);
    } else if (OP == OP_STOKES_AN || OP == OP_STOKES_SD) {
      const PT qx = PT(pin[i]), qy = PT(pin[M + i]);
      const PT c0 = ws * (qx * nx + qy * ny);  // Q·n
      const PT c1 = ws * (PT(2) * qx * nx);    // A_xx
      const PT c2 = ws * (PT(2) * qy * ny);    // A_yy
      const PT c3 = ws * (qx * ny + qy * nx);  // A_xy
      add(0, c0 * pp);
      if (OP == OP_STOKES_AN) {
        const PT ddx = it.dpx * py, ddy = px * it.dpy;
        // g_x = ∂_x S(A_xx) + ∂_y S(A_xy), g_y = ∂_x S(A_xy) + ∂_y S(A_yy); the completed method
        // adds (η/μ) S(Q) to the projected source
        const PT ce = p.eta_src * ws * pp;
        add(1, c1 * ddx + c3 * ddy + ce * qx);
        add(2, c3 * ddx + c2 * ddy + ce * qy);
      } else {
        add(1, c1 * pp);
        add(2, c2 * pp);
        add(3, c3 * pp);
      }
    } else if (OP == OP_STOKES_T) {
      // ψ_l = Σ_j μ_{l,j} Φ(x − X_j): the transpose of S*, unweighted
      add(0, PT(pin[i]) * pp);
      add(1, PT(pin[M + i]) * pp);
    } else {
      // plain spread of W (A*: weight Δs/h^d), or of λ (Aᵀ: weight 1, Δs/h^d moves to the gather)
      add(0, PT(pin[i]) * (p.trans ? PT(1) : ws) * pp);
    }
  }
  __syncthreads();

  if constexpr (!PF) {
#pragma unroll
    for (int v = 0; v < V; ++v) tw[v].load(p.tw, j0 + v * QT);
  }
  // forward FFT of every (field, row pair) sequence; each lane reads and writes back only its own
  // positions, so only the exchanges inside need barriers
#pragma unroll
  for (int k = 0; k < NB / NGRP; ++k) {
    const int f = g + k * NGRP;
    cplx<T>* sb = buf + ((size_t)f * half + rp) * PN;
    cplx<T> x[1][V][8];
    if (active) {
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int s = 0; s < 8; ++s) x[0][v][s] = Prec2<T>::acc_load(sb, ppos_strided<F::Q>(j0 + v * QT, s));
    }
    f8_fft<T, false, L, V, 1>(x, sb, 0, j0, tw, active);
    if (active) {
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int s = 0; s < 8; ++s) sb[ppos_strided<F::Q>(j0 + v * QT, s)] = x[0][v][s];
    }
  }
  __syncthreads();

  // unpack Z = FFT(a + i b) of the row pair (2j, 2j + 1) into A = FFT(a) (even row) and
  // B = FFT(b) (odd row), k = 0..n/2, packed format: thread t takes wavenumber k = t mod n/2 of
  // one (field, row pair), reads Z_k and Z_{n−k} once and writes A_k and B_k, adjacent in the
  // band-major block (offset k·R + 2j), with one store
  const cplx<T>* res = buf;
  constexpr int nh = n >> 1, lnh = L - 1;
  for (int t = threadIdx.x; t < NB * half * nh; t += blockDim.x) {
    const int k = t & (nh - 1), q2 = t >> lnh;
    const int f = q2 / half, jj = q2 - f * half;
    const int zb = (f * half + jj) * PN;
    const int fo = SPLIT ? p.fsel : f;  // the spectrum field written
    cplx<T> a, b;
    if (k == 0) {
      const cplx<T> z0 = res[zb], zh = res[zb + ppos(nh)];
      a = mk(z0.x, zh.x);
      b = mk(z0.y, zh.y);
    } else {
      const cplx<T> zk = res[zb + ppos(k)], zc = res[zb + ppos(n - k)];
      a = mk(T(0.5) * (zk.x + zc.x), T(0.5) * (zk.y - zc.y));
      b = mk(T(0.5) * (zk.y + zc.y), T(0.5) * (zc.x - zk.x));
    }
    store_pair(p.spec + ((fo * n + r0) * nh + k * R + 2 * jj), a, b);
  }
}

template <typename T, int OP, int L>
__global__ void __launch_bounds__(kMaxThreads2d) k_spread_rowfft(RowParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  spread_rowfft_body<T, OP, L>(p, blockIdx.x, gridDim.x, smem_raw);
}
// one input field (p.fsel) per launch
template <typename T, int OP, int L>
__global__ void __launch_bounds__(kMaxThreads2d) k_spread_rowfft1(RowParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  spread_rowfft_body<T, OP, L, true, true>(p, blockIdx.x, gridDim.x, smem_raw);
}

// ------------------------------------------------------------------------------------------
// Fourier symbols: NIN transformed fields in → NOUT out; lap = |k̃|² (sum of the per-axis
// Laplacian symbols), dkx, dky the per-axis derivative symbols
// ------------------------------------------------------------------------------------------
// a/b: the hardware reciprocal estimate in FP32 (within 2 ulp, well inside the FP32 application's
// rounding), IEEE division in FP64, a corrected quotient in float-float
__device__ __forceinline__ float sym_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double sym_div(double a, double b) { return a / b; }
__device__ __forceinline__ ff sym_div(ff a, ff b) { return a / b; }

template <typename T, int OP>
__device__ __forceinline__ void apply_symbol(const ColParams<T>& p, T lap, T dkx, T dky, const cplx<T>* in,
                                             cplx<T>* out) {
  if (OP == OP_SCALAR_AN || OP == OP_SCALAR_SD || OP == OP_ADJ_AN || OP == OP_ADJ_SD || OP == OP_SL) {
    // −L⁻¹ ↦ 1/(|k|² + λ), zero mode dropped when λ = 0 (Δ₀⁻¹)
    const T den = lap + p.lam;
    const T sig = den != T(0) ? sym_div(p.scale, den) : T(0);
    if (OP == OP_SCALAR_AN || OP == OP_ADJ_AN || OP == OP_SL) {
      out[0] = cscale(in[0], sig);
    } else if (OP == OP_SCALAR_SD) {
      // ∇·F ↦ i(k̃_x F̂_x + k̃_y F̂_y)
      const cplx<T> d = cadd(cscale(in[0], dkx), cscale(in[1], dky));
      out[0] = cscale(cmuli(d), sig);
    } else {
      const cplx<T> v = cscale(in[0], sig);
      out[0] = cscale(cmuli(v), dkx);
      out[1] = cscale(cmuli(v), dky);
    }
  } else if (OP == OP_STOKES_T) {
    // transpose of the Stokes multiplier (conjugate symbol): v̂_s = −i k̃·ψ̂/|k|², v̂_g = P̂ψ̂/|k|²
    const T inv = lap != T(0) ? sym_div(T(1), lap) : T(0);
    const cplx<T> kp = cadd(cscale(in[0], dkx), cscale(in[1], dky));
    const T sc = inv * p.scale;
    // Brinkman (λ > 0): the projected part carries μ/(μ|k|² + λ) in place of 1/|k|²
    const T sg = p.lam > T(0) ? sym_div(p.mu, p.mu * lap + p.lam) * p.scale : sc;
    out[0] = cscale(cmuli(kp), -sc);
    out[1] = cscale(csub(in[0], cscale(kp, dkx * inv)), sg);
    out[2] = cscale(csub(in[1], cscale(kp, dky * inv)), sg);
  } else {
    // Stokes, interior, η = 0: û = (i k̃ ŝ + P̂ ĝ)/|k|², P̂ = I − k̃k̃ᵀ/|k|²
    const T inv = lap != T(0) ? sym_div(T(1), lap) : T(0);
    cplx<T> gx, gy;
    if (OP == OP_STOKES_AN) {
      gx = in[1];
      gy = in[2];
    } else {  // ĝ_l = i k̃_m Â_lm with fields A11, A22, A12 in slots 1, 2, 3
      gx = cmuli(cadd(cscale(in[1], dkx), cscale(in[3], dky)));
      gy = cmuli(cadd(cscale(in[3], dkx), cscale(in[2], dky)));
    }
    const cplx<T> kg = cadd(cscale(gx, dkx), cscale(gy, dky));
    const cplx<T> is = cmuli(in[0]);
    const T sc = inv * p.scale;
    if (p.lam > T(0)) {
      // Brinkman (Sec. 6.3.2): û = i k̃ ŝ/|k|² + μ P̂ ĝ/(μ|k|² + λ), defined at k = 0 as well
      const T sg = sym_div(p.mu, p.mu * lap + p.lam) * p.scale;
      out[0] = cadd(cscale(is, dkx * sc), cscale(csub(gx, cscale(kg, dkx * inv)), sg));
      out[1] = cadd(cscale(is, dky * sc), cscale(csub(gy, cscale(kg, dky * inv)), sg));
    } else {
      out[0] = cscale(cadd(cscale(is, dkx), csub(gx, cscale(kg, dkx * inv))), sc);
      out[1] = cscale(cadd(cscale(is, dky), csub(gy, cscale(kg, dky * inv))), sc);
    }
  }
}

// symbol at (kx, ky) for a column other than the packed one
template <typename T, int OP, int NI, int NO>
__device__ __forceinline__ void symbol_point(const ColParams<T>& p, T lapx, T derx, T lapy, T dery,
                                             const cplx<T> (&in)[NI], cplx<T> (&out)[NO]) {
  apply_symbol<T, OP>(p, lapx + lapy, derx, dery, in, out);
}

// symbol on the packed kx = 0 | kx = n/2 column at ky, from P(ky) and P(−ky) of every input field:
// P = Â + i B̂ with Â, B̂ Hermitian in ky; output Â' + i B̂' at ky
template <typename T, int OP, int NI, int NO>
__device__ __forceinline__ void symbol_packed(const ColParams<T>& p, T lap0, T der0, T lapn, T dern, T lapy,
                                              T dery, const cplx<T> (&P)[NI], const cplx<T> (&Pm)[NI],
                                              cplx<T> (&out)[NO]) {
  cplx<T> A[NI], B[NI], oA[NO], oB[NO];
#pragma unroll
  for (int f = 0; f < NI; ++f) {
    // Â(j) = (P(j) + conj P(−j))/2, B̂(j) = −i (P(j) − conj P(−j))/2
    A[f] = mk(T(0.5) * (P[f].x + Pm[f].x), T(0.5) * (P[f].y - Pm[f].y));
    B[f] = mk(T(0.5) * (P[f].y + Pm[f].y), T(0.5) * (Pm[f].x - P[f].x));
  }
  apply_symbol<T, OP>(p, lap0 + lapy, der0, dery, A, oA);
  apply_symbol<T, OP>(p, lapn + lapy, dern, dery, B, oB);
#pragma unroll
  for (int f = 0; f < NO; ++f) out[f] = cadd(oA[f], cmuli(oB[f]));
}

// ------------------------------------------------------------------------------------------
// kernel 2: FFT along y, symbol, inverse FFT along y, for C kx columns per CTA
// ------------------------------------------------------------------------------------------
// offset of element (row m) of column k of field f in the band-major half spectra
// (a geometry's half spectra hold at most 4·8192·4096 < 2^31 elements, so 32-bit offsets suffice)
template <int L>
__device__ __forceinline__ int col_at(int f, int m, int k, int R) {
  constexpr int n = 1 << L, nh = n / 2;
  return (f * n + (m & ~(R - 1))) * nh + k * R + (m & (R - 1));
}
// row j + s·Q of a lane (j < Q = n/8): with R ≤ Q (the planner keeps it so) the rows j + s·Q
// lie in bands s·Q/R apart at the same offset, so the element is col_at(f, j, k, R) + s·Q·n/2
template <int L>
__device__ __forceinline__ int col_at_s(int f, int j, int s, int k, int R) {
  constexpr int Q = (1 << L) / 8, nh = (1 << L) / 2;
  return col_at<L>(f, j, k, R) + s * (Q * nh);
}

template <typename T, int OP, int L, bool PF = true>
__device__ __forceinline__ void colpass_body(const ColParams<T>& p, int unit, unsigned char* smem_raw) {
  constexpr int NIN = Traits<OP>::NIN;
  constexpr int NOUT = Traits<OP>::NOUT;
  constexpr int NMAX = NIN > NOUT ? NIN : NOUT;
  using CF = Cfg2<T, L, NMAX>;
  using F = F8<L, CF::V>;
  constexpr int n = F::N, nh = n / 2, V = CF::V, QT = CF::QT, NGRP = CF::NGRP, Q = F::Q;
  const int C = p.C, R = p.R;
  const int k0 = unit * C;
  // thread (group g, column c, lane j0), the group's C columns interleaved across threads
  int g, c, j0;
  col_lane_2d<QT>(C, g, c, j0);
  const bool active = g < NGRP;
  const int kx = k0 + c;
  // sequence (field f, column c) at buf + (f·C + c)·PN
  const int PN = col_stride_2d(L, C, (int)sizeof(cplx<T>));
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  typename CF::TW tw[V];
#pragma unroll
  for (int v = 0; v < V; ++v) tw[v].load(p.tw, j0 + v * QT);
  // per-axis symbols: kx of this column (the packed column also needs kx = n/2) and, with one
  // field in and out, ky of the lane's rows, loaded before the wait; with more fields the ky
  // values are read at use (registers go to the fields)
  constexpr bool PREF = PF && NIN == 1 && NOUT == 1;
  const bool packed = k0 == 0;  // uniform over the CTA: column 0 holds kx = 0 and kx = n/2
  T lapx = T(0), derx = T(0), lapn = T(0), dern = T(0);
  T lapy[PREF ? V : 1][8], dery[PREF ? V : 1][8];
  if (active) {
    lapx = p.lap1[kx];
    derx = p.der1[kx];
    lapn = p.lap1[nh];
    dern = p.der1[nh];
    if constexpr (PREF) {
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          lapy[v][s] = p.lap1[j0 + v * QT + s * Q];
          dery[v][s] = p.der1[j0 + v * QT + s * Q];
        }
    }
  }
  // The stop flag is final before the wait: it is written by the GMRES step (or the cycle start)
  // at least two kernels back, which has completed once the direct predecessor (the spread,
  // which always waits) passed its own wait and triggered this launch. So no dependent load
  // follows the wait, and a slot after the stop returns without waiting: the kernels after it
  // only read the same final flag.
  const bool stopped = p.stop && *p.stop;
  if (stopped) return;
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();  // after the wait (see the spread kernel)

  if constexpr (NIN == 1 && NOUT == 1) {
    // one field in and out: the symbol is applied to the registers between the transforms
    cplx<T>* sb = buf + (size_t)c * PN;
    cplx<T> x[1][V][8];
    if (active) {
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int s = 0; s < 8; ++s) x[0][v][s] = p.spec[col_at_s<L>(0, j0 + v * QT, s, kx, R)];
    }
    f8_fft<T, false, L, V, 1>(x, sb, 0, j0, tw, active);
    if (packed) {
      // the packed column needs P(−ky): every lane stores its own positions (free of conflicts
      // with the last exchange, which read only those), then reads the partner's
      if (active) {
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int s = 0; s < 8; ++s) sb[ppos_strided<Q>(j0 + v * QT, s)] = x[0][v][s];
      }
      __syncthreads();
    }
    if (active) {
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          const cplx<T> in[1] = {x[0][v][s]};
          cplx<T> out[1];
          const int ky = j0 + v * QT + s * Q;
          const T ly = PREF ? lapy[PREF ? v : 0][s] : p.lap1[ky], dy = PREF ? dery[PREF ? v : 0][s] : p.der1[ky];
          if (kx == 0) {
            const cplx<T> pm[1] = {sb[ppos((n - ky) & (n - 1))]};
            symbol_packed<T, OP>(p, lapx, derx, lapn, dern, ly, dy, in, pm, out);
          } else {
            symbol_point<T, OP>(p, lapx, derx, ly, dy, in, out);
          }
          x[0][v][s] = out[0];
        }
    }
    // (the inverse transform's first exchange barrier orders the partner reads before its writes)
    f8_fft<T, true, L, V, 1>(x, sb, 0, j0, tw, active);
    if (active) {
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int s = 0; s < 8; ++s) p.spec[col_at_s<L>(0, j0 + v * QT, s, kx, R)] = x[0][v][s];
    }
  } else {
    // forward transforms of the NIN input fields, results left in shared memory
#pragma unroll
    for (int k = 0; k < (NIN + NGRP - 1) / NGRP; ++k) {
      const int f = g + k * NGRP;
      const bool act = active && f < NIN;
      cplx<T>* sb = buf + ((size_t)f * C + c) * PN;
      cplx<T> x[1][V][8];
      if (act) {
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int s = 0; s < 8; ++s) x[0][v][s] = p.spec[col_at_s<L>(f, j0 + v * QT, s, kx, R)];
      }
      f8_fft<T, false, L, V, 1>(x, sb, 0, j0, tw, act);
      if (act) {
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int s = 0; s < 8; ++s) sb[ppos_strided<Q>(j0 + v * QT, s)] = x[0][v][s];
      }
    }
    __syncthreads();
    // symbol at the points of the lane's positions, split over the groups (point s to group
    // s mod NGRP), in place; the packed column reads its partners (P(−ky)) and writes after a
    // second barrier
    if (!packed) {
      if (active) {
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int s = 0; s < 8; ++s) {
            if (s % NGRP != g) continue;
            const int ky = j0 + v * QT + s * Q;
            cplx<T> in[NIN], o[NOUT];
#pragma unroll
            for (int f = 0; f < NIN; ++f) in[f] = buf[((size_t)f * C + c) * PN + ppos(ky)];
            symbol_point<T, OP>(p, lapx, derx, p.lap1[ky], p.der1[ky], in, o);
#pragma unroll
            for (int f = 0; f < NOUT; ++f) buf[((size_t)f * C + c) * PN + ppos(ky)] = o[f];
          }
      }
    } else {
      cplx<T> o[V][8][NOUT];
      if (active) {
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int s = 0; s < 8; ++s) {
            if (s % NGRP != g) continue;
            const int ky = j0 + v * QT + s * Q;
            cplx<T> in[NIN];
#pragma unroll
            for (int f = 0; f < NIN; ++f) in[f] = buf[((size_t)f * C + c) * PN + ppos(ky)];
            if (kx == 0) {
              cplx<T> pm[NIN];
#pragma unroll
              for (int f = 0; f < NIN; ++f) pm[f] = buf[((size_t)f * C + c) * PN + ppos((n - ky) & (n - 1))];
              symbol_packed<T, OP>(p, lapx, derx, lapn, dern, p.lap1[ky], p.der1[ky], in, pm, o[v][s]);
            } else {
              symbol_point<T, OP>(p, lapx, derx, p.lap1[ky], p.der1[ky], in, o[v][s]);
            }
          }
      }
      __syncthreads();
      if (active) {
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int s = 0; s < 8; ++s) {
            if (s % NGRP != g) continue;
#pragma unroll
            for (int f = 0; f < NOUT; ++f) buf[((size_t)f * C + c) * PN + ppos_strided<Q>(j0 + v * QT, s)] = o[v][s][f];
          }
      }
    }
    __syncthreads();
    // inverse transforms of the NOUT output fields, straight to the half spectra
#pragma unroll
    for (int k = 0; k < (NOUT + NGRP - 1) / NGRP; ++k) {
      const int f = g + k * NGRP;
      const bool act = active && f < NOUT;
      cplx<T>* sb = buf + ((size_t)f * C + c) * PN;
      cplx<T> x[1][V][8];
      if (act) {
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int s = 0; s < 8; ++s) x[0][v][s] = sb[ppos_strided<Q>(j0 + v * QT, s)];
      }
      f8_fft<T, true, L, V, 1>(x, sb, 0, j0, tw, act);
      if (act) {
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int s = 0; s < 8; ++s) p.spec[col_at_s<L>(f, j0 + v * QT, s, kx, R)] = x[0][v][s];
      }
    }
  }
}

// Persistent batched column pass of a one-field operator (the scalar operator's batches): a
// CTA takes the units blockIdx.x, blockIdx.x + gridDim.x, … of this size's range (all of one
// grid size, so equal work: a static round-robin balances them) and loads the next unit's
// columns into registers before it transforms the current one, so that one unit's HBM latency
// overlaps the previous unit's transforms.
template <typename T, int L>
__device__ __forceinline__ void colpass1_load(const ColParams<T>& p, int unit, int c, int j0, bool active,
                                              cplx<T> (&x)[1][Cfg2<T, L, 1>::V][8]) {
  using CF = Cfg2<T, L, 1>;
  constexpr int V = CF::V, QT = CF::QT;
  const int kx = unit * p.C + c;
  if (active) {
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int s = 0; s < 8; ++s) x[0][v][s] = p.spec[col_at_s<L>(0, j0 + v * QT, s, kx, p.R)];
  }
}

template <typename T, int OP, int L>
__global__ void __launch_bounds__(kMaxThreads2d) kbp_colpass(const ColParams<T>* __restrict__ P, const int2* units,
                                                             int nunits) {
  static_assert(Traits<OP>::NIN == 1 && Traits<OP>::NOUT == 1, "one field in and out");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using CF = Cfg2<T, L, 1>;
  using F = F8<L, CF::V>;
  constexpr int n = F::N, nh = n / 2, V = CF::V, QT = CF::QT, Q = F::Q, PN = F::PN;
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  int u = blockIdx.x;
  if (u >= nunits) return;
  const int q = threadIdx.x / QT, j0 = threadIdx.x - q * QT;
  TwTable<T, L> tw[V];
#pragma unroll
  for (int v = 0; v < V; ++v) tw[v].load(P[units[u].x].tw, j0 + v * QT);
  int2 cu = units[u];
  ColParams<T> p = P[cu.x];
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
  cplx<T> x[1][V][8];
  colpass1_load<T, L>(p, cu.y, q % p.C, j0, q < p.C && !(p.stop && *p.stop), x);
  for (;;) {
    const int c = q % p.C, k0 = cu.y * p.C, kx = k0 + c;
    const bool stopped = p.stop && *p.stop;  // uniform over the CTA
    const bool active = q < p.C && !stopped;
    // the next unit: its parameters and its columns, loaded before this unit's transforms
    const int un = u + gridDim.x;
    const bool more = un < nunits;
    int2 nu = make_int2(0, 0);
    ColParams<T> pn = p;
    cplx<T> xn[1][V][8];
    if (more) {
      nu = units[un];
      pn = P[nu.x];
      colpass1_load<T, L>(pn, nu.y, q % pn.C, j0, q < pn.C && !(pn.stop && *pn.stop), xn);
    }
    if (!stopped) {
      cplx<T>* sb = buf + (size_t)(q < p.C ? c : 0) * PN;
      f8_fft<T, false, L, V, 1>(x, sb, 0, j0, tw, active);
      const T lapx = p.lap1[kx], derx = p.der1[kx], lapn = p.lap1[nh], dern = p.der1[nh];
      if (k0 == 0) {
        if (active) {
#pragma unroll
          for (int v = 0; v < V; ++v)
#pragma unroll
            for (int s = 0; s < 8; ++s) sb[ppos_strided<Q>(j0 + v * QT, s)] = x[0][v][s];
        }
        __syncthreads();
      }
      if (active) {
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int s = 0; s < 8; ++s) {
            const cplx<T> in[1] = {x[0][v][s]};
            cplx<T> out[1];
            const int ky = j0 + v * QT + s * Q;
            if (kx == 0) {
              const cplx<T> pm[1] = {sb[ppos((n - ky) & (n - 1))]};
              symbol_packed<T, OP>(p, lapx, derx, lapn, dern, p.lap1[ky], p.der1[ky], in, pm, out);
            } else {
              symbol_point<T, OP>(p, lapx, derx, p.lap1[ky], p.der1[ky], in, out);
            }
            x[0][v][s] = out[0];
          }
      }
      f8_fft<T, true, L, V, 1>(x, sb, 0, j0, tw, active);
      if (active) {
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int s = 0; s < 8; ++s) p.spec[col_at_s<L>(0, j0 + v * QT, s, kx, p.R)] = x[0][v][s];
      }
    }
    if (!more) break;
    __syncthreads();  // this unit's shared-memory reads are done before the next unit's writes
    u = un;
    cu = nu;
    p = pn;
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int s = 0; s < 8; ++s) x[0][v][s] = xn[0][v][s];
  }
}

template <typename T, int OP, int L>
__global__ void __launch_bounds__(kMaxThreads2d) k_colpass(ColParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  colpass_body<T, OP, L>(p, blockIdx.x, smem_raw);
}

// ------------------------------------------------------------------------------------------
// kernel 2, one field at a time: for grids whose columns of every field do not fit shared memory
// together, the column stage runs as the forward transform of each input field (in place), one
// pointwise symbol launch over the whole spectrum, and the inverse transform of each output field
// ------------------------------------------------------------------------------------------
template <typename T, int L, bool INV>
__global__ void __launch_bounds__(kMaxThreads2d) k_colfft(ColParams<T> p, int field) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using CF = Cfg2<T, L, 1>;
  using F = F8<L, CF::V>;
  constexpr int V = CF::V, QT = CF::QT;
  const int C = p.C, R = p.R, kx0 = blockIdx.x * C;
  int g, c, j0;
  col_lane_2d<QT>(C, g, c, j0);
  const bool active = g < 1;
  const int kx = kx0 + c;
  cplx<T>* sb = reinterpret_cast<cplx<T>*>(smem_raw) + (size_t)c * col_stride_2d(L, C, (int)sizeof(cplx<T>));
  typename CF::TW tw[V];
#pragma unroll
  for (int v = 0; v < V; ++v) tw[v].load(p.tw, j0 + v * QT);
  const bool stopped = p.stop && *p.stop;  // final before the wait (see the column pass)
  if (stopped) return;
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
  cplx<T> x[1][V][8];
  if (active) {
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int s8 = 0; s8 < 8; ++s8) x[0][v][s8] = p.spec[col_at_s<L>(field, j0 + v * QT, s8, kx, R)];
  }
  f8_fft<T, INV, L, V, 1>(x, sb, 0, j0, tw, active);
  if (active) {
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int s8 = 0; s8 < 8; ++s8) p.spec[col_at_s<L>(field, j0 + v * QT, s8, kx, R)] = x[0][v][s8];
  }
}

// The Fourier symbol at every (ky, kx) of the transformed spectra, NIN fields in and NOUT out, in
// place, one thread per point in memory order (band b, column kx, row r of the band); the packed
// kx = 0 | n/2 column is taken in pairs (ky, −ky) by the thread of the smaller ky.
template <typename T, int OP, int L>
__global__ void __launch_bounds__(256) k_symbol2d(ColParams<T> p) {
  constexpr int NIN = Traits<OP>::NIN, NOUT = Traits<OP>::NOUT;
  constexpr int n = 1 << L, nh = n / 2;
  const bool stopped = p.stop && *p.stop;  // final before the wait (see the column pass)
  if (stopped) return;
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
  const int R = p.R;
  const size_t fstride = (size_t)n * nh;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * nh; idx += gridDim.x * blockDim.x) {
    const int r = idx & (R - 1), kx = (idx / R) & (nh - 1), ky = (idx / (nh * R)) * R + r;
    if (kx == 0 && ky > nh) continue;
    cplx<T> in[NIN], o[NOUT];
#pragma unroll
    for (int f = 0; f < NIN; ++f) in[f] = p.spec[f * fstride + idx];
    if (kx != 0) {
      symbol_point<T, OP>(p, p.lap1[kx], p.der1[kx], p.lap1[ky], p.der1[ky], in, o);
#pragma unroll
      for (int f = 0; f < NOUT; ++f) p.spec[f * fstride + idx] = o[f];
    } else {
      const int ky2 = (n - ky) & (n - 1);
      const int idx2 = (ky2 & ~(R - 1)) * nh + (ky2 & (R - 1));  // (ky2, kx = 0)
      cplx<T> pm[NIN], o2[NOUT];
#pragma unroll
      for (int f = 0; f < NIN; ++f) pm[f] = p.spec[f * fstride + idx2];
      const T lap0 = p.lap1[0], der0 = p.der1[0], lapn = p.lap1[nh], dern = p.der1[nh];
      symbol_packed<T, OP>(p, lap0, der0, lapn, dern, p.lap1[ky], p.der1[ky], in, pm, o);
      if (ky2 != ky) symbol_packed<T, OP>(p, lap0, der0, lapn, dern, p.lap1[ky2], p.der1[ky2], pm, in, o2);
#pragma unroll
      for (int f = 0; f < NOUT; ++f) p.spec[f * fstride + idx] = o[f];
      if (ky2 != ky) {
#pragma unroll
        for (int f = 0; f < NOUT; ++f) p.spec[f * fstride + idx2] = o2[f];
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// kernel 2, staged form (FP32): persistent CTAs walk the column units of one grid size (of one
// problem, or of every problem of that size in a batch). Each unit's C columns of all input fields,
// and its problem's symbol tables, are copied into shared memory by the tensor memory accelerator
// NS units ahead of their use, so that the loads of the next units overlap the transforms of the
// current one; the column values then come from shared memory instead of scattered global loads.
// ------------------------------------------------------------------------------------------
// A stage holds one unit as the tensor map's boxes land: field f, band b = m/R, column c, row
// m mod R of the band at complex offset (f·(n/R) + b)·C·R + c·R + (m mod R) = f·n·C + (m/R)·C·R +
// c·R + (m mod R); then lap1[0 … n) and der1[0 … n) (floats). The tensor map of a problem's FP32
// half spectra has dimensions (x: R·n floats of a band, y: n/R bands, z: fields) and a box of
// (2·C·R, min(n/R, 256), 1): one copy per field and 256 bands.
struct ColStageArgs {
  const ColParams<float>* P;  // batch: parameter block per problem (NULL: the single problem)
  const CUtensorMap* maps;    // batch: tensor map per problem, in global memory
  const int2* units;          // batch: (problem, column unit) of this grid size
  int nunits;                 // units to walk
  int stages;                 // NS (2 … 4)
  int stage_bytes;            // bytes per stage (a multiple of 128)
  int* err;                   // set to 1 when a stage's copies do not arrive within the wait limit
};

template <int OP, int L>
__global__ void __launch_bounds__(kMaxThreads2d)
    kt_colpass(const __grid_constant__ ColParams<float> p1, const __grid_constant__ CUtensorMap map1,
               const ColStageArgs A) {
  using T = float;
  constexpr int NIN = Traits<OP>::NIN;
  constexpr int NOUT = Traits<OP>::NOUT;
  constexpr int NMAX = NIN > NOUT ? NIN : NOUT;
  using CF = Cfg2<T, L, NMAX>;
  using F = F8<L, CF::V>;
  constexpr int n = F::N, nh = n / 2, V = CF::V, QT = CF::QT, NGRP = CF::NGRP, Q = F::Q;
  // the stages start on a 128-byte boundary (the launch adds 128 bytes of slack for it)
  extern __shared__ __align__(16) unsigned char smem_stage[];
  unsigned char* base = smem_stage + ((128u - (smem_addr(smem_stage) & 127u)) & 127u);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base);  // NS barriers in the first 128 bytes
  unsigned char* stages = base + 128;
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(stages + (size_t)A.stages * A.stage_bytes);
  const int NS = A.stages;
  const int cnt = (int)blockIdx.x < A.nunits ? (A.nunits - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  if (cnt == 0) return;  // (the host launches at most one CTA per unit)

  auto unit_of = [&](int i, const ColParams<T>*& q, const CUtensorMap*& m, int& cu) {
    const int u = (int)blockIdx.x + i * (int)gridDim.x;
    if (A.P) {
      const int2 t = A.units[u];
      q = A.P + t.x;
      m = A.maps + t.x;
      cu = t.y;
    } else {
      q = &p1;
      m = &map1;
      cu = u;
    }
  };
  // thread 0: start the copies of this CTA's unit i into stage s
  auto issue = [&](int i, int s) {
    const ColParams<T>* q;
    const CUtensorMap* m;
    int cu;
    unit_of(i, q, m, cu);
    const int C = q->C, R = q->R, nb = n / R, box1 = nb < 256 ? nb : 256;
    unsigned char* st = stages + (size_t)s * A.stage_bytes;
    const uint32_t dbytes = (uint32_t)NIN * C * n * sizeof(cplx<T>);
    mbar_arrive_expect_tx(&bar[s], dbytes + 2u * n * sizeof(T));
    if (A.P) tmap_acquire(m);
    for (int f = 0; f < NIN; ++f)
      for (int y0 = 0; y0 < nb; y0 += box1)
        tma_load_3d(st + ((size_t)f * nb + y0) * C * R * sizeof(cplx<T>), m, &bar[s], 2 * cu * C * R, y0, f);
    bulk_load(st + dbytes, q->lap1, n * sizeof(T), &bar[s]);
    bulk_load(st + dbytes + n * sizeof(T), q->der1, n * sizeof(T), &bar[s]);
  };

  // prologue independent of the previous kernel: barriers and twiddles (every problem of one
  // size has the same twiddle values)
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bar[s], 1);
    mbar_init_fence();
  }
  typename CF::TW tw[V];
  {
    const ColParams<T>* q0;
    const CUtensorMap* m0;
    int c0;
    unit_of(0, q0, m0, c0);
    // (every unit of a launch has the same column group C, so a lane keeps its twiddles)
    int gg, cc, jj;
    col_lane_2d<QT>(q0->C, gg, cc, jj);
    const cplx<T>* twp = q0->tw;
#pragma unroll
    for (int v = 0; v < V; ++v) tw[v].load(twp, jj + v * QT);
  }
  __syncthreads();
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();  // after the wait (see the spread kernel)
  if (threadIdx.x == 0)
    for (int i = 0; i < NS && i < cnt; ++i) issue(i, i);

  for (int i = 0; i < cnt; ++i) {
    const int s = i % NS;
    const bool ok = mbar_wait_bounded(&bar[s], (uint32_t)((i / NS) & 1));
    if (__syncthreads_or(!ok)) {
      // the copies did not arrive: record it, wait (bounded) for the copies still in flight, stop
      if (threadIdx.x == 0) {
        if (A.err) atomicExch(A.err, 1);
        for (int k = i; k < i + NS && k < cnt; ++k) mbar_wait_bounded(&bar[k % NS], (uint32_t)((k / NS) & 1));
      }
      return;
    }
    const ColParams<T>* q;
    const CUtensorMap* m;
    int cu;
    unit_of(i, q, m, cu);
    const ColParams<T> qv = *q;
    const int C = qv.C, R = qv.R, k0 = cu * C;
    int g, c, j0;
    col_lane_2d<QT>(C, g, c, j0);
    const bool active = g < NGRP;
    const int kx = k0 + c;
    const int PN = col_stride_2d(L, C, (int)sizeof(cplx<T>));
    const bool packed = k0 == 0;
    const bool stopped = qv.stop && *qv.stop;  // uniform over the CTA (one problem per unit)
    const unsigned char* st = stages + (size_t)s * A.stage_bytes;
    const cplx<T>* sx = reinterpret_cast<const cplx<T>*>(st);
    const T* slap = reinterpret_cast<const T*>(st + (size_t)NIN * C * n * sizeof(cplx<T>));
    const T* sder = slap + n;
    // staged element (field f, row j + s·Q, column c) = sx[f·n·C + xb(j) + s·Q·C]
    auto xb = [&](int j) { return (j / R) * C * R + c * R + (j & (R - 1)); };
    const T lapx = slap[kx], derx = sder[kx], lapn = slap[nh], dern = sder[nh];
    cplx<T> x[1][V][8];
    if constexpr (NIN == 1 && NOUT == 1) {
      cplx<T>* sb = buf + (size_t)c * PN;
      if (!stopped) {
        if (active) {
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const int b = xb(j0 + v * QT);
#pragma unroll
            for (int s8 = 0; s8 < 8; ++s8) x[0][v][s8] = sx[b + s8 * Q * C];
          }
        }
        f8_fft<T, false, L, V, 1>(x, sb, 0, j0, tw, active);
        if (packed) {
          if (active) {
#pragma unroll
            for (int v = 0; v < V; ++v)
#pragma unroll
              for (int s8 = 0; s8 < 8; ++s8) sb[ppos_strided<Q>(j0 + v * QT, s8)] = x[0][v][s8];
          }
          __syncthreads();
        }
        if (active) {
#pragma unroll
          for (int v = 0; v < V; ++v)
#pragma unroll
            for (int s8 = 0; s8 < 8; ++s8) {
              const cplx<T> in[1] = {x[0][v][s8]};
              cplx<T> out[1];
              const int ky = j0 + v * QT + s8 * Q;
              if (kx == 0) {
                const cplx<T> pm[1] = {sb[ppos((n - ky) & (n - 1))]};
                symbol_packed<T, OP>(qv, lapx, derx, lapn, dern, slap[ky], sder[ky], in, pm, out);
              } else {
                symbol_point<T, OP>(qv, lapx, derx, slap[ky], sder[ky], in, out);
              }
              x[0][v][s8] = out[0];
            }
        }
      }
      // stage s is read: its next copies may start
      __syncthreads();
      if (threadIdx.x == 0 && i + NS < cnt) issue(i + NS, s);
      if (!stopped) {
        f8_fft<T, true, L, V, 1>(x, sb, 0, j0, tw, active);
        if (active) {
#pragma unroll
          for (int v = 0; v < V; ++v)
#pragma unroll
            for (int s8 = 0; s8 < 8; ++s8) qv.spec[col_at_s<L>(0, j0 + v * QT, s8, kx, R)] = x[0][v][s8];
        }
      }
    } else {
      if (!stopped) {
        // forward transforms of the NIN input fields, results left in the exchange buffers
#pragma unroll
        for (int k = 0; k < (NIN + NGRP - 1) / NGRP; ++k) {
          const int f = g + k * NGRP;
          const bool act = active && f < NIN;
          cplx<T>* sb = buf + ((size_t)f * C + c) * PN;
          if (act) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
              const int b = f * n * C + xb(j0 + v * QT);
#pragma unroll
              for (int s8 = 0; s8 < 8; ++s8) x[0][v][s8] = sx[b + s8 * Q * C];
            }
          }
          f8_fft<T, false, L, V, 1>(x, sb, 0, j0, tw, act);
          if (act) {
#pragma unroll
            for (int v = 0; v < V; ++v)
#pragma unroll
              for (int s8 = 0; s8 < 8; ++s8) sb[ppos_strided<Q>(j0 + v * QT, s8)] = x[0][v][s8];
          }
        }
        __syncthreads();
        // symbol at the points of the lane's positions, split over the groups (point s to group
        // s mod NGRP), in place; the packed column reads its partners first and writes after a
        // second barrier
        if (!packed) {
          if (active) {
#pragma unroll
            for (int v = 0; v < V; ++v)
#pragma unroll
              for (int s8 = 0; s8 < 8; ++s8) {
                if (s8 % NGRP != g) continue;
                const int ky = j0 + v * QT + s8 * Q;
                cplx<T> in[NIN], o[NOUT];
#pragma unroll
                for (int f = 0; f < NIN; ++f) in[f] = buf[((size_t)f * C + c) * PN + ppos(ky)];
                symbol_point<T, OP>(qv, lapx, derx, slap[ky], sder[ky], in, o);
#pragma unroll
                for (int f = 0; f < NOUT; ++f) buf[((size_t)f * C + c) * PN + ppos(ky)] = o[f];
              }
          }
        } else {
          cplx<T> o[V][8][NOUT];
          if (active) {
#pragma unroll
            for (int v = 0; v < V; ++v)
#pragma unroll
              for (int s8 = 0; s8 < 8; ++s8) {
                if (s8 % NGRP != g) continue;
                const int ky = j0 + v * QT + s8 * Q;
                cplx<T> in[NIN];
#pragma unroll
                for (int f = 0; f < NIN; ++f) in[f] = buf[((size_t)f * C + c) * PN + ppos(ky)];
                if (kx == 0) {
                  cplx<T> pm[NIN];
#pragma unroll
                  for (int f = 0; f < NIN; ++f) pm[f] = buf[((size_t)f * C + c) * PN + ppos((n - ky) & (n - 1))];
                  symbol_packed<T, OP>(qv, lapx, derx, lapn, dern, slap[ky], sder[ky], in, pm, o[v][s8]);
                } else {
                  symbol_point<T, OP>(qv, lapx, derx, slap[ky], sder[ky], in, o[v][s8]);
                }
              }
          }
          __syncthreads();
          if (active) {
#pragma unroll
            for (int v = 0; v < V; ++v)
#pragma unroll
              for (int s8 = 0; s8 < 8; ++s8) {
                if (s8 % NGRP != g) continue;
#pragma unroll
                for (int f = 0; f < NOUT; ++f)
                  buf[((size_t)f * C + c) * PN + ppos_strided<Q>(j0 + v * QT, s8)] = o[v][s8][f];
              }
          }
        }
      }
      // stage s is read (and the symbol's results are written): its next copies may start
      __syncthreads();
      if (threadIdx.x == 0 && i + NS < cnt) issue(i + NS, s);
      if (!stopped) {
        // inverse transforms of the NOUT output fields, straight to the half spectra
#pragma unroll
        for (int k = 0; k < (NOUT + NGRP - 1) / NGRP; ++k) {
          const int f = g + k * NGRP;
          const bool act = active && f < NOUT;
          cplx<T>* sb = buf + ((size_t)f * C + c) * PN;
          if (act) {
#pragma unroll
            for (int v = 0; v < V; ++v)
#pragma unroll
              for (int s8 = 0; s8 < 8; ++s8) x[0][v][s8] = sb[ppos_strided<Q>(j0 + v * QT, s8)];
          }
          f8_fft<T, true, L, V, 1>(x, sb, 0, j0, tw, act);
          if (act) {
#pragma unroll
            for (int v = 0; v < V; ++v)
#pragma unroll
              for (int s8 = 0; s8 < 8; ++s8) qv.spec[col_at_s<L>(f, j0 + v * QT, s8, kx, R)] = x[0][v][s8];
          }
        }
      }
    }
    // the next unit's first exchange writes follow its own wait barrier, which orders them after
    // this unit's last reads of the exchange buffers
  }
}

// ------------------------------------------------------------------------------------------
// kernel 3: inverse FFT along x, then interpolation (or write the grid)
// ------------------------------------------------------------------------------------------
// Z_m = A_m + i B_m (m = 0..n−1) for the row pair (r0 + 2j, r0 + 2j + 1) of field f, rebuilt from
// the band-major half spectra (A_{n−k} = conj A_k): A_k at band offset k·R + 2j, B_k next to it.
template <typename T, int L>
__device__ __forceinline__ cplx<T> row_z(const cplx<T>* __restrict__ spec, int f, int r0, int jj, int R, int m) {
  constexpr int n = 1 << L, nh = n / 2;
  const cplx<T>* band = spec + ((f * n + r0) * nh + 2 * jj);
  cplx<T> A, B;
  if (m == 0 || m == nh) {
    load_pair(band, A, B);
    return m == 0 ? mk(A.x, B.x) : mk(A.y, B.y);
  }
  const int k = m < nh ? m : n - m;
  load_pair(band + k * R, A, B);
  return m < nh ? mk(A.x - B.y, A.y + B.x) : mk(A.x + B.y, B.x - A.y);
}

// One gather work item (point, stencil row): the point-table values it needs
template <typename T>
struct GatherItem {
  int lr, i, bx;
  T py, dy, ws, nx, ny;
  T px[4], dx[4];
};
template <typename T>
__device__ __forceinline__ GatherItem<typename Prec2<T>::PT> gather_item(const RowParams<T>& p, const PointRanges& pr,
                                                                         int t, int r0) {
  const int n = p.n, M = p.M;
  const int s = pr.at(t >> 2);
  const int ay = t & 3;
  GatherItem<typename Prec2<T>::PT> it;
  it.lr = (((p.base[M + s] + ay) & (n - 1)) - r0) & (n - 1);
  it.i = p.perm[s];
  it.bx = p.base[s];
  it.py = p.phi[(1 * 4 + ay) * M + s];
  it.dy = p.dphi[(1 * 4 + ay) * M + s];
  it.ws = p.wscale[s];
  it.nx = p.nrm[s];
  it.ny = p.nrm[M + s];
#pragma unroll
  for (int ax = 0; ax < 4; ++ax) {
    it.px[ax] = p.phi[(0 * 4 + ax) * M + s];
    it.dx[ax] = p.dphi[(0 * 4 + ax) * M + s];
  }
  return it;
}

// SPLIT: one output field (p.fsel) per launch (see the spread kernel); its contribution to every
// boundary component is added to Y (the operator is linear in the interpolated fields).
template <typename T, int OP, int GMODE, int L, bool PF = true, bool SPLIT = false>
__device__ __forceinline__ void rowifft_gather_body(const RowParams<T>& p, int unit, unsigned char* smem_raw) {
  constexpr int NOUT = Traits<OP>::NOUT;
  constexpr int NB = SPLIT ? 1 : NOUT;  // fields held in shared memory
  using CF = Cfg2<T, L, NB>;
  using F = F8<L, CF::V>;
  using PT = typename Prec2<T>::PT;
  constexpr int n = F::N, V = CF::V, QT = CF::QT, NGRP = CF::NGRP, Q = F::Q;
  const int R = p.R, half = R >> 1, M = p.M;
  // sequences and lanes as in the spread kernel (row pairs interleaved across threads)
  const int PN = row_stride_2d(L, half, (int)sizeof(cplx<T>));
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  const int r0 = unit * R;
  // FFT lanes: thread (group g, row pair rp, lane j0); threads past NGRP·half·QT only gather
  int g, rp, j0;
  row_lane_2d<QT, row_interleave_2d(L, sizeof(T) == 4)>(half, g, rp, j0);
  const bool active = g < NGRP;
  typename CF::TW tw[V];
#pragma unroll
  for (int v = 0; v < V; ++v) tw[v].load(p.tw, j0 + v * QT);
  // the points whose stencil meets the band and this thread's first work item (4 per point),
  // loaded before the wait: the point tables are constant
  const PointRanges pr = band_points(p.cell_start, n, r0, R);
  const int nitems = GMODE == G_GRID ? 0 : pr.cnt * 4;
  GatherItem<PT> it0 = {};
  if (PF && (int)threadIdx.x < nitems) it0 = gather_item(p, pr, threadIdx.x, r0);
  // the stop flag and the Krylov index (the output column) are final before the wait: the GMRES
  // step that writes them is three kernels back and completed before the column pass was
  // launched (see the column pass)
  const bool stopped = p.stop && *p.stop;
  if (stopped) return;
  const double* pin;
  double* pout;
  resolve_io(p, pin, pout);
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();  // after the wait (see the spread kernel)

  // inverse FFT of every (field, row pair) sequence, its first stage fed from the half spectra
#pragma unroll
  for (int k = 0; k < NB / NGRP; ++k) {
    const int f = g + k * NGRP;
    cplx<T>* sb = buf + ((size_t)f * half + rp) * PN;
    cplx<T> x[1][V][8];
    const int fs = SPLIT ? p.fsel : f;  // the spectrum field read
    if (active) {
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int s = 0; s < 8; ++s) x[0][v][s] = row_z<T, L>(p.spec, fs, r0, rp, R, j0 + v * QT + s * Q);
    }
    f8_fft<T, true, L, V, 1>(x, sb, 0, j0, tw, active);
    if (active) {
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int s = 0; s < 8; ++s) sb[ppos_strided<Q>(j0 + v * QT, s)] = x[0][v][s];
    }
  }
  __syncthreads();
  // real values: field f, local row lr, column x at element e = (f·half + lr/2)·n + x, part lr & 1
  const T* u = reinterpret_cast<const T*>(buf);

  if (GMODE == G_GRID) {
    for (int t = threadIdx.x; t < NB * R * n; t += blockDim.x) {
      const int f = t / (R * n);
      const int rem = t - f * R * n;
      const int lr = rem / n, x = rem - lr * n;
      const int fo = SPLIT ? p.fsel : f;  // the grid field written
      // the completed method's field is u₀ + ū (ū after the density in the input vector)
      const double ub = p.aug ? p.in[(size_t)Traits<OP>::C * M + fo] : 0.0;
      p.grid[((size_t)fo * n + r0 + lr) * n + x] =
          double(Prec2<T>::to_pt(u[2 * ((f * half + (lr >> 1)) * PN + ppos(x)) + (lr & 1)])) + ub;
    }
    return;
  }

  // one thread per (point, stencil row in the band): the row's partial sum is added to Y
  // (the next item's table values are loaded before this item's sums, as in the spread)
  GatherItem<PT> cur = it0;
  if (!PF && (int)threadIdx.x < nitems) cur = gather_item(p, pr, threadIdx.x, r0);
  for (int t = threadIdx.x; t < nitems; t += blockDim.x) {
    GatherItem<PT> nxt = {};
    if (t + (int)blockDim.x < nitems) nxt = gather_item(p, pr, t + blockDim.x, r0);
    const GatherItem<PT> it = cur;
    cur = nxt;
    const int lr = it.lr;
    if (lr >= R) continue;
    const int i = it.i;
    const int bx = it.bx;
    const PT py = it.py;
    const PT dy = (OP == OP_ADJ_AN || OP == OP_STOKES_T) ? it.dy : PT(0);
    // value of sequence lr/2 + field·half at column x (part lr & 1)
    const int eb = 2 * (lr >> 1) * PN + (lr & 1), fs2 = 2 * half * PN;
    auto uval = [&](int f, int x) { return Prec2<T>::to_pt(u[eb + f * fs2 + 2 * ppos(x)]); };
    if constexpr (SPLIT) {
      // the value, x-gradient and y-gradient gathers of field p.fsel (first slot)
      PT a = 0, gx = 0, gy = 0;
#pragma unroll
      for (int ax = 0; ax < 4; ++ax) {
        const int col = (bx + ax) & (n - 1);
        const PT px = it.px[ax], v0 = uval(0, col);
        a += v0 * px * py;
        if (OP == OP_STOKES_T) {
          gx += v0 * it.dx[ax] * py;
          gy += v0 * px * dy;
        }
      }
      const int fs = p.fsel;
      if (OP == OP_STOKES_AN || OP == OP_STOKES_SD) {
        atomicAdd(pout + (size_t)fs * M + i, double(a));  // field l is velocity component l
      } else if (OP == OP_ADJ_SD) {
        // −n_m S*(∂_m v) with field m = ∂_m v
        double val = -(fs == 0 ? double(it.nx) : double(it.ny)) * double(a);
        if (p.trans) val *= double(it.ws);
        atomicAdd(pout + i, val);
      } else if (OP == OP_STOKES_T) {
        // field 0 = v_s (a_s), 1 = v_gx (G_xx, G_xy), 2 = v_gy (G_yx, G_yy): their terms of
        // (Δs/h²)[n_l a_s + Σ_k n_k (G_lk + G_kl)]
        const double ws = double(it.ws), nx = double(it.nx), ny = double(it.ny);
        double ox, oy;
        if (fs == 0) {
          ox = nx * double(a);
          oy = ny * double(a);
        } else if (fs == 1) {
          ox = 2.0 * nx * double(gx) + ny * double(gy);
          oy = nx * double(gy);
        } else {
          ox = ny * double(gx);
          oy = nx * double(gx) + 2.0 * ny * double(gy);
        }
        atomicAdd(pout + i, ws * ox);
        atomicAdd(pout + M + i, ws * oy);
      } else {
        atomicAdd(pout + i, double(a));
      }
      continue;
    }
    if (OP == OP_STOKES_T) {
      // a_s = Σ v_s Φ, G_mk = Σ v_gm ∂_kΦ; out_l += (Δs/h²)[n_l a_s + Σ_k n_k (G_lk + G_kl)]
      PT as = 0, gxx = 0, gxy = 0, gyx = 0, gyy = 0;
#pragma unroll
      for (int ax = 0; ax < 4; ++ax) {
        const int col = (bx + ax) & (n - 1);
        const PT px = it.px[ax], dx = it.dx[ax];
        const PT vs = uval(0, col);
        const PT vx = uval(1, col);
        const PT vy = uval(2, col);
        as += vs * px * py;
        gxx += vx * dx * py;
        gxy += vx * px * dy;
        gyx += vy * dx * py;
        gyy += vy * px * dy;
      }
      const double ws = double(it.ws), nx = double(it.nx), ny = double(it.ny);
      const double cross = double(gxy) + double(gyx);
      atomicAdd(pout + i, ws * (nx * double(as) + 2.0 * nx * double(gxx) + ny * cross));
      atomicAdd(pout + M + i, ws * (ny * double(as) + nx * cross + 2.0 * ny * double(gyy)));
      continue;
    }
    PT acc0 = 0, acc1 = 0;
#pragma unroll
    for (int ax = 0; ax < 4; ++ax) {
      const int col = (bx + ax) & (n - 1);
      const PT px = it.px[ax];
      const PT v0 = uval(0, col);
      if (OP == OP_ADJ_AN) {
        acc0 += v0 * it.dx[ax] * py;
        acc1 += v0 * px * dy;
      } else {
        const PT pp = px * py;
        acc0 += v0 * pp;
        if (NOUT == 2) acc1 += uval(1, col) * pp;
      }
    }
    if (OP == OP_STOKES_AN || OP == OP_STOKES_SD) {
      atomicAdd(pout + i, double(acc0));
      atomicAdd(pout + M + i, double(acc1));
    } else if (OP == OP_ADJ_AN || OP == OP_ADJ_SD) {
      // analytic: (S̃)* v = n · (kernel-gradient gather of v); spectral: −Σ_m n_m S*(∂_m v)
      double val = double(it.nx) * double(acc0) + double(it.ny) * double(acc1);
      if (OP == OP_ADJ_SD) val = -val;
      if (p.trans) val *= double(it.ws);  // Δs/h^d · (S̃)* … for Aᵀ
      atomicAdd(pout + i, val);
    } else {
      atomicAdd(pout + i, double(acc0));
    }
  }
}

template <typename T, int OP, int GMODE, int L>
__global__ void __launch_bounds__(kMaxThreads2d) k_rowifft_gather(RowParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rowifft_gather_body<T, OP, GMODE, L>(p, blockIdx.x, smem_raw);
}
// one output field (p.fsel) per launch
template <typename T, int OP, int GMODE, int L>
__global__ void __launch_bounds__(kMaxThreads2d) k_rowifft_gather1(RowParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rowifft_gather_body<T, OP, GMODE, L, true, true>(p, blockIdx.x, smem_raw);
}

// ------------------------------------------------------------------------------------------
// batched launches: one grid per stage covers every problem of a batch; CTA i runs work unit
// units[i] = (problem, unit) with that problem's parameter block and transform size
// ------------------------------------------------------------------------------------------
// One batched kernel per stage and grid size: a CTA runs unit units[i] = (problem, unit) of a
// problem of this size with that problem's parameter block (the bodies load twiddles, symbol rows
// and the first gather item where they are used, which keeps registers down and occupancy up).
template <typename T, int OP, int L>
__global__ void __launch_bounds__(kMaxThreads2d) kb_spread_rowfft(const RowParams<T>* __restrict__ P, const int2* units,
                                                                  const double* in_base, double* out_base) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 u = units[blockIdx.x];
  RowParams<T> p = P[u.x];
  p.in = in_base + p.io_off;
  p.out = out_base + p.io_off;
  spread_rowfft_body<T, OP, L, false>(p, u.y, p.n / p.R, smem_raw);
}

template <typename T, int OP, int L>
__global__ void __launch_bounds__(kMaxThreads2d) kb_colpass(const ColParams<T>* __restrict__ P, const int2* units) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 u = units[blockIdx.x];
  const ColParams<T> p = P[u.x];
  colpass_body<T, OP, L, false>(p, u.y, smem_raw);
}

template <typename T, int OP, int L>
__global__ void __launch_bounds__(kMaxThreads2d) kb_rowifft_gather(const RowParams<T>* __restrict__ P, const int2* units,
                                                                   const double* in_base, double* out_base) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 u = units[blockIdx.x];
  RowParams<T> p = P[u.x];
  p.in = in_base + p.io_off;
  p.out = out_base + p.io_off;
  rowifft_gather_body<T, OP, G_INTERP, L, false>(p, u.y, smem_raw);
}

// ------------------------------------------------------------------------------------------
// shared memory and thread counts (host and device)
// ------------------------------------------------------------------------------------------
__host__ __device__ constexpr size_t padded_seq_2d(int L) { return (size_t(1) << L) + (size_t(1) << L) / 8; }
// row kernels: one padded sequence per field and row pair, then 32 doubles of reduction slots
// (the completed method's constraint rows in the spread kernel)
constexpr size_t kRowReduceBytes2d = 32 * sizeof(double);
template <typename T>
__host__ __device__ constexpr size_t smem_rows_2d(int nf, int R, int L) {
  return (size_t)nf * (R / 2) * row_stride_2d(L, R / 2, 2 * sizeof(T)) * 2 * sizeof(T) + kRowReduceBytes2d;
}
template <typename T>
__host__ __device__ constexpr size_t smem_cols_2d(int nf, int C, int L) {
  return (size_t)nf * C * col_stride_2d(L, C, 2 * sizeof(T)) * 2 * sizeof(T);
}

// Launch of one application's three kernels for a compile-time size (defined in the per-size
// translation units apply2d_n*.cu).
struct Launch2D {
  int R, C;                 // rows per band, kx columns per CTA
  size_t smem_row, smem_col, smem_gather;
  int threads_row, threads_col, threads_gather;
  bool pdl;
  int grid_mode;            // G_INTERP or G_GRID
  bool split;               // one field per launch (the shapes above are those of one field)
};

template <typename T, int OP, int L>
ibdl_status launch_apply_2d(Geometry* g, const RowParams<T>& rp, const ColParams<T>& cp, const Launch2D& lc,
                            cudaStream_t s);
template <typename T, int OP, int L>
ibdl_status set_attrs_2d();

}  // namespace ibdl
