// Two-dimensional IBDL operator: spread → FFT → Fourier symbol → inverse FFT → interpolate.
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
// Packed half spectrum: for a real row a, A_k (k = 0..n/2) is stored in n/2 slots with slot 0
// holding (A_0, A_{n/2}), both real. Along y, the kx = 0 and kx = n/2 columns are therefore one
// complex column a + i b with a, b real columns; the column pass separates them by Hermitian
// symmetry before the symbol and repacks after it.
//
// Band-major storage: the n rows of a field form bands of R rows (the row kernels' work unit),
// and element (row, k) of field f sits at (f·n + band·R)·(n/2) + k·R + (row mod R). A row band is
// one contiguous block, and a column reads R contiguous values per band (128 bytes at R = 16 in
// FP32) whatever the number of columns a CTA takes.
#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <vector>
#include <type_traits>
#include <utility>

#include "fft.cuh"

namespace ibdl {

enum { OP_SCALAR_AN = 0, OP_SCALAR_SD = 1, OP_STOKES_AN = 2, OP_STOKES_SD = 3, OP_ADJ_AN = 4,
       OP_ADJ_SD = 5, OP_STOKES_T = 6, OP_SL = 7 };

// grid fields entering / leaving the Fourier stage, and boundary components in / out
template <int OP>
struct Traits;
template <>
struct Traits<OP_SCALAR_AN> { static constexpr int NIN = 1, NOUT = 1, C = 1; };  // f = S̃Q
// (NMAX = max(NIN, NOUT) sizes the shared buffers of the column pass)
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

constexpr int kThreads = 512;

template <typename T>
struct RowParams {
  int n, log2n, R;
  int M;
  const int* cell_start;
  const int* base;
  const int* perm;
  const T* phi;
  const T* dphi;
  const T* wscale;
  const T* nrm;
  const double* in;   // [c][M] density
  double* out;        // [c][M] result (first kernel stores ½·in, last kernel adds S*u)
  cplx<T>* spec;      // [nf][n][n/2]
  const cplx<T>* tw;  // [n]
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
  T eta_src;              // weight of the ηSQ source: η (scalar) or η/μ (Stokes, projected part)
  int tw_smem;            // 1: the twiddles are staged in shared memory; 0: read from p.tw (large n)
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
  int n, log2n, C, lc;
  int R;  // rows per band of the band-major spectrum
  T lam, scale;
  T mu;   // viscosity (Brinkman: L = μΔ − λ)
  const T* lap1;
  const T* der1;
  cplx<T>* spec;
  const cplx<T>* tw;
  const int* stop;
  int tw_smem;  // 1: twiddles and symbol tables staged in shared memory; 0: read from global (large n)
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
__device__ __forceinline__ SpreadItem<T> spread_item(const RowParams<T>& p, const PointRanges& pr, int t, int r0) {
  const int n = p.n, M = p.M;
  const int s = pr.at(t >> 4);
  const int ay = (t >> 2) & 3, ax = t & 3;
  SpreadItem<T> it;
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

template <typename T, int OP>
__device__ __forceinline__ void spread_rowfft_body(const RowParams<T>& p, int unit, int nunits,
                                                   unsigned char* smem_raw) {
  constexpr int NIN = Traits<OP>::NIN;
  constexpr int NC = Traits<OP>::C;
  const int n = p.n, R = p.R, half = R >> 1, M = p.M;
  const int seqs = NIN * half;
  cplx<T>* tws_s = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* bufA = tws_s + (p.tw_smem ? n : 0);
  cplx<T>* bufB = bufA + padded((size_t)seqs * n);
  const cplx<T>* tws = p.tw_smem ? tws_s : p.tw;
  // accumulation view: field f, local row lr, column x → complex element e = (f·half + lr/2)·n + x
  // of the padded buffer, real part for even lr and imaginary part for odd lr
  T* acc = reinterpret_cast<T*>(bufA);
  const int r0 = unit * R;
  // prologue independent of the previous kernel, then wait for it (programmatic launch)
  for (int i = threadIdx.x; i < (int)padded((size_t)seqs * n) * 2; i += blockDim.x) acc[i] = T(0);
  if (p.tw_smem) load_twiddles(tws_s, p.tw, n);
  // the points whose stencil meets the band, and this thread's first work item (16 per point)
  const PointRanges pr = band_points(p.cell_start, n, r0, R);
  const int nitems = p.grid_in ? 0 : pr.cnt * 16;
  SpreadItem<T> it0 = {};
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

  // jump term: out = ±½·in (the gather kernel adds S*u afterwards); none for grid input
  if (!p.grid_in)
    for (int i = unit * blockDim.x + threadIdx.x; i < NC * M; i += nunits * blockDim.x)
      pout[i] = p.jump * pin[i] + (p.aug ? pin[NC * M + i / M] : 0.0);
  if (p.aug && unit == 0) {
    // constraint rows of the completed method: η Σ_i Δs_i Q_{l,i} (Δs = wscale·h^d); the
    // partial sums use the second FFT buffer, which the FFT's first stage writes later
    double* red = reinterpret_cast<double*>(bufB);
    for (int l = 0; l < NC; ++l) {
      double v = 0.0;
      for (int s = threadIdx.x; s < M; s += blockDim.x) v += double(p.wscale[s]) * pin[(size_t)l * M + p.perm[s]];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
      __syncthreads();
      if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) pout[NC * M + l] = p.eta * p.hd * t;
      }
      __syncthreads();
    }
  }
  __syncthreads();

  if (p.grid_in) {
    for (int t = threadIdx.x; t < NIN * R * n; t += blockDim.x) {
      const int f = t / (R * n);
      const int rem = t - f * R * n;
      const int lr = rem / n, x = rem - lr * n;
      acc[2 * pidx((f * half + (lr >> 1)) * n + x) + (lr & 1)] = T(p.grid_in[((size_t)f * n + r0 + lr) * n + x]);
    }
  }

  // one thread per (point, stencil node): 16 work items per point whose stencil meets the band
  for (int t = threadIdx.x; t < nitems; t += blockDim.x) {
    const SpreadItem<T> it = t == (int)threadIdx.x ? it0 : spread_item(p, pr, t, r0);
    const int lr = it.lr;
    if (lr >= R) continue;
    const int i = it.i;
    const T px = it.px, py = it.py, ws = it.ws, nx = it.nx, ny = it.ny;
    const int e = (lr >> 1) * n + it.col;  // field 0; field f adds f·half·n
    const int odd = lr & 1;
    const T pp = px * py;
    if (OP == OP_SCALAR_AN) {
      const T q = T(pin[i]) * ws;
      const T ddx = it.dpx * py, ddy = px * it.dpy;
      // dipole source n·∇δ_h, plus ηδ_h for the completed method
      atomicAdd(acc + 2 * pidx(e) + odd, q * (nx * ddx + ny * ddy + p.eta_src * pp));
    } else if (OP == OP_SCALAR_SD) {
      const T q = T(pin[i]) * ws * pp;
      atomicAdd(acc + 2 * pidx(e) + odd, q * nx);
      atomicAdd(acc + 2 * pidx(e + half * n) + odd, q * ny);
    } else if (OP == OP_STOKES_AN || OP == OP_STOKES_SD) {
      const T qx = T(pin[i]), qy = T(pin[M + i]);
      const T c0 = ws * (qx * nx + qy * ny);  // Q·n
      const T c1 = ws * (T(2) * qx * nx);     // A_xx
      const T c2 = ws * (T(2) * qy * ny);     // A_yy
      const T c3 = ws * (qx * ny + qy * nx);  // A_xy
      atomicAdd(acc + 2 * pidx(e) + odd, c0 * pp);
      if (OP == OP_STOKES_AN) {
        const T ddx = it.dpx * py, ddy = px * it.dpy;
        // g_x = ∂_x S(A_xx) + ∂_y S(A_xy), g_y = ∂_x S(A_xy) + ∂_y S(A_yy); the completed method
        // adds (η/μ) S(Q) to the projected source
        const T ce = p.eta_src * ws * pp;
        atomicAdd(acc + 2 * pidx(e + half * n) + odd, c1 * ddx + c3 * ddy + ce * qx);
        atomicAdd(acc + 2 * pidx(e + 2 * half * n) + odd, c3 * ddx + c2 * ddy + ce * qy);
      } else {
        atomicAdd(acc + 2 * pidx(e + half * n) + odd, c1 * pp);
        atomicAdd(acc + 2 * pidx(e + 2 * half * n) + odd, c2 * pp);
        atomicAdd(acc + 2 * pidx(e + 3 * half * n) + odd, c3 * pp);
      }
    } else if (OP == OP_STOKES_T) {
      // ψ_l = Σ_j μ_{l,j} Φ(x − X_j): the transpose of S*, unweighted
      atomicAdd(acc + 2 * pidx(e) + odd, T(pin[i]) * pp);
      atomicAdd(acc + 2 * pidx(e + half * n) + odd, T(pin[M + i]) * pp);
    } else {
      // plain spread of W (A*: weight Δs/h^d), or of λ (Aᵀ: weight 1, Δs/h^d moves to the gather)
      atomicAdd(acc + 2 * pidx(e) + odd, T(pin[i]) * (p.trans ? T(1) : ws) * pp);
    }
  }
  __syncthreads();

  const cplx<T>* res = fft_run<T, false>(bufA, bufB, p.log2n, seqs, tws);

  // unpack Z = FFT(a + i b) of the row pair (2j, 2j + 1) into A = FFT(a) (even rows) and
  // B = FFT(b) (odd rows), k = 0..n/2, packed format; thread t writes element t of the field's
  // band-major block, k·R + rr, so consecutive threads write consecutive addresses
  const int nh = n >> 1, lnh = p.log2n - 1, lR = __ffs(R) - 1;
  for (int t = threadIdx.x; t < NIN * nh * R; t += blockDim.x) {
    const int rr = t & (R - 1), k = (t >> lR) & (nh - 1), f = t >> (lR + lnh);
    const int zb = (f * half + (rr >> 1)) * n;
    cplx<T> v;
    if (k == 0) {
      const cplx<T> z0 = res[pidx(zb)], zh = res[pidx(zb + nh)];
      v = (rr & 1) ? mk(z0.y, zh.y) : mk(z0.x, zh.x);
    } else {
      const cplx<T> zk = res[pidx(zb + k)], zc = res[pidx(zb + n - k)];
      v = (rr & 1) ? mk(T(0.5) * (zk.y + zc.y), T(0.5) * (zc.x - zk.x))
                   : mk(T(0.5) * (zk.x + zc.x), T(0.5) * (zk.y - zc.y));
    }
    p.spec[((size_t)f * n + r0) * nh + (t - f * (nh << lR))] = v;
  }
}

template <typename T, int OP>
__global__ void __launch_bounds__(kThreads) k_spread_rowfft(RowParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  spread_rowfft_body<T, OP>(p, blockIdx.x, gridDim.x, smem_raw);
}

// ------------------------------------------------------------------------------------------
// Fourier symbols: NIN transformed fields in → NOUT out at wavenumber indices (kx, ky)
// ------------------------------------------------------------------------------------------
template <typename T, int OP>
__device__ __forceinline__ void apply_symbol(const ColParams<T>& p, const T* lap1, const T* der1, int kx, int ky,
                                             const cplx<T>* in, cplx<T>* out) {
  const T lap = lap1[kx] + lap1[ky];
  const T dkx = der1[kx], dky = der1[ky];
  if (OP == OP_SCALAR_AN || OP == OP_SCALAR_SD || OP == OP_ADJ_AN || OP == OP_ADJ_SD || OP == OP_SL) {
    // −L⁻¹ ↦ 1/(|k|² + λ), zero mode dropped when λ = 0 (Δ₀⁻¹)
    const T den = lap + p.lam;
    const T sig = den != T(0) ? p.scale / den : T(0);
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
    const T inv = lap != T(0) ? T(1) / lap : T(0);
    const cplx<T> kp = cadd(cscale(in[0], dkx), cscale(in[1], dky));
    const T sc = inv * p.scale;
    // Brinkman (λ > 0): the projected part carries μ/(μ|k|² + λ) in place of 1/|k|²
    const T sg = p.lam > T(0) ? p.mu / (p.mu * lap + p.lam) * p.scale : sc;
    out[0] = cscale(cmuli(kp), -sc);
    out[1] = cscale(csub(in[0], cscale(kp, dkx * inv)), sg);
    out[2] = cscale(csub(in[1], cscale(kp, dky * inv)), sg);
  } else {
    // Stokes, interior, η = 0: û = (i k̃ ŝ + P̂ ĝ)/|k|², P̂ = I − k̃k̃ᵀ/|k|²
    const T inv = lap != T(0) ? T(1) / lap : T(0);
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
      const T sg = p.mu / (p.mu * lap + p.lam) * p.scale;
      out[0] = cadd(cscale(is, dkx * sc), cscale(csub(gx, cscale(kg, dkx * inv)), sg));
      out[1] = cadd(cscale(is, dky * sc), cscale(csub(gy, cscale(kg, dky * inv)), sg));
    } else {
      out[0] = cscale(cadd(cscale(is, dkx), csub(gx, cscale(kg, dkx * inv))), sc);
      out[1] = cscale(cadd(cscale(is, dky), csub(gy, cscale(kg, dky * inv))), sc);
    }
  }
}

// ------------------------------------------------------------------------------------------
// kernel 2: FFT along y, symbol, inverse FFT along y, for C kx columns per CTA
// ------------------------------------------------------------------------------------------
// element m of column sequence bi = f·C + c, straight from / to the band-major half spectra
template <typename T>
struct ColumnIO {
  cplx<T>* spec;
  int n, nh, k0, lc, C, R;
  __device__ __forceinline__ size_t at(int bi, int m) const {
    return ((size_t)(bi >> lc) * n + (m & ~(R - 1))) * nh + (size_t)(k0 + (bi & (C - 1))) * R + (m & (R - 1));
  }
  __device__ __forceinline__ cplx<T> load(int bi, int m) const { return spec[at(bi, m)]; }
  __device__ __forceinline__ void store(int bi, int m, cplx<T> v) const { spec[at(bi, m)] = v; }
};

template <typename T, int OP>
__device__ __forceinline__ void colpass_body(const ColParams<T>& p, int unit, unsigned char* smem_raw) {
  constexpr int NIN = Traits<OP>::NIN;
  constexpr int NOUT = Traits<OP>::NOUT;
  constexpr int NMAX = NIN > NOUT ? NIN : NOUT;
  const int n = p.n, C = p.C, nh = n >> 1;
  cplx<T>* tws_s = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* bufA = tws_s + (p.tw_smem ? n : 0);
  cplx<T>* bufB = bufA + padded((size_t)NMAX * C * n);
  T* lap1_s = reinterpret_cast<T*>(bufB + padded((size_t)NMAX * C * n));
  T* der1_s = lap1_s + n;
  const cplx<T>* tws = p.tw_smem ? tws_s : p.tw;
  const T* lap1 = p.tw_smem ? lap1_s : p.lap1;
  const T* der1 = p.tw_smem ? der1_s : p.der1;
  const int k0 = unit * C;
  if (p.tw_smem) {
    load_twiddles(tws_s, p.tw, n);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      lap1_s[i] = p.lap1[i];
      der1_s[i] = p.der1[i];
    }
  }
  // The stop flag is final before the wait: it is written by the GMRES step (or the cycle start)
  // at least two kernels back, which has completed once the direct predecessor passed its own
  // wait and triggered this launch. So no dependent load follows the wait.
  const bool stopped = p.stop && *p.stop;
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();  // after the wait (see the spread kernel)
  if (stopped) return;
  __syncthreads();
  const ColumnIO<T> cio{p.spec, n, nh, k0, p.lc, C, p.R};
  // forward transform along y: the first stage reads the half spectra directly
  cplx<T>* res = fft_run<T, false>(bufA, bufB, p.log2n, NIN * C, tws, cio, NoIO());
  cplx<T>* other = res == bufA ? bufB : bufA;

  for (int t = threadIdx.x; t < (C << p.log2n); t += blockDim.x) {
    const int c = t >> p.log2n, ky = t & (n - 1);
    const int kx = k0 + c;
    cplx<T> in[NIN], out[NOUT];
    if (kx != 0) {
#pragma unroll
      for (int f = 0; f < NIN; ++f) in[f] = res[pidx((f * C + c) * n + ky)];
      apply_symbol<T, OP>(p, lap1, der1, kx, ky, in, out);
#pragma unroll
      for (int f = 0; f < NOUT; ++f) res[pidx((f * C + c) * n + ky)] = out[f];
    } else if (ky <= nh) {
      // packed kx = 0 | kx = n/2 column: P = Â + i B̂ with Â, B̂ Hermitian in ky
      const int j = ky, jp = (n - ky) & (n - 1);
      cplx<T> Aj[NIN], Ajp[NIN], Bj[NIN], Bjp[NIN];
#pragma unroll
      for (int f = 0; f < NIN; ++f) {
        const cplx<T> P = res[pidx((f * C + c) * n + j)];
        const cplx<T> Pp = res[pidx((f * C + c) * n + jp)];
        // Â(j) = (P(j) + conj P(−j))/2, B̂(j) = −i (P(j) − conj P(−j))/2
        Aj[f] = mk(T(0.5) * (P.x + Pp.x), T(0.5) * (P.y - Pp.y));
        Bj[f] = mk(T(0.5) * (P.y + Pp.y), T(0.5) * (Pp.x - P.x));
        Ajp[f] = mk(T(0.5) * (Pp.x + P.x), T(0.5) * (Pp.y - P.y));
        Bjp[f] = mk(T(0.5) * (Pp.y + P.y), T(0.5) * (P.x - Pp.x));
      }
      cplx<T> oA[NOUT], oB[NOUT], oAp[NOUT], oBp[NOUT];
      apply_symbol<T, OP>(p, lap1, der1, 0, j, Aj, oA);
      apply_symbol<T, OP>(p, lap1, der1, nh, j, Bj, oB);
      apply_symbol<T, OP>(p, lap1, der1, 0, jp, Ajp, oAp);
      apply_symbol<T, OP>(p, lap1, der1, nh, jp, Bjp, oBp);
#pragma unroll
      for (int f = 0; f < NOUT; ++f) {
        res[pidx((f * C + c) * n + j)] = cadd(oA[f], cmuli(oB[f]));
        if (jp != j) res[pidx((f * C + c) * n + jp)] = cadd(oAp[f], cmuli(oBp[f]));
      }
    }
  }
  __syncthreads();
  // inverse transform along y: the last stage writes the half spectra directly
  fft_run<T, true>(res, other, p.log2n, NOUT * C, tws, NoIO(), cio);
}

template <typename T, int OP>
__global__ void __launch_bounds__(kThreads) k_colpass(ColParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  colpass_body<T, OP>(p, blockIdx.x, smem_raw);
}

// ------------------------------------------------------------------------------------------
// kernel 3: inverse FFT along x, then interpolation (or write the grid)
// ------------------------------------------------------------------------------------------
// Z_m = A_m + i B_m (m = 0..n−1) for the row pair (r0 + 2j, r0 + 2j + 1) of field f, sequence
// sq = f·half + j, rebuilt on the fly from the band-major half spectra (A_{n−k} = conj A_k):
// A_k at band offset k·R + 2j, B_k next to it.
template <typename T>
struct RowZLoad {
  const cplx<T>* spec;
  int n, nh, r0, half, R;
  __device__ __forceinline__ cplx<T> load(int sq, int m) const {
    const int f = sq / half, j = sq - f * half;
    const cplx<T>* band = spec + ((size_t)f * n + r0) * nh + 2 * j;
    if (m == 0 || m == nh) {
      const cplx<T> A = band[0], B = band[1];
      return m == 0 ? mk(A.x, B.x) : mk(A.y, B.y);
    }
    if (m < nh) {
      const cplx<T> A = band[(size_t)m * R], B = band[(size_t)m * R + 1];
      return mk(A.x - B.y, A.y + B.x);
    }
    const cplx<T> A = band[(size_t)(n - m) * R], B = band[(size_t)(n - m) * R + 1];
    return mk(A.x + B.y, B.x - A.y);
  }
};

// One gather work item (point, stencil row): the point-table values it needs
template <typename T>
struct GatherItem {
  int lr, i, bx;
  T py, dy, ws, nx, ny;
  T px[4], dx[4];
};
template <typename T>
__device__ __forceinline__ GatherItem<T> gather_item(const RowParams<T>& p, const PointRanges& pr, int t, int r0) {
  const int n = p.n, M = p.M;
  const int s = pr.at(t >> 2);
  const int ay = t & 3;
  GatherItem<T> it;
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

template <typename T, int OP, int GMODE>
__device__ __forceinline__ void rowifft_gather_body(const RowParams<T>& p, int unit, unsigned char* smem_raw) {
  constexpr int NOUT = Traits<OP>::NOUT;
  const int n = p.n, R = p.R, half = R >> 1, M = p.M, nh = n >> 1;
  const int seqs = NOUT * half;
  cplx<T>* tws_s = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* bufA = tws_s + (p.tw_smem ? n : 0);
  cplx<T>* bufB = bufA + padded((size_t)seqs * n);
  const cplx<T>* tws = p.tw_smem ? tws_s : p.tw;
  const int r0 = unit * R;
  if (p.tw_smem) load_twiddles(tws_s, p.tw, n);
  // the points whose stencil meets the band and this thread's first work item (4 per point),
  // loaded before the wait: the point tables are constant
  const PointRanges pr = band_points(p.cell_start, n, r0, R);
  const int nitems = GMODE == G_GRID ? 0 : pr.cnt * 4;
  GatherItem<T> it0 = {};
  if ((int)threadIdx.x < nitems) it0 = gather_item(p, pr, threadIdx.x, r0);
  // the stop flag and the Krylov index (the output column) are final before the wait: the GMRES
  // step that writes them is three kernels back (see the column pass)
  const bool stopped = p.stop && *p.stop;
  const double* pin;
  double* pout;
  resolve_io(p, pin, pout);
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();  // after the wait (see the spread kernel)
  if (stopped) return;
  __syncthreads();
  const RowZLoad<T> zl{p.spec, n, nh, r0, half, R};
  const cplx<T>* res = fft_run<T, true>(bufA, bufB, p.log2n, seqs, tws, zl, NoIO());
  // real values: field f, local row lr, column x at element e = (f·half + lr/2)·n + x, part lr & 1
  const T* u = reinterpret_cast<const T*>(res);

  if (GMODE == G_GRID) {
    for (int t = threadIdx.x; t < NOUT * R * n; t += blockDim.x) {
      const int f = t / (R * n);
      const int rem = t - f * R * n;
      const int lr = rem / n, x = rem - lr * n;
      // the completed method's field is u₀ + ū (ū after the density in the input vector)
      const double ub = p.aug ? p.in[(size_t)Traits<OP>::C * M + f] : 0.0;
      p.grid[((size_t)f * n + r0 + lr) * n + x] = double(u[2 * pidx((f * half + (lr >> 1)) * n + x) + (lr & 1)]) + ub;
    }
    return;
  }

  // one thread per (point, stencil row in the band): the row's partial sum is added to Y
  for (int t = threadIdx.x; t < nitems; t += blockDim.x) {
    const GatherItem<T> it = t == (int)threadIdx.x ? it0 : gather_item(p, pr, t, r0);
    const int lr = it.lr;
    if (lr >= R) continue;
    const int i = it.i;
    const int bx = it.bx;
    const T py = it.py;
    const T dy = (OP == OP_ADJ_AN || OP == OP_STOKES_T) ? it.dy : T(0);
    const int eb = (lr >> 1) * n, odd = lr & 1;
    if (OP == OP_STOKES_T) {
      // a_s = Σ v_s Φ, G_mk = Σ v_gm ∂_kΦ; out_l += (Δs/h²)[n_l a_s + Σ_k n_k (G_lk + G_kl)]
      T as = 0, gxx = 0, gxy = 0, gyx = 0, gyy = 0;
#pragma unroll
      for (int ax = 0; ax < 4; ++ax) {
        const int col = (bx + ax) & (n - 1);
        const T px = it.px[ax], dx = it.dx[ax];
        const T vs = u[2 * pidx(eb + col) + odd];
        const T vx = u[2 * pidx(eb + half * n + col) + odd];
        const T vy = u[2 * pidx(eb + 2 * half * n + col) + odd];
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
    T acc0 = 0, acc1 = 0;
#pragma unroll
    for (int ax = 0; ax < 4; ++ax) {
      const int col = (bx + ax) & (n - 1);
      const T px = it.px[ax];
      const T v0 = u[2 * pidx(eb + col) + odd];
      if (OP == OP_ADJ_AN) {
        acc0 += v0 * it.dx[ax] * py;
        acc1 += v0 * px * dy;
      } else {
        const T pp = px * py;
        acc0 += v0 * pp;
        if (NOUT == 2) acc1 += u[2 * pidx(eb + half * n + col) + odd] * pp;
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

template <typename T, int OP, int GMODE>
__global__ void __launch_bounds__(kThreads) k_rowifft_gather(RowParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rowifft_gather_body<T, OP, GMODE>(p, blockIdx.x, smem_raw);
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
template <typename T>
static RowParams<T> row_params(Geometry* g, const double* in, double* out, const int* stop, double* grid) {
  const int pi = std::is_same<T, float>::value ? 1 : 0;
  RowParams<T> rp;
  rp.n = g->n;
  rp.log2n = __builtin_ctz(g->n);
  rp.R = g->rows_per_cta[pi];
  rp.M = (int)g->M;
  rp.cell_start = g->cell_start;
  rp.base = g->base;
  rp.perm = g->perm;
  const PointTable<T>& tb = *reinterpret_cast<const PointTable<T>*>(pi ? (const void*)&g->t32 : (const void*)&g->t64);
  rp.phi = tb.phi;
  rp.dphi = tb.dphi;
  rp.wscale = tb.wscale;
  rp.nrm = tb.nrm;
  rp.in = in;
  rp.out = out;
  rp.spec = reinterpret_cast<cplx<T>*>(g->spec);
  rp.tw = reinterpret_cast<const cplx<T>*>(pi ? (const void*)g->tw32 : (const void*)g->tw64);
  rp.stop = stop;
  rp.grid = grid;
  rp.idx = nullptr;
  rp.vstride = 0;
  rp.io_off = 0;
  rp.trans = 0;
  rp.grid_in = nullptr;
  rp.jump = g->bc == IBDL_BC_NEUMANN ? -0.5 : 0.5;
  rp.aug = g->naug > 0;
  rp.eta = g->eta;
  rp.hd = g->h * g->h;
  rp.eta_src = T(g->naug ? (g->pde == IBDL_PDE_STOKES ? g->eta / g->mu : g->eta) : 0.0);
  rp.tw_smem = 1;
  return rp;
}

template <typename T>
static ColParams<T> col_params(Geometry* g, const int* stop) {
  const int pi = std::is_same<T, float>::value ? 1 : 0;
  ColParams<T> cp;
  cp.n = g->n;
  cp.log2n = __builtin_ctz(g->n);
  cp.C = g->cols_per_cta[pi];
  cp.lc = __builtin_ctz(cp.C ? cp.C : 1);
  cp.R = g->rows_per_cta[pi];
  cp.lam = T(g->lambda);
  cp.mu = T(g->mu);
  cp.scale = T(1.0 / ((double)g->n * (double)g->n));
  cp.lap1 = reinterpret_cast<const T*>(pi ? (const void*)g->lap32 : (const void*)g->lap64);
  cp.der1 = reinterpret_cast<const T*>(pi ? (const void*)g->der32 : (const void*)g->der64);
  cp.spec = reinterpret_cast<cplx<T>*>(g->spec);
  cp.tw = reinterpret_cast<const cplx<T>*>(pi ? (const void*)g->tw32 : (const void*)g->tw64);
  cp.stop = stop;
  cp.tw_smem = 1;
  return cp;
}

// shared memory: two padded FFT buffers, plus (staged) the twiddles (n) and, in the column pass,
// the two symbol tables. Large grids leave the tables in global memory (L1-cached reads) so the
// buffers fit: FP64 to 4096², FP32 to 8192² for the scalar operator, 2048² / 4096² for Stokes.
template <typename T, int OP>
static size_t smem_spread(const Geometry* g, int R, bool staged = true) {
  return ((staged ? g->n : 0) + 2 * padded((size_t)Traits<OP>::NIN * (R / 2) * g->n)) * sizeof(cplx<T>);
}
template <typename T, int OP>
static size_t smem_gather(const Geometry* g, int R, bool staged = true) {
  return ((staged ? g->n : 0) + 2 * padded((size_t)Traits<OP>::NOUT * (R / 2) * g->n)) * sizeof(cplx<T>);
}
template <typename T, int OP>
static size_t smem_col(const Geometry* g, int C, bool staged = true) {
  const int nmax = Traits<OP>::NIN > Traits<OP>::NOUT ? Traits<OP>::NIN : Traits<OP>::NOUT;
  return ((staged ? g->n : 0) + 2 * padded((size_t)nmax * C * g->n)) * sizeof(cplx<T>) +
         (staged ? 2 * g->n * sizeof(T) : 0);
}

static const size_t kSmemLimit = 227 * 1024;

// Programmatic dependent launch: the kernel may start while the previous kernel on the stream
// drains; it runs its prologue and then waits in cudaGridDependencySynchronize(). IBDL_NO_PDL=1
// turns it off.
static bool use_pdl() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("IBDL_NO_PDL");
    v = (e && atoi(e) != 0) ? 0 : 1;
  }
  return v == 1;
}

template <typename... KArgs, typename... Args>
static cudaError_t launch_k(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s, bool pdl,
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

template <typename T, int OP>
static ibdl_status set_attrs() {
  IBDL_CUDA(cudaFuncSetAttribute(k_spread_rowfft<T, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
  IBDL_CUDA(cudaFuncSetAttribute(k_colpass<T, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
  IBDL_CUDA(cudaFuncSetAttribute(k_rowifft_gather<T, OP, G_INTERP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
  IBDL_CUDA(cudaFuncSetAttribute(k_rowifft_gather<T, OP, G_GRID>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
  return IBDL_OK;
}

template <typename T>
static ibdl_status set_attrs_all() {
  IBDL_TRY((set_attrs<T, OP_SCALAR_AN>()));
  IBDL_TRY((set_attrs<T, OP_SCALAR_SD>()));
  IBDL_TRY((set_attrs<T, OP_STOKES_AN>()));
  IBDL_TRY((set_attrs<T, OP_STOKES_SD>()));
  IBDL_TRY((set_attrs<T, OP_ADJ_AN>()));
  IBDL_TRY((set_attrs<T, OP_ADJ_SD>()));
  IBDL_TRY((set_attrs<T, OP_STOKES_T>()));
  IBDL_TRY((set_attrs<T, OP_SL>()));
  return IBDL_OK;
}

// run_op mode bits: RUN_LAPLACE solves the plain Laplace problem (λ → 0) without the completed
// method's terms; RUN_NO_AUG only drops those terms
enum { RUN_LAPLACE = 1, RUN_NO_AUG = 2 };

template <typename T, int OP>
static ibdl_status run_op(Geometry* g, const double* in, double* out, cudaStream_t s, const int* stop,
                          double* grid, const int* idx = nullptr, int vstride = 0, int trans = 0,
                          const double* grid_in = nullptr, int mode = 0) {
  const int pi = std::is_same<T, float>::value ? 1 : 0;
  const int R = g->rows_per_cta[pi], C = g->cols_per_cta[pi];
  if (R == 0 || C == 0)
    return fail(IBDL_ERR_UNSUPPORTED, "grid too large for the shared-memory FFT at this precision");
  // stage the twiddles (and symbol tables) in shared memory when they fit beside the buffers
  const bool row_staged = smem_spread<T, OP>(g, R) <= kSmemLimit && smem_gather<T, OP>(g, R) <= kSmemLimit;
  const bool col_staged = smem_col<T, OP>(g, C) <= kSmemLimit;
  const size_t s1 = smem_spread<T, OP>(g, R, row_staged), s2 = smem_col<T, OP>(g, C, col_staged),
               s3 = smem_gather<T, OP>(g, R, row_staged);
  if (s1 > kSmemLimit || s2 > kSmemLimit || s3 > kSmemLimit)
    return fail(IBDL_ERR_UNSUPPORTED, "grid too large for the shared-memory FFT at this precision");
  RowParams<T> rp = row_params<T>(g, in, out, stop, grid);
  rp.idx = idx;
  rp.vstride = vstride;
  rp.trans = trans;
  rp.grid_in = grid_in;
  if (OP == OP_SL) rp.jump = 0.0;
  if (OP != OP_SCALAR_AN && OP != OP_STOKES_AN) {  // the completed method exists for these two only
    rp.aug = 0;
    rp.eta_src = T(0);
  }
  rp.tw_smem = row_staged ? 1 : 0;
  ColParams<T> cp = col_params<T>(g, stop);
  cp.tw_smem = col_staged ? 1 : 0;
  if (mode & RUN_LAPLACE) cp.lam = T(0);  // the plain Laplace problem (indicator)
  if (mode & (RUN_LAPLACE | RUN_NO_AUG)) {  // no completed-method terms
    rp.aug = 0;
    rp.eta_src = T(0);
  }
  const int st0 = pi ? IBDL_STAGE_SPREAD_ROWFFT_FP32 : IBDL_STAGE_SPREAD_ROWFFT_FP64;
  if (g->timing) timing_mark(g, s, -1);
  const int nt = g->threads[pi] ? g->threads[pi] : kThreads;
  IBDL_CUDA(launch_k(k_spread_rowfft<T, OP>, g->n / R, nt, s1, s, !g->timing, rp));
  if (g->timing) timing_mark(g, s, st0);
  IBDL_CUDA(launch_k(k_colpass<T, OP>, (g->n / 2) / C, nt, s2, s, !g->timing, cp));
  if (g->timing) timing_mark(g, s, st0 + 1);
  if (grid)
    IBDL_CUDA(launch_k(k_rowifft_gather<T, OP, G_GRID>, g->n / R, nt, s3, s, !g->timing, rp));
  else
    IBDL_CUDA(launch_k(k_rowifft_gather<T, OP, G_INTERP>, g->n / R, nt, s3, s, !g->timing, rp));
  if (g->timing) timing_mark(g, s, st0 + 2);
  g->launches += 3;
  IBDL_CUDA(cudaGetLastError());
  return IBDL_OK;
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
  return precision == IBDL_FP32 ? apply_t<float>(g, V, V, s, stop, nullptr, idx, nd, op)
                                : apply_t<double>(g, V, V, s, stop, nullptr, idx, nd, op);
}

ibdl_status apply_2d(Geometry* g, int precision, const double* Q, double* Y, cudaStream_t s, const int* stop,
                     int op) {
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
// batched launches: one grid per stage covers every problem of a batch; CTA i runs work unit
// units[i] = (problem, unit) with that problem's parameter block
// ------------------------------------------------------------------------------------------
template <typename T, int OP>
__global__ void __launch_bounds__(kThreads) kb_spread_rowfft(const RowParams<T>* __restrict__ P, const int2* units,
                                                             const double* in_base, double* out_base) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 u = units[blockIdx.x];
  RowParams<T> p = P[u.x];
  p.in = in_base + p.io_off;
  p.out = out_base + p.io_off;
  spread_rowfft_body<T, OP>(p, u.y, p.n / p.R, smem_raw);
}

template <typename T, int OP>
__global__ void __launch_bounds__(kThreads) kb_colpass(const ColParams<T>* __restrict__ P, const int2* units) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 u = units[blockIdx.x];
  const ColParams<T> p = P[u.x];
  colpass_body<T, OP>(p, u.y, smem_raw);
}

template <typename T, int OP>
__global__ void __launch_bounds__(kThreads) kb_rowifft_gather(const RowParams<T>* __restrict__ P, const int2* units,
                                                              const double* in_base, double* out_base) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 u = units[blockIdx.x];
  RowParams<T> p = P[u.x];
  p.in = in_base + p.io_off;
  p.out = out_base + p.io_off;
  rowifft_gather_body<T, OP, G_INTERP>(p, u.y, smem_raw);
}

template <typename T, int OP>
static ibdl_status batch_launch(Batch* B, int mode, const double* in_base, double* out_base, cudaStream_t s) {
  const int pi = std::is_same<T, float>::value ? 1 : 0;
  static bool attrs = false;
  if (!attrs) {
    IBDL_CUDA(cudaFuncSetAttribute(kb_spread_rowfft<T, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
    IBDL_CUDA(cudaFuncSetAttribute(kb_colpass<T, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
    IBDL_CUDA(cudaFuncSetAttribute(kb_rowifft_gather<T, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
    attrs = true;
  }
  const RowParams<T>* rp = static_cast<const RowParams<T>*>(B->rowp[pi][mode]);
  const ColParams<T>* cp = static_cast<const ColParams<T>*>(B->colp[pi]);
  kb_spread_rowfft<T, OP><<<B->nrow_units[pi], kThreads, B->smem_row[pi], s>>>(rp, B->row_units[pi], in_base, out_base);
  IBDL_CUDA(launch_k(kb_colpass<T, OP>, B->ncol_units[pi], kThreads, B->smem_col[pi], s, true, cp,
                     (const int2*)B->col_units[pi]));
  IBDL_CUDA(launch_k(kb_rowifft_gather<T, OP>, B->nrow_units[pi], kThreads, B->smem_gather[pi], s, true, rp,
                     (const int2*)B->row_units[pi], in_base, out_base));
  B->launches += 3;
  IBDL_CUDA(cudaGetLastError());
  return IBDL_OK;
}

template <typename T>
static ibdl_status batch_apply_t(Batch* B, int mode, const double* in_base, double* out_base, cudaStream_t s) {
  if (B->pde == IBDL_PDE_STOKES)
    return B->dipole == IBDL_DIPOLE_ANALYTIC ? batch_launch<T, OP_STOKES_AN>(B, mode, in_base, out_base, s)
                                             : batch_launch<T, OP_STOKES_SD>(B, mode, in_base, out_base, s);
  return B->dipole == IBDL_DIPOLE_ANALYTIC ? batch_launch<T, OP_SCALAR_AN>(B, mode, in_base, out_base, s)
                                           : batch_launch<T, OP_SCALAR_SD>(B, mode, in_base, out_base, s);
}

ibdl_status batch_apply_2d(Batch* B, int precision, int mode, const double* in_base, double* out_base, cudaStream_t s) {
  return precision == IBDL_FP32 ? batch_apply_t<float>(B, mode, in_base, out_base, s)
                                : batch_apply_t<double>(B, mode, in_base, out_base, s);
}

template <typename T, int OP>
static void batch_smem(Batch* B, Geometry* g, int pi) {
  const int R = g->rows_per_cta[pi], C = g->cols_per_cta[pi];
  const size_t a = smem_spread<T, OP>(g, R), b = smem_col<T, OP>(g, C), c = smem_gather<T, OP>(g, R);
  if (a > B->smem_row[pi]) B->smem_row[pi] = a;
  if (b > B->smem_col[pi]) B->smem_col[pi] = b;
  if (c > B->smem_gather[pi]) B->smem_gather[pi] = c;
}

template <typename T>
static void batch_smem_any(Batch* B, Geometry* g, int pi) {
  if (B->pde == IBDL_PDE_STOKES) {
    if (B->dipole == IBDL_DIPOLE_ANALYTIC) batch_smem<T, OP_STOKES_AN>(B, g, pi); else batch_smem<T, OP_STOKES_SD>(B, g, pi);
  } else {
    if (B->dipole == IBDL_DIPOLE_ANALYTIC) batch_smem<T, OP_SCALAR_AN>(B, g, pi); else batch_smem<T, OP_SCALAR_SD>(B, g, pi);
  }
}

template <typename T>
static ibdl_status batch_prepare_t(Batch* B, const int* kptr /* device &st[b].k, stride in bytes */, size_t kstride) {
  const int pi = std::is_same<T, float>::value ? 1 : 0;
  std::vector<RowParams<T>> user(B->count), kry(B->count);
  std::vector<ColParams<T>> col(B->count);
  std::vector<int2> ru, cu;
  for (int b = 0; b < B->count; ++b) {
    Geometry* g = B->geoms[b];
    if (g->rows_per_cta[pi] == 0 || g->cols_per_cta[pi] == 0)
      return fail(IBDL_ERR_UNSUPPORTED, "a batch problem's grid is too large for the shared-memory FFT");
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
    for (int u = 0; u < g->n / g->rows_per_cta[pi]; ++u) ru.push_back(make_int2(b, u));
    for (int u = 0; u < (g->n / 2) / g->cols_per_cta[pi]; ++u) cu.push_back(make_int2(b, u));
    batch_smem_any<T>(B, g, pi);
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
  return IBDL_OK;
}

// Band height R (rows per CTA, even) and kx columns per CTA C, per precision, within the
// shared-memory limit for the widest field count this geometry uses.
// ------------------------------------------------------------------------------------------
// autotuner: time candidate launch shapes of the 2-D application on a geometry's own data and
// keep the fastest; results are cached per (n, fields in, fields out, pde, dipole, precision)
// so geometries created later with the same key start from the tuned shape
// ------------------------------------------------------------------------------------------
struct TuneKey {
  int n, nf_in, nf_out, pde, dipole, pi;
  bool operator==(const TuneKey& o) const {
    return n == o.n && nf_in == o.nf_in && nf_out == o.nf_out && pde == o.pde && dipole == o.dipole && pi == o.pi;
  }
};
struct TuneVal {
  int R, C, threads;
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

static TuneKey tune_key(const Geometry* g, int pi) { return {g->n, g->nf_in, g->nf_out, g->pde, g->dipole, pi}; }

// Candidates R ∈ {2..16}, C ∈ {1..8} that fit shared memory and keep R ≤ n/2, and (unless
// fixed_threads) 256 or 512 threads; each timed as the median of 5 applications after one warm-up.
ibdl_status autotune_2d(Geometry* g, int pi, bool fixed_threads, cudaStream_t s, const double* Q, double* Y) {
  const int nf = g->nf_in > g->nf_out ? g->nf_in : g->nf_out;
  const size_t cs = pi ? sizeof(float2) : sizeof(double2);
  // feasible without the staged tables (each launch stages them when they fit)
  auto row_bytes = [&](int r) { return 2 * padded((size_t)nf * (r / 2) * g->n) * cs; };
  auto col_bytes = [&](int c) { return 2 * padded((size_t)nf * c * g->n) * cs; };
  const int saved_R = g->rows_per_cta[pi], saved_C = g->cols_per_cta[pi], saved_T = g->threads[pi];
  const int saved_timing = g->timing;
  g->timing = 0;
  cudaEvent_t e0, e1;
  IBDL_CUDA(cudaEventCreate(&e0));
  IBDL_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  TuneVal bestv{saved_R, saved_C, saved_T};
  ibdl_status err = IBDL_OK;
  const int threads_opts[2] = {256, 512};
  for (int R = 2; R <= 16 && err == IBDL_OK; R *= 2) {
    if (R > g->n / 2 || row_bytes(R) > kSmemLimit) continue;
    for (int C = 1; C <= 8 && err == IBDL_OK; C *= 2) {
      if (C > g->n / 2 || col_bytes(C) > kSmemLimit) continue;
      for (int ti = 0; ti < 2 && err == IBDL_OK; ++ti) {
        const int T = fixed_threads ? 0 : threads_opts[ti];
        if (fixed_threads && ti == 1) break;
        g->rows_per_cta[pi] = R;
        g->cols_per_cta[pi] = C;
        g->threads[pi] = T;
        float ms[5];
        err = apply_2d(g, pi ? IBDL_FP32 : IBDL_FP64, Q, Y, s, nullptr);
        for (int k = 0; k < 5 && err == IBDL_OK; ++k) {
          cudaEventRecord(e0, s);
          err = apply_2d(g, pi ? IBDL_FP32 : IBDL_FP64, Q, Y, s, nullptr);
          cudaEventRecord(e1, s);
          if (cudaEventSynchronize(e1) != cudaSuccess) err = fail(IBDL_ERR_CUDA, "autotune: event synchronize");
          cudaEventElapsedTime(&ms[k], e0, e1);
        }
        if (err != IBDL_OK) break;
        std::sort(ms, ms + 5);
        if (ms[2] < best) {
          best = ms[2];
          bestv = {R, C, T};
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g->timing = saved_timing;
  g->rows_per_cta[pi] = bestv.R;
  g->cols_per_cta[pi] = bestv.C;
  g->threads[pi] = bestv.threads;
  if (err == IBDL_OK) tuned_store(tune_key(g, pi), bestv);
  return err;
}

// Shapes from the volume rule: about `target` complex elements of FFT per CTA, at least 16 row
// bands and 16 column groups, R ≤ n/2 (distinct wrapped band rows), within shared memory.
void shape_for_target_2d(Geometry* g, int pi, int row_target, int col_target) {
  const int nf = g->nf_in > g->nf_out ? g->nf_in : g->nf_out;
  const int n = g->n;
  auto clampp2 = [](int v, int lo, int hi) {
    v = v < lo ? lo : (v > hi ? hi : v);
    int r = 1;
    while (r * 2 <= v) r *= 2;
    return r;
  };
  const size_t cs = pi ? sizeof(float2) : sizeof(double2);
  auto row_bytes = [&](int r) { return (g->n + 2 * padded((size_t)nf * (r / 2) * g->n)) * cs; };
  auto col_bytes = [&](int c) { return (g->n + 2 * padded((size_t)nf * c * g->n)) * cs + 2 * g->n * cs / 2; };
  int R = clampp2(2 * (row_target / (n * g->nf_in)), 2, n / 16 > 2 ? n / 16 : 2);
  while (R > 2 && row_bytes(R) > kSmemLimit) R /= 2;
  int C = clampp2(col_target / (n * nf), 1, n / 32 > 1 ? n / 32 : 1);
  while (C > 1 && col_bytes(C) > kSmemLimit) C /= 2;
  if (row_bytes(R) <= kSmemLimit && col_bytes(C) <= kSmemLimit) {
    g->rows_per_cta[pi] = R;
    g->cols_per_cta[pi] = C;
  }
}

ibdl_status plan_2d(Geometry* g) {
  static bool attrs = false;  // opt in to large dynamic shared memory once per kernel instance
  if (!attrs) {
    IBDL_TRY(set_attrs_all<double>());
    IBDL_TRY(set_attrs_all<float>());
    attrs = true;
  }
  // Work units sized by FFT volume: about 2048 complex elements per CTA in FP32 and 1024 in FP64
  // (one radix-8 butterfly per thread per stage or fewer), keeping at least 16 row bands and 16
  // column groups per problem; R ≤ n/2 keeps the wrapped band rows [r0 − 3, r0 + R) distinct.
  const int nf = g->nf_in > g->nf_out ? g->nf_in : g->nf_out;
  const int n = g->n;
  auto clampp2 = [](int v, int lo, int hi) {
    v = v < lo ? lo : (v > hi ? hi : v);
    int r = 1;
    while (r * 2 <= v) r *= 2;
    return r;
  };
  for (int pi = 0; pi < 2; ++pi) {
    const size_t cs = pi ? sizeof(float2) : sizeof(double2);
    const int target = pi ? 2048 : 1024;
    int R = clampp2(2 * (target / (n * g->nf_in)), 2, n / 16 > 2 ? n / 16 : 2);
    // feasible without the staged tables (each launch stages them when they fit)
    auto row_bytes = [&](int r) { return 2 * padded((size_t)nf * (r / 2) * g->n) * cs; };
    auto col_bytes = [&](int c) { return 2 * padded((size_t)nf * c * g->n) * cs; };
    while (R > 2 && row_bytes(R) > kSmemLimit) R /= 2;
    if (row_bytes(R) > kSmemLimit) R = 0;
    int C = clampp2(target / (n * nf), 1, n / 32 > 1 ? n / 32 : 1);
    while (C > 1 && col_bytes(C) > kSmemLimit) C /= 2;
    if (col_bytes(C) > kSmemLimit) C = 0;
    if ((g->n / 2) % (C ? C : 1)) C = 1;
    // launch-shape overrides for tuning experiments (IBDL_PLAN_R, IBDL_PLAN_C, IBDL_THREADS)
    if (const char* e = getenv("IBDL_PLAN_R")) {
      const int v = atoi(e);
      // R ≤ n/2 keeps the wrapped band rows [r0 − 3, r0 + R) distinct (no point counted twice)
      if (v >= 2 && v <= g->n / 2 && (v & (v - 1)) == 0 && row_bytes(v) <= kSmemLimit) R = v;
    }
    if (const char* e = getenv("IBDL_PLAN_C")) {
      const int v = atoi(e);
      if (v >= 1 && v <= g->n / 2 && (v & (v - 1)) == 0 && col_bytes(v) <= kSmemLimit) C = v;
    }
    g->rows_per_cta[pi] = R;
    g->cols_per_cta[pi] = C;
    g->threads[pi] = 0;
    TuneVal tv;
    if (tuned_lookup(tune_key(g, pi), &tv)) {
      g->rows_per_cta[pi] = tv.R;
      g->cols_per_cta[pi] = tv.C;
      g->threads[pi] = tv.threads;
    }
  }
  if (const char* e = getenv("IBDL_THREADS")) {
    const int v = atoi(e);
    if (v >= 32 && v <= kThreads && v % 32 == 0) g->threads[0] = g->threads[1] = v;
  }
  if (g->rows_per_cta[0] == 0 && g->rows_per_cta[1] == 0)
    return fail(IBDL_ERR_UNSUPPORTED, "grid too large for the shared-memory FFT");
  return IBDL_OK;
}

}  // namespace ibdl
