// Shared-memory Stockham FFT and the regularised-delta kernels used by the IBDL kernels.
#pragma once

#include <type_traits>

#include "ibdl_internal.cuh"

namespace ibdl {

// ------------------------------------------------------------------------------------------
// Batched complex FFT of power-of-two length n in shared memory (Stockham autosort: every
// stage reads one buffer and writes the other, so no bit reversal is needed).
//
// Stage with current sub-transform length p and radix R: butterfly i ∈ [0, n/R) of every
// sequence reads x[i + r·n/R] (r < R), multiplies input r by ω^{r·k} with k = i mod p and
// ω = e^{∓2πi/(pR)}, takes the R-point DFT, and writes output t to y[(i − k)·R + k + t·p].
// Radix-8 stages run while at least three factors of two remain, then one radix-4 or radix-2.
//
// tw[j] = e^{−2πi j/n} (the kernels stage it in shared memory); the inverse transform (INV)
// uses conjugates and is unnormalised. Sequences are `nb` runs of n contiguous elements,
// sequence b starting at b·bstride. Returns the buffer that holds the result (a or b). All
// threads of the block must call it.
// ------------------------------------------------------------------------------------------
template <typename T, bool INV>
__device__ __forceinline__ void dft2(cplx<T>* u) {
  const cplx<T> t = u[0];
  u[0] = cadd(t, u[1]);
  u[1] = csub(t, u[1]);
}

// multiply by −i (forward) or +i (inverse)
template <typename T, bool INV>
__device__ __forceinline__ cplx<T> rot90(cplx<T> a) {
  return INV ? mk(-a.y, a.x) : mk(a.y, -a.x);
}

template <typename T, bool INV>
__device__ __forceinline__ void dft4(cplx<T>& a0, cplx<T>& a1, cplx<T>& a2, cplx<T>& a3) {
  const cplx<T> t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3);
  const cplx<T> t3 = rot90<T, INV>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a1 = cadd(t1, t3);
  a2 = csub(t0, t2);
  a3 = csub(t1, t3);
}

// 8-point DFT as two 4-point DFTs: X_{2k} = DFT4(u_r + u_{r+4}), X_{2k+1} = DFT4((u_r − u_{r+4}) ω₈^r)
template <typename T, bool INV>
__device__ __forceinline__ void dft8(cplx<T>* u) {
  const T c = T(0.70710678118654752440);
  cplx<T> a0 = cadd(u[0], u[4]), a1 = cadd(u[1], u[5]), a2 = cadd(u[2], u[6]), a3 = cadd(u[3], u[7]);
  cplx<T> b0 = csub(u[0], u[4]), b1 = csub(u[1], u[5]), b2 = csub(u[2], u[6]), b3 = csub(u[3], u[7]);
  b1 = INV ? mk((b1.x - b1.y) * c, (b1.x + b1.y) * c) : mk((b1.x + b1.y) * c, (b1.y - b1.x) * c);
  b2 = rot90<T, INV>(b2);
  b3 = INV ? mk(-(b3.x + b3.y) * c, (b3.x - b3.y) * c) : mk((b3.y - b3.x) * c, -(b3.x + b3.y) * c);
  dft4<T, INV>(a0, a1, a2, a3);
  dft4<T, INV>(b0, b1, b2, b3);
  u[0] = a0;
  u[1] = b0;
  u[2] = a1;
  u[3] = b1;
  u[4] = a2;
  u[5] = b2;
  u[6] = a3;
  u[7] = b3;
}

// Shared-memory FFT buffers are padded with one element after every eight, which keeps the
// radix-8 stride-8 writes of the first stages free of bank conflicts for 8- and 16-byte elements.
__device__ __forceinline__ int pidx(int x) { return x + (x >> 3); }
__host__ __device__ constexpr size_t padded(size_t x) { return x + (x >> 3); }

// element m of sequence bi in a padded shared-memory buffer of sequences of length 2^log2n
template <typename T>
struct SmemIO {
  cplx<T>* buf;
  int log2n;
  __device__ __forceinline__ cplx<T> load(int bi, int m) const { return buf[pidx((bi << log2n) + m)]; }
  __device__ __forceinline__ void store(int bi, int m, cplx<T> v) const { buf[pidx((bi << log2n) + m)] = v; }
};

struct NoIO {};

// One Stockham stage reading through `ld` and writing through `st`.
template <typename T, bool INV, int LR, class LD, class ST>
__device__ __forceinline__ void fft_stage(const LD& ld, const ST& st, int log2n, int lp, int nb,
                                          const cplx<T>* __restrict__ tw) {
  constexpr int R = 1 << LR;
  const int lq = log2n - LR;
  const int q = 1 << lq;
  const int p = 1 << lp;
  const int total = nb << lq;
  const int tws = 1 << (log2n - lp - LR);  // n / (pR)
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int bi = t >> lq, i = t & (q - 1), k = i & (p - 1);
    cplx<T> u[R];
#pragma unroll
    for (int r = 0; r < R; ++r) u[r] = ld.load(bi, i + r * q);
    if (k) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cplx<T> w = tw[r * k * tws];
        if (INV) w.y = -w.y;
        u[r] = cmul(u[r], w);
      }
    }
    if (LR == 3)
      dft8<T, INV>(u);
    else if (LR == 2)
      dft4<T, INV>(u[0], u[1], u[2], u[3]);
    else
      dft2<T, INV>(u);
    const int j = ((i - k) << LR) + k;
#pragma unroll
    for (int r = 0; r < R; ++r) st.store(bi, j + r * p, u[r]);
  }
}

template <typename T, bool INV, int LR, class FL, class LS>
__device__ __forceinline__ void fft_stage_dispatch(bool first, bool last, const SmemIO<T>& in, const SmemIO<T>& out,
                                                   const FL& fl, const LS& ls, int log2n, int lp, int nb,
                                                   const cplx<T>* tw) {
  constexpr bool HF = !std::is_same<FL, NoIO>::value, HL = !std::is_same<LS, NoIO>::value;
  if constexpr (HF && HL) {
    if (first && last) {
      fft_stage<T, INV, LR>(fl, ls, log2n, lp, nb, tw);
      return;
    }
  }
  if constexpr (HF) {
    if (first) {
      fft_stage<T, INV, LR>(fl, out, log2n, lp, nb, tw);
      return;
    }
  }
  if constexpr (HL) {
    if (last) {
      fft_stage<T, INV, LR>(in, ls, log2n, lp, nb, tw);
      return;
    }
  }
  fft_stage<T, INV, LR>(in, out, log2n, lp, nb, tw);
}

// All stages of `nb` transforms of length 2^log2n. Stage 0 reads through `fl` (or from the padded
// buffer a), the last stage writes through `ls` (or to its padded target buffer); in between the
// stages ping-pong between a and b. Returns the padded buffer the last stage wrote (meaningful
// when `ls` is NoIO). All threads of the block must call it.
template <typename T, bool INV, class FL = NoIO, class LS = NoIO>
__device__ cplx<T>* fft_run(cplx<T>* a, cplx<T>* b, int log2n, int nb, const cplx<T>* __restrict__ tw,
                            const FL& fl = FL(), const LS& ls = LS()) {
  int lp = 0;
  int s = log2n;
  cplx<T>* src = a;
  cplx<T>* dst = b;
  bool first = true;
  while (s > 0) {
    const int lr = s >= 3 ? 3 : s;
    const bool last = s == lr;
    const SmemIO<T> in{src, log2n}, out{dst, log2n};
    if (lr == 3)
      fft_stage_dispatch<T, INV, 3>(first, last, in, out, fl, ls, log2n, lp, nb, tw);
    else if (lr == 2)
      fft_stage_dispatch<T, INV, 2>(first, last, in, out, fl, ls, log2n, lp, nb, tw);
    else
      fft_stage_dispatch<T, INV, 1>(first, last, in, out, fl, ls, log2n, lp, nb, tw);
    __syncthreads();
    cplx<T>* tmp = src;
    src = dst;
    dst = tmp;
    lp += lr;
    s -= lr;
    first = false;
  }
  return src;
}

// copy the n-entry twiddle table into shared memory (caller synchronises before use)
template <typename T>
__device__ __forceinline__ void load_twiddles(cplx<T>* dst, const cplx<T>* __restrict__ src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// ------------------------------------------------------------------------------------------
// One-dimensional 4-point kernels φ of δ_h (Sec. 2.2.2) and their derivatives, FP64.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double phi_cos(double r) {
  return fabs(r) < 2.0 ? 0.25 * (1.0 + cospi(0.5 * r)) : 0.0;
}
__device__ __forceinline__ double dphi_cos(double r) {
  return fabs(r) < 2.0 ? -0.125 * 3.14159265358979323846 * sinpi(0.5 * r) : 0.0;
}
// Peskin: (3 − 2a + √(1 + 4a − 4a²))/8 on a ≤ 1, (5 − 2a − √(−7 + 12a − 4a²))/8 on 1 < a < 2
__device__ __forceinline__ double phi_sqrt(double r) {
  const double a = fabs(r);
  if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) * 0.125;
  if (a < 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) * 0.125;
  return 0.0;
}
__device__ __forceinline__ double dphi_sqrt(double r) {
  const double a = fabs(r);
  double d = 0.0;
  if (a <= 1.0)
    d = (-2.0 + (2.0 - 4.0 * a) / sqrt(1.0 + 4.0 * a - 4.0 * a * a)) * 0.125;
  else if (a < 2.0)
    d = (-2.0 - (6.0 - 4.0 * a) / sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) * 0.125;
  return r < 0.0 ? -d : d;
}
// second derivatives (even in r); at the joins |r| = 1 (√ form) and |r| = 2 the inner piece's value
__device__ __forceinline__ double ddphi_cos(double r) {
  const double c = 3.14159265358979323846 * 3.14159265358979323846 / 16.0;
  return fabs(r) < 2.0 ? -c * cospi(0.5 * r) : 0.0;
}
__device__ __forceinline__ double ddphi_sqrt(double r) {
  const double a = fabs(r);
  if (a <= 1.0) {
    const double q = 1.0 + 4.0 * a - 4.0 * a * a, sq = sqrt(q);
    return (-4.0 / sq - (2.0 - 4.0 * a) * (4.0 - 8.0 * a) / (2.0 * q * sq)) * 0.125;
  }
  if (a < 2.0) {
    const double q = -7.0 + 12.0 * a - 4.0 * a * a, sq = sqrt(q);
    return (4.0 / sq + (6.0 - 4.0 * a) * (12.0 - 8.0 * a) / (2.0 * q * sq)) * 0.125;
  }
  return 0.0;
}

}  // namespace ibdl
