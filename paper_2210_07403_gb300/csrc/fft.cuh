// Shared-memory Stockham FFT and the regularised-delta kernels used by the IBDL kernels.
#pragma once

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

template <typename T, bool INV, int LR>
__device__ __forceinline__ void stockham_stage(const cplx<T>* __restrict__ src, cplx<T>* __restrict__ dst, int log2n,
                                               int lp, int nb, int bstride, const cplx<T>* __restrict__ tw) {
  constexpr int R = 1 << LR;
  const int lq = log2n - LR;
  const int q = 1 << lq;
  const int p = 1 << lp;
  const int total = nb << lq;
  const int tws = 1 << (log2n - lp - LR);  // n / (pR)
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int bi = t >> lq, i = t & (q - 1), k = i & (p - 1);
    const cplx<T>* x = src + bi * bstride;
    cplx<T> u[R];
#pragma unroll
    for (int r = 0; r < R; ++r) u[r] = x[i + r * q];
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
    cplx<T>* y = dst + bi * bstride;
    const int j = ((i - k) << LR) + k;
#pragma unroll
    for (int r = 0; r < R; ++r) y[j + r * p] = u[r];
  }
}

template <typename T, bool INV>
__device__ cplx<T>* fft_stockham(cplx<T>* a, cplx<T>* b, int log2n, int nb, int bstride,
                                 const cplx<T>* __restrict__ tw) {
  int lp = 0;  // log2 of the current sub-transform length
  int s = log2n;
  cplx<T>* src = a;
  cplx<T>* dst = b;
  while (s > 0) {
    if (s >= 3) {
      stockham_stage<T, INV, 3>(src, dst, log2n, lp, nb, bstride, tw);
      lp += 3;
      s -= 3;
    } else if (s == 2) {
      stockham_stage<T, INV, 2>(src, dst, log2n, lp, nb, bstride, tw);
      lp += 2;
      s -= 2;
    } else {
      stockham_stage<T, INV, 1>(src, dst, log2n, lp, nb, bstride, tw);
      lp += 1;
      s -= 1;
    }
    __syncthreads();
    cplx<T>* tmp = src;
    src = dst;
    dst = tmp;
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

}  // namespace ibdl
