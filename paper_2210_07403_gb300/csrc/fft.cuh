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
// Radix-4 stages run while at least two factors of two remain, then one radix-2 stage.
//
// tw[j] = e^{−2πi j/n}; the inverse transform (INV) uses conjugates and is unnormalised.
// Sequences are `nb` runs of n contiguous elements, sequence b starting at b·bstride.
// Returns the buffer that holds the result (a or b). All threads of the block must call it.
// ------------------------------------------------------------------------------------------
template <typename T, bool INV>
__device__ cplx<T>* fft_stockham(cplx<T>* a, cplx<T>* b, int log2n, int nb, int bstride,
                                 const cplx<T>* __restrict__ tw) {
  const int n = 1 << log2n;
  int p = 1;
  int lp = 0;  // log2 p
  int s = log2n;
  cplx<T>* src = a;
  cplx<T>* dst = b;
  while (s > 0) {
    if (s >= 2) {
      const int lq = log2n - 2;
      const int q = 1 << lq;
      const int total = nb << lq;
      const int tws = n >> (lp + 2);  // n / (4p)
      for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int bi = t >> lq;
        const int i = t & (q - 1);
        const int k = i & (p - 1);
        const cplx<T>* x = src + bi * bstride;
        cplx<T> u0 = x[i], u1 = x[i + q], u2 = x[i + 2 * q], u3 = x[i + 3 * q];
        if (k) {
          cplx<T> w1 = tw[k * tws], w2 = tw[2 * k * tws], w3 = tw[3 * k * tws];
          if (INV) {
            w1.y = -w1.y;
            w2.y = -w2.y;
            w3.y = -w3.y;
          }
          u1 = cmul(u1, w1);
          u2 = cmul(u2, w2);
          u3 = cmul(u3, w3);
        }
        const cplx<T> t0 = cadd(u0, u2), t1 = csub(u0, u2), t2 = cadd(u1, u3);
        cplx<T> t3 = csub(u1, u3);
        // forward: multiply (u1 − u3) by −i; inverse: by +i
        t3 = INV ? mk(-t3.y, t3.x) : mk(t3.y, -t3.x);
        cplx<T>* y = dst + bi * bstride;
        const int j = ((i - k) << 2) + k;
        y[j] = cadd(t0, t2);
        y[j + p] = cadd(t1, t3);
        y[j + 2 * p] = csub(t0, t2);
        y[j + 3 * p] = csub(t1, t3);
      }
      p <<= 2;
      lp += 2;
      s -= 2;
    } else {
      const int lq = log2n - 1;
      const int q = 1 << lq;
      const int total = nb << lq;
      const int tws = n >> (lp + 1);
      for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int bi = t >> lq;
        const int i = t & (q - 1);
        const int k = i & (p - 1);
        const cplx<T>* x = src + bi * bstride;
        cplx<T> u0 = x[i], u1 = x[i + q];
        if (k) {
          cplx<T> w = tw[k * tws];
          if (INV) w.y = -w.y;
          u1 = cmul(u1, w);
        }
        cplx<T>* y = dst + bi * bstride;
        const int j = ((i - k) << 1) + k;
        y[j] = cadd(u0, u1);
        y[j + p] = csub(u0, u1);
      }
      p <<= 1;
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
