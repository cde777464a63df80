// Register-resident FFT of power-of-two length N = 2^L (L = 4 … 13), the transform of the 2-D
// IBDL kernels. The transform length is a compile-time constant, so every index, stride and loop
// below folds to constants.
//
// Layout. A sequence is handled by Q = N/8 lanes; lane j holds the eight elements
// x[j + s·Q], s = 0 … 7, in registers, both on entry and on exit (the transform of element
// j + s·Q). A thread may hold V lanes of a sequence (j, j + Q/V, …) and FL sequences at once.
//
// Stages (Stockham autosort, no bit reversal): radix-8 stages with sub-transform lengths
// p = 1, 8, 64, … first, then one radix-2 or radix-4 stage when L is not a multiple of 3. A
// radix-8 stage with length p: butterfly j takes x[j + r·Q] (r < 8), multiplies input r by
// ω^{r·k}, k = j mod p, ω = e^{∓2πi/(8p)}, takes the 8-point DFT and writes output t to
// y[(j − k)·8 + k + t·p]. The tail stage (radix R, length N/R) runs 8/R butterflies per lane,
// i = j + m·Q, on the lane's own registers and leaves output t of butterfly m in x[m + t·8/R]:
// the same positions j + s·Q. Between stages the lanes exchange through one padded shared-memory
// buffer per sequence (N + N/8 elements: one pad after every eight keeps the stride-8 writes of the
// first stage free of bank conflicts).
//
// Twiddles come from the table tw[m] = e^{−2πi m/N}: held in registers per lane (read once,
// before a kernel's dependency wait) or read from the table at each use.
#pragma once

#include <type_traits>
#include <utility>

#include "fft.cuh"

namespace ibdl {

template <int I, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < E) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, E>(f);
  }
}

template <int L, int V_>
struct F8 {
  static_assert(L >= 4 && L <= 13, "transform lengths 16 … 8192");
  static constexpr int N = 1 << L;
  static constexpr int Q = N / 8;                        // lanes of a sequence
  static constexpr int S8 = L / 3;                       // radix-8 stages
  static constexpr int LT = L % 3;                       // log2 of the tail radix (0: none)
  static constexpr int RT = 1 << LT;
  static constexpr int NST = S8 + (LT ? 1 : 0);          // stages
  static constexpr int V = V_;                           // lanes per thread
  static_assert(Q % V == 0, "lanes per thread must divide Q");
  static constexpr int QT = Q / V;                       // threads per sequence
  // twiddles per lane: 7 per radix-8 stage after the first, (RT − 1) per tail butterfly
  static constexpr int NTW = (S8 - 1) * 7 + (LT ? (RT - 1) * (8 / RT) : 0);
  static constexpr int PN = N + N / 8;                   // padded sequence length in shared memory
};

__host__ __device__ constexpr int ipow8(int s) { return s == 0 ? 1 : 8 * ipow8(s - 1); }

// table index of the twiddle of stage S, tail butterfly m (0 for radix-8 stages), input r, lane j
template <int L, int S>
__device__ __forceinline__ int tw_index(int j, int m, int r) {
  constexpr int S8 = L / 3, N = 1 << L, Q = N / 8;
  if constexpr (S < S8) {
    constexpr int p = ipow8(S);
    return r * (j & (p - 1)) * (N / (8 * p));
  } else {
    return r * (j + m * Q);
  }
}

// the twiddles of one lane, in registers
template <typename T, int L>
struct TwRegs {
  static constexpr int S8 = L / 3, LT = L % 3, RT = 1 << LT;
  static constexpr int NTW = (S8 - 1) * 7 + (LT ? (RT - 1) * (8 / RT) : 0);
  cplx<T> w[NTW > 0 ? NTW : 1];
  template <int S>
  __host__ __device__ static constexpr int off(int m, int r) {
    return S < S8 ? (S - 1) * 7 + (r - 1) : (S8 - 1) * 7 + m * (RT - 1) + (r - 1);
  }
  __device__ __forceinline__ void load(const cplx<T>* __restrict__ tab, int j) {
    static_for<1, S8>([&](auto st) {
      constexpr int S = decltype(st)::value;
#pragma unroll
      for (int r = 1; r < 8; ++r) w[off<S>(0, r)] = tab[tw_index<L, S>(j, 0, r)];
    });
    if constexpr (LT > 0) {
#pragma unroll
      for (int m = 0; m < 8 / RT; ++m)
#pragma unroll
        for (int r = 1; r < RT; ++r) w[off<S8>(m, r)] = tab[tw_index<L, S8>(j, m, r)];
    }
  }
  template <int S>
  __device__ __forceinline__ cplx<T> get(int m, int r) const { return w[off<S>(m, r)]; }
};

// the twiddles of one lane, read from the table (global memory, L1-cached) at each use
template <typename T, int L>
struct TwTable {
  const cplx<T>* __restrict__ tab;
  int j;
  __device__ __forceinline__ void load(const cplx<T>* __restrict__ t, int lane) {
    tab = t;
    j = lane;
  }
  template <int S>
  __device__ __forceinline__ cplx<T> get(int m, int r) const { return tab[tw_index<L, S>(j, m, r)]; }
};

// a·w (forward) or a·conj(w) (inverse)
template <typename T, bool INV>
__device__ __forceinline__ cplx<T> cmul_tw(cplx<T> a, cplx<T> w) {
  return INV ? mk(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y) : mk(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}

// stage S on one lane's registers
template <typename T, bool INV, int L, int S, class TW>
__device__ __forceinline__ void f8_stage(cplx<T> (&x)[8], const TW& tw) {
  constexpr int S8 = L / 3, LT = L % 3, RT = 1 << LT;
  if constexpr (S < S8) {
    if constexpr (S > 0) {
#pragma unroll
      for (int r = 1; r < 8; ++r) x[r] = cmul_tw<T, INV>(x[r], tw.template get<S>(0, r));
    }
    dft8<T, INV>(x);
  } else {
    constexpr int MB = 8 / RT;
#pragma unroll
    for (int m = 0; m < MB; ++m) {
      cplx<T> u[RT];
#pragma unroll
      for (int r = 0; r < RT; ++r) u[r] = x[m + r * MB];
#pragma unroll
      for (int r = 1; r < RT; ++r) u[r] = cmul_tw<T, INV>(u[r], tw.template get<S>(m, r));
      if constexpr (RT == 4)
        dft4<T, INV>(u[0], u[1], u[2], u[3]);
      else
        dft2<T, INV>(u);
#pragma unroll
      for (int t = 0; t < RT; ++t) x[m + t * MB] = u[t];
    }
  }
}

// padded position of element e of a sequence (see pidx); e < N
__device__ __forceinline__ int ppos(int e) { return e + (e >> 3); }
// padded position of j + s·Q: ppos(j) + s·(Q + Q/8) when Q is a multiple of 8 (n ≥ 64)
template <int Q>
__device__ __forceinline__ int ppos_strided(int j, int s) {
  if constexpr (Q % 8 == 0)
    return ppos(j) + s * (Q + Q / 8);
  else
    return ppos(j + s * Q);
}

// The same transform for one sequence with the radix-8 stages as a loop over a runtime
// sub-length p and the twiddles read from the table (index r·k·n/(8p), k = j mod p): one copy of
// the stage code instead of one per stage. For float-float, whose unrolled stages would not fit
// the instruction cache.
template <typename T, bool INV, int L, int V>
__device__ __forceinline__ void f8_fft_rolled(cplx<T> (&x)[1][V][8], cplx<T>* buf, int j0,
                                              const cplx<T>* __restrict__ tab, bool active) {
  using F = F8<L, V>;
#pragma unroll 1
  for (int S = 0; S < F::S8; ++S) {
    const int p = 1 << (3 * S);
    if (active) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        if (S > 0) {
          const int step = ((j0 + v * F::QT) & (p - 1)) << (L - 3 - 3 * S);
#pragma unroll
          for (int r = 1; r < 8; ++r) x[0][v][r] = cmul_tw<T, INV>(x[0][v][r], tab[r * step]);
        }
        dft8<T, INV>(x[0][v]);
      }
    }
    if (S + 1 < F::NST) {
      __syncthreads();
      if (active) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int j = j0 + v * F::QT, k = j & (p - 1);
          const int base = (j - k) * 8 + k;
#pragma unroll
          for (int t = 0; t < 8; ++t) buf[ppos(base + t * p)] = x[0][v][t];
        }
      }
      __syncthreads();
      if (active) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int j = j0 + v * F::QT;
#pragma unroll
          for (int s = 0; s < 8; ++s) x[0][v][s] = buf[ppos(j + s * F::Q)];
        }
      }
    }
  }
  if constexpr (F::LT > 0) {
    if (active) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        TwTable<T, L> tw;
        tw.load(tab, j0 + v * F::QT);
        f8_stage<T, INV, L, F::S8>(x[0][v], tw);
      }
    }
  }
}

// Transform of the FL sequences whose lanes j0 + v·QT (v < V) this thread holds: x[f][v][s] is
// element j + s·Q on entry and its transform on exit. buf + f·fstride is the padded shared buffer
// of sequence f. Every thread of the block must call it (it synchronises the block); `active` is
// false for threads that hold no sequence. Each lane reads its inputs before the call and writes
// its results after it only at its own positions j + s·Q, so neither needs a barrier against the
// exchanges inside.
template <typename T, bool INV, int L, int V, int FL, class TW>
__device__ __forceinline__ void f8_fft(cplx<T> (&x)[FL][V][8], cplx<T>* buf, int fstride, int j0,
                                       const TW (&tw)[V], bool active) {
  using F = F8<L, V>;
  if constexpr (FL == 1 && std::is_same<TW, TwTable<T, L>>::value && sizeof(T) == 8 && !std::is_same<T, double>::value) {
    // float-float (8-byte elements that are not double): the stage loop
    f8_fft_rolled<T, INV, L, V>(reinterpret_cast<cplx<T>(&)[1][V][8]>(x), buf, j0, tw[0].tab, active);
    return;
  }
  static_for<0, F::NST>([&](auto st) {
    constexpr int S = decltype(st)::value;
    if (active) {
#pragma unroll
      for (int f = 0; f < FL; ++f)
#pragma unroll
        for (int v = 0; v < V; ++v) f8_stage<T, INV, L, S>(x[f][v], tw[v]);
    }
    if constexpr (S + 1 < F::NST) {
      constexpr int p = ipow8(S);
      __syncthreads();
      if (active) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int j = j0 + v * F::QT, k = j & (p - 1);
          // base + t·p (t < 8) keeps base's low three bits when p ≥ 8 (and is 8j + t when
          // p = 1), so its padded position is ppos(base) plus a constant per t
          const int pb = ppos((j - k) * 8 + k);
          constexpr int dt = p == 1 ? 1 : p + p / 8;
#pragma unroll
          for (int f = 0; f < FL; ++f)
#pragma unroll
            for (int t = 0; t < 8; ++t) buf[f * fstride + pb + t * dt] = x[f][v][t];
        }
      }
      __syncthreads();
      if (active) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int j = j0 + v * F::QT;
#pragma unroll
          for (int f = 0; f < FL; ++f)
#pragma unroll
            for (int s = 0; s < 8; ++s) x[f][v][s] = buf[f * fstride + ppos_strided<F::Q>(j, s)];
        }
      }
    }
  });
}

}  // namespace ibdl
