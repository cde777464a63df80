// The Arnoldi step of GMRES (Sec. 5.3.2) on one thread-block cluster, FP64.
//
// Step j orthogonalises w = A v_j (stored at V_{j+1}) against V_0..V_j by classical Gram–Schmidt
// whose second pass comes from the basis' Gram matrix (one cluster reduction per step; see
// arnoldi_body), normalises it, applies the stored Givens rotations to the new Hessenberg
// column, forms the new rotation and updates the residual estimate |g_{j+1}|.
//
// CTA r of the cluster owns the slice [r·slice, (r+1)·slice) of every vector. Written for
// GB300's FP64 unit: each SM sub-partition accepts one FP64 warp instruction about every 76
// cycles whatever the number of active lanes, and a dependent FP64 operation waits about 65
// cycles (square root and division are sequences of them). So
//   - with STAGED the CTA copies its slice of V_0..V_j into shared memory before it waits for the
//     application (programmatic launch), and every CTA copies the Gram block of v_0..v_{j−1}:
//     those vectors, the Gram matrix and the rotation state are final by then;
//   - dot products give L lanes to each basis vector (all lanes busy), each lane two
//     accumulators over a strided part of the slice, then an 8-way tree of the partial sums;
//     no shuffle reductions (a full-warp FP64 add per level);
//   - vector updates spread the sum over basis vectors across all threads in groups;
//   - 1/√x comes from the single-precision estimate refined by two Newton–Raphson steps in
//     FP64, taken once per CTA;
//   - the old rotations are applied by one warp as a scan of the affine recurrence
//     x_{i+1} = −s_i x_i + c_i h_{i+1} (x_0 = h_0), whose values give the rotated column
//     H_i = c_i x_i + s_i h_{i+1}; 5 shuffle levels replace the 2j dependent operations;
//   - that warp, about 2 µs of dependent FP64 operations, runs beside the vector update (named
//     barriers hand it ‖w₂‖), and short reductions (the ranks' partial sums, the Gram product)
//     are spread over several warps so that no single SM sub-partition issues them all.
// Partial sums of the cluster are combined through distributed shared memory. One cluster barrier
// per step, and a split arrive/wait one so no CTA exits while another may still read its shared
// memory. On the 512² Stokes star the step takes 12.4 µs standalone (14.4 µs with the rotation
// after the update, 16.8 µs with CGS2's two reductions), and the solves keep their iteration
// counts.
#pragma once

#include <cooperative_groups.h>

namespace ibdl {

namespace cg = cooperative_groups;

enum { KMAX = 64 };
enum { ST_RUNNING = 0, ST_CONVERGED = 1, ST_BREAKDOWN = 2, ST_NONFINITE = 3 };

struct GmresState {
  int stop;    // nonzero: every queued kernel returns at once
  int status;  // ST_*
  int k;       // Arnoldi steps completed in this cycle
  int kmax;    // steps allowed in this cycle (≤ restart length and the remaining budget)
  int body_iters;  // loop bodies run by the captured cycle (a guard on the device-side loop)
  int pad2;
  double res;      // |g_k|, the GMRES residual estimate
  double beta;     // ‖r0‖ of the cycle
  double target;   // absolute tolerance on the residual
  double rnorm;    // ‖r‖ from k_residual
  double cs[KMAX], sn[KMAX], g[KMAX + 1];
  double H[(KMAX + 1) * KMAX];  // column j at H[j·(m+1) + i]
  double bnorm;                 // ‖U_b‖, recorded by the first cycle of a refinement solve
  double G[KMAX * KMAX];        // Gram matrix v_iᵀv_k of the basis, G[i·KMAX + k] (filled one column per step)
};

struct HostStatus {
  int stop, status, k, kmax, body_iters, pad2;
  double res, beta, target, rnorm;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int ATH = 512;
constexpr int ALEAD = ATH - 32;  // the thread of CTA 0 that returns a step's result (lane 0 of the rotation warp)

// dynamic shared memory (doubles) of a step: w's slice, then (staged) m + 1 basis rows, then the
// (m + 1)² Gram block
__host__ __device__ constexpr size_t arnoldi_dyn_doubles(int m, int slice, bool staged) {
  return (size_t)(staged ? m + 2 : 1) * (size_t)slice + (size_t)(m + 1) * (size_t)(m + 1);
}

// 1/√x for finite x > 2^−1000, by Newton–Raphson iteration for the reciprocal square root,
// y ← y + (y/2)(1 − x y²), started from the single-precision estimate; x is first scaled by
// 4^−k into [1, 4) so that estimate neither underflows nor overflows. Two steps take the
// estimate's ~1e−7 relative error below FP64 rounding.
__device__ __forceinline__ double rsqrt_newton(double x) {
  const int hi = __double2hiint(x), lo = __double2loint(x);
  const int k = (((hi >> 20) & 0x7ff) - 1023) >> 1;
  const double m = __hiloint2double(hi - k * (1 << 21), lo);
  double y = (double)rsqrtf((float)m);
  double r = fma(-m * y, y, 1.0);
  y = fma(0.5 * y, r, y);
  r = fma(-m * y, y, 1.0);
  y = fma(0.5 * y, r, y);
  return __hiloint2double(__double2hiint(y) - k * (1 << 20), __double2loint(y));
}

// named barrier `id` over `n` threads (n a multiple of 32); id 0 is __syncthreads'
__device__ __forceinline__ void bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void bar_arrive(int id, int n) { asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// ws[e] −= Σ_{i≤j} h[i]·V_i[e] over the slice, the sum over i split into groups of threads; run by
// threads 0..NT−1, which synchronise on named barrier 1
template <int NT>
__device__ __forceinline__ void slice_update(const double* rows, size_t rstride, double* ws, int cnt, int j,
                                             const double* h, double* pw) {
  const int tid = threadIdx.x;
  auto vat = [&](int i, int e) -> double { return rows[(size_t)i * rstride + e]; };
  const int G = cnt > 0 ? min(8, NT / cnt) : 0;
  if (G <= 1) {
    for (int e = tid; e < cnt; e += NT) {
      double a0 = ws[e], a1 = 0.0;
      int i = 0;
      for (; i + 1 <= j; i += 2) {
        a0 -= h[i] * vat(i, e);
        a1 -= h[i + 1] * vat(i + 1, e);
      }
      if (i <= j) a0 -= h[i] * vat(i, e);
      ws[e] = a0 + a1;
    }
    bar_sync(1, NT);
    return;
  }
  const int g = tid / cnt, e = tid - g * cnt;
  if (g < G) {
    double a0 = 0.0, a1 = 0.0;
    int i = g;
    for (; i + G <= j; i += 2 * G) {
      a0 += h[i] * vat(i, e);
      a1 += h[i + G] * vat(i + G, e);
    }
    if (i <= j) a0 += h[i] * vat(i, e);
    pw[g * cnt + e] = a0 + a1;
  }
  bar_sync(1, NT);
  if (tid < cnt) {
    double s = 0.0;
    for (int q = 0; q < G; ++q) s += pw[q * cnt + tid];
    ws[tid] -= s;
  }
  bar_sync(1, NT);
}

// Dot products of the pairs (a_d, b_d) over the slice, d < ndots: d ≤ j: (V_d, w); d = j + 1:
// (w, w); j + 2 ≤ d ≤ 2j + 2: (V_{d−j−2}, V_j) (the last one V_j·V_j). Lanes, accumulators and the
// tree of partial sums as in slice_dots.
__device__ __forceinline__ void slice_dots_pairs(const double* rows, size_t rstride, const double* ws, int cnt,
                                                 int j, int ndots, double* pw, double* pw2, double* out) {
  const int tid = threadIdx.x;
  const int L = min(64, ATH / ndots), R = (L + 7) >> 3;
  if (tid < ndots * L) {
    const int d = tid / L, l = tid - d * L;
    const double* a;
    const double* b;
    if (d <= j) {
      a = rows + (size_t)d * rstride;
      b = ws;
    } else if (d == j + 1) {
      a = ws;
      b = ws;
    } else {
      a = rows + (size_t)(d - j - 2) * rstride;
      b = rows + (size_t)j * rstride;
    }
    double a0 = 0.0, a1 = 0.0;
    int e = l;
    for (; e + L < cnt; e += 2 * L) {
      a0 += a[e] * b[e];
      a1 += a[e + L] * b[e + L];
    }
    if (e < cnt) a0 += a[e] * b[e];
    pw[tid] = a0 + a1;
  }
  __syncthreads();
  if (tid < ndots * R) {
    const int d = tid / R, r = tid - d * R;
    const int b0 = d * L + 8 * r, b1 = min(d * L + L, b0 + 8);
    double a0 = 0.0, a1 = 0.0;
    int q = b0;
    for (; q + 1 < b1; q += 2) {
      a0 += pw[q];
      a1 += pw[q + 1];
    }
    if (q < b1) a0 += pw[q];
    pw2[tid] = a0 + a1;
  }
  __syncthreads();
  if (tid < ndots) {
    double a0 = 0.0, a1 = 0.0;
    int r = 0;
    for (; r + 1 < R; r += 2) {
      a0 += pw2[tid * R + r];
      a1 += pw2[tid * R + r + 1];
    }
    if (r < R) a0 += pw2[tid * R + r];
    out[tid] = a0 + a1;
  }
}

// Returns −1 (every thread) when the step was skipped because the cycle had already stopped;
// otherwise, on CTA 0 thread ALEAD, 1 if this step stopped the cycle and 0 if it continues.
// Control flow is uniform over the cluster (the skip decision reads state no kernel of the
// running application writes).
//
// Classical Gram–Schmidt with the second pass taken from the Gram matrix G = VᵀV of the basis:
// with t = V_jᵀw, CGS2's second coefficients are V_jᵀ(w − V_j t) = t − G t, so the new column is
// h = (2I − G)t and w₂ = w − V_j h needs one projection and one update. G's new column
// (v_iᵀv_j, i ≤ j) comes from the same cluster reduction as t and ‖w‖², so a step makes one
// reduction instead of two; ‖w₂‖² = ‖w‖² − hᵀt to second order in G − I. The rounding of the single
// subtraction leaves v_{j+1} off orthogonal by about ε‖w‖/‖w₂‖; the next step's G sees it and
// corrects the projection, so the departure does not accumulate.
template <bool STAGED, int CL>
__device__ __forceinline__ int arnoldi_body(GmresState* st, double* V, int j, int nd, int m, int slice) {
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double dsm[];
  __shared__ double part[2 * KMAX + 4], t[KMAX + 2], gc[KMAX + 2], h[KMAX + 2];
  __shared__ double pw[ATH], pw2[2 * KMAX + 8];
  __shared__ double csl[KMAX], snl[KMAX], sc[8], qsum[4 * (2 * KMAX + 4)];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rank = (int)cluster.block_rank();
  const int lo = rank * slice;
  const int cnt = nd - lo < slice ? (nd - lo > 0 ? nd - lo : 0) : slice;
  double* ws = dsm;
  double* Vs = dsm + slice;
  double* Gs = dsm + (STAGED ? (size_t)(m + 2) * slice : (size_t)slice);  // [(m+1)][(m+1)]
  const double* rows = STAGED ? Vs : V + lo;
  const size_t rstride = STAGED ? (size_t)slice : (size_t)nd;

  // prologue: everything but w is final while the application that writes V_{j+1} still runs
  // (every kernel triggers its dependents only after its own wait, so the step before that
  // application has completed)
  if (j < 0) j = st->k;
  const bool skip = st->stop || j >= st->kmax || j >= m;
  // a slot after the stop: return without waiting (the kernels after it read the same final state)
  if (skip) return -1;
  {
    if (STAGED)
      for (int q = tid; q < (j + 1) * cnt; q += ATH) {
        const int i = q / cnt, e = q - i * cnt;
        Vs[(size_t)i * slice + e] = V[(size_t)i * nd + lo + e];
      }
    for (int q = tid; q < j * j; q += ATH) {  // the Gram block of v_0..v_{j−1}
      const int a = q / j, b = q - a * j;
      Gs[a * (m + 1) + b] = st->G[a * KMAX + b];
    }
    if (rank == 0) {
      if (tid < j) {
        csl[tid] = st->cs[tid];
        snl[tid] = st->sn[tid];
      }
      if (tid == 0) {
        sc[0] = st->g[j];
        sc[4] = st->target;
        sc[5] = (double)st->kmax;
      }
    }
  }
  cudaGridDependencySynchronize();  // programmatic launch: wait for the application
  cudaTriggerProgrammaticLaunchCompletion();
  double* w = V + (size_t)(j + 1) * nd + lo;
  for (int e = tid; e < cnt; e += ATH) ws[e] = w[e];
  __syncthreads();

  // one reduction: t = V_jᵀw, ‖w‖², and G's column j (v_iᵀv_j, i ≤ j)
  const int ndots = 2 * j + 3;
  slice_dots_pairs(rows, rstride, ws, cnt, j, ndots, pw, pw2, part);
  cluster.sync();
  {  // the CL ranks' partial sums: quarter qq of the ranks per thread, then the four quarters
    constexpr int QR = CL % 4 == 0 ? 4 : 1, PER = CL / QR;
    for (int q = tid; q < QR * ndots; q += ATH) {
      const int qq = q / ndots, d = q - qq * ndots;
      double v[PER];
#pragma unroll
      for (int r = 0; r < PER; ++r) v[r] = cluster.map_shared_rank(part, qq * PER + r)[d];
#pragma unroll
      for (int s2 = PER / 2; s2 > 0; s2 >>= 1)
#pragma unroll
        for (int r = 0; r < s2; ++r) v[r] += v[r + s2];
      qsum[qq * ndots + d] = v[0];
    }
    // every remote read of this step is done: arrive now, wait before leaving
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    __syncthreads();
    if (tid < ndots) {
      double v = qsum[tid];
      if (QR == 4) v = (v + qsum[ndots + tid]) + (qsum[2 * ndots + tid] + qsum[3 * ndots + tid]);
      if (tid <= j)
        t[tid] = v;
      else if (tid == j + 1)
        sc[6] = v;
      else
        gc[tid - j - 2] = v;
    }
  }
  __syncthreads();
  {  // h = (2I − G) t: lanes own the rows, warps 4c..4c+3 split the k range of row chunk c in four
    const int nr = j + 1, chunks = (nr + 31) >> 5, K4 = (nr + 3) >> 2;
    if (warp < 4 * chunks) {
      const int i = 32 * (warp >> 2) + lane;
      const int k0 = (warp & 3) * K4, k1 = min(nr, k0 + K4);
      // G is symmetric: read G[k][i] so that the lanes' rows are contiguous
      auto gik = [&](int k) -> double {
        return (i < j && k < j) ? Gs[k * (m + 1) + i] : (i == j ? gc[k] : gc[i]);
      };
      double a0 = 0.0, a1 = 0.0;
      if (i < nr) {
        int k = k0;
        for (; k + 1 < k1; k += 2) {
          a0 += gik(k) * t[k];
          a1 += gik(k + 1) * t[k + 1];
        }
        if (k < k1) a0 += gik(k) * t[k];
      }
      pw[warp * 32 + lane] = a0 + a1;
    }
    __syncthreads();
    if (tid < nr) {
      const double* pr = pw + (tid >> 5) * 128 + (tid & 31);
      h[tid] = 2.0 * t[tid] - ((pr[0] + pr[32]) + (pr[64] + pr[96]));
    }
    __syncthreads();
  }

  // Three roles from here, so that the rotation (one warp of CTA 0, a chain of dependent FP64
  // operations) runs beside the vector update instead of after it:
  //   warps 0..WQ−1: w₂ = w − V_j h over the slice, then v_{j+1} = w₂ / ‖w₂‖;
  //   warp WQ: ‖w₂‖ and its reciprocal (named barrier 2 to the update warps, 3 to warp WG);
  //   warp WG (CTA 0): the old rotations on h, then, with ‖w₂‖, the new rotation and the status.
  constexpr int WQ = ATH / 32 - 2, WG = ATH / 32 - 1;
  int ret = 0;
  if (warp == WQ) {
    double q = 0.0;
    for (int i = lane; i <= j; i += 32) q += h[i] * t[i];
    q = warp_sum(q);
    if (lane == 0) {
      const double hn2 = sc[6] - q;
      const double y = hn2 > 0x1p-1000 && hn2 <= 1e300 ? rsqrt_newton(hn2) : 0.0;
      sc[1] = isfinite(hn2) ? hn2 * y : hn2;  // NaN/Inf passed on to the status test
      sc[2] = y;
    }
    __syncwarp();
    bar_arrive(2, ATH);
    if (rank == 0) bar_arrive(3, 64);
  } else if (warp == WG) {
    bar_arrive(2, ATH);
    if (rank == 0) {
      // old rotations on the new column by a scan over the affine maps f_i(x) = −s_i x + c_i h_{i+1}
      const int i0 = 2 * lane, i1 = i0 + 1;
      double a0 = 1.0, b0 = 0.0, a1 = 1.0, b1 = 0.0;
      if (i0 < j) {
        a0 = -snl[i0];
        b0 = csl[i0] * h[i0 + 1];
      }
      if (i1 < j) {
        a1 = -snl[i1];
        b1 = csl[i1] * h[i1 + 1];
      }
      double A = a1 * a0, B = a1 * b0 + b1;  // f_{i1} ∘ f_{i0}
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const double Ap = __shfl_up_sync(0xffffffffu, A, off), Bp = __shfl_up_sync(0xffffffffu, B, off);
        if (lane >= off) {
          B = A * Bp + B;
          A = A * Ap;
        }
      }
      double Ae = __shfl_up_sync(0xffffffffu, A, 1), Be = __shfl_up_sync(0xffffffffu, B, 1);
      if (lane == 0) {
        Ae = 1.0;
        Be = 0.0;
      }
      const double x0 = h[0];
      const double xa = Ae * x0 + Be;  // x_{i0}
      const double xb = a0 * xa + b0;  // x_{i1}
      double* hc = st->H + (size_t)j * (m + 1);
      if (i0 < j) hc[i0] = csl[i0] * xa + snl[i0] * h[i0 + 1];
      if (i1 < j) hc[i1] = csl[i1] * xb + snl[i1] * h[i1 + 1];
      __syncwarp();
      bar_sync(3, 64);  // ‖w₂‖ from warp WQ
      if (j == i0 || j == i1) {
        // the new rotation zeroes hn below x_j
        const double hn = sc[1];
        const double a = j == i0 ? xa : xb, b = hn;
        const double q = a * a + b * b;
        const double ir = q > 0x1p-1000 && q <= 1e300 ? rsqrt_newton(q) : (q > 0.0 ? 1.0 / sqrt(q) : 0.0);
        const double r = q * ir;
        const double c = q > 0.0 ? a * ir : 1.0, sn = b * ir;
        hc[j] = r;
        hc[j + 1] = 0.0;
        st->cs[j] = c;
        st->sn[j] = sn;
        const double gj = sc[0];
        st->g[j + 1] = -sn * gj;
        st->g[j] = c * gj;
        const double res = fabs(sn * gj);
        st->res = res;
        st->k = j + 1;
        int stop = 0;
        if (!isfinite(res) || !isfinite(hn) || !isfinite(a)) {
          st->status = ST_NONFINITE;
          stop = 1;
        } else if (res <= sc[4]) {
          st->status = ST_CONVERGED;
          stop = 1;
        } else if (hn == 0.0) {
          st->status = ST_BREAKDOWN;
          stop = 1;
        } else if (j + 1 >= (int)sc[5]) {
          stop = 1;  // cycle full
        }
        if (stop) st->stop = 1;
        sc[3] = stop;
      }
      __syncwarp();
      if (lane == 0) ret = (int)sc[3];
    }
  } else {
    slice_update<WQ * 32>(rows, rstride, ws, cnt, j, h, pw);
    bar_sync(2, ATH);
    const double inv = sc[2];
    for (int e = tid; e < cnt; e += WQ * 32) w[e] = ws[e] * inv;
    if (rank == 0 && tid <= j) {  // G's column and row j for the later steps of the cycle
      st->G[tid * KMAX + j] = gc[tid];
      st->G[j * KMAX + tid] = gc[tid];
    }
  }
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
  return (rank == 0 && tid == ALEAD) ? ret : 0;
}

}  // namespace ibdl
