// Derivatives of the IBDL operator and of values at probe points (analytic dipole spread).
//
// Both operators are A Q = S*(K[sources(Q)]) + ½Q with K a Fourier multiplier (Sec. 5.3.2:
// K = −L⁻¹ on f = Σ_i (Δs_i/h^d) Q_i n_i·∇Φ(x − X_i); Sec. 6.3.3: the Stokes multiplier on
// s = Σ_i (Δs_i/h^d)(Q_i·n_i)Φ and g_m = Σ_i (Δs_i/h^d) Σ_k A_mk,i ∂_kΦ, A = Q nᵀ + n Qᵀ), with
// (S*u)_i = Σ_g u_g Φ(x_g − X_i) and Φ = Π_m φ((x − X)_m/h). For a grid field v = Kᵀψ:
//   ⟨v, sources(Q)⟩ has the Q-gradient (the spread transpose)
//       scalar  (Δs_i/h^d) n_i·Σ_g v ∇Φ
//       Stokes  (Δs_i/h^d)[n_l a_s + Σ_k n_k (G_lk + G_kl)],  a_s = Σ_g v_s Φ, G_mk = Σ_g v_gm ∂_kΦ
//   and derivatives in X_i, n_i, Δs_i through the point's kernel weights (∇∇Φ for X).
// The solve gradient: for λ = A⁻ᵀ ∂J/∂Q, ∂J/∂p = −∂(λᵀAQ)/∂p = −(⟨v, sources(Q)⟩ terms with
// ψ = Σ λ Φ) + Σ_l λ_l Σ_g u_l ∇Φ (interpolation term, u = K[sources(Q)]).
// Probes: E Q = (S*_P u)(p) at probe points p; Eᵀν and ∂(νᵀEQ)/∂p are the ⟨v, sources(Q)⟩
// terms with ψ = Σ_p ν_p Φ(x − p).
// One thread per boundary point gathers over its 4^d stencil from FP64 grid fields.
#include "fft.cuh"

namespace ibdl {

struct PointDerivParams {
  int n, M;
  size_t cells;              // n^d
  const int* base;           // sorted tables of the geometry
  const int* perm;
  const double* phi;
  const double* dphi;
  const double* ddphi;
  const double* wscale;      // Δs/h^d
  const double* nrm;
  double hd;                 // h^d
  const double* Q;           // [c][M], original order
  const double* v;           // Kᵀψ: scalar [1][cells], Stokes [1 + d][cells] (v_s, v_g)
  const double* u;           // optional forward field [c][cells] for the interpolation term
  const double* mu;          // with u: [c][M]
  double sgn;                // multiplies every output
  double* dQ;                // optional outputs: [c][M], [d][M], [d][M], [M]
  double* dX;
  double* dn;
  double* dw;
};

template <int D, bool STOKES>
__global__ void __launch_bounds__(128) k_point_derivs(PointDerivParams p) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.M) return;
  const int M = p.M, i = p.perm[s];
  constexpr int NV = STOKES ? 1 + D : 1, NU = STOKES ? D : 1;
  double p0[D][4], p1[D][4], p2[D][4];
  int node[D][4];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const int b = p.base[j * M + s];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      p0[j][a] = p.phi[(j * 4 + a) * M + s];
      p1[j][a] = p.dphi[(j * 4 + a) * M + s];
      p2[j][a] = p.ddphi[(j * 4 + a) * M + s];
      node[j][a] = (b + a) & (p.n - 1);
    }
  }
  // per field: value gather (Stokes v_s only), gradient and Hessian gathers
  double a0 = 0.0, G[NV][D] = {}, H[NV][D][D] = {}, Gu[NU][D] = {};
  constexpr int NN = D == 2 ? 16 : 64;
#pragma unroll
  for (int t = 0; t < NN; ++t) {
    int a[D];
    size_t idx = 0;
#pragma unroll
    for (int j = D - 1; j >= 0; --j) {
      a[j] = (t >> (2 * j)) & 3;
      idx = idx * p.n + node[j][a[j]];
    }
    double w0 = 1.0, w1[D], w2[D][D];
#pragma unroll
    for (int j = 0; j < D; ++j) w0 *= p0[j][a[j]];
#pragma unroll
    for (int m = 0; m < D; ++m) {
      w1[m] = 1.0;
#pragma unroll
      for (int j = 0; j < D; ++j) w1[m] *= j == m ? p1[j][a[j]] : p0[j][a[j]];
#pragma unroll
      for (int l = 0; l < D; ++l) {
        double h = 1.0;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          if (l == m)
            h *= j == m ? p2[j][a[j]] : p0[j][a[j]];
          else
            h *= (j == m || j == l) ? p1[j][a[j]] : p0[j][a[j]];
        }
        w2[m][l] = h;
      }
    }
#pragma unroll
    for (int f = 0; f < NV; ++f) {
      const double vg = p.v[f * p.cells + idx];
      if (f == 0) a0 += vg * w0;
#pragma unroll
      for (int m = 0; m < D; ++m) {
        G[f][m] += vg * w1[m];
#pragma unroll
        for (int l = 0; l < D; ++l) H[f][m][l] += vg * w2[m][l];
      }
    }
    if (p.u) {
#pragma unroll
      for (int f = 0; f < NU; ++f) {
        const double ug = p.u[f * p.cells + idx];
#pragma unroll
        for (int m = 0; m < D; ++m) Gu[f][m] += ug * w1[m];
      }
    }
  }
  double nv[D];
#pragma unroll
  for (int m = 0; m < D; ++m) nv[m] = p.nrm[m * M + s];
  const double ws = p.wscale[s];
  double dX[D], dn[D], dw;
  if (!STOKES) {
    const double q = p.Q[i];
    double ng = 0.0;
#pragma unroll
    for (int m = 0; m < D; ++m) {
      double hn = 0.0;
#pragma unroll
      for (int l = 0; l < D; ++l) hn += H[0][m][l] * nv[l];
      dX[m] = -ws * q * hn;
      dn[m] = ws * q * G[0][m];
      ng += nv[m] * G[0][m];
    }
    dw = q * ng / p.hd;
    if (p.dQ) p.dQ[i] = p.sgn * ws * ng;
  } else {
    // G[0] = ∇-gather of v_s, G[1 + m][k] = Σ v_gm ∂_kΦ, H[1 + m][k][j] = Σ v_gm ∂_k∂_jΦ
    double q[D], c = 0.0;
#pragma unroll
    for (int m = 0; m < D; ++m) {
      q[m] = p.Q[(size_t)m * M + i];
      c += q[m] * nv[m];
    }
    double AG = 0.0;
#pragma unroll
    for (int m = 0; m < D; ++m)
#pragma unroll
      for (int k = 0; k < D; ++k) AG += (q[m] * nv[k] + q[k] * nv[m]) * G[1 + m][k];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double ah = 0.0, gq = 0.0;
#pragma unroll
      for (int m = 0; m < D; ++m) {
        gq += q[m] * (G[1 + m][j] + G[1 + j][m]);
#pragma unroll
        for (int k = 0; k < D; ++k) ah += (q[m] * nv[k] + q[k] * nv[m]) * H[1 + m][k][j];
      }
      dX[j] = -ws * (c * G[0][j] + ah);
      dn[j] = ws * (q[j] * a0 + gq);
    }
    dw = (c * a0 + AG) / p.hd;
    if (p.dQ) {
#pragma unroll
      for (int l = 0; l < D; ++l) {
        double t = nv[l] * a0;
#pragma unroll
        for (int k = 0; k < D; ++k) t += nv[k] * (G[1 + l][k] + G[1 + k][l]);
        p.dQ[(size_t)l * M + i] = p.sgn * ws * t;
      }
    }
  }
  if (p.u) {
#pragma unroll
    for (int l = 0; l < NU; ++l) {
      const double ml = p.mu[(size_t)l * M + i];
#pragma unroll
      for (int m = 0; m < D; ++m) dX[m] -= ml * Gu[l][m];
    }
  }
#pragma unroll
  for (int m = 0; m < D; ++m) {
    if (p.dX) p.dX[(size_t)m * M + i] = p.sgn * dX[m];
    if (p.dn) p.dn[(size_t)m * M + i] = p.sgn * dn[m];
  }
  if (p.dw) p.dw[i] = p.sgn * dw;
}

// ------------------------------------------------------------------------------------------
// probes: φ weights computed from the raw coordinates (FP64), 4×4 stencil, periodic wrap
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void probe_stencil(const double* P, int np, int pidx, double ox, double oy, double h,
                                             int n, int delta, int node[2][4], double w[2][4]) {
  const double org[2] = {ox, oy};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const double xi = (P[(size_t)j * np + pidx] - org[j]) / h;
    const long long b = (long long)floor(xi) - 1;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const double r = (double)(b + a) - xi;
      w[j][a] = delta == IBDL_DELTA_SQRT ? phi_sqrt(r) : phi_cos(r);
      long long m = (b + a) % n;
      node[j][a] = (int)(m < 0 ? m + n : m);
    }
  }
}

// U[c][np] = Σ_g u_c(x_g) Φ(x_g − p)
__global__ void k_probe_interp(const double* __restrict__ P, int np, int c, const double* __restrict__ u, size_t cells,
                               int n, double ox, double oy, double h, int delta, double* __restrict__ U) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  int node[2][4];
  double w[2][4];
  probe_stencil(P, np, k, ox, oy, h, n, delta, node, w);
  for (int f = 0; f < c; ++f) {
    double acc = 0.0;
#pragma unroll
    for (int ay = 0; ay < 4; ++ay)
#pragma unroll
      for (int ax = 0; ax < 4; ++ax)
        acc += u[f * cells + (size_t)node[1][ay] * n + node[0][ax]] * w[0][ax] * w[1][ay];
    U[(size_t)f * np + k] = acc;
  }
}

// ψ_c(x_g) += Σ_p ν_c,p Φ(x_g − p) (ψ zeroed by the caller)
__global__ void k_probe_spread(const double* __restrict__ P, int np, int c, const double* __restrict__ nu, size_t cells,
                               int n, double ox, double oy, double h, int delta, double* __restrict__ psi) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  int node[2][4];
  double w[2][4];
  probe_stencil(P, np, k, ox, oy, h, n, delta, node, w);
  for (int f = 0; f < c; ++f) {
    const double v = nu[(size_t)f * np + k];
#pragma unroll
    for (int ay = 0; ay < 4; ++ay)
#pragma unroll
      for (int ax = 0; ax < 4; ++ax)
        atomicAdd(psi + f * cells + (size_t)node[1][ay] * n + node[0][ax], v * w[0][ax] * w[1][ay]);
  }
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
static size_t grid_cells(const Geometry* g) {
  size_t cells = (size_t)g->n * g->n;
  if (g->dim == 3) cells *= g->n;
  return cells;
}

// grid workspace: c forward fields followed by the adjoint fields (1 scalar, 1 + d Stokes)
static ibdl_status vjp_workspace(Geometry* g, double** u, double** v) {
  const size_t cells = grid_cells(g);
  const int nv = g->pde == IBDL_PDE_STOKES ? 1 + g->dim : 1;
  if (!g->vjp_buf) IBDL_CUDA(cudaMalloc((void**)&g->vjp_buf, (g->ncomp + nv) * cells * sizeof(double)));
  *u = g->vjp_buf;
  *v = g->vjp_buf + g->ncomp * cells;
  return IBDL_OK;
}

static PointDerivParams deriv_params(Geometry* g, const double* Q, const double* v, double sgn) {
  PointDerivParams p = {};
  p.n = g->n;
  p.M = (int)g->M;
  p.cells = grid_cells(g);
  p.base = g->base;
  p.perm = g->perm;
  p.phi = g->t64.phi;
  p.dphi = g->t64.dphi;
  p.ddphi = g->ddphi64;
  p.wscale = g->t64.wscale;
  p.nrm = g->t64.nrm;
  p.hd = g->dim == 2 ? g->h * g->h : g->h * g->h * g->h;
  p.Q = Q;
  p.v = v;
  p.sgn = sgn;
  return p;
}

static ibdl_status launch_derivs(Geometry* g, const PointDerivParams& p, cudaStream_t s) {
  const int tb = 128, grid = (p.M + tb - 1) / tb;
  if (p.M == 0) return IBDL_OK;
  if (g->pde == IBDL_PDE_STOKES)
    k_point_derivs<2, true><<<grid, tb, 0, s>>>(p);
  else if (g->dim == 2)
    k_point_derivs<2, false><<<grid, tb, 0, s>>>(p);
  else
    k_point_derivs<3, false><<<grid, tb, 0, s>>>(p);
  g->launches += 1;
  IBDL_CUDA(cudaGetLastError());
  return IBDL_OK;
}

static ibdl_status check_derivs(const Geometry* g) {
  if (g->dipole != IBDL_DIPOLE_ANALYTIC)
    return fail(IBDL_ERR_UNSUPPORTED, "derivatives: analytic dipole spread only");
  if (!g->ddphi64) return fail(IBDL_ERR_UNSUPPORTED, "derivatives need the second-derivative table");
  return IBDL_OK;
}

ibdl_status solve_vjp_impl(Geometry* g, const double* Q, const double* lam, double* dX, double* dn, double* dw,
                           cudaStream_t s) {
  IBDL_TRY(check_derivs(g));
  double *u, *v;
  IBDL_TRY(vjp_workspace(g, &u, &v));
  IBDL_TRY(g->dim == 2 ? field_pair_2d(g, Q, lam, u, v, s) : field_pair_3d(g, Q, lam, u, v, s));
  PointDerivParams p = deriv_params(g, Q, v, -1.0);
  p.u = u;
  p.mu = lam;
  p.dX = dX;
  p.dn = dn;
  p.dw = dw;
  return launch_derivs(g, p, s);
}

ibdl_status probe_evaluate_impl(Geometry* g, const double* P, int np, const double* Q, double* U, cudaStream_t s) {
  if (g->dim != 2) return fail(IBDL_ERR_UNSUPPORTED, "probes: 2-D only");
  double *u, *v;
  IBDL_TRY(vjp_workspace(g, &u, &v));
  IBDL_TRY(field_2d(g, Q, u, s));
  if (np == 0) return IBDL_OK;
  k_probe_interp<<<(np + 127) / 128, 128, 0, s>>>(P, np, g->ncomp, u, grid_cells(g), g->n, g->origin[0],
                                                  g->origin[1], g->h, g->delta, U);
  g->launches += 1;
  IBDL_CUDA(cudaGetLastError());
  return IBDL_OK;
}

ibdl_status probe_vjp_impl(Geometry* g, const double* P, int np, const double* Q, const double* nu, double* dQ,
                           double* dX, double* dn, double* dw, cudaStream_t s) {
  if (g->dim != 2) return fail(IBDL_ERR_UNSUPPORTED, "probes: 2-D only");
  IBDL_TRY(check_derivs(g));
  double *psi, *v;
  IBDL_TRY(vjp_workspace(g, &psi, &v));
  const size_t cells = grid_cells(g);
  IBDL_CUDA(cudaMemsetAsync(psi, 0, g->ncomp * cells * sizeof(double), s));
  if (np > 0) {
    k_probe_spread<<<(np + 127) / 128, 128, 0, s>>>(P, np, g->ncomp, nu, cells, g->n, g->origin[0], g->origin[1],
                                                    g->h, g->delta, psi);
    g->launches += 1;
    IBDL_CUDA(cudaGetLastError());
  }
  IBDL_TRY(transform_T_2d(g, psi, v, s));
  PointDerivParams p = deriv_params(g, Q, v, 1.0);
  p.dQ = dQ;
  p.dX = dX;
  p.dn = dn;
  p.dw = dw;
  return launch_derivs(g, p, s);
}

}  // namespace ibdl
