// Boundary derivatives of a solve (scalar operator, analytic dipole spread).
//
// For Q = A⁻¹U_b and an objective J with g = ∂J/∂Q, the adjoint state is λ = A⁻ᵀ g
// (ibdl_solve_transpose) and ∂J/∂p = −∂(λᵀ A Q)/∂p for the boundary points X, normals n and
// weights Δs. The operator is A Q = S*u + ½Q, u = −L⁻¹ S̃Q (Sec. 5.3.2), with
//   (S*u)_j = Σ_g u_g Φ(x_g − X_j),  (S̃Q)_g = Σ_k Δs_k Q_k n_k·∇δ_h(x_g − X_k),
// Φ = Π_m φ((x − X)_m/h) and δ_h = Φ/h^d (Sec. 2.2.2). With v = −L⁻¹(Σ_j λ_j δ_h(x − X_j))
// (−L⁻¹ has a real even symbol, so it is symmetric), λᵀS*u = h^d vᵀ S̃Q and
//   ∂(λᵀAQ)/∂X_i = −λ_i Σ_g u_g ∇Φ(x_g − X_i) − Δs_i Q_i Σ_g v_g ∇∇Φ(x_g − X_i) n_i,
//   ∂(λᵀAQ)/∂n_i = Δs_i Q_i Σ_g v_g ∇Φ(x_g − X_i),
//   ∂(λᵀAQ)/∂Δs_i = Q_i n_i · Σ_g v_g ∇Φ(x_g − X_i).
// u and v are the grid fields of the forward and the transposed operator (FP64); one thread
// per boundary point then gathers ∇u, ∇v and ∇∇v over its 4^d stencil nodes.
#include "fft.cuh"

namespace ibdl {

template <int D>
__global__ void __launch_bounds__(256) k_boundary_vjp(int n, int M, const int* __restrict__ base,
                                                      const int* __restrict__ perm, const double* __restrict__ phi,
                                                      const double* __restrict__ dphi, const double* __restrict__ ddphi,
                                                      const double* __restrict__ wscale, double hd,
                                                      const double* __restrict__ nrm, const double* __restrict__ u,
                                                      const double* __restrict__ v, const double* __restrict__ Q,
                                                      const double* __restrict__ lam, double* __restrict__ dX,
                                                      double* __restrict__ dn, double* __restrict__ dw) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= M) return;
  const int i = perm[s];
  double p0[D][4], p1[D][4], p2[D][4];
  int node[D][4];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const int b = base[j * M + s];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      p0[j][a] = phi[(j * 4 + a) * M + s];
      p1[j][a] = dphi[(j * 4 + a) * M + s];
      p2[j][a] = ddphi[(j * 4 + a) * M + s];
      node[j][a] = (b + a) & (n - 1);
    }
  }
  double Gu[D] = {}, Gv[D] = {}, Hv[D][D] = {};
  constexpr int NN = D == 2 ? 16 : 64;
  for (int t = 0; t < NN; ++t) {
    int a[D];
    size_t idx = 0;
#pragma unroll
    for (int j = D - 1; j >= 0; --j) {
      a[j] = (t >> (2 * j)) & 3;
      idx = idx * n + node[j][a[j]];
    }
    const double ug = u[idx], vg = v[idx];
#pragma unroll
    for (int m = 0; m < D; ++m) {
      double dm = 1.0;
#pragma unroll
      for (int j = 0; j < D; ++j) dm *= j == m ? p1[j][a[j]] : p0[j][a[j]];
      Gu[m] += ug * dm;
      Gv[m] += vg * dm;
#pragma unroll
      for (int l = m; l < D; ++l) {
        double h = 1.0;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          if (l == m)
            h *= j == m ? p2[j][a[j]] : p0[j][a[j]];
          else
            h *= (j == m || j == l) ? p1[j][a[j]] : p0[j][a[j]];
        }
        Hv[m][l] += vg * h;
      }
    }
  }
  double nv[D];
#pragma unroll
  for (int m = 0; m < D; ++m) nv[m] = nrm[m * M + s];
  const double q = Q[i];
  const double wq = wscale[s] * hd * q;  // Δs_i Q_i
  const double li = lam[i];
  double ndotg = 0.0;
#pragma unroll
  for (int m = 0; m < D; ++m) {
    double hn = 0.0;
#pragma unroll
    for (int l = 0; l < D; ++l) hn += (l >= m ? Hv[m][l] : Hv[l][m]) * nv[l];
    // ∂J/∂p = −∂(λᵀAQ)/∂p
    if (dX) dX[(size_t)m * M + i] = li * Gu[m] + wq * hn;
    if (dn) dn[(size_t)m * M + i] = -wq * Gv[m];
    ndotg += nv[m] * Gv[m];
  }
  if (dw) dw[i] = -q * ndotg;
}

ibdl_status solve_vjp_impl(Geometry* g, const double* Q, const double* lam, double* dX, double* dn, double* dw,
                           cudaStream_t s) {
  if (g->pde != IBDL_PDE_SCALAR || g->dipole != IBDL_DIPOLE_ANALYTIC)
    return fail(IBDL_ERR_UNSUPPORTED, "boundary derivatives: scalar PDE with the analytic dipole only");
  if (!g->ddphi64) return fail(IBDL_ERR_UNSUPPORTED, "boundary derivatives need the second-derivative table");
  size_t cells = (size_t)g->n * g->n;
  if (g->dim == 3) cells *= g->n;
  if (!g->vjp_buf) IBDL_CUDA(cudaMalloc((void**)&g->vjp_buf, 2 * cells * sizeof(double)));
  double* u = g->vjp_buf;
  double* v = g->vjp_buf + cells;
  IBDL_TRY(g->dim == 2 ? field_pair_2d(g, Q, lam, u, v, s) : field_pair_3d(g, Q, lam, u, v, s));
  const int M = (int)g->M, tb = 128;
  const double hd = g->dim == 2 ? g->h * g->h : g->h * g->h * g->h;
  if (g->dim == 2)
    k_boundary_vjp<2><<<(M + tb - 1) / tb, tb, 0, s>>>(g->n, M, g->base, g->perm, g->t64.phi, g->t64.dphi, g->ddphi64,
                                                       g->t64.wscale, hd, g->t64.nrm, u, v, Q, lam, dX, dn, dw);
  else
    k_boundary_vjp<3><<<(M + tb - 1) / tb, tb, 0, s>>>(g->n, M, g->base, g->perm, g->t64.phi, g->t64.dphi, g->ddphi64,
                                                       g->t64.wscale, hd, g->t64.nrm, u, v, Q, lam, dX, dn, dw);
  g->launches += 1;
  IBDL_CUDA(cudaGetLastError());
  return IBDL_OK;
}

}  // namespace ibdl
