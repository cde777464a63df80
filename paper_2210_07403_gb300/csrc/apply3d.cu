// Three-dimensional IBDL operator, host side: launch plans, the application of each operator and
// grid arithmetic, field evaluation, adjoints and the source term. The kernels are in
// apply3d_kernels.cuh; each grid size n = 2^L is compiled in its own unit (apply3d_n*.cu) and
// reached through launch_apply_3d<T, OP, L>.
#include <cstdlib>
#include <type_traits>

#include <algorithm>

#include "apply3d_kernels.cuh"

namespace ibdl {

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
// the per-size launches (defined in apply3d_n*.cu)
IBDL_DECLARE_3D(4)
IBDL_DECLARE_3D(5)
IBDL_DECLARE_3D(6)
IBDL_DECLARE_3D(7)
IBDL_DECLARE_3D(8)

template <typename T, int OP, int L>
static ibdl_status launch3_for_size(int lg, Geometry* g, const Row3Params& rp, const Col3Params& cp, int R, int C,
                                    int Cz, bool grid, cudaStream_t s) {
  if constexpr (L > 8) {
    return fail(IBDL_ERR_UNSUPPORTED, "3-D grid size outside 16 … 256");
  } else {
    if (lg == L) return launch_apply_3d<T, OP, L>(g, rp, cp, R, C, Cz, grid, s);
    return launch3_for_size<T, OP, L + 1>(lg, g, rp, cp, R, C, Cz, grid, s);
  }
}

ibdl_status plan_3d(Geometry* g) {
  // Work units sized by FFT volume per CTA: R y-rows per row band, C kx columns per y-pass CTA,
  // Cz per z-pass CTA (which holds 2·Cz columns: ky and −ky).
  const int nf = g->nf_in > g->nf_out ? g->nf_in : g->nf_out;
  const int n = g->n;
  auto clampp2 = [](int v, int lo, int hi) { v = v < lo ? lo : (v > hi ? hi : v); int r = 1; while (r * 2 <= v) r *= 2; return r; };
  for (int pi = 0; pi < 3; ++pi) {
    const bool f32 = pi == 1;
    // FP32 CTAs take about 2048 complex elements, FP64 (and float-float, the same element size)
    // about 1024 (measured on the 128³ sphere); R ≤ n/2 keeps the wrapped band rows
    // [y0 − 3, y0 + R) distinct (no point counted twice)
    const int target = f32 ? 2048 : 1024;
    int R = clampp2(2 * (target / (n * nf)), 2, n / 2);
    int C = clampp2(target / (n * nf), 1, n / 2);
    int Cz = clampp2(target / 2 / (n * nf), 1, n / 2);
    // the column passes interleave a pass's kThreads3/(n/8) sequences across the threads of each
    // warp: fewer sequences than that leave every warp partly idle, and an FP64 warp instruction
    // costs its issue slot whatever the number of active lanes, so a y pass holds at least
    // that many columns (fields × C) and a z pass that many (fields × 2 × Cz)
    const int sp = kThreads3 / (n / 8);
    C = std::max(C, clampp2(sp / nf, 1, n / 2));
    Cz = std::max(Cz, clampp2(sp / (2 * nf), 1, n / 2));
    if (const char* e = getenv("IBDL_PLAN3_R")) R = clampp2(atoi(e), 2, n / 2);
    if (const char* e = getenv("IBDL_PLAN3_C")) C = clampp2(atoi(e), 1, n / 2);
    if (const char* e = getenv("IBDL_PLAN3_CZ")) Cz = clampp2(atoi(e), 1, n / 2);
    auto rb = [&](int r) { return f32 ? smem_rows3<float>(n, nf, r) : smem_rows3<double>(n, nf, r); };
    auto yb = [&](int c) { return f32 ? smem_y3<float>(n, nf, c) : smem_y3<double>(n, nf, c); };
    auto zb = [&](int c) { return f32 ? smem_z3<float>(n, nf, c) : smem_z3<double>(n, nf, c); };
    while (R > 2 && rb(R) > kSmemLimit3) R /= 2;
    while (C > 1 && yb(C) > kSmemLimit3) C /= 2;
    while (Cz > 1 && zb(Cz) > kSmemLimit3) Cz /= 2;
    if (rb(R) > kSmemLimit3 || yb(C) > kSmemLimit3 || zb(Cz) > kSmemLimit3) R = C = Cz = 0;
    g->rows_per_cta[pi] = R;
    g->cols_per_cta[pi] = C;
    g->zcols_per_cta[pi] = Cz;
  }
  if (g->rows_per_cta[0] == 0 && g->rows_per_cta[1] == 0)
    return fail(IBDL_ERR_UNSUPPORTED, "3-D grid too large for the shared-memory FFT");
  return IBDL_OK;
}

template <typename T, int OP>
static ibdl_status run_op3(Geometry* g, const double* in, double* out, cudaStream_t s, const int* stop, double* grid,
                           const int* idx = nullptr, int vstride = 0, int trans = 0, bool laplace = false,
                           const double* grid_in = nullptr) {
  constexpr bool is_ff = std::is_same<T, ff>::value;
  const int pi = std::is_same<T, float>::value ? 1 : (is_ff ? 2 : 0);
  const int R = g->rows_per_cta[pi], C = g->cols_per_cta[pi], Cz = g->zcols_per_cta[pi];
  if (R == 0 || C == 0 || Cz == 0)
    return fail(IBDL_ERR_UNSUPPORTED, "3-D grid too large for the shared-memory FFT at this precision");
  const int n = g->n;
  if (is_ff && !g->twff) return fail(IBDL_ERR_UNSUPPORTED, "this geometry has no float-float tables");
  // point tables: FP32 for FP32 grids, FP64 for FP64 and float-float grids
  using PT = typename Prec3<T>::PT;
  const PointTable<PT>& tb =
      *reinterpret_cast<const PointTable<PT>*>(pi == 1 ? (const void*)&g->t32 : (const void*)&g->t64);
  Row3Params rp;
  rp.n = n;
  rp.log2n = __builtin_ctz(n);
  rp.R = R;
  rp.M = (int)g->M;
  rp.cell_start = g->cell_start;
  rp.base = g->base;
  rp.perm = g->perm;
  rp.phi = tb.phi;
  rp.dphi = tb.dphi;
  rp.wscale = tb.wscale;
  rp.nrm = tb.nrm;
  rp.in = in;
  rp.out = out;
  rp.spec = g->spec;
  rp.tw = pi == 1 ? (const void*)g->tw32 : (pi == 2 ? (const void*)g->twff : (const void*)g->tw64);
  rp.stop = stop;
  rp.grid = grid;
  rp.idx = idx;
  rp.vstride = vstride;
  rp.trans = trans;
  rp.jump = g->bc == IBDL_BC_NEUMANN ? -0.5 : 0.5;
  rp.grid_in = grid_in;
  Col3Params cp;
  cp.n = n;
  cp.log2n = rp.log2n;
  cp.C = C;
  cp.lc = __builtin_ctz(C);
  cp.lam = laplace ? 0.0 : g->lambda;
  cp.scale = 1.0 / ((double)n * n * n);
  cp.lap1 = pi == 1 ? (const void*)g->lap32 : (pi == 2 ? (const void*)g->lapff : (const void*)g->lap64);
  cp.der1 = pi == 1 ? (const void*)g->der32 : (pi == 2 ? (const void*)g->derff : (const void*)g->der64);
  cp.spec = g->spec;
  cp.tw = rp.tw;
  cp.stop = stop;
  cp.nf = 1;  // (the launch sets the fields of each y pass)
  return launch3_for_size<T, OP, 4>(rp.log2n, g, rp, cp, R, C, Cz, grid != nullptr, s);
}

template <typename T>
static ibdl_status apply3_t(Geometry* g, const double* Q, double* Y, cudaStream_t s, const int* stop, double* grid,
                            const int* idx = nullptr, int vstride = 0, int op = OPK_A) {
  if (g->pde != IBDL_PDE_SCALAR) return fail(IBDL_ERR_UNSUPPORTED, "3-D: scalar PDE only");
  if (op == OPK_AT)
    return g->dipole == IBDL_DIPOLE_ANALYTIC ? run_op3<T, OP3_ADJ_AN>(g, Q, Y, s, stop, grid, idx, vstride, 1)
                                             : run_op3<T, OP3_ADJ_SD>(g, Q, Y, s, stop, grid, idx, vstride, 1);
  return g->dipole == IBDL_DIPOLE_ANALYTIC ? run_op3<T, OP3_SCALAR_AN>(g, Q, Y, s, stop, grid, idx, vstride)
                                           : run_op3<T, OP3_SCALAR_SD>(g, Q, Y, s, stop, grid, idx, vstride);
}

ibdl_status apply_3d(Geometry* g, int precision, const double* Q, double* Y, cudaStream_t s, const int* stop,
                     int op) {
  if (precision == IBDL_FP32X2) return apply3_t<ff>(g, Q, Y, s, stop, nullptr, nullptr, 0, op);
  return precision == IBDL_FP32 ? apply3_t<float>(g, Q, Y, s, stop, nullptr, nullptr, 0, op)
                                : apply3_t<double>(g, Q, Y, s, stop, nullptr, nullptr, 0, op);
}

ibdl_status apply_3d_indexed(Geometry* g, int precision, double* V, const int* idx, int nd, cudaStream_t s,
                             const int* stop, int op) {
  if (precision == IBDL_FP32X2) return apply3_t<ff>(g, V, V, s, stop, nullptr, idx, nd, op);
  return precision == IBDL_FP32 ? apply3_t<float>(g, V, V, s, stop, nullptr, idx, nd, op)
                                : apply3_t<double>(g, V, V, s, stop, nullptr, idx, nd, op);
}

// u = −L⁻¹S̃Q and v = −L⁻¹(Σ_j λ_j Φ(x − X_j)), FP64 on [n][n][n]
ibdl_status field_pair_3d(Geometry* g, const double* Q, const double* lam, double* u, double* v, cudaStream_t s) {
  IBDL_TRY(apply3_t<double>(g, Q, g->tmp_m, s, nullptr, u));
  return apply3_t<double>(g, lam, g->tmp_m, s, nullptr, v, nullptr, 0, OPK_AT);
}

// u = −Δ₀⁻¹S̃Q (mean-zero), the geometry's λ ignored
ibdl_status laplace_field_3d(Geometry* g, const double* Q, double* u, cudaStream_t s) {
  return g->dipole == IBDL_DIPOLE_ANALYTIC
             ? run_op3<double, OP3_SCALAR_AN>(g, Q, g->tmp_m, s, nullptr, u, nullptr, 0, 0, true)
             : run_op3<double, OP3_SCALAR_SD>(g, Q, g->tmp_m, s, nullptr, u, nullptr, 0, 0, true);
}

ibdl_status field_3d(Geometry* g, const double* Q, double* u, cudaStream_t s) {
  return apply3_t<double>(g, Q, g->tmp_m, s, nullptr, u);
}

namespace {

__global__ void k3_negate(const double* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = -a[i];
}

__global__ void k3_axpy(double* __restrict__ y, const double* __restrict__ x, double a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

}  // namespace

// the source term g̃ of the scalar 3-D problem: u_g = L⁻¹g̃ from −g̃ through the −L⁻¹ symbol of the
// forward op's Fourier stage; rhs[0..M) −= S*u_g (rhs may be NULL), grid += u_g (grid may be NULL)
ibdl_status source_terms_3d(Geometry* g, const double* gsrc, double* rhs, double* grid, cudaStream_t s) {
  const int64_t cells = (int64_t)g->n * g->n * g->n;
  const int M = (int)g->M;
  // −g̃ [n³] | u_g [n³] | S*u_g [M]
  if (!g->src_buf) IBDL_CUDA(cudaMalloc((void**)&g->src_buf, sizeof(double) * (2 * cells + M)));
  double* f = g->src_buf;
  double* ug = f + cells;
  double* w = ug + cells;
  const int blocks = (int)std::min<int64_t>((cells + 255) / 256, 152 * 8);
  k3_negate<<<blocks, 256, 0, s>>>(gsrc, f, cells);
  IBDL_CUDA(cudaGetLastError());
  g->launches += 1;
  if (rhs) {
    IBDL_CUDA(cudaMemsetAsync(w, 0, sizeof(double) * M, s));
    IBDL_TRY((run_op3<double, OP3_SCALAR_AN>(g, nullptr, w, s, nullptr, nullptr, nullptr, 0, 0, false, f)));
    k3_axpy<<<(M + 255) / 256, 256, 0, s>>>(rhs, w, -1.0, M);
    IBDL_CUDA(cudaGetLastError());
    g->launches += 1;
  }
  if (grid) {
    IBDL_TRY((run_op3<double, OP3_SCALAR_AN>(g, nullptr, w, s, nullptr, ug, nullptr, 0, 0, false, f)));
    k3_axpy<<<blocks, 256, 0, s>>>(grid, ug, 1.0, cells);
    IBDL_CUDA(cudaGetLastError());
    g->launches += 1;
  }
  return IBDL_OK;
}

ibdl_status adjoint_3d(Geometry* g, int precision, const double* W, double* Z, cudaStream_t s) {
  if (g->pde != IBDL_PDE_SCALAR) return fail(IBDL_ERR_UNSUPPORTED, "adjoint: scalar PDE only");
  if (precision == IBDL_FP32)
    return g->dipole == IBDL_DIPOLE_ANALYTIC ? run_op3<float, OP3_ADJ_AN>(g, W, Z, s, nullptr, nullptr)
                                             : run_op3<float, OP3_ADJ_SD>(g, W, Z, s, nullptr, nullptr);
  return g->dipole == IBDL_DIPOLE_ANALYTIC ? run_op3<double, OP3_ADJ_AN>(g, W, Z, s, nullptr, nullptr)
                                           : run_op3<double, OP3_ADJ_SD>(g, W, Z, s, nullptr, nullptr);
}

}  // namespace ibdl
