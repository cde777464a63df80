// extern "C" entry points of include/ibdl.h: argument checks, then the launchers.
#include <cstring>
#include <string>

#include "ibdl_internal.cuh"

struct ibdl_geometry {
  ibdl::Geometry* g;
};

namespace ibdl {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

ibdl_status fail(ibdl_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

ibdl_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? IBDL_ERR_NO_MEMORY : IBDL_ERR_CUDA;
}

ibdl_status create_geometry(const ibdl_geometry_desc* d, cudaStream_t s, Geometry** out);
ibdl_status destroy_geometry(Geometry* g);

// Device (or managed) memory check for caller buffers handed to kernels: a host pointer
// passed to a kernel would fault, so it is rejected here instead.
static ibdl_status check_device_ptr(const void* p, const char* name) {
  if (!p) return fail(IBDL_ERR_INVALID_ARG, std::string(name) + " is NULL");
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(IBDL_ERR_INVALID_ARG, std::string(name) + " is not a CUDA device pointer");
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return fail(IBDL_ERR_INVALID_ARG, std::string(name) + " is not a CUDA device pointer");
  return IBDL_OK;
}

static bool ranges_overlap(const void* a, const void* b, size_t bytes) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + bytes && pb < pa + bytes;
}

// [a, a + abytes) and [b, b + bbytes) intersect
static bool spans_overlap(const void* a, size_t abytes, const void* b, size_t bbytes) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + bbytes && pb < pa + abytes;
}

}  // namespace ibdl

using namespace ibdl;

extern "C" {

ibdl_status ibdl_create_geometry(const ibdl_geometry_desc* desc, void* stream, ibdl_geometry** out) {
  set_error("");
  if (!out) return fail(IBDL_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  Geometry* g = nullptr;
  ibdl_status st = create_geometry(desc, static_cast<cudaStream_t>(stream), &g);
  if (st != IBDL_OK) return st;
  *out = new ibdl_geometry{g};
  return IBDL_OK;
}

ibdl_status ibdl_destroy_geometry(ibdl_geometry* geom) {
  set_error("");
  if (!geom) return IBDL_OK;
  ibdl_status st = destroy_geometry(geom->g);
  delete geom;
  return st;
}

ibdl_status ibdl_apply(ibdl_geometry* geom, int precision, const double* Q, double* Y, void* stream) {
  set_error("");
  if (!geom || !geom->g) return fail(IBDL_ERR_INVALID_ARG, "geometry is NULL");
  if (precision != IBDL_FP64 && precision != IBDL_FP32 && precision != IBDL_FP32X2)
    return fail(IBDL_ERR_INVALID_ARG, "precision must be IBDL_FP64, IBDL_FP32 or IBDL_FP32X2");
  Geometry* g = geom->g;
  IBDL_TRY(check_device_ptr(Q, "Q"));
  IBDL_TRY(check_device_ptr(Y, "Y"));
  if (ranges_overlap(Q, Y, sizeof(double) * geom_nd(g))) return fail(IBDL_ERR_INVALID_ARG, "Q and Y overlap");
  return apply_any(g, precision, Q, Y, static_cast<cudaStream_t>(stream), nullptr);
}

ibdl_status ibdl_adjoint(ibdl_geometry* geom, int precision, const double* W, double* Z, void* stream) {
  set_error("");
  if (!geom || !geom->g) return fail(IBDL_ERR_INVALID_ARG, "geometry is NULL");
  if (geom->g->naug) return fail(IBDL_ERR_UNSUPPORTED, "ibdl_adjoint: not for the completed method (eta > 0)");
  if (precision != IBDL_FP64 && precision != IBDL_FP32) return fail(IBDL_ERR_INVALID_ARG, "precision must be IBDL_FP64 or IBDL_FP32");
  Geometry* g = geom->g;
  if (g->pde != IBDL_PDE_SCALAR) return fail(IBDL_ERR_UNSUPPORTED, "ibdl_adjoint: scalar PDE only");
  IBDL_TRY(check_device_ptr(W, "W"));
  IBDL_TRY(check_device_ptr(Z, "Z"));
  if (ranges_overlap(W, Z, sizeof(double) * g->M)) return fail(IBDL_ERR_INVALID_ARG, "W and Z overlap");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return g->dim == 2 ? adjoint_2d(g, precision, W, Z, s) : adjoint_3d(g, precision, W, Z, s);
}

void ibdl_default_solve_opts(ibdl_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->rtol = 1e-8;
  o->restart = 50;
  o->maxit = 200;
  o->precision = IBDL_FP64;
  o->inner_rtol = 1e-4;
  o->max_refine = 6;
  o->io_on_host = 0;
  o->residual = IBDL_FP32X2;
}

}  // extern "C"

namespace ibdl {

// shared argument checks and dispatch of ibdl_solve (op = A) and ibdl_solve_transpose (op = Aᵀ)
static ibdl_status solve_entry(ibdl_geometry* geom, const double* b, double* x, const ibdl_solve_opts* opts,
                               ibdl_solve_info* info, void* stream, int op, const char* bname, const char* xname,
                               const double* gsrc = nullptr) {
  set_error("");
  if (info) std::memset(info, 0, sizeof(*info));
  if (!geom || !geom->g) return fail(IBDL_ERR_INVALID_ARG, "geometry is NULL");
  ibdl_solve_opts o;
  if (opts)
    o = *opts;
  else
    ibdl_default_solve_opts(&o);
  if (!(o.rtol > 0) || !(o.rtol < 1)) return fail(IBDL_ERR_INVALID_ARG, "rtol must be in (0, 1)");
  if (o.restart < 1 || o.restart > 64) return fail(IBDL_ERR_INVALID_ARG, "restart must be in [1, 64]");
  if (o.maxit < 1) return fail(IBDL_ERR_INVALID_ARG, "maxit must be >= 1");
  if (o.precision != IBDL_FP64 && o.precision != IBDL_FP32 && o.precision != IBDL_MIXED)
    return fail(IBDL_ERR_INVALID_ARG, "unknown precision");
  if (o.precision == IBDL_MIXED && (!(o.inner_rtol > 0) || !(o.inner_rtol < 1) || o.max_refine < 1))
    return fail(IBDL_ERR_INVALID_ARG, "mixed precision needs inner_rtol in (0, 1) and max_refine >= 1");
  if (o.residual != IBDL_FP64 && o.residual != IBDL_FP32X2)
    return fail(IBDL_ERR_INVALID_ARG, "residual must be IBDL_FP64 or IBDL_FP32X2");
  if (!b || !x) return fail(IBDL_ERR_INVALID_ARG, std::string(bname) + " and " + xname + " are required");
  if (op == OPK_AT && geom->g->naug)
    return fail(IBDL_ERR_UNSUPPORTED, "ibdl_solve_transpose: not for the completed method (eta > 0)");
  if (op == OPK_AT && geom->g->pde == IBDL_PDE_STOKES && geom->g->dipole != IBDL_DIPOLE_ANALYTIC)
    return fail(IBDL_ERR_UNSUPPORTED, "ibdl_solve_transpose: Stokes with the analytic dipole only");
  if (!o.io_on_host) {
    IBDL_TRY(check_device_ptr(b, bname));
    IBDL_TRY(check_device_ptr(x, xname));
  }
  const int64_t before = geom->g->launches;
  ibdl_status st = solve_impl(geom->g, b, x, &o, info, static_cast<cudaStream_t>(stream), op, gsrc);
  if (info) info->kernel_launches = geom->g->launches - before;
  return st;
}

// Optional derivative outputs dX [d][M], dn [d][M], dw [M], dQ [c][M]: device pointers that
// overlap neither each other nor the inputs.
static ibdl_status check_outputs(const Geometry* g, double* dX, double* dn, double* dw, double* dQ,
                                 const void* const* ins, const size_t* ib, int nin, const char* in_names) {
  const size_t vb = sizeof(double) * g->M;
  double* outs[4] = {dX, dn, dw, dQ};
  const size_t ob[4] = {vb * g->dim, vb * g->dim, vb, vb * g->ncomp};
  const char* names[4] = {"dX", "dn", "dw", "dQ"};
  for (int k = 0; k < 4; ++k) {
    if (!outs[k]) continue;
    IBDL_TRY(check_device_ptr(outs[k], names[k]));
    for (int j = 0; j < nin; ++j)
      if (ins[j] && spans_overlap(outs[k], ob[k], ins[j], ib[j]))
        return fail(IBDL_ERR_INVALID_ARG, std::string(names[k]) + " overlaps " + in_names);
    for (int l = 0; l < k; ++l)
      if (outs[l] && spans_overlap(outs[k], ob[k], outs[l], ob[l]))
        return fail(IBDL_ERR_INVALID_ARG, std::string(names[k]) + " overlaps " + names[l]);
  }
  return IBDL_OK;
}

}  // namespace ibdl

extern "C" {

ibdl_status ibdl_solve(ibdl_geometry* geom, const double* Ub, double* Q, const ibdl_solve_opts* opts,
                       ibdl_solve_info* info, void* stream) {
  return solve_entry(geom, Ub, Q, opts, info, stream, OPK_A, "U_b", "Q");
}

// the source term g̃: device FP64 [c][n^dim]; NULL = none
static ibdl_status check_source(ibdl_geometry* geom, const double* g_grid) {
  if (!g_grid) return IBDL_OK;
  if (!geom || !geom->g) return fail(IBDL_ERR_INVALID_ARG, "geometry is NULL");
  return check_device_ptr(g_grid, "g_grid");
}

ibdl_status ibdl_solve_forced(ibdl_geometry* geom, const double* Ub, const double* g_grid, double* Q,
                              const ibdl_solve_opts* opts, ibdl_solve_info* info, void* stream) {
  set_error("");
  IBDL_TRY(check_source(geom, g_grid));
  return solve_entry(geom, Ub, Q, opts, info, stream, OPK_A, "U_b", "Q", g_grid);
}

ibdl_status ibdl_evaluate_field_forced(ibdl_geometry* geom, const double* Q, const double* g_grid, double* u_grid,
                                       void* stream) {
  set_error("");
  IBDL_TRY(check_source(geom, g_grid));
  if (g_grid && u_grid) {
    const Geometry* g = geom->g;
    const size_t grid_bytes = sizeof(double) * g->ncomp * (size_t)g->n * g->n * (g->dim == 3 ? g->n : 1);
    if (spans_overlap(u_grid, grid_bytes, g_grid, grid_bytes)) return fail(IBDL_ERR_INVALID_ARG, "u_grid and g_grid overlap");
  }
  IBDL_TRY(ibdl_evaluate_field(geom, Q, u_grid, stream));
  if (!g_grid) return IBDL_OK;
  return source_terms(geom->g, g_grid, nullptr, u_grid, static_cast<cudaStream_t>(stream));
}

ibdl_status ibdl_solve_transpose(ibdl_geometry* geom, const double* G, double* lambda, const ibdl_solve_opts* opts,
                                 ibdl_solve_info* info, void* stream) {
  return solve_entry(geom, G, lambda, opts, info, stream, OPK_AT, "G", "lambda");
}

ibdl_status ibdl_apply_transpose(ibdl_geometry* geom, int precision, const double* G, double* Z, void* stream) {
  set_error("");
  if (!geom || !geom->g) return fail(IBDL_ERR_INVALID_ARG, "geometry is NULL");
  if (geom->g->naug) return fail(IBDL_ERR_UNSUPPORTED, "ibdl_apply_transpose: not for the completed method (eta > 0)");
  if (precision != IBDL_FP64 && precision != IBDL_FP32 && precision != IBDL_FP32X2)
    return fail(IBDL_ERR_INVALID_ARG, "precision must be IBDL_FP64, IBDL_FP32 or IBDL_FP32X2");
  Geometry* g = geom->g;
  if (g->pde == IBDL_PDE_STOKES && g->dipole != IBDL_DIPOLE_ANALYTIC)
    return fail(IBDL_ERR_UNSUPPORTED, "ibdl_apply_transpose: Stokes with the analytic dipole only");
  IBDL_TRY(check_device_ptr(G, "G"));
  IBDL_TRY(check_device_ptr(Z, "Z"));
  if (ranges_overlap(G, Z, sizeof(double) * g->ncomp * g->M)) return fail(IBDL_ERR_INVALID_ARG, "G and Z overlap");
  return apply_any(g, precision, G, Z, static_cast<cudaStream_t>(stream), nullptr, OPK_AT);
}

ibdl_status ibdl_single_layer(ibdl_geometry* geom, int precision, const double* V, double* Z, void* stream) {
  set_error("");
  if (!geom || !geom->g) return fail(IBDL_ERR_INVALID_ARG, "geometry is NULL");
  if (geom->g->naug) return fail(IBDL_ERR_UNSUPPORTED, "ibdl_single_layer: not for the completed method (eta > 0)");
  if (precision != IBDL_FP64 && precision != IBDL_FP32) return fail(IBDL_ERR_INVALID_ARG, "precision must be IBDL_FP64 or IBDL_FP32");
  Geometry* g = geom->g;
  if (g->pde != IBDL_PDE_SCALAR || g->dim != 2) return fail(IBDL_ERR_UNSUPPORTED, "ibdl_single_layer: scalar PDE in 2-D only");
  IBDL_TRY(check_device_ptr(V, "V"));
  IBDL_TRY(check_device_ptr(Z, "Z"));
  if (ranges_overlap(V, Z, sizeof(double) * g->M)) return fail(IBDL_ERR_INVALID_ARG, "V and Z overlap");
  return single_layer_2d(g, precision, V, Z, static_cast<cudaStream_t>(stream));
}

ibdl_status ibdl_solve_vjp(ibdl_geometry* geom, const double* Q, const double* lambda, double* dX, double* dn,
                           double* dw, void* stream) {
  set_error("");
  if (!geom || !geom->g) return fail(IBDL_ERR_INVALID_ARG, "geometry is NULL");
  if (geom->g->naug) return fail(IBDL_ERR_UNSUPPORTED, "ibdl_solve_vjp: not for the completed method (eta > 0)");
  Geometry* g = geom->g;
  if (g->dipole != IBDL_DIPOLE_ANALYTIC)
    return fail(IBDL_ERR_UNSUPPORTED, "ibdl_solve_vjp: analytic dipole only");
  IBDL_TRY(check_device_ptr(Q, "Q"));
  IBDL_TRY(check_device_ptr(lambda, "lambda"));
  if (!dX && !dn && !dw) return IBDL_OK;
  const size_t cb = sizeof(double) * g->ncomp * g->M;
  const void* ins[2] = {Q, lambda};
  const size_t ib[2] = {cb, cb};
  IBDL_TRY(check_outputs(g, dX, dn, dw, nullptr, ins, ib, 2, "Q or lambda"));
  return solve_vjp_impl(g, Q, lambda, dX, dn, dw, static_cast<cudaStream_t>(stream));
}

ibdl_status ibdl_probe_evaluate(ibdl_geometry* geom, const double* P, int n_probes, const double* Q, double* U,
                                void* stream) {
  set_error("");
  if (!geom || !geom->g) return fail(IBDL_ERR_INVALID_ARG, "geometry is NULL");
  if (geom->g->naug) return fail(IBDL_ERR_UNSUPPORTED, "ibdl_probe_evaluate: not for the completed method (eta > 0)");
  Geometry* g = geom->g;
  if (g->dim != 2) return fail(IBDL_ERR_UNSUPPORTED, "ibdl_probe_evaluate: 2-D only");
  if (n_probes < 0) return fail(IBDL_ERR_INVALID_ARG, "n_probes must be >= 0");
  IBDL_TRY(check_device_ptr(Q, "Q"));
  if (n_probes > 0) {
    IBDL_TRY(check_device_ptr(P, "P"));
    IBDL_TRY(check_device_ptr(U, "U"));
    if (spans_overlap(U, sizeof(double) * g->ncomp * n_probes, Q, sizeof(double) * g->ncomp * g->M) ||
        spans_overlap(U, sizeof(double) * g->ncomp * n_probes, P, sizeof(double) * 2 * n_probes))
      return fail(IBDL_ERR_INVALID_ARG, "U overlaps Q or P");
  }
  return probe_evaluate_impl(g, P, n_probes, Q, U, static_cast<cudaStream_t>(stream));
}

ibdl_status ibdl_probe_vjp(ibdl_geometry* geom, const double* P, int n_probes, const double* Q, const double* nu,
                           double* dQ, double* dX, double* dn, double* dw, void* stream) {
  set_error("");
  if (!geom || !geom->g) return fail(IBDL_ERR_INVALID_ARG, "geometry is NULL");
  if (geom->g->naug) return fail(IBDL_ERR_UNSUPPORTED, "ibdl_probe_vjp: not for the completed method (eta > 0)");
  Geometry* g = geom->g;
  if (g->dim != 2) return fail(IBDL_ERR_UNSUPPORTED, "ibdl_probe_vjp: 2-D only");
  if (g->dipole != IBDL_DIPOLE_ANALYTIC) return fail(IBDL_ERR_UNSUPPORTED, "ibdl_probe_vjp: analytic dipole only");
  if (n_probes < 0) return fail(IBDL_ERR_INVALID_ARG, "n_probes must be >= 0");
  IBDL_TRY(check_device_ptr(Q, "Q"));
  if (n_probes > 0) {
    IBDL_TRY(check_device_ptr(P, "P"));
    IBDL_TRY(check_device_ptr(nu, "nu"));
  }
  if (!dQ && !dX && !dn && !dw) return IBDL_OK;
  const void* ins[3] = {Q, nu, P};
  const size_t ib[3] = {sizeof(double) * g->ncomp * g->M, sizeof(double) * g->ncomp * n_probes,
                        sizeof(double) * 2 * n_probes};
  IBDL_TRY(check_outputs(g, dX, dn, dw, dQ, ins, ib, n_probes > 0 ? 3 : 1, "Q, nu or P"));
  return probe_vjp_impl(g, P, n_probes, Q, nu, dQ, dX, dn, dw, static_cast<cudaStream_t>(stream));
}

ibdl_status ibdl_evaluate_field(ibdl_geometry* geom, const double* Q, double* u_grid, void* stream) {
  set_error("");
  if (!geom || !geom->g) return fail(IBDL_ERR_INVALID_ARG, "geometry is NULL");
  IBDL_TRY(check_device_ptr(Q, "Q"));
  IBDL_TRY(check_device_ptr(u_grid, "u_grid"));
  Geometry* g = geom->g;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return g->dim == 2 ? field_2d(g, Q, u_grid, s) : field_3d(g, Q, u_grid, s);
}

ibdl_status ibdl_geometry_sizes(const ibdl_geometry* geom, int* ncomp, int64_t* n_points) {
  set_error("");
  if (!geom || !geom->g) return fail(IBDL_ERR_INVALID_ARG, "geometry is NULL");
  if (ncomp) *ncomp = geom->g->ncomp;
  if (n_points) *n_points = geom->g->M;
  return IBDL_OK;
}

ibdl_status ibdl_launch_plan(const ibdl_geometry* geom, int precision, int* rows, int* cols, int* threads,
                             int* staged, int* split) {
  set_error("");
  if (!geom || !geom->g) return fail(IBDL_ERR_INVALID_ARG, "geometry is NULL");
  if (precision != IBDL_FP64 && precision != IBDL_FP32 && precision != IBDL_FP32X2)
    return fail(IBDL_ERR_INVALID_ARG, "precision must be IBDL_FP64, IBDL_FP32 or IBDL_FP32X2");
  const Geometry* g = geom->g;
  if (g->dim != 2) return fail(IBDL_ERR_UNSUPPORTED, "launch plans are reported for 2-D geometries");
  const int pi = prec_slot(precision);
  if (rows) *rows = g->rows_per_cta[pi];
  if (cols) *cols = g->cols_per_cta[pi];
  if (threads) *threads = g->threads[pi];
  if (staged) *staged = pi == 1 ? g->col_stage : 0;
  if (split) *split = g->split[pi];
  return IBDL_OK;
}

ibdl_status ibdl_autotune(ibdl_geometry* geom, int precision_mask, void* stream) {
  set_error("");
  if (!geom || !geom->g) return fail(IBDL_ERR_INVALID_ARG, "geometry is NULL");
  if (precision_mask < 1 || precision_mask > 7) return fail(IBDL_ERR_INVALID_ARG, "precision_mask must be in 1 … 7");
  Geometry* g = geom->g;
  if (g->dim != 2) return IBDL_OK;  // 3-D shapes come from the volume rule only
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t nd = (size_t)geom_nd(g);
  double* buf = nullptr;
  IBDL_CUDA(cudaMalloc((void**)&buf, sizeof(double) * 2 * nd));
  ibdl_status st = IBDL_OK;
  if (cudaMemsetAsync(buf, 0, sizeof(double) * nd, s) != cudaSuccess) st = fail(IBDL_ERR_CUDA, "memset");
  for (int pi = 0; pi < 3 && st == IBDL_OK; ++pi)
    if ((precision_mask & (1 << pi)) && !(pi == 2 && (g->n > 4096 || !g->twff)))  // float-float: to 4096²
      st = autotune_2d(g, pi, false, s, buf, buf + nd);
  cudaStreamSynchronize(s);
  cudaFree(buf);
  return st;
}

ibdl_status ibdl_set_stage_timing(ibdl_geometry* geom, int enable) {
  set_error("");
  if (!geom || !geom->g) return fail(IBDL_ERR_INVALID_ARG, "geometry is NULL");
  return set_stage_timing(geom->g, enable);
}

ibdl_status ibdl_get_stage_times(ibdl_geometry* geom, double* ms, int64_t* launches) {
  set_error("");
  if (!geom || !geom->g) return fail(IBDL_ERR_INVALID_ARG, "geometry is NULL");
  if (!ms || !launches) return fail(IBDL_ERR_INVALID_ARG, "ms and launches are required");
  return get_stage_times(geom->g, ms, launches);
}

const char* ibdl_last_error(void) { return ibdl::g_last_error.c_str(); }

}  // extern "C"

ibdl_status ibdl_indicator(ibdl_geometry* geom, double* chi, uint8_t* flags, void* stream) {
  set_error("");
  if (!geom || !geom->g) return fail(IBDL_ERR_INVALID_ARG, "geometry is NULL");
  Geometry* g = geom->g;
  IBDL_TRY(check_device_ptr(chi, "chi"));
  IBDL_TRY(check_device_ptr(flags, "flags"));
  size_t cells = (size_t)g->n * g->n;
  if (g->dim == 3) cells *= g->n;
  if (spans_overlap(chi, sizeof(double) * cells, flags, cells)) return fail(IBDL_ERR_INVALID_ARG, "chi and flags overlap");
  return indicator_impl(g, chi, flags, static_cast<cudaStream_t>(stream));
}

ibdl_status ibdl_near_boundary(ibdl_geometry* geom, const double* Ub, const double* u, const uint8_t* omega, double m1,
                               double m2, double* out, void* stream) {
  set_error("");
  if (!geom || !geom->g) return fail(IBDL_ERR_INVALID_ARG, "geometry is NULL");
  Geometry* g = geom->g;
  if (g->dim != 2) return fail(IBDL_ERR_UNSUPPORTED, "ibdl_near_boundary: 2-D only");
  if (g->M < 3) return fail(IBDL_ERR_INVALID_ARG, "ibdl_near_boundary: needs at least three boundary points");
  if (!(m1 > 0) || !(m1 < 0.5 * g->n)) return fail(IBDL_ERR_INVALID_ARG, "m1 must lie in (0, n/2)");
  if (!(m2 > 0) || !std::isfinite(m2)) return fail(IBDL_ERR_INVALID_ARG, "m2 must be positive and finite");
  IBDL_TRY(check_device_ptr(Ub, "Ub"));
  IBDL_TRY(check_device_ptr(u, "u"));
  IBDL_TRY(check_device_ptr(omega, "omega"));
  IBDL_TRY(check_device_ptr(out, "out"));
  const size_t cells = (size_t)g->n * g->n;
  const size_t ob = sizeof(double) * g->ncomp * cells;
  if (spans_overlap(out, ob, u, ob) || spans_overlap(out, ob, Ub, sizeof(double) * g->ncomp * g->M) ||
      spans_overlap(out, ob, omega, cells))
    return fail(IBDL_ERR_INVALID_ARG, "out overlaps Ub, u or omega");
  return near_boundary_impl(g, Ub, u, omega, m1, m2, out, static_cast<cudaStream_t>(stream));
}
