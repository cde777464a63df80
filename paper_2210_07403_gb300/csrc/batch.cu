// Batches of independent 2-D problems: creation, destruction and the C entry points. Every
// problem is an ordinary geometry (its own sorted tables, spectra and symbols); the batch adds
// the per-problem parameter blocks and (problem, unit) tables of the batched launches, and the
// batched GMRES state.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ibdl_internal.cuh"

struct ibdl_batch {
  ibdl::Batch* b;
};

namespace ibdl {
ibdl_status create_geometry(const ibdl_geometry_desc* d, cudaStream_t s, Geometry** out);
ibdl_status destroy_geometry(Geometry* g);

static void free_batch(Batch* B) {
  if (!B) return;
  cudaDeviceSynchronize();
  if (B->geoms) {
    for (int i = 0; i < B->count; ++i)
      if (B->geoms[i]) destroy_geometry(B->geoms[i]);
    delete[] B->geoms;
  }
  for (int p = 0; p < 3; ++p) {
    for (int m = 0; m < 2; ++m)
      if (B->rowp[p][m]) cudaFree(B->rowp[p][m]);
    if (B->colp[p]) cudaFree(B->colp[p]);
    if (B->row_units[p]) cudaFree(B->row_units[p]);
    if (B->col_units[p]) cudaFree(B->col_units[p]);
    if (p < 2 && B->exec[p]) cudaGraphExecDestroy(B->exec[p]);
  }
  void* dev[] = {B->V,      B->st,    B->ctl,  B->vec,     B->target, B->active,
                 B->d_off,  B->d_voff, B->d_nd, B->d_slice, B->tmaps};
  for (void* p : dev)
    if (p) cudaFree(p);
  if (B->host_st) cudaFreeHost(B->host_st);
  delete[] B->off;
  delete[] B->voff;
  delete B;
}

static ibdl_status check_dev(const void* p, const char* name) {
  if (!p) return fail(IBDL_ERR_INVALID_ARG, std::string(name) + " is NULL");
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return fail(IBDL_ERR_INVALID_ARG, std::string(name) + " is not a CUDA device pointer");
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return fail(IBDL_ERR_INVALID_ARG, std::string(name) + " is not a CUDA device pointer");
  return IBDL_OK;
}

}  // namespace ibdl

using namespace ibdl;

extern "C" {

ibdl_status ibdl_create_batch(const ibdl_geometry_desc* descs, int count, void* stream, ibdl_batch** out) {
  set_error("");
  if (!out) return fail(IBDL_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!descs) return fail(IBDL_ERR_INVALID_ARG, "descs is NULL");
  if (count < 1 || count > 65536) return fail(IBDL_ERR_INVALID_ARG, "count must be in [1, 65536]");
  for (int i = 0; i < count; ++i) {
    if (descs[i].dim != 2) return fail(IBDL_ERR_UNSUPPORTED, "batches hold 2-D problems only");
    if (descs[i].eta != 0) return fail(IBDL_ERR_UNSUPPORTED, "batches do not hold completed problems (eta > 0)");
    if (descs[i].pde != descs[0].pde || descs[i].dipole != descs[0].dipole)
      return fail(IBDL_ERR_INVALID_ARG, "all problems of a batch need the same pde and dipole form");
  }
  Batch* B = new Batch();
  std::memset(B, 0, sizeof(Batch));
  B->count = count;
  B->pde = descs[0].pde;
  B->dipole = descs[0].dipole;
  B->ncomp = descs[0].pde == IBDL_PDE_STOKES ? 2 : 1;
  B->geoms = new Geometry*[count]();
  {
    const char* e = getenv("IBDL_BATCH_PERSISTENT");
    B->persistent = (e && atoi(e) != 0) ? 1 : 0;
  }
  {
    // the FP32 column pass: IBDL_COL_STAGED if set, else direct until the batch autotuner chooses
    const int e = col_stage_env();
    B->col_stage_forced = e >= 0;
    B->col_stage = e > 0 ? 1 : 0;
  }
  B->off = new int64_t[count + 1];
  B->voff = new int64_t[count];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  B->off[0] = 0;
  for (int i = 0; i < count; ++i) {
    ibdl_status st = create_geometry(descs + i, s, &B->geoms[i]);
    if (st != IBDL_OK) {
      const std::string msg = "problem " + std::to_string(i) + ": " + ibdl_last_error();
      free_batch(B);
      return fail(st, msg);
    }
    B->off[i + 1] = B->off[i] + B->geoms[i]->ncomp * B->geoms[i]->M;
    B->max_log2n = std::max(B->max_log2n, __builtin_ctz(B->geoms[i]->n));
  }
  B->total = B->off[count];
  ibdl_status st = batch_prepare_2d(B);
  if (st != IBDL_OK) {
    free_batch(B);
    return st;
  }
  *out = new ibdl_batch{B};
  return IBDL_OK;
}

ibdl_status ibdl_destroy_batch(ibdl_batch* batch) {
  set_error("");
  if (!batch) return IBDL_OK;
  free_batch(batch->b);
  delete batch;
  return IBDL_OK;
}

ibdl_status ibdl_batch_sizes(const ibdl_batch* batch, int* count, int64_t* offsets, int64_t* total) {
  set_error("");
  if (!batch || !batch->b) return fail(IBDL_ERR_INVALID_ARG, "batch is NULL");
  const Batch* B = batch->b;
  if (count) *count = B->count;
  if (offsets)
    for (int i = 0; i <= B->count; ++i) offsets[i] = B->off[i];
  if (total) *total = B->total;
  return IBDL_OK;
}

ibdl_status ibdl_batch_autotune(ibdl_batch* batch, int precision_mask, void* stream) {
  set_error("");
  if (!batch || !batch->b) return fail(IBDL_ERR_INVALID_ARG, "batch is NULL");
  if (precision_mask < 1 || precision_mask > 7) return fail(IBDL_ERR_INVALID_ARG, "precision_mask must be in 1 … 7");
  Batch* B = batch->b;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* buf = nullptr;
  IBDL_CUDA(cudaMalloc((void**)&buf, sizeof(double) * 2 * B->total));
  ibdl_status st = IBDL_OK;
  if (cudaMemsetAsync(buf, 0, sizeof(double) * B->total, s) != cudaSuccess) st = fail(IBDL_ERR_CUDA, "memset");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // three knobs for the whole batch: the FFT volume per CTA of the row kernels and of the column
  // kernel (the band-major spectra make tall row bands and narrow column groups a useful pair),
  // and the row kernels' least thread count, timed on the batched application itself
  // (throughput, not one problem's latency)
  const int targets[5] = {512, 1024, 2048, 4096, 8192};
  const int floors[2] = {0, 256};
  for (int pi = 0; pi < 3 && st == IBDL_OK; ++pi) {
    if (!(precision_mask & (1 << pi))) continue;
    if (pi == 2 && B->max_log2n > 12) continue;  // float-float batches exist to 4096²
    float best = 1e30f;
    int best_t = targets[0], best_c = targets[0], best_f = 0;
    for (int ti = 0; ti < 50 && st == IBDL_OK; ++ti) {
      const int tr = targets[(ti / 2) / 5], tc = targets[(ti / 2) % 5], fl = floors[ti % 2];
      for (int i = 0; i < B->count; ++i) shape_for_target_2d(B->geoms[i], pi, tr, tc, fl);
      st = batch_prepare_2d(B);
      if (st != IBDL_OK) break;
      float ms[3];
      st = batch_apply_2d(B, slot_precision(pi), 0, buf, buf + B->total, s);
      for (int k = 0; k < 3 && st == IBDL_OK; ++k) {
        cudaEventRecord(e0, s);
        st = batch_apply_2d(B, slot_precision(pi), 0, buf, buf + B->total, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(IBDL_ERR_CUDA, "batch autotune: event synchronize");
        cudaEventElapsedTime(&ms[k], e0, e1);
      }
      if (st != IBDL_OK) break;
      std::sort(ms, ms + 3);
      if (ms[1] < best) {
        best = ms[1];
        best_t = tr;
        best_c = tc;
        best_f = fl;
      }
    }
    if (st == IBDL_OK)
      for (int i = 0; i < B->count; ++i) shape_for_target_2d(B->geoms[i], pi, best_t, best_c, best_f);
    if (st == IBDL_OK && pi == 1 && !B->col_stage_forced) {
      // FP32: the direct or the staged column pass at the chosen shapes, whichever is faster
      float t[2] = {1e30f, 1e30f};
      for (int mode = 0; mode < 2 && st == IBDL_OK; ++mode) {
        B->col_stage = mode;
        st = batch_prepare_2d(B);
        if (st != IBDL_OK) break;
        float ms[3];
        st = batch_apply_2d(B, IBDL_FP32, 0, buf, buf + B->total, s);
        for (int k = 0; k < 3 && st == IBDL_OK; ++k) {
          cudaEventRecord(e0, s);
          st = batch_apply_2d(B, IBDL_FP32, 0, buf, buf + B->total, s);
          cudaEventRecord(e1, s);
          if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(IBDL_ERR_CUDA, "batch autotune: event synchronize");
          cudaEventElapsedTime(&ms[k], e0, e1);
        }
        if (st != IBDL_OK) break;
        std::sort(ms, ms + 3);
        t[mode] = ms[1];
      }
      B->col_stage = t[1] < t[0] ? 1 : 0;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(buf);
  if (st != IBDL_OK) return st;
  // rebuild the unit tables and parameter blocks (and the captured cycles) for the chosen shapes
  for (int p = 0; p < 2; ++p)
    if (B->exec[p]) {
      cudaGraphExecDestroy(B->exec[p]);
      B->exec[p] = nullptr;
    }
  return batch_prepare_2d(B);
}

ibdl_status ibdl_batch_apply(ibdl_batch* batch, int precision, const double* Q, double* Y, void* stream) {
  set_error("");
  if (!batch || !batch->b) return fail(IBDL_ERR_INVALID_ARG, "batch is NULL");
  if (precision != IBDL_FP64 && precision != IBDL_FP32 && precision != IBDL_FP32X2)
    return fail(IBDL_ERR_INVALID_ARG, "precision must be IBDL_FP64, IBDL_FP32 or IBDL_FP32X2");
  IBDL_TRY(check_dev(Q, "Q"));
  IBDL_TRY(check_dev(Y, "Y"));
  const int64_t T = batch->b->total;
  if (Q + T > Y && Y + T > Q) return fail(IBDL_ERR_INVALID_ARG, "Q and Y overlap");
  return batch_apply_2d(batch->b, precision, 0, Q, Y, static_cast<cudaStream_t>(stream));
}

ibdl_status ibdl_batch_solve(ibdl_batch* batch, const double* Ub, double* Q, const ibdl_solve_opts* opts,
                             ibdl_solve_info* infos, void* stream) {
  set_error("");
  if (!batch || !batch->b) return fail(IBDL_ERR_INVALID_ARG, "batch is NULL");
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
  if (!Ub || !Q) return fail(IBDL_ERR_INVALID_ARG, "U_b and Q are required");
  if (!o.io_on_host) {
    IBDL_TRY(check_dev(Ub, "U_b"));
    IBDL_TRY(check_dev(Q, "Q"));
  }
  Batch* B = batch->b;
  const int64_t before = B->launches;
  ibdl_status st = batch_solve_impl(B, Ub, Q, &o, infos, static_cast<cudaStream_t>(stream));
  if (infos)
    for (int i = 0; i < B->count; ++i) infos[i].kernel_launches = B->launches - before;
  return st;
}

}  // extern "C"
