// Tile autotuner of the per-mode solve kernel (sp_autotune): times every tile
// shape (solved modes per block x threads per block) on the context's own
// workspaces and keeps the fastest for the tangent and for the FP64 step.
// The shapes differ only in how modes are grouped into blocks; each mode's
// arithmetic is the same, so the choice never changes a result.
#include <vector>

#include "sp_internal.h"

extern "C" sp_status sp_autotune(sp_ctx* c, int n_dir, sp_tune_report* rep, void* stream) {
  if (!c || n_dir < 1) return sp_fail(c, SP_EINVAL, "sp_autotune: bad arguments");
  if (c->geom != 0) return sp_fail(c, SP_EINVAL, "sp_autotune: plane Couette contexts only");
  if (n_dir > c->cfg.max_batch) return sp_fail(c, SP_EINVAL, "sp_autotune: n_dir exceeds max_batch");
  cudaStream_t st = (cudaStream_t)stream;
  int tm[SP_TUNE_MAX], th[SP_TUNE_MAX];
  const int ns = sp_solve_shapes(c, tm, th);
  sp_tune_report r{};
  r.n_shapes = ns;
  const size_t L = c->state_len;
  double* buf = nullptr;
  if (cudaMalloc((void**)&buf, 2 * (size_t)n_dir * L * 8) != cudaSuccess) {
    cudaGetLastError();
    return sp_fail(c, SP_ENOMEM, "sp_autotune: scratch allocation");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  sp_status s = SP_OK;
  auto cleanup = [&]() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
  };
  if ((s = sp_cuda(c, cudaEventCreate(&e0), "event")) != SP_OK || (s = sp_cuda(c, cudaEventCreate(&e1), "event")) != SP_OK) {
    cleanup();
    return s;
  }
  // the product workspace is scratch between calls; zero it and the scratch states
  const size_t ws3_bytes = (size_t)n_dir * 3 * c->NY * c->Mm * 16;
  if ((s = sp_cuda(c, cudaMemsetAsync(c->ws3, 0, ws3_bytes, st), "memset")) != SP_OK ||
      (s = sp_cuda(c, cudaMemsetAsync(buf, 0, 2 * (size_t)n_dir * L * 8, st), "memset")) != SP_OK) {
    cleanup();
    return s;
  }
  const bool f32 = c->cfg.prec == SP_MIXED;
  constexpr int kReps = 5;
  for (int pass = 0; pass < 2 && s == SP_OK; ++pass) {
    const bool fp32 = pass == 0 ? f32 : false;
    const int nd = pass == 0 ? n_dir : 1;
    double* ms = pass == 0 ? r.ms_tangent : r.ms_step;
    for (int i = 0; i < ns; ++i) {
      r.tile[i] = tm[i];
      r.threads[i] = th[i];
      cudaError_t e = launch_solve(c, fp32, c->ws3, buf, buf + (size_t)n_dir * L, nd, st, i);  // warm-up
      if (e == cudaErrorInvalidConfiguration) {
        cudaGetLastError();
        ms[i] = -1.0;
        continue;
      }
      if ((s = sp_cuda(c, e, "sp_autotune: solve")) != SP_OK) break;
      cudaEventRecord(e0, st);
      for (int k = 0; k < kReps && e == cudaSuccess; ++k)
        e = launch_solve(c, fp32, c->ws3, buf, buf + (size_t)n_dir * L, nd, st, i);
      cudaEventRecord(e1, st);
      if ((s = sp_cuda(c, e, "sp_autotune: solve")) != SP_OK) break;
      if ((s = sp_cuda(c, cudaEventSynchronize(e1), "sp_autotune: sync")) != SP_OK) break;
      float t = 0;
      cudaEventElapsedTime(&t, e0, e1);
      ms[i] = t / kReps;
    }
  }
  cleanup();
  if (s != SP_OK) return s;
  auto best = [&](const double* ms) {
    int b = 0;
    for (int i = 1; i < ns; ++i)
      if (ms[i] >= 0 && (ms[b] < 0 || ms[i] < ms[b])) b = i;
    return b;
  };
  r.chosen_tangent = best(r.ms_tangent);
  r.chosen_step = best(r.ms_step);
  c->solve_shape_tan = r.chosen_tangent;
  c->solve_shape_step = r.chosen_step;
  if (rep) *rep = r;
  return SP_OK;
}

extern "C" sp_status sp_set_solve_shape(sp_ctx* c, int tangent_shape, int step_shape) {
  if (!c) return SP_EINVAL;
  const int ns = sp_solve_shapes(c, nullptr, nullptr);
  if (tangent_shape < -1 || tangent_shape >= ns || step_shape < -1 || step_shape >= ns)
    return sp_fail(c, SP_EINVAL, "sp_set_solve_shape: index out of range");
  if (tangent_shape >= 0) c->solve_shape_tan = tangent_shape;
  if (step_shape >= 0) c->solve_shape_step = step_shape;
  return SP_OK;
}

extern "C" sp_status sp_set_tensor_cores(sp_ctx* c, int inverse, int forward) {
  if (!c) return SP_EINVAL;
  c->use_yinv_tc = inverse ? 1 : 0;
  c->use_rhs_tc = forward ? 1 : 0;
  return SP_OK;
}
