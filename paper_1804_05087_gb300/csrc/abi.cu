// The C ABI (include/stokesprec.h): context lifetime, the BEFE step, its
// tangent and finite-difference actions, inner products and seeding.
#include <chrono>
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "hookstep.h"
#include "sp_internal.h"

static thread_local std::string g_create_error;

sp_status sp_fail(sp_ctx* c, sp_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

sp_status sp_cuda(sp_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return SP_OK;
  if (c) c->err = std::string(what) + ": " + cudaGetErrorString(e);
  return SP_ECUDA;
}

static cudaEvent_t take_event(sp_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

cudaError_t sp_traced(sp_ctx* c, int stage, cudaStream_t st, cudaError_t (*fn)(void*), void* arg) {
  if (!c->trace) return fn(arg);
  cudaEvent_t e0 = take_event(c), e1 = take_event(c);
  if (!e0 || !e1) return cudaErrorMemoryAllocation;
  cudaEventRecord(e0, st);
  cudaError_t r = fn(arg);
  cudaEventRecord(e1, st);
  c->trace_ev[stage].emplace_back(e0, e1);
  return r;
}

static void trace_reset(sp_ctx* c) {
  for (auto& v : c->trace_ev) {
    for (auto& p : v) {
      c->ev_pool.push_back(p.first);
      c->ev_pool.push_back(p.second);
    }
    v.clear();
  }
}

extern "C" sp_status sp_trace_enable(sp_ctx* c, int on) {
  if (!c) return SP_EINVAL;
  trace_reset(c);
  c->trace = on != 0;
  return SP_OK;
}

extern "C" sp_status sp_trace_read(sp_ctx* c, double* ms, long long* launches, int n) {
  if (!c || n < 0 || n > SP_NSTAGE || (n > 0 && (!ms || !launches))) return sp_fail(c, SP_EINVAL, "sp_trace_read");
  for (int s = 0; s < n; ++s) {
    double acc = 0;
    for (auto& p : c->trace_ev[s]) {
      if (cudaEventSynchronize(p.second) != cudaSuccess) return sp_cuda(c, cudaGetLastError(), "trace sync");
      float t = 0;
      cudaEventElapsedTime(&t, p.first, p.second);
      acc += t;
    }
    ms[s] = acc;
    launches[s] = (long long)c->trace_ev[s].size();
  }
  return SP_OK;
}

static bool good_fft_len(int n) {
  if (n < 4 || n % 2) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

static void drop_newton_graphs(sp_ctx* c);

static void free_ctx(sp_ctx* c) {
  void* ptrs[] = {c->Th, c->TDh, c->Cfh, c->yv, c->lam6, c->Th_f, c->TDh_f, c->Cfh_f, c->twx, c->twz, c->base32t,
                  c->twx_f, c->twz_f, c->ops, c->ws6, c->ws3, c->base64, c->base32, c->U0,
                  c->G0, c->tmp, c->red, c->kry, c->wsG, c->pb_fac, c->pb_uh, c->pb_dinv, c->fd_w1, c->fd_c1, c->dzU,
                  c->traj, c->nbuf, c->traj_base, c->chain, c->Tp, c->TDp, c->tq,
                  c->Tp_f, c->TDp_f, c->tq_f, c->Cq, c->Cq_f, c->yinv_tc_mat, c->rhs_tc_mat};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->red_host) cudaFreeHost(c->red_host);
  if (c->kry_host) cudaFreeHost(c->kry_host);
  if (c->hbuf) cudaFree(c->hbuf);
  for (cudaEvent_t e : {c->hev_start, c->hev_in[0], c->hev_in[1], c->hev_comp[0], c->hev_comp[1], c->hev_out[0],
                        c->hev_out[1]})
    if (e) cudaEventDestroy(e);
  drop_newton_graphs(c);
  for (cudaEvent_t e : c->nev) cudaEventDestroy(e);
  c->nev.clear();
  if (c->nev_in) cudaEventDestroy(c->nev_in);
  if (c->nstream) cudaStreamDestroy(c->nstream);
  if (c->hs_in) cudaStreamDestroy(c->hs_in);
  if (c->hs_out) cudaStreamDestroy(c->hs_out);
  trace_reset(c);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  c->ev_pool.clear();
}

static bool alloc_workspaces(sp_ctx* c);

extern "C" sp_status sp_create(const sp_config* cfg, sp_ctx** out) {
  if (!out) return SP_EINVAL;
  *out = nullptr;
  if (!cfg) return SP_EINVAL;
  sp_ctx* c = new (std::nothrow) sp_ctx();
  if (!c) return SP_ENOMEM;
  c->cfg = *cfg;
  auto bail = [&](sp_status s, const std::string& m) {
    g_create_error = "sp_create: " + m;
    free_ctx(c);
    delete c;
    return s;
  };
  if (!good_fft_len(cfg->nx) || !good_fft_len(cfg->nz)) return bail(SP_EINVAL, "nx, nz");
  if (cfg->ny < 5 || cfg->ny % 2 == 0 || cfg->ny > 257) return bail(SP_EINVAL, "ny");
  if (!(cfg->lx > 0) || !(cfg->lz > 0) || !(cfg->re > 0) || !(cfg->dt > 0)) return bail(SP_EINVAL, "params");
  if (cfg->prec != SP_FP64 && cfg->prec != SP_MIXED) return bail(SP_EINVAL, "prec");
  if (cfg->max_batch < 1) return bail(SP_EINVAL, "max_batch");
  if (cfg->lam_adv != 0 && cfg->lam_adv != 1) return bail(SP_EINVAL, "lam_adv");
  c->nx = cfg->nx; c->ny = cfg->ny; c->nz = cfg->nz;
  c->N = cfg->ny - 1;
  c->NH = c->N / 2 + 1;
  c->Kx = (cfg->nx - 1) / 3;
  c->Kz = (cfg->nz - 1) / 3;
  c->MX = 2 * c->Kx + 1;
  c->MZ = c->Kz + 1;
  c->NY = cfg->ny;
  c->Mm = c->MX * c->MZ;
  c->n_unique = (c->Kx + 1) * c->MZ + c->Kx * (c->MZ - 1);
  c->alpha = 2.0 * M_PI / cfg->lx;
  c->beta = 2.0 * M_PI / cfg->lz;
  c->nu = 1.0 / cfg->re;
  c->dt = cfg->dt;
  c->cplx_per_state = (size_t)3 * c->Mm * c->NY;
  c->state_len = 2 * c->cplx_per_state;
  if (cudaGetDevice(&c->dev) != cudaSuccess) return bail(SP_ECUDA, "no device");
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->dev);
  if (c->sm_count <= 0) c->sm_count = 1;
  if (sp_build_plan(c) != SP_OK) return bail(SP_EINVAL, c->err);
  if (!sp_xz_fits(c)) return bail(SP_EINVAL, "grid too large for the plane kernel");
  c->field_cplx = c->cplx_per_state;
  if (!alloc_workspaces(c)) return bail(SP_ENOMEM, "workspace allocation");
  *out = c;
  return SP_OK;
}

static bool alloc_workspaces(sp_ctx* c) {
  const size_t B = (size_t)c->cfg.max_batch;
  const size_t plane6 = (size_t)6 * c->NY * c->Mm * 16, plane3 = (size_t)3 * c->NY * c->Mm * 16;
  const size_t grid = (size_t)c->NY * c->nx * c->nz;
  c->red_blocks = 2 * c->sm_count;
  bool ok = cudaMalloc(&c->ws6, B * plane6) == cudaSuccess && cudaMalloc(&c->ws3, B * plane3) == cudaSuccess &&
            cudaMalloc((void**)&c->base64, 6 * grid * 8) == cudaSuccess &&
            cudaMalloc((void**)&c->base32, 6 * grid * 4) == cudaSuccess &&
            cudaMalloc((void**)&c->base32t, 6 * grid * 4) == cudaSuccess &&
            cudaMalloc((void**)&c->U0, c->state_len * 8) == cudaSuccess &&
            cudaMalloc((void**)&c->G0, c->state_len * 8) == cudaSuccess &&
            cudaMalloc((void**)&c->tmp, B * c->state_len * 8) == cudaSuccess &&
            cudaMalloc((void**)&c->red, (size_t)64 * c->red_blocks * 8 + 4096) == cudaSuccess &&
            cudaMallocHost((void**)&c->red_host, (size_t)64 * c->red_blocks * 8 + 4096) == cudaSuccess;
  const size_t gplane = sp_xz_global_plane_bytes(c);
  if (ok && gplane) ok = cudaMalloc(&c->wsG, B * gplane) == cudaSuccess;
  if (ok && c->geom == 1) ok = cudaMalloc((void**)&c->dzU, c->state_len * 8) == cudaSuccess;
  if (!ok) cudaGetLastError();
  return ok;
}

extern "C" sp_status sp_pipe_create(const sp_pipe_config* cfg, sp_ctx** out) {
  if (!out) return SP_EINVAL;
  *out = nullptr;
  if (!cfg) return SP_EINVAL;
  sp_ctx* c = new (std::nothrow) sp_ctx();
  if (!c) return SP_ENOMEM;
  auto bail = [&](sp_status s, const std::string& m) {
    g_create_error = "sp_pipe_create: " + m;
    free_ctx(c);
    delete c;
    return s;
  };
  c->geom = 1;
  c->pcfg = *cfg;
  if (cfg->nr < 12 || cfg->nr > 512) return bail(SP_EINVAL, "nr");
  if (cfg->mt < 1 || cfg->kz < 1 || cfg->sym < 1) return bail(SP_EINVAL, "mt, kz, sym");
  if (!good_fft_len(cfg->nz) || !good_fft_len(cfg->ntheta)) return bail(SP_EINVAL, "nz, ntheta");
  if (cfg->ntheta < 3 * cfg->mt + 1 || cfg->nz < 3 * cfg->kz + 1) return bail(SP_EINVAL, "grid below the 2/3 rule");
  if (!(cfg->alpha > 0) || !(cfg->re > 0) || !(cfg->dt > 0)) return bail(SP_EINVAL, "params");
  if (cfg->prec != SP_FP64 && cfg->prec != SP_MIXED) return bail(SP_EINVAL, "prec");
  if (cfg->max_batch < 1) return bail(SP_EINVAL, "max_batch");
  // the periodic directions map onto the Couette slots: "x" = z (full), "z" = theta (half)
  c->cfg.nx = cfg->nz;
  c->cfg.nz = cfg->ntheta;
  c->cfg.ny = cfg->nr;
  c->cfg.re = cfg->re;
  c->cfg.dt = cfg->dt;
  c->cfg.prec = cfg->prec;
  c->cfg.max_batch = cfg->max_batch;
  c->cfg.lx = 2.0 * M_PI / cfg->alpha;
  c->cfg.lz = 2.0 * M_PI / cfg->sym;
  c->nx = cfg->nz; c->nz = cfg->ntheta; c->ny = cfg->nr;
  c->NY = cfg->nr;
  c->Kx = cfg->kz;
  c->Kz = cfg->mt;
  c->MX = 2 * c->Kx + 1;
  c->MZ = c->Kz + 1;
  c->Mm = c->MX * c->MZ;
  c->n_unique = (c->Kx + 1) * c->MZ + c->Kx * (c->MZ - 1);
  c->alpha = cfg->alpha;
  c->beta = cfg->sym;
  c->nu = 1.0 / cfg->re;
  c->dt = cfg->dt;
  c->field_cplx = (size_t)3 * c->Mm * c->NY;
  c->cplx_per_state = c->field_cplx + 1;
  c->state_len = 2 * c->cplx_per_state;
  if (cudaGetDevice(&c->dev) != cudaSuccess) return bail(SP_ECUDA, "no device");
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->dev);
  if (c->sm_count <= 0) c->sm_count = 1;
  if (sp_build_pipe_plan(c) != SP_OK) return bail(SP_EINVAL, c->err);
  if (!sp_xz_fits(c)) return bail(SP_EINVAL, "grid too large for the plane kernel");
  if (!alloc_workspaces(c)) return bail(SP_ENOMEM, "workspace allocation");
  *out = c;
  return SP_OK;
}

extern "C" sp_status sp_destroy(sp_ctx* c) {
  if (!c) return SP_EINVAL;
  free_ctx(c);
  delete c;
  return SP_OK;
}

extern "C" const char* sp_last_error(const sp_ctx* c) {
  if (!c) return g_create_error.c_str();  // the last failed sp_create on this thread
  return c->err.c_str();
}

extern "C" size_t sp_state_len(const sp_ctx* c) { return c ? c->state_len : 0; }

extern "C" sp_status sp_dims(const sp_ctx* c, int* kx, int* kz, int* ny) {
  if (!c) return SP_EINVAL;
  if (kx) *kx = c->Kx;
  if (kz) *kz = c->Kz;
  if (ny) *ny = c->NY;
  return SP_OK;
}

// ---------------------------------------------------------------- internals
static sp_status step_batch(sp_ctx* c, const double* U, double* G, int n, cudaStream_t st) {
  for (int d0 = 0; d0 < n; d0 += c->cfg.max_batch) {
    const int nb = std::min(c->cfg.max_batch, n - d0);
    const double* u = U + (size_t)d0 * c->state_len;
    double* g = G + (size_t)d0 * c->state_len;
    sp_status s;
    if (c->geom == 1) {
      if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_pvals(c, false, u, c->ws6, nb, st); }),
                       "pvals")) != SP_OK)
        return s;
      if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st,
                                 [&] { return launch_xz(c, false, XZ_STEP, c->ws6, c->ws3, nb, st); }),
                       "xz step")) != SP_OK)
        return s;
      if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st,
                                 [&] { return launch_psolve(c, false, false, c->ws3, u, g, nb, st); }),
                       "psolve")) != SP_OK)
        return s;
      continue;
    }
    if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_yinv(c, false, u, c->ws6, nb, st); }), "yinv")) != SP_OK) return s;
    if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_xz(c, false, XZ_STEP, c->ws6, c->ws3, nb, st); }), "xz step")) != SP_OK) return s;
    if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_solve(c, false, c->ws3, u, g, nb, st, c->solve_shape_step); }), "solve")) != SP_OK) return s;
  }
  return SP_OK;
}

static sp_status inner_many(sp_ctx* c, const double* V, int k, const double* w, double* out, cudaStream_t st) {
  const int nb = c->red_blocks;
  for (int i0 = 0; i0 < k; i0 += 64) {
    const int kk = std::min(64, k - i0);
    sp_status s = sp_cuda(c, launch_multi_inner(c, V + (size_t)i0 * c->state_len, kk, w, c->red, nb, st),
                          "inner");
    if (s != SP_OK) return s;
    s = sp_cuda(c, cudaMemcpyAsync(c->red_host, c->red, (size_t)kk * nb * 8, cudaMemcpyDeviceToHost, st),
                "inner copy");
    if (s != SP_OK) return s;
    s = sp_cuda(c, cudaStreamSynchronize(st), "inner sync");
    if (s != SP_OK) return s;
    for (int i = 0; i < kk; ++i) {
      double acc = 0.0;
      for (int b = 0; b < nb; ++b) acc += c->red_host[(size_t)i * nb + b];
      out[i0 + i] = acc;
    }
  }
  return SP_OK;
}

// ---------------------------------------------------------------- entry points
extern "C" sp_status sp_step(sp_ctx* c, const double* U, double* G, void* stream) {
  if (!c || !U || !G || U == G) return sp_fail(c, SP_EINVAL, "sp_step: bad pointers");
  return step_batch(c, U, G, 1, (cudaStream_t)stream);
}

extern "C" sp_status sp_set_base(sp_ctx* c, const double* U, void* stream) {
  if (!c || !U) return sp_fail(c, SP_EINVAL, "sp_set_base: bad pointers");
  cudaStream_t st = (cudaStream_t)stream;
  sp_status s;
  if ((s = sp_cuda(c, cudaMemcpyAsync(c->U0, U, c->state_len * 8, cudaMemcpyDeviceToDevice, st), "copy")) != SP_OK)
    return s;
  if (c->geom == 1) {
    if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_pvals(c, false, c->U0, c->ws6, 1, st); }),
                     "pvals")) != SP_OK)
      return s;
    if ((s = sp_cuda(c, launch_pipe_dz(c, c->U0, c->dzU, st), "dz")) != SP_OK) return s;
  } else {
    // one pass of curl, values and inverse transforms serves both the base fields and the
    // step's product G(U) (the same arithmetic as sp_step)
    if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_yinv(c, false, c->U0, c->ws6, 1, st); }), "yinv")) != SP_OK) return s;
    if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_xz(c, false, XZ_STEP_BASE, c->ws6, c->ws3, 1, st); }), "xz step+base")) != SP_OK) return s;
    if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_base_to_f32(c, st); }), "base f32")) != SP_OK) return s;
    if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_solve(c, false, c->ws3, c->U0, c->G0, 1, st, c->solve_shape_step); }), "solve")) != SP_OK) return s;
    c->has_base = 1;
    c->traj_n = 1;
    return SP_OK;
  }
  if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_xz(c, false, XZ_BASE, c->ws6, nullptr, 1, st); }), "xz base")) != SP_OK) return s;
  if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_base_to_f32(c, st); }), "base f32")) != SP_OK) return s;
  if ((s = step_batch(c, c->U0, c->G0, 1, st)) != SP_OK) return s;
  c->has_base = 1;
  c->traj_n = 1;
  return SP_OK;
}

// pipe: the speed slot of a tangent holds the phase condition <d/dz U, du>
static sp_status pipe_phase(sp_ctx* c, const double* du, double* out, int n_dir, cudaStream_t st) {
  const int nb = (int)std::max<size_t>(1, std::min<size_t>(c->red_blocks, (c->cplx_per_state + 1023) / 1024));
  for (int d = 0; d < n_dir; ++d) {
    double* slot = out + (size_t)d * c->state_len + 2 * c->field_cplx;
    sp_status s = sp_cuda(c, cudaMemsetAsync(slot, 0, 16, st), "phase clear");
    if (s != SP_OK) return s;
    if ((s = sp_cuda(c, launch_dev_dots(c, c->dzU, 1, du + (size_t)d * c->state_len, c->red, nb, slot, nullptr, st),
                     "phase")) != SP_OK)
      return s;
  }
  return SP_OK;
}

// The tangent's per-mode solve of one pass: the O(N) chains (k_rhs, then k_chain) on
// contexts built for large batches, else the dense per-mode operators (k_solve).
// bytes of the context's ws3 (max_batch planes of three complex fields)
static size_t ws3_bytes(const sp_ctx* c) { return (size_t)c->cfg.max_batch * 3 * c->NY * c->Mm * 16; }

sp_status sp_tangent_solve(sp_ctx* c, bool f32, void* vals, size_t vals_bytes, const double* du, double* out,
                           void* work, int nb, cudaStream_t st) {
  // the O(N) chains use vals (consumed by their right-hand-side launch) as their scratch
  if (c->use_chain && chain_scratch_bytes(c, nb) <= vals_bytes) {
    sp_status s = sp_cuda(c, traced(c, SP_STAGE_RHS, st, [&] { return launch_chain_rhs(c, f32, vals, du, work, nb, st); }),
                          "rhs");
    if (s != SP_OK) return s;
    return sp_cuda(c, traced(c, SP_STAGE_SOLVE, st, [&] { return launch_chain_solve(c, du, out, work, vals, nb, st); }),
                   "chain solve");
  }
  return sp_cuda(c, traced(c, SP_STAGE_SOLVE, st, [&] { return launch_solve(c, f32, vals, du, out, nb, st); }), "solve");
}

extern "C" sp_status sp_jvp(sp_ctx* c, const double* du, double* Jdu, int n_dir, void* stream) {
  if (!c || !du || !Jdu || n_dir < 0 || du == Jdu) return sp_fail(c, SP_EINVAL, "sp_jvp: bad arguments");
  if (!c->has_base) return sp_fail(c, SP_EINVAL, "sp_jvp: call sp_set_base first");
  cudaStream_t st = (cudaStream_t)stream;
  const bool f32 = c->cfg.prec == SP_MIXED;
  for (int d0 = 0; d0 < n_dir; d0 += c->cfg.max_batch) {
    const int nb = std::min(c->cfg.max_batch, n_dir - d0);
    const double* u = du + (size_t)d0 * c->state_len;
    double* g = Jdu + (size_t)d0 * c->state_len;
    sp_status s;
    if (c->geom == 1) {
      if ((s = sp_cuda(c, traced(c, SP_STAGE_YINV, st, [&] { return launch_pvals(c, f32, u, c->ws6, nb, st); }),
                       "pvals")) != SP_OK)
        return s;
      if ((s = sp_cuda(c, traced(c, SP_STAGE_XZ, st,
                                 [&] { return launch_xz(c, f32, XZ_TANGENT, c->ws6, c->ws3, nb, st); }),
                       "xz tangent")) != SP_OK)
        return s;
      if ((s = sp_cuda(c, traced(c, SP_STAGE_SOLVE, st,
                                 [&] { return launch_psolve(c, f32, true, c->ws3, u, g, nb, st); }),
                       "psolve")) != SP_OK)
        return s;
      if ((s = pipe_phase(c, u, g, nb, st)) != SP_OK) return s;
      continue;
    }
    if ((s = sp_cuda(c, traced(c, SP_STAGE_YINV, st, [&] { return launch_yinv(c, f32, u, c->ws6, nb, st); }), "yinv")) != SP_OK) return s;
    if ((s = sp_cuda(c, traced(c, SP_STAGE_XZ, st, [&] { return launch_xz(c, f32, XZ_TANGENT, c->ws6, c->ws3, nb, st); }), "xz tangent")) != SP_OK) return s;
    if ((s = sp_tangent_solve(c, f32, c->ws3, ws3_bytes(c), u, g, c->ws6, nb, st)) != SP_OK) return s;
  }
  return SP_OK;
}

// ---------------------------------------------------------------- host buffers
// Tangent of directions that live in host memory: chunk i is copied in on one
// stream, computed on the caller's stream and copied out on another, with two
// device slots, so the copies of neighbouring chunks overlap the computation.
static sp_status host_pipeline_setup(sp_ctx* c, int chunk) {
  if (!c->hs_in) {
    bool ok = cudaStreamCreateWithFlags(&c->hs_in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&c->hs_out, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&c->hev_start, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < 2 && ok; ++k)
      ok = cudaEventCreateWithFlags(&c->hev_in[k], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&c->hev_comp[k], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&c->hev_out[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      return sp_fail(c, SP_ECUDA, "sp_jvp_host: stream/event creation");
    }
  }
  if (c->hchunk < chunk) {
    if (c->hbuf) cudaFree(c->hbuf);
    c->hbuf = nullptr;
    c->hchunk = 0;
    if (cudaMalloc((void**)&c->hbuf, (size_t)4 * chunk * c->state_len * 8) != cudaSuccess) {
      cudaGetLastError();
      return sp_fail(c, SP_ENOMEM, "sp_jvp_host: device slots");
    }
    c->hchunk = chunk;
  }
  return SP_OK;
}

extern "C" sp_status sp_jvp_host(sp_ctx* c, const double* du, double* Jdu, int n_dir, int chunk, void* stream) {
  if (!c || !du || !Jdu || n_dir < 0 || du == Jdu) return sp_fail(c, SP_EINVAL, "sp_jvp_host: bad arguments");
  if (!c->has_base) return sp_fail(c, SP_EINVAL, "sp_jvp_host: call sp_set_base first");
  if (n_dir == 0) return SP_OK;
  // default: quarters of the batch (a chunk of 64 at 256 directions keeps the batched kernels
  // efficient, while the first copy in and the last copy out stay short)
  if (chunk <= 0) chunk = std::max(1, std::min(c->cfg.max_batch, (n_dir + 3) / 4));
  chunk = std::min(chunk, c->cfg.max_batch);
  sp_status s = host_pipeline_setup(c, chunk);
  if (s != SP_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t L = c->state_len;
  double* din[2] = {c->hbuf, c->hbuf + (size_t)c->hchunk * L};
  double* dout[2] = {c->hbuf + (size_t)2 * c->hchunk * L, c->hbuf + (size_t)3 * c->hchunk * L};
  // the copies start after the caller's earlier work on `stream`
  if ((s = sp_cuda(c, cudaEventRecord(c->hev_start, st), "event")) != SP_OK) return s;
  if ((s = sp_cuda(c, cudaStreamWaitEvent(c->hs_in, c->hev_start, 0), "wait")) != SP_OK) return s;
  if ((s = sp_cuda(c, cudaStreamWaitEvent(c->hs_out, c->hev_start, 0), "wait")) != SP_OK) return s;
  const int nchunks = (n_dir + chunk - 1) / chunk;
  for (int i = 0; i < nchunks; ++i) {
    const int k = i & 1, d0 = i * chunk, nb = std::min(chunk, n_dir - d0);
    const size_t bytes = (size_t)nb * L * 8;
    // slot k is free for input once chunk i-2 was computed, for output once it was copied out
    if (i >= 2 && (s = sp_cuda(c, cudaStreamWaitEvent(c->hs_in, c->hev_comp[k], 0), "wait")) != SP_OK) return s;
    if ((s = sp_cuda(c, cudaMemcpyAsync(din[k], du + (size_t)d0 * L, bytes, cudaMemcpyHostToDevice, c->hs_in),
                     "copy in")) != SP_OK)
      return s;
    if ((s = sp_cuda(c, cudaEventRecord(c->hev_in[k], c->hs_in), "event")) != SP_OK) return s;
    if ((s = sp_cuda(c, cudaStreamWaitEvent(st, c->hev_in[k], 0), "wait")) != SP_OK) return s;
    if (i >= 2 && (s = sp_cuda(c, cudaStreamWaitEvent(st, c->hev_out[k], 0), "wait")) != SP_OK) return s;
    if ((s = sp_jvp(c, din[k], dout[k], nb, st)) != SP_OK) return s;
    if ((s = sp_cuda(c, cudaEventRecord(c->hev_comp[k], st), "event")) != SP_OK) return s;
    if ((s = sp_cuda(c, cudaStreamWaitEvent(c->hs_out, c->hev_comp[k], 0), "wait")) != SP_OK) return s;
    if ((s = sp_cuda(c, cudaMemcpyAsync(Jdu + (size_t)d0 * L, dout[k], bytes, cudaMemcpyDeviceToHost, c->hs_out),
                     "copy out")) != SP_OK)
      return s;
    if ((s = sp_cuda(c, cudaEventRecord(c->hev_out[k], c->hs_out), "event")) != SP_OK) return s;
  }
  // the caller's stream completes after the last copy out
  for (int k = 0; k < std::min(2, nchunks); ++k)
    if ((s = sp_cuda(c, cudaStreamWaitEvent(st, c->hev_out[k], 0), "wait")) != SP_OK) return s;
  return SP_OK;
}

static sp_status vjp_impl(sp_ctx* c, const double* r, double* JTr, int n_dir, bool weighted, cudaStream_t st,
                          const char* who) {
  if (!c || !r || !JTr || n_dir < 0 || r == JTr) return sp_fail(c, SP_EINVAL, std::string(who) + ": bad arguments");
  if (c->geom != 0) return sp_fail(c, SP_EINVAL, std::string(who) + ": the adjoint is built for plane Couette only");
  if (c->cfg.lam_adv) return sp_fail(c, SP_EINVAL, std::string(who) + ": the adjoint is built for the Stokes step only");
  if (!c->has_base) return sp_fail(c, SP_EINVAL, std::string(who) + ": call sp_set_base first");
  const bool f32 = c->cfg.prec == SP_MIXED;
  for (int d0 = 0; d0 < n_dir; d0 += c->cfg.max_batch) {
    const int nb = std::min(c->cfg.max_batch, n_dir - d0);
    const double* rr = r + (size_t)d0 * c->state_len;
    double* g = JTr + (size_t)d0 * c->state_len;
    sp_status s;
    if ((s = sp_cuda(c, traced(c, SP_STAGE_SOLVE, st,
                               [&] { return launch_solve_adj(c, f32, rr, g, c->ws3, nb, weighted, st); }),
                     "solve adjoint")) != SP_OK)
      return s;
    if ((s = sp_cuda(c, traced(c, SP_STAGE_XZ, st, [&] { return launch_xz(c, f32, XZ_ADJOINT, c->ws3, c->ws6, nb, st); }),
                     "xz adjoint")) != SP_OK)
      return s;
    if ((s = sp_cuda(c, traced(c, SP_STAGE_YINV, st, [&] { return launch_yinv_adj(c, f32, c->ws6, g, nb, st); }),
                     "yinv adjoint")) != SP_OK)
      return s;
    if ((s = sp_cuda(c, traced(c, SP_STAGE_VEC, st, [&] { return launch_finish_adj(c, rr, g, nb, weighted, st); }),
                     "finish adjoint")) != SP_OK)
      return s;
  }
  return SP_OK;
}

extern "C" sp_status sp_vjp(sp_ctx* c, const double* r, double* JTr, int n_dir, void* stream) {
  return vjp_impl(c, r, JTr, n_dir, true, (cudaStream_t)stream, "sp_vjp");
}

extern "C" sp_status sp_vjp_euclid(sp_ctx* c, const double* g, double* JTg, int n_dir, void* stream) {
  return vjp_impl(c, g, JTg, n_dir, false, (cudaStream_t)stream, "sp_vjp_euclid");
}

extern "C" sp_status sp_inner(sp_ctx* c, const double* a, const double* b, int n, double* out_host, void* stream) {
  if (!c || !a || !b || !out_host || n < 0) return sp_fail(c, SP_EINVAL, "sp_inner: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  for (int i = 0; i < n; ++i) {
    sp_status s = inner_many(c, a + (size_t)i * c->state_len, 1, b + (size_t)i * c->state_len, out_host + i, st);
    if (s != SP_OK) return s;
  }
  return SP_OK;
}

// ---------------------------------------------------------------- multi-step map
// G^int = B^n - I (Eq. Gint): n BEFE steps of the context's dt. The tangent is the
// chain rule along the trajectory U_k = B^k(U): d_{k+1} = d_k + G_{U_k} d_k, so
// G^int_U du = d_n - d_0. The trajectory states are stored by sp_set_base_n; the
// total fields of each U_k are recomputed from them at every tangent step.
static sp_status ensure_buf(sp_ctx* c, double** buf, int* cap, int n, const char* what) {
  if (*cap >= n) return SP_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  if (cudaMalloc((void**)buf, (size_t)n * c->state_len * 8) != cudaSuccess) {
    cudaGetLastError();
    return sp_fail(c, SP_ENOMEM, what);
  }
  *cap = n;
  return SP_OK;
}

static sp_status step_n(sp_ctx* c, const double* U, double* G, int n, cudaStream_t st) {
  if (n == 1) return step_batch(c, U, G, 1, st);
  int cap = c->nbuf ? 2 : 0;
  sp_status s = ensure_buf(c, &c->nbuf, &cap, 2, "multi-step scratch");
  if (s != SP_OK) return s;
  double* X = c->nbuf;
  double* D = c->nbuf + c->state_len;
  const size_t L = c->state_len;
  if ((s = sp_cuda(c, cudaMemcpyAsync(X, U, L * 8, cudaMemcpyDeviceToDevice, st), "copy")) != SP_OK) return s;
  for (int k = 0; k < n; ++k) {
    if ((s = step_batch(c, X, D, 1, st)) != SP_OK) return s;
    if ((s = sp_cuda(c, launch_axpby(X, 1.0, X, 1.0, D, L, st), "axpby")) != SP_OK) return s;
  }
  return sp_cuda(c, launch_axpby(G, 1.0, X, -1.0, U, L, st), "axpby");
}

// total fields of state X on the grid (FP64 and the float copies)
static sp_status base_fields(sp_ctx* c, const double* X, cudaStream_t st) {
  sp_status s;
  if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_yinv(c, false, X, c->ws6, 1, st); }), "yinv")) != SP_OK)
    return s;
  if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_xz(c, false, XZ_BASE, c->ws6, nullptr, 1, st); }),
                   "xz base")) != SP_OK)
    return s;
  return sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_base_to_f32(c, st); }), "base f32");
}

extern "C" sp_status sp_step_n(sp_ctx* c, const double* U, double* G, int n, void* stream) {
  if (!c || !U || !G || U == G || n < 1) return sp_fail(c, SP_EINVAL, "sp_step_n: bad arguments");
  if (n > 1 && c->geom != 0) return sp_fail(c, SP_EINVAL, "sp_step_n: n > 1 needs a plane Couette context");
  return step_n(c, U, G, n, (cudaStream_t)stream);
}

// bytes of one trajectory step's base fields in the precision of the tangent
static size_t base_slot_bytes(const sp_ctx* c) {
  const size_t grid = (size_t)6 * c->NY * c->nx * c->nz;
  return c->cfg.prec == SP_MIXED ? 2 * grid * 4 : grid * 8;
}

// copy the base fields of the tangent's precision to (save = true) or from trajectory slot k
static sp_status base_slot(sp_ctx* c, int k, bool save, cudaStream_t st) {
  const size_t grid = (size_t)6 * c->NY * c->nx * c->nz;
  unsigned char* slot = c->traj_base + (size_t)k * base_slot_bytes(c);
  auto cp = [&](void* live, unsigned char* p, size_t bytes) {
    return save ? cudaMemcpyAsync(p, live, bytes, cudaMemcpyDeviceToDevice, st)
                : cudaMemcpyAsync(live, p, bytes, cudaMemcpyDeviceToDevice, st);
  };
  if (c->cfg.prec == SP_MIXED) {
    cudaError_t e = cp(c->base32, slot, grid * 4);
    if (e == cudaSuccess) e = cp(c->base32t, slot + grid * 4, grid * 4);
    return sp_cuda(c, e, "trajectory base fields");
  }
  return sp_cuda(c, cp(c->base64, slot, grid * 8), "trajectory base fields");
}

extern "C" sp_status sp_set_base_n(sp_ctx* c, const double* U, int n, void* stream) {
  if (!c || !U || n < 1) return sp_fail(c, SP_EINVAL, "sp_set_base_n: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  sp_status s;
  if (n == 1) return sp_set_base(c, U, stream);  // any geometry
  if (c->geom != 0) return sp_fail(c, SP_EINVAL, "sp_set_base_n: n > 1 needs a plane Couette context");
  if ((s = ensure_buf(c, &c->traj, &c->traj_cap, n, "trajectory allocation")) != SP_OK) return s;
  const size_t L = c->state_len;
  // base fields of every step, if they fit in a quarter of the free memory
  c->traj_base_n = 0;
  const size_t need = base_slot_bytes(c) * (size_t)n;
  if (c->traj_base_bytes < need) {
    size_t freeb = 0, totb = 0;
    if (cudaMemGetInfo(&freeb, &totb) == cudaSuccess && need <= freeb / 4) {
      if (c->traj_base) cudaFree(c->traj_base);
      c->traj_base = nullptr;
      c->traj_base_bytes = 0;
      if (cudaMalloc((void**)&c->traj_base, need) == cudaSuccess) c->traj_base_bytes = need;
      else cudaGetLastError();
    }
  }
  const bool keep = c->traj_base_bytes >= need;
  if ((s = sp_cuda(c, cudaMemcpyAsync(c->traj, U, L * 8, cudaMemcpyDeviceToDevice, st), "copy")) != SP_OK) return s;
  if ((s = sp_cuda(c, cudaMemcpyAsync(c->U0, U, L * 8, cudaMemcpyDeviceToDevice, st), "copy")) != SP_OK) return s;
  double* D = c->G0;  // step increments, then G^int(U) for the finite-difference action
  for (int k = 0; k < n; ++k) {
    const double* Xk = c->traj + (size_t)k * L;
    if (keep) {
      // one pass gives the step's product and the base fields of U_k (as in sp_set_base)
      if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_yinv(c, false, Xk, c->ws6, 1, st); }), "yinv")) != SP_OK) return s;
      if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_xz(c, false, XZ_STEP_BASE, c->ws6, c->ws3, 1, st); }), "xz step+base")) != SP_OK) return s;
      if (c->cfg.prec == SP_MIXED &&
          (s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_base_to_f32(c, st); }), "base f32")) != SP_OK)
        return s;
      if ((s = base_slot(c, k, true, st)) != SP_OK) return s;
      if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_solve(c, false, c->ws3, Xk, D, 1, st, c->solve_shape_step); }), "solve")) != SP_OK) return s;
    } else if ((s = step_batch(c, Xk, D, 1, st)) != SP_OK) {
      return s;
    }
    if (k + 1 < n &&
        (s = sp_cuda(c, launch_axpby(c->traj + (size_t)(k + 1) * L, 1.0, Xk, 1.0, D, L, st), "axpby")) != SP_OK)
      return s;
  }
  // D = U_n - U_{n-1}; G0 = U_n - U_0 = (U_{n-1} - U_0) + D
  const double* Xl = c->traj + (size_t)(n - 1) * L;
  if ((s = sp_cuda(c, launch_axpby(D, 1.0, D, 1.0, Xl, L, st), "axpby")) != SP_OK) return s;
  if ((s = sp_cuda(c, launch_axpby(D, 1.0, D, -1.0, U, L, st), "axpby")) != SP_OK) return s;
  c->traj_n = n;
  c->traj_base_n = keep ? n : 0;
  c->has_base = 0;  // the single-step base fields are overwritten along the trajectory
  return SP_OK;
}

extern "C" sp_status sp_jvp_n(sp_ctx* c, const double* du, double* Jdu, int n_dir, void* stream) {
  if (!c || !du || !Jdu || n_dir < 0 || du == Jdu) return sp_fail(c, SP_EINVAL, "sp_jvp_n: bad arguments");
  if (c->traj_n < 1) return sp_fail(c, SP_EINVAL, "sp_jvp_n: call sp_set_base_n first");
  if (c->traj_n == 1) return sp_jvp(c, du, Jdu, n_dir, stream);
  cudaStream_t st = (cudaStream_t)stream;
  const bool f32 = c->cfg.prec == SP_MIXED;
  const size_t L = c->state_len;
  sp_status s;
  for (int d0 = 0; d0 < n_dir; d0 += c->cfg.max_batch) {
    const int nb = std::min(c->cfg.max_batch, n_dir - d0);
    const double* u = du + (size_t)d0 * L;
    double* g = Jdu + (size_t)d0 * L;  // holds d_k
    if ((s = sp_cuda(c, cudaMemcpyAsync(g, u, (size_t)nb * L * 8, cudaMemcpyDeviceToDevice, st), "copy")) != SP_OK)
      return s;
    for (int k = 0; k < c->traj_n; ++k) {
      if (c->traj_base_n == c->traj_n) s = base_slot(c, k, false, st);
      else s = base_fields(c, c->traj + (size_t)k * L, st);
      if (s != SP_OK) return s;
      if ((s = sp_cuda(c, traced(c, SP_STAGE_YINV, st, [&] { return launch_yinv(c, f32, g, c->ws6, nb, st); }), "yinv")) != SP_OK)
        return s;
      if ((s = sp_cuda(c, traced(c, SP_STAGE_XZ, st, [&] { return launch_xz(c, f32, XZ_TANGENT, c->ws6, c->ws3, nb, st); }),
                       "xz tangent")) != SP_OK)
        return s;
      if ((s = sp_tangent_solve(c, f32, c->ws3, ws3_bytes(c), g, c->tmp, c->ws6, nb, st)) != SP_OK) return s;
      if ((s = sp_cuda(c, launch_axpby(g, 1.0, g, 1.0, c->tmp, (size_t)nb * L, st), "axpby")) != SP_OK) return s;
    }
    if ((s = sp_cuda(c, launch_axpby(g, 1.0, g, -1.0, u, (size_t)nb * L, st), "axpby")) != SP_OK) return s;
  }
  return SP_OK;
}

extern "C" sp_status sp_jvp_fd(sp_ctx* c, const double* du, double* Jdu, int n_dir, void* stream) {
  if (!c || !du || !Jdu || n_dir < 0 || du == Jdu) return sp_fail(c, SP_EINVAL, "sp_jvp_fd: bad arguments");
  if (!c->has_base && c->traj_n < 2) return sp_fail(c, SP_EINVAL, "sp_jvp_fd: call sp_set_base first");
  cudaStream_t st = (cudaStream_t)stream;
  double nU;
  sp_status s = inner_many(c, c->U0, 1, c->U0, &nU, st);
  if (s != SP_OK) return s;
  nU = std::sqrt(nU);
  for (int d = 0; d < n_dir; ++d) {
    const double* u = du + (size_t)d * c->state_len;
    double* g = Jdu + (size_t)d * c->state_len;
    double nd;
    if ((s = inner_many(c, u, 1, u, &nd, st)) != SP_OK) return s;
    nd = std::sqrt(nd);
    if (!(nd > 0)) {
      if ((s = sp_cuda(c, cudaMemsetAsync(g, 0, c->state_len * 8, st), "memset")) != SP_OK) return s;
      continue;
    }
    const double eps = 1e-7 * (1.0 + nU) / nd;
    if ((s = sp_cuda(c, launch_axpby(c->tmp, 1.0, c->U0, eps, u, c->state_len, st), "axpby")) != SP_OK) return s;
    if ((s = step_n(c, c->tmp, g, c->traj_n > 1 ? c->traj_n : 1, st)) != SP_OK) return s;
    if ((s = sp_cuda(c, launch_axpby(g, 1.0 / eps, g, -1.0 / eps, c->G0, c->state_len, st), "axpby")) != SP_OK)
      return s;
    if (c->geom == 1 && (s = pipe_phase(c, u, g, 1, st)) != SP_OK) return s;
  }
  return sp_cuda(c, cudaStreamSynchronize(st), "fd sync");
}

extern "C" sp_status sp_seed_state(sp_ctx* c, const double* ra, const double* rb, const double* rc, double amp,
                                   double* U, void* stream) {
  if (!c || !ra || !rb || !rc || !U) return sp_fail(c, SP_EINVAL, "sp_seed_state: bad pointers");
  if (c->geom != 0) return sp_fail(c, SP_EINVAL, "sp_seed_state: plane Couette only (pipe: sp_pipe_seed_state)");
  cudaStream_t st = (cudaStream_t)stream;
  sp_status s = sp_cuda(c, launch_seed(c, ra, rb, rc, U, st), "seed");
  if (s != SP_OK) return s;
  double n2;
  if ((s = inner_many(c, U, 1, U, &n2, st)) != SP_OK) return s;
  if (n2 > 0) {
    if ((s = sp_cuda(c, launch_scale(U, amp / std::sqrt(n2), c->state_len, st), "scale")) != SP_OK) return s;
  }
  return sp_cuda(c, cudaStreamSynchronize(st), "seed sync");
}

extern "C" sp_status sp_pipe_seed_state(sp_ctx* c, const double* streak, const double* pol, int npoly, double amp,
                                        double frac, double c0, double* U, void* stream) {
  if (!c || !streak || !pol || !U || npoly < 1 || npoly > 32) return sp_fail(c, SP_EINVAL, "sp_pipe_seed_state: bad arguments");
  if (c->geom != 1) return sp_fail(c, SP_EINVAL, "sp_pipe_seed_state: not a pipe context");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t npol = (size_t)c->Mm * npoly * 2, nst = (size_t)c->MZ;
  // device copies of the random shapes live in the tail of the ws3 workspace
  double* dstreak = reinterpret_cast<double*>(c->ws3);
  double* dpol = dstreak + ((nst + 1) / 2) * 2 + 2;  // even offset: pol is read as double2 (16-byte aligned)
  double* B = c->tmp;
  sp_status s;
  if ((s = sp_cuda(c, cudaMemcpyAsync(dstreak, streak, nst * 8, cudaMemcpyHostToDevice, st), "seed copy")) != SP_OK)
    return s;
  if ((s = sp_cuda(c, cudaMemcpyAsync(dpol, pol, npol * 8, cudaMemcpyHostToDevice, st), "seed copy")) != SP_OK) return s;
  if ((s = sp_cuda(c, launch_pipe_seed(c, dstreak, dpol, npoly, U, B, st), "pipe seed")) != SP_OK) return s;
  double na, nb2;
  if ((s = inner_many(c, U, 1, U, &na, st)) != SP_OK) return s;
  if ((s = inner_many(c, B, 1, B, &nb2, st)) != SP_OK) return s;
  const double sa = na > 0 ? amp / std::sqrt(na) : 0.0, sb = nb2 > 0 ? frac * amp / std::sqrt(nb2) : 0.0;
  if ((s = sp_cuda(c, launch_axpby(U, sa, U, sb, B, c->state_len, st), "seed combine")) != SP_OK) return s;
  const double cc[2] = {c0, 0.0};
  if ((s = sp_cuda(c, cudaMemcpyAsync(U + 2 * c->field_cplx, cc, 16, cudaMemcpyHostToDevice, st), "speed")) != SP_OK)
    return s;
  return sp_cuda(c, cudaStreamSynchronize(st), "seed sync");
}

// ================================================================= Newton
namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

// ---------------------------------------------------------------- BiCGSTAB(l)
// Newton with BiCGSTAB(l) (Sleijpen & Fokkema, 1993) for G_U du = G(U): no Krylov
// basis is kept, so no part of the work grows like K^2 (Sec. 3.6). Each outer
// iteration takes l BiCG steps (two actions each) and then minimises the residual
// over the l new directions (modified Gram-Schmidt on the small space). Without a
// Hessenberg matrix there is no hookstep: the trust region acts along the single
// direction X (step s X, s = min(1, delta/|X|)), with the predicted residual
// |G - s J X| from one more action and the hookstep's radius update.
// Short-recurrence Krylov solvers for the Newton system J x = F (Sec. 3.6: no K^2 term).
// Work vectors are states of the context; scalars live on the host.
struct ShortKrylov {
  sp_ctx* c;
  const sp_newton_opts* o;
  sp_newton_report* rep;
  cudaStream_t st;
  size_t L;
  const double* shadow = nullptr;      // caller's shadow vector(s) (device), or null
  std::vector<double>* hist = nullptr;  // |r| at every residual update, or null
  void record(double rn) const {
    if (hist) hist->push_back(rn);
  }
  sp_status dot(const double* a, const double* b, double* out) const { return inner_many(c, a, 1, b, out, st); }
  sp_status dots(const double* V, int k, const double* w, double* out) const { return inner_many(c, V, k, w, out, st); }
  sp_status axpby(double* out, double a, const double* x, double b, const double* y) const {
    return sp_cuda(c, launch_axpby(out, a, x, b, y, L, st), "axpby");
  }
  sp_status copy(double* out, const double* x) const {
    return sp_cuda(c, cudaMemcpyAsync(out, x, L * 8, cudaMemcpyDeviceToDevice, st), "copy");
  }
  sp_status zero(double* x) const { return sp_cuda(c, cudaMemsetAsync(x, 0, L * 8, st), "zero"); }
  sp_status act(const double* in, double* out) const {
    rep->total_jvps++;
    return o->use_fd ? sp_jvp_fd(c, in, out, 1, st) : sp_jvp(c, in, out, 1, st);
  }
};

static int bicgstab_ell(const sp_newton_opts* o) { return std::max(1, std::min(8, o->ell > 0 ? o->ell : 2)); }
static int idr_s(const sp_newton_opts* o) { return std::max(1, std::min(8, o->ell > 0 ? o->ell : 4)); }

// BiCGSTAB(ell) (Sleijpen and Fokkema): ell BiCG steps, then a minimal-residual polynomial of
// degree ell. W: 2 (ell + 1) + 1 vectors. Solves J X = F from X = 0 to |r| <= eta |F|.
static sp_status bicgstab_solve(const ShortKrylov& k, double* W, const double* F, double nF, double* X, double* Xb) {
  const int ell = bicgstab_ell(k.o);
  const size_t L = k.L;
  double* R = W;                                   // r_0 .. r_l
  double* Uv = W + (size_t)(ell + 1) * L;          // u_0 .. u_l
  double* Rt = W + (size_t)2 * (ell + 1) * L;      // shadow residual
  auto r = [&](int i) { return R + (size_t)i * L; };
  auto u = [&](int i) { return Uv + (size_t)i * L; };
  const int max_act = std::max(2, k.o->max_krylov);
  sp_status s;
  std::vector<double> tau((size_t)(ell + 1) * (ell + 1)), sigma(ell + 1), gp(ell + 1), g(ell + 1), gpp(ell + 1);
  if ((s = k.copy(r(0), F)) != SP_OK || (s = k.copy(Rt, k.shadow ? k.shadow : F)) != SP_OK ||
      (s = k.zero(u(0))) != SP_OK || (s = k.zero(X)) != SP_OK)
    return s;
  double rho0 = 1.0, alpha = 0.0, omega = 1.0, rn = nF, best = nF;
  k.record(nF);
  if ((s = k.zero(Xb)) != SP_OK) return s;
  int acts = 0;
  bool broke = false;
  while (acts < max_act && rn > k.o->eta * nF && !broke) {
    rho0 = -omega * rho0;
    for (int j = 0; j < ell && !broke; ++j) {
      double rho1;
      if ((s = k.dot(Rt, r(j), &rho1)) != SP_OK) return s;
      if (rho0 == 0.0 || !std::isfinite(rho1)) { broke = true; break; }
      const double beta = alpha * rho1 / rho0;
      rho0 = rho1;
      for (int i = 0; i <= j; ++i)
        if ((s = k.axpby(u(i), 1.0, r(i), -beta, u(i))) != SP_OK) return s;
      if ((s = k.act(u(j), u(j + 1))) != SP_OK) return s;
      double gam;
      if ((s = k.dot(Rt, u(j + 1), &gam)) != SP_OK) return s;
      if (gam == 0.0 || !std::isfinite(gam)) { broke = true; break; }
      alpha = rho0 / gam;
      for (int i = 0; i <= j; ++i)
        if ((s = k.axpby(r(i), 1.0, r(i), -alpha, u(i + 1))) != SP_OK) return s;
      if ((s = k.act(r(j), r(j + 1))) != SP_OK) return s;
      if ((s = k.axpby(X, 1.0, X, alpha, u(0))) != SP_OK) return s;
      acts += 2;
    }
    if (broke) break;
    // minimal residual over r_1 .. r_l
    for (int j = 1; j <= ell; ++j) {
      for (int i = 1; i < j; ++i) {
        double t;
        if ((s = k.dot(r(j), r(i), &t)) != SP_OK) return s;
        tau[(size_t)i * (ell + 1) + j] = t / sigma[i];
        if ((s = k.axpby(r(j), 1.0, r(j), -tau[(size_t)i * (ell + 1) + j], r(i))) != SP_OK) return s;
      }
      if ((s = k.dot(r(j), r(j), &sigma[j])) != SP_OK) return s;
      double t0r;
      if ((s = k.dot(r(0), r(j), &t0r)) != SP_OK) return s;
      if (!(sigma[j] > 0.0)) { broke = true; break; }
      gp[j] = t0r / sigma[j];
    }
    if (broke) break;
    g[ell] = gp[ell];
    omega = g[ell];
    for (int j = ell - 1; j >= 1; --j) {
      double acc = gp[j];
      for (int i = j + 1; i <= ell; ++i) acc -= tau[(size_t)j * (ell + 1) + i] * g[i];
      g[j] = acc;
    }
    for (int j = 1; j < ell; ++j) {
      double acc = g[j + 1];
      for (int i = j + 1; i < ell; ++i) acc += tau[(size_t)j * (ell + 1) + i] * g[i + 1];
      gpp[j] = acc;
    }
    if ((s = k.axpby(X, 1.0, X, g[1], r(0))) != SP_OK) return s;
    if ((s = k.axpby(r(0), 1.0, r(0), -gp[ell], r(ell))) != SP_OK) return s;
    if ((s = k.axpby(u(0), 1.0, u(0), -g[ell], u(ell))) != SP_OK) return s;
    for (int j = 1; j < ell; ++j) {
      if ((s = k.axpby(u(0), 1.0, u(0), -g[j], u(j))) != SP_OK) return s;
      if ((s = k.axpby(X, 1.0, X, gpp[j], r(j))) != SP_OK) return s;
      if ((s = k.axpby(r(0), 1.0, r(0), -gp[j], r(j))) != SP_OK) return s;
    }
    if ((s = k.dot(r(0), r(0), &rn)) != SP_OK) return s;
    rn = std::sqrt(rn);
    k.record(rn);
    if (!std::isfinite(rn) || omega == 0.0) broke = true;
    if (std::isfinite(rn) && rn < best) {
      best = rn;
      if ((s = k.copy(Xb, X)) != SP_OK) return s;
    }
  }
  // a broken, stagnating or diverging recurrence hands back its best iterate
  if ((broke || !(std::isfinite(rn) && rn <= best)) && best < nF) return k.copy(X, Xb);
  return SP_OK;
}

// IDR(s) with biorthogonalised bases (van Gijzen and Sonneveld's variant): each cycle
// builds s directions U_k (G_k = J U_k) whose residual updates keep r orthogonal to the
// shadow space P, then one minimal-residual step (omega, with the 0.7 safeguard).
// W: 3 s + 3 vectors; P (s orthonormal seeded vectors) is built once per solve.
static sp_status idr_solve(const ShortKrylov& k, double* W, const double* F, double nF, double* X, double* Xb) {
  const int sdim = idr_s(k.o);
  const size_t L = k.L;
  double* P = W;
  double* G = W + (size_t)sdim * L;
  double* Us = W + (size_t)2 * sdim * L;
  double* r = W + (size_t)3 * sdim * L;
  double* v = r + L;
  double* t = v + L;
  auto pv = [&](int i) { return P + (size_t)i * L; };
  auto gv = [&](int i) { return G + (size_t)i * L; };
  auto uv = [&](int i) { return Us + (size_t)i * L; };
  const int max_act = std::max(2, k.o->max_krylov);
  sp_status s;
  // shadow space: the caller's s vectors as given, else seeded normal vectors
  // orthonormalised by modified Gram-Schmidt
  if (k.shadow) {
    if ((s = k.copy(P, k.shadow)) != SP_OK) return s;
    for (int i = 1; i < sdim; ++i)
      if ((s = k.copy(pv(i), k.shadow + (size_t)i * L)) != SP_OK) return s;
  } else {
    std::vector<double> h((size_t)sdim * L);
    uint64_t z = 0x9E3779B97F4A7C15ull;
    for (size_t i = 0; i < h.size(); ++i) {  // splitmix64 + Box-Muller
      auto next = [&]() {
        z += 0x9E3779B97F4A7C15ull;
        uint64_t x = z;
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        x ^= x >> 31;
        return ((x >> 11) + 0.5) * (1.0 / 9007199254740992.0);
      };
      const double u1 = next(), u2 = next();
      h[i] = std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
    }
    if ((s = sp_cuda(k.c, cudaMemcpyAsync(P, h.data(), h.size() * 8, cudaMemcpyHostToDevice, k.st), "P")) != SP_OK)
      return s;
    if ((s = sp_cuda(k.c, cudaStreamSynchronize(k.st), "P sync")) != SP_OK) return s;
    for (int i = 0; i < sdim; ++i) {
      for (int j = 0; j < i; ++j) {
        double d;
        if ((s = k.dot(pv(j), pv(i), &d)) != SP_OK || (s = k.axpby(pv(i), 1.0, pv(i), -d, pv(j))) != SP_OK)
          return s;
      }
      double n2;
      if ((s = k.dot(pv(i), pv(i), &n2)) != SP_OK) return s;
      if (!(n2 > 0.0)) return sp_fail(k.c, SP_ENAN, "IDR: degenerate shadow space");
      if ((s = k.axpby(pv(i), 1.0 / std::sqrt(n2), pv(i), 0.0, nullptr)) != SP_OK) return s;
    }
  }
  if ((s = k.copy(r, F)) != SP_OK || (s = k.zero(X)) != SP_OK) return s;
  for (int i = 0; i < sdim; ++i)
    if ((s = k.zero(gv(i))) != SP_OK || (s = k.zero(uv(i))) != SP_OK) return s;
  std::vector<double> M((size_t)sdim * sdim, 0.0), f(sdim), cc(sdim), col(sdim);
  for (int i = 0; i < sdim; ++i) M[(size_t)i * sdim + i] = 1.0;
  double om = 1.0, rn = nF, best = nF;
  k.record(nF);
  if ((s = k.zero(Xb)) != SP_OK) return s;
  auto keep_best = [&]() -> sp_status {
    if (std::isfinite(rn) && rn < best) {
      best = rn;
      return k.copy(Xb, X);
    }
    return SP_OK;
  };
  int acts = 0;
  bool broke = false;
  while (acts < max_act && rn > k.o->eta * nF && !broke) {
    if ((s = k.dots(P, sdim, r, f.data())) != SP_OK) return s;
    for (int kk = 0; kk < sdim && !broke; ++kk) {
      // M(kk:s, kk:s) c = f(kk:s), lower triangular
      for (int i = kk; i < sdim; ++i) {
        double acc = f[i];
        for (int j = kk; j < i; ++j) acc -= M[(size_t)i * sdim + j] * cc[j];
        cc[i] = acc / M[(size_t)i * sdim + i];
      }
      // v = r - G(:, kk:s) c;  U_kk = om v + U(:, kk:s) c
      if ((s = k.copy(v, r)) != SP_OK) return s;
      for (int i = kk; i < sdim; ++i)
        if ((s = k.axpby(v, 1.0, v, -cc[i], gv(i))) != SP_OK) return s;
      if ((s = k.axpby(t, om, v, cc[kk], uv(kk))) != SP_OK) return s;
      for (int i = kk + 1; i < sdim; ++i)
        if ((s = k.axpby(t, 1.0, t, cc[i], uv(i))) != SP_OK) return s;
      if ((s = k.copy(uv(kk), t)) != SP_OK) return s;
      if ((s = k.act(uv(kk), gv(kk))) != SP_OK) return s;
      ++acts;
      // biorthogonalise: P_i . G_kk = 0 for i < kk
      for (int i = 0; i < kk; ++i) {
        double d;
        if ((s = k.dot(pv(i), gv(kk), &d)) != SP_OK) return s;
        const double alpha = d / M[(size_t)i * sdim + i];
        if ((s = k.axpby(gv(kk), 1.0, gv(kk), -alpha, gv(i))) != SP_OK) return s;
        if ((s = k.axpby(uv(kk), 1.0, uv(kk), -alpha, uv(i))) != SP_OK) return s;
      }
      if ((s = k.dots(pv(kk), sdim - kk, gv(kk), col.data())) != SP_OK) return s;
      for (int i = kk; i < sdim; ++i) M[(size_t)i * sdim + kk] = col[i - kk];
      const double mkk = M[(size_t)kk * sdim + kk];
      if (mkk == 0.0 || !std::isfinite(mkk)) { broke = true; break; }
      const double beta = f[kk] / mkk;
      if ((s = k.axpby(r, 1.0, r, -beta, gv(kk))) != SP_OK) return s;
      if ((s = k.axpby(X, 1.0, X, beta, uv(kk))) != SP_OK) return s;
      if ((s = k.dot(r, r, &rn)) != SP_OK) return s;
      rn = std::sqrt(rn);
      k.record(rn);
      if (!std::isfinite(rn)) { broke = true; break; }
      if ((s = keep_best()) != SP_OK) return s;
      if (rn <= k.o->eta * nF || acts >= max_act) break;
      for (int i = kk + 1; i < sdim; ++i) f[i] -= beta * M[(size_t)i * sdim + kk];
    }
    if (broke || rn <= k.o->eta * nF || acts >= max_act) break;
    // dimension reduction: t = J r, om minimises |r - om t| (kept away from 0)
    if ((s = k.act(r, t)) != SP_OK) return s;
    ++acts;
    double tt, tr;
    if ((s = k.dot(t, t, &tt)) != SP_OK || (s = k.dot(t, r, &tr)) != SP_OK) return s;
    if (!(tt > 0.0) || !std::isfinite(tr)) break;
    om = tr / tt;
    const double rho = std::fabs(tr) / (std::sqrt(tt) * rn);
    if (rho < 0.7) om *= 0.7 / rho;
    if (om == 0.0 || !std::isfinite(om)) break;
    if ((s = k.axpby(X, 1.0, X, om, r)) != SP_OK) return s;
    if ((s = k.axpby(r, 1.0, r, -om, t)) != SP_OK) return s;
    if ((s = k.dot(r, r, &rn)) != SP_OK) return s;
    rn = std::sqrt(rn);
    k.record(rn);
    if (!std::isfinite(rn)) break;
    if ((s = keep_best()) != SP_OK) return s;
  }
  // a broken, stagnating or diverging recurrence hands back its best iterate
  if ((broke || !(std::isfinite(rn) && rn <= best)) && best < nF) return k.copy(X, Xb);
  return SP_OK;
}

// Newton with a short-recurrence linear solver (krylov = 1: BiCGSTAB(ell), 2: IDR(s)) and a
// trust region along the computed direction X (the hookstep's radius update): the step
// s X with s = min(1, delta/|X|), its predicted residual |F - s J X| from one more action.
static void drop_newton_graphs(sp_ctx* c);

// work vectors of the short-recurrence solvers: the solver's own plus five
static sp_status short_vectors(sp_ctx* c, const sp_newton_opts* o, int* nsolve) {
  *nsolve = o->krylov == 2 ? 3 * idr_s(o) + 3 : 2 * (bicgstab_ell(o) + 1) + 1;
  const int nvec = *nsolve + 5;
  if (c->kry_cap < nvec) {
    drop_newton_graphs(c);  // they hold pointers into the old basis
    if (c->kry) cudaFree(c->kry);
    if (c->kry_host) cudaFreeHost(c->kry_host);
    c->kry = nullptr;
    c->kry_host = nullptr;  // no GMRES scratch in this allocation: sp_newton_gmres reallocates
    c->kry_cap = 0;
    if (cudaMalloc((void**)&c->kry, (size_t)nvec * c->state_len * 8) != cudaSuccess) {
      cudaGetLastError();
      return sp_fail(c, SP_ENOMEM, "short-recurrence Krylov vectors");
    }
    c->kry_cap = nvec;
  }
  return SP_OK;
}

static sp_status newton_short(sp_ctx* c, double* U, const sp_newton_opts* o, sp_newton_report* rep, cudaStream_t st) {
  const size_t L = c->state_len;
  int nsolve;
  sp_status sv = short_vectors(c, o, &nsolve);
  if (sv != SP_OK) return sv;
  double* W = c->kry;
  double* X = c->kry + (size_t)nsolve * L;  // the Newton correction
  double* F = X + L;                        // G(U)
  double* Ut = F + L;                       // trial state
  double* JX = Ut + L;                      // J X
  double* Xb = JX + L;                      // best iterate of the linear solve
  const ShortKrylov k{c, o, rep, st, L};
  const double t0 = now_ms();
  sp_status s;
  if ((s = step_batch(c, U, F, 1, st)) != SP_OK) return s;
  rep->total_steps++;
  double nF;
  if ((s = k.dot(F, F, &nF)) != SP_OK) return s;
  nF = std::sqrt(nF);
  rep->norm_F0 = nF;
  double nU;
  if ((s = k.dot(U, U, &nU)) != SP_OK) return s;
  double delta = o->delta0 > 0 ? o->delta0 : 0.1 * std::max(std::sqrt(nU), 1.0);
  sp_status result = SP_ENOTCONV;
  for (int it = 0; it <= o->max_newton; ++it) {
    if (!std::isfinite(nF)) { result = SP_ENAN; break; }
    if (nF < o->tol) { result = SP_OK; break; }
    if (it == o->max_newton) break;
    if ((s = sp_set_base(c, U, st)) != SP_OK) return s;
    rep->total_steps++;
    s = o->krylov == 2 ? idr_solve(k, W, F, nF, X, Xb) : bicgstab_solve(k, W, F, nF, X, Xb);
    if (s != SP_OK) return s;
    if ((s = k.act(X, JX)) != SP_OK) return s;
    double xx, fj, jj;
    if ((s = k.dot(X, X, &xx)) != SP_OK || (s = k.dot(F, JX, &fj)) != SP_OK || (s = k.dot(JX, JX, &jj)) != SP_OK)
      return s;
    const double nX = std::sqrt(xx);
    rep->newton_len = nX;
    bool accepted = false;
    double nT = nF;
    for (int trial = 0; trial < 12 && nX > 0 && std::isfinite(nX); ++trial) {
      rep->hook_trials++;
      const double sc = std::min(1.0, delta / nX);
      const double pred = std::sqrt(std::max(0.0, nF * nF - 2.0 * sc * fj + sc * sc * jj));
      if ((s = k.axpby(Ut, 1.0, U, -sc, X)) != SP_OK) return s;
      if ((s = step_batch(c, Ut, F, 1, st)) != SP_OK) return s;
      rep->total_steps++;
      if ((s = k.dot(F, F, &nT)) != SP_OK) return s;
      nT = std::sqrt(nT);
      if (trust_update(nF, pred, nT, sc * nX, &delta)) {
        accepted = true;
        break;
      }
    }
    if (!accepted) {
      if ((s = step_batch(c, U, F, 1, st)) != SP_OK) return s;
      break;
    }
    if ((s = k.copy(U, Ut)) != SP_OK) return s;
    nF = nT;
    rep->newton_iters++;
  }
  if ((s = sp_cuda(c, cudaStreamSynchronize(st), "newton sync")) != SP_OK) return s;
  rep->norm_F = nF;
  rep->delta = delta;
  rep->lin_rel = -1.0;
  rep->t_total_ms = now_ms() - t0;
  rep->t_action_ms = -1.0;  // not split for the short-recurrence solvers
  if (result == SP_ENOTCONV) c->err = "Newton did not reach the tolerance";
  return result;
}

static void drop_newton_graphs(sp_ctx* c) {
  for (auto& kv : c->ngraphs) cudaGraphExecDestroy(kv.second);
  c->ngraphs.clear();
}

extern "C" sp_status sp_krylov_solve(sp_ctx* c, const double* F, double* X, int krylov, int param, int max_act,
                                     double eta, const double* shadow, double* hist, int max_hist, int* n_hist,
                                     int* n_act, void* stream) {
  if (!c || !F || !X || (krylov != 1 && krylov != 2) || max_act < 1 || !(eta >= 0.0) || max_hist < 0 ||
      (max_hist > 0 && !hist))
    return sp_fail(c, SP_EINVAL, "sp_krylov_solve: bad arguments");
  if (param < 1 || param > 8) return sp_fail(c, SP_EINVAL, "sp_krylov_solve: l or s must be in 1..8");
  if (!c->has_base) return sp_fail(c, SP_EINVAL, "sp_krylov_solve: no linearisation point (sp_set_base)");
  if (F == X) return sp_fail(c, SP_EINVAL, "sp_krylov_solve: F and X must not alias");
  sp_newton_opts o{};
  o.krylov = krylov;
  o.ell = param;
  o.max_krylov = max_act;
  o.eta = eta;
  int nsolve;
  sp_status s = short_vectors(c, &o, &nsolve);
  if (s != SP_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t L = c->state_len;
  double* W = c->kry;
  double* Xd = c->kry + (size_t)nsolve * L;
  double* Xb = Xd + L;
  sp_newton_report rep{};
  std::vector<double> h;
  ShortKrylov k{c, &o, &rep, st, L};
  k.shadow = shadow;
  k.hist = &h;
  if ((s = sp_cuda(c, cudaStreamSynchronize(st), "krylov sync")) != SP_OK) return s;
  double nF;
  if ((s = k.dot(F, F, &nF)) != SP_OK) return s;
  nF = std::sqrt(nF);
  s = krylov == 2 ? idr_solve(k, W, F, nF, Xd, Xb) : bicgstab_solve(k, W, F, nF, Xd, Xb);
  if (s != SP_OK) return s;
  if ((s = k.copy(X, Xd)) != SP_OK) return s;
  if ((s = sp_cuda(c, cudaStreamSynchronize(st), "krylov sync")) != SP_OK) return s;
  const int nh = (int)std::min<size_t>(h.size(), (size_t)max_hist);
  for (int i = 0; i < nh; ++i) hist[i] = h[i];
  if (n_hist) *n_hist = (int)h.size();
  if (n_act) *n_act = rep.total_jvps;
  return SP_OK;
}

extern "C" sp_status sp_newton_gmres(sp_ctx* c, double* U, const sp_newton_opts* o, sp_newton_report* rep,
                                     void* stream) {
  if (!c || !U || !o) return sp_fail(c, SP_EINVAL, "sp_newton_gmres: bad arguments");
  if (o->use_gradient && c->geom != 0)
    return sp_fail(c, SP_EINVAL, "sp_newton_gmres: use_gradient needs the adjoint (plane Couette only)");
  if (o->use_gradient && c->cfg.lam_adv)
    return sp_fail(c, SP_EINVAL, "sp_newton_gmres: use_gradient needs the adjoint of the Stokes step (lam_adv = 0)");
  if (o->krylov < 0 || o->krylov > 2) return sp_fail(c, SP_EINVAL, "sp_newton_gmres: krylov must be 0, 1 or 2");
  if (o->krylov != 0) {
    if (o->use_gradient || o->int_steps > 1)
      return sp_fail(c, SP_EINVAL, "sp_newton_gmres: BiCGSTAB(l) and IDR(s) take single-step actions without use_gradient");
    sp_newton_report rr{};
    sp_status s2 = newton_short(c, U, o, &rr, (cudaStream_t)stream);
    if (rep) *rep = rr;
    return s2;
  }
  const int ns = o->int_steps > 1 ? o->int_steps : 1;  // 1: G^Stokes; > 1: G^int = B^ns - I
  if (ns > 1 && (c->geom != 0 || o->use_gradient))
    return sp_fail(c, SP_EINVAL, "sp_newton_gmres: int_steps > 1 needs a plane Couette context, no use_gradient");
  const int K = o->max_krylov;
  if (K < 1 || K > 4096 || o->max_newton < 0) return sp_fail(c, SP_EINVAL, "sp_newton_gmres: bad options");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t L = c->state_len;
  // one partial sum per ~1024 complex values, at most red_blocks
  const int nb = (int)std::max<size_t>(1, std::min<size_t>(c->red_blocks, (c->cplx_per_state + 1023) / 1024));
  // device scratch after the basis: partials, hA, hB, hn/inv
  const size_t extra = (size_t)(K + 2) * nb + 3 * (size_t)(K + 3) + 24 + (size_t)orth_small_blocks(c);
  if (c->kry_cap < K + 5 || !c->kry_host) {
    drop_newton_graphs(c);  // they hold pointers into the old basis
    if (c->kry) cudaFree(c->kry);
    if (c->kry_host) cudaFreeHost(c->kry_host);
    c->kry = nullptr;
    c->kry_host = nullptr;
    c->kry_cap = 0;
    if (cudaMalloc((void**)&c->kry, ((size_t)(K + 5) * L + extra) * 8) != cudaSuccess ||
        cudaMallocHost((void**)&c->kry_host, ((size_t)4 * (K + 3) + 4) * 8) != cudaSuccess) {
      cudaGetLastError();
      return sp_fail(c, SP_ENOMEM, "Krylov basis allocation");
    }
    c->kry_cap = K + 5;
  }
  // the layout follows the capacity, so captured graphs stay valid for smaller K
  const int Kc = c->kry_cap - 5;
  double* V = c->kry;                            // Kc+2 basis vectors
  double* F = c->kry + (size_t)(Kc + 2) * L;     // residual
  double* Ut = c->kry + (size_t)(Kc + 3) * L;    // trial state
  double* Zg = c->kry + (size_t)(Kc + 4) * L;    // gradient direction (use_gradient)
  double* dpart = c->kry + (size_t)(Kc + 5) * L; // partial sums
  double* dhA = dpart + (size_t)(Kc + 2) * nb;   // first Gram-Schmidt pass
  double* dhB = dhA + (Kc + 3);                  // second pass
  double* dhn = dhB + (Kc + 3);                  // [0] = |w|, [1] = 1/|w|, then y
  double* dwn = dhn + (Kc + 6);                  // |w| before the first pass, scratch
  int* dflag = reinterpret_cast<int*>(dwn + 4);  // second Gram-Schmidt pass needed
  double* dnorm = dwn + 8;                         // partial norms of the small-state column
  // pinned: two copies of hA | hB | hn, column j in copy j mod 2, so that the host reads column j
  // while column j + 1 is computed
  // (a buffer of its own: the actions of column j + 1 may use the context's reduction buffer)
  const size_t hstride = (size_t)2 * (Kc + 3) + 2;
  double* hbuf = c->kry_host;
  // CUDA graphs of the Arnoldi steps: tangent actions only, on the context's own stream
  bool graphs = o->use_graphs && !o->use_fd && ns == 1 && !c->trace;
  if (graphs && !c->nstream) {
    if (cudaStreamCreateWithFlags(&c->nstream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->nev_in, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      graphs = false;
    }
  }
  if (graphs) {  // the private stream starts after the caller's earlier work
    cudaEventRecord(c->nev_in, st);
    cudaStreamWaitEvent(c->nstream, c->nev_in, 0);
    st = c->nstream;
  }
  while ((int)c->nev.size() < 3 * (Kc + 2)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return sp_fail(c, SP_ECUDA, "events");
    c->nev.push_back(e);
  }
  sp_newton_report r{};
  const double t0 = now_ms();
  sp_status s;
  auto norm = [&](const double* x, double* out) { return inner_many(c, x, 1, x, out, st); };
  if ((s = step_n(c, U, F, ns, st)) != SP_OK) return s;
  r.total_steps += ns;
  double nF;
  if ((s = norm(F, &nF)) != SP_OK) return s;
  nF = std::sqrt(nF);
  r.norm_F0 = nF;
  double nU;
  if ((s = norm(U, &nU)) != SP_OK) return s;
  double delta = o->delta0 > 0 ? o->delta0 : 0.1 * std::max(std::sqrt(nU), 1.0);
  // H: unrotated Hessenberg (column-major, ld K+1); R: the same after the Givens rotations
  const int LD = K + 2;  // leading dimension of H and R (one extra row and column for the gradient)
  std::vector<double> H((size_t)LD * (K + 1)), R((size_t)LD * (K + 1)), g(K + 2), cs(K + 1), sn(K + 1);
  sp_status result = SP_ENOTCONV;
  for (int it = 0; it <= o->max_newton; ++it) {
    if (!std::isfinite(nF)) { result = SP_ENAN; break; }
    if (nF < o->tol) { result = SP_OK; break; }
    if (it == o->max_newton) break;
    if ((s = sp_set_base_n(c, U, ns, st)) != SP_OK) return s;
    r.total_steps += ns;
    // GMRES without restarts; classical Gram-Schmidt applied twice, all reductions on the device
    if ((s = sp_cuda(c, launch_axpby(V, 1.0 / nF, F, 0.0, nullptr, L, st), "v0")) != SP_OK) return s;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = nF;
    int k = 0;
    // orthogonalise w = (action on column j) against V[0..j] (CGS2 on the device), normalise it
    // into V[j+1], and update column j of H, its Givens-rotated copy R and the residual g
    // device part of one Arnoldi column (capturable): classical Gram-Schmidt twice, normalisation,
    // the column to the host. For large states the second pass runs only when the first one lost
    // too much (|w'| < |w|/sqrt(2), decided on the device): it halves the basis traffic. Small
    // states are bound by FP64 work and launch latency: orth.cu (the same selective second pass).
    const bool selective = L >= 65536;
    const bool small = !selective && orth_small_applies(c, nb);
    auto enqueue_orth = [&](int j, double* w) -> sp_status {
      sp_status q;
      double* hb = hbuf + (size_t)(j & 1) * hstride;
      if (small)
        return sp_cuda(c, launch_orth_small(c, V, j + 1, w, dpart, nb, dhA, dhB, dhn, hb, Kc + 3, dflag, dnorm, st),
                       "column");
      const int* gate = selective ? dflag : nullptr;
      if ((q = sp_cuda(c, launch_dev_dots(c, V, j + 1, w, dpart, nb, dhA, nullptr, st), "dots")) != SP_OK) return q;
      if (selective) {
        if ((q = sp_cuda(c, launch_dev_norm(c, w, dpart, nb, dwn, dwn + 1, st), "norm")) != SP_OK) return q;
        if ((q = sp_cuda(c, launch_reorth_decide(dhA, j + 1, dwn, dflag, dhB, st), "decide")) != SP_OK) return q;
      }
      if ((q = sp_cuda(c, launch_multi_axpy(c, V, j + 1, dhA, w, st), "axpy")) != SP_OK) return q;
      if ((q = sp_cuda(c, launch_dev_dots(c, V, j + 1, w, dpart, nb, dhB, nullptr, st, gate), "dots")) != SP_OK)
        return q;
      if ((q = sp_cuda(c, launch_multi_axpy(c, V, j + 1, dhB, w, st, gate), "axpy")) != SP_OK) return q;
      if ((q = sp_cuda(c, launch_dev_norm(c, w, dpart, nb, dhn, dhn + 1, st), "norm")) != SP_OK) return q;
      if ((q = sp_cuda(c, launch_scale_dev(c, w, dhn + 1, st), "scale")) != SP_OK) return q;
      if ((q = sp_cuda(c, cudaMemcpyAsync(hb, dhA, (size_t)(j + 1) * 8, cudaMemcpyDeviceToHost, st), "h")) != SP_OK)
        return q;
      if ((q = sp_cuda(c, cudaMemcpyAsync(hb + Kc + 3, dhB, (size_t)(j + 1) * 8, cudaMemcpyDeviceToHost, st), "h")) !=
          SP_OK)
        return q;
      return sp_cuda(c, cudaMemcpyAsync(hb + 2 * (Kc + 3), dhn, 8, cudaMemcpyDeviceToHost, st), "h");
    };
    // host part (after the stream is synchronised): column j of H, its Givens-rotated copy R, g
    auto finish_orth = [&](int j) -> double {
      const double* hb = hbuf + (size_t)(j & 1) * hstride;
      const double hn = hb[2 * (Kc + 3)];
      double* Hc = H.data() + (size_t)j * LD;
      double* Rc = R.data() + (size_t)j * LD;
      for (int i = 0; i <= j; ++i) Hc[i] = hb[i] + hb[Kc + 3 + i];
      Hc[j + 1] = hn;
      givens_column(Hc, Rc, j, cs.data(), sn.data(), g.data());
      return hn;
    };
    auto orth_column = [&](int j, double* w, double* hn_out) -> sp_status {
      sp_status q;
      if ((q = enqueue_orth(j, w)) != SP_OK) return q;
      if ((q = sp_cuda(c, cudaStreamSynchronize(st), "orth sync")) != SP_OK) return q;
      *hn_out = finish_orth(j);
      return SP_OK;
    };
    // one Arnoldi step on the device: the action on v_j, then its column; events bracket both
    auto enqueue_step = [&](int j, bool capturing) -> sp_status {
      double* vj = V + (size_t)j * L;
      double* w = V + (size_t)(j + 1) * L;
      cudaEvent_t* ev = c->nev.data() + 3 * (size_t)j;
      auto rec = [&](cudaEvent_t e) {
        return capturing ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal) : cudaEventRecord(e, st);
      };
      sp_status q;
      if ((q = sp_cuda(c, rec(ev[0]), "event")) != SP_OK) return q;
      if (o->use_fd) q = sp_jvp_fd(c, vj, w, 1, st);
      else q = ns > 1 ? sp_jvp_n(c, vj, w, 1, st) : sp_jvp(c, vj, w, 1, st);
      if (q != SP_OK) return q;
      if ((q = sp_cuda(c, rec(ev[1]), "event")) != SP_OK) return q;
      if ((q = enqueue_orth(j, w)) != SP_OK) return q;
      return sp_cuda(c, rec(ev[2]), "event");
    };
    // Column j + 1 is launched before the host reads column j: the stopping test then runs while
    // the device works. When the test stops at column j, column j + 1 is computed and discarded.
    auto launch_step = [&](int j) -> sp_status {
      bool launched = false;
      if (graphs) {
        auto itg = c->ngraphs.find(j);
        if (itg == c->ngraphs.end()) {
          cudaGraph_t graph = nullptr;
          cudaGraphExec_t exec = nullptr;
          bool ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
          const sp_status cs_ = ok ? enqueue_step(j, true) : SP_ECUDA;
          const cudaError_t ce = cudaStreamEndCapture(st, &graph);
          ok = ok && cs_ == SP_OK && ce == cudaSuccess && graph &&
               cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
          if (graph) cudaGraphDestroy(graph);
          if (!ok) {  // not capturable here: continue with plain launches
            cudaGetLastError();
            if (exec) cudaGraphExecDestroy(exec);
            graphs = false;
          } else {
            itg = c->ngraphs.emplace(j, exec).first;
          }
        }
        if (graphs) {
          sp_status q = sp_cuda(c, cudaGraphLaunch(itg->second, st), "graph launch");
          if (q != SP_OK) return q;
          launched = true;
        }
      }
      return launched ? SP_OK : enqueue_step(j, false);
    };
    if ((s = launch_step(0)) != SP_OK) return s;
    for (int j = 0; j < K; ++j) {
      const bool ahead = j + 1 < K;
      if (ahead && (s = launch_step(j + 1)) != SP_OK) return s;
      cudaEvent_t* ev = c->nev.data() + 3 * (size_t)j;
      if ((s = sp_cuda(c, cudaEventSynchronize(ev[2]), "arnoldi sync")) != SP_OK) return s;
      const double hn = finish_orth(j);
      float ta = 0, tb = 0;
      if (cudaEventElapsedTime(&ta, ev[0], ev[1]) == cudaSuccess) r.t_action_ms += ta;
      else cudaGetLastError();  // timing is best effort; keep the error state clean
      if (cudaEventElapsedTime(&tb, ev[1], ev[2]) == cudaSuccess) r.t_orth_ms += tb;
      else cudaGetLastError();
      r.total_jvps++;
      k = j + 1;
      if (!std::isfinite(hn)) return sp_fail(c, SP_ENAN, "non-finite Arnoldi vector");
      if (std::fabs(g[k]) <= o->eta * nF || hn == 0.0) {
        if (ahead) r.spec_jvps++;
        break;
      }
    }
    // optional extra direction: the steepest-descent direction J^* F of |F|^2 / 2,
    // made orthogonal to the Krylov basis; one more (flexible) Arnoldi column
    bool grad_col = false;
    if (o->use_gradient && k >= 1) {
      if ((s = sp_vjp(c, F, Zg, 1, st)) != SP_OK) return s;
      double* w = V + (size_t)(k + 1) * L;
      for (int pass = 0; pass < 2; ++pass) {
        if ((s = sp_cuda(c, launch_dev_dots(c, V, k + 1, Zg, dpart, nb, dhA, nullptr, st), "dots")) != SP_OK) return s;
        if ((s = sp_cuda(c, launch_multi_axpy(c, V, k + 1, dhA, Zg, st), "axpy")) != SP_OK) return s;
      }
      // z must also be orthogonal to v_k (the last Krylov vector) for the update formula below
      if ((s = sp_cuda(c, launch_dev_norm(c, Zg, dpart, nb, dhn, dhn + 1, st), "norm")) != SP_OK) return s;
      if ((s = sp_cuda(c, cudaMemcpyAsync(hbuf, dhn, 16, cudaMemcpyDeviceToHost, st), "zn")) != SP_OK) return s;
      if ((s = sp_cuda(c, cudaStreamSynchronize(st), "zn sync")) != SP_OK) return s;
      if (hbuf[0] > 1e-12 * nF && std::isfinite(hbuf[0])) {
        if ((s = sp_cuda(c, launch_scale_dev(c, Zg, dhn + 1, st), "scale")) != SP_OK) return s;
        if ((s = sp_jvp(c, Zg, w, 1, st)) != SP_OK) return s;
        r.total_jvps++;
        double hn = 0;
        if ((s = orth_column(k, w, &hn)) != SP_OK) return s;
        if (std::isfinite(hn)) {
          grad_col = true;
          k = k + 1;
        }
      }
    }
    // hookstep: minimise |g - R y| (R = rotated k x k Hessenberg) subject to |y| <= delta.
    // The constrained minimiser is y(mu) = (R^T R + mu I)^-1 R^T g with mu >= 0 chosen so that
    // |y(mu)| = delta; R^T R = Q T Q^T (tridiagonal T) makes every |y(mu)| an O(k) solve.
    r.lin_rel = std::fabs(g[k]) / nF;
    Hookstep hs;
    hs.init(R.data(), LD, k, g.data());
    r.newton_len = hs.ny0;
    bool accepted = false;
    double nT = nF;
    for (int trial = 0; trial < 12; ++trial) {
      r.hook_trials++;
      double pred = 0, ylen = 0;
      const std::vector<double> y = hs.solve(delta, &pred, &ylen);
      if ((s = sp_cuda(c, cudaMemcpyAsync(Ut, U, L * 8, cudaMemcpyDeviceToDevice, st), "copy")) != SP_OK) return s;
      if ((s = sp_cuda(c, cudaMemcpyAsync(dhn + 2, y.data(), (size_t)k * 8, cudaMemcpyHostToDevice, st), "y copy")) !=
          SP_OK)
        return s;
      // U_trial = U - sum y_i z_i with z_i = v_i (Krylov) and, last, the gradient direction
      const int kv = grad_col ? k - 1 : k;
      if ((s = sp_cuda(c, launch_multi_axpy(c, V, kv, dhn + 2, Ut, st), "update")) != SP_OK) return s;
      if (grad_col)
        if ((s = sp_cuda(c, launch_multi_axpy(c, Zg, 1, dhn + 2 + kv, Ut, st), "update")) != SP_OK) return s;
      if ((s = step_n(c, Ut, F, ns, st)) != SP_OK) return s;
      r.total_steps += ns;
      if ((s = norm(F, &nT)) != SP_OK) return s;
      nT = std::sqrt(nT);
      if (!trust_update(nF, pred, nT, ylen, &delta)) continue;
      accepted = true;
      break;
    }
    if (!accepted) {
      if ((s = step_n(c, U, F, ns, st)) != SP_OK) return s;
      break;
    }
    if ((s = sp_cuda(c, cudaMemcpyAsync(U, Ut, L * 8, cudaMemcpyDeviceToDevice, st), "accept")) != SP_OK) return s;
    nF = nT;
    r.newton_iters++;
  }
  if ((s = sp_cuda(c, cudaStreamSynchronize(st), "newton sync")) != SP_OK) return s;
  r.norm_F = nF;
  r.delta = delta;
  r.t_total_ms = now_ms() - t0;
  if (rep) *rep = r;
  if (result == SP_ENOTCONV) c->err = "Newton did not reach the tolerance";
  return result;
}
