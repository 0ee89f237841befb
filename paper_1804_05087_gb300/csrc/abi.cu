// The C ABI (include/stokesprec.h): context lifetime, the BEFE step, its
// tangent and finite-difference actions, inner products and seeding.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

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

static void free_ctx(sp_ctx* c) {
  void* ptrs[] = {c->Th, c->TDh, c->Cfh, c->yv, c->Th_f, c->TDh_f, c->Cfh_f, c->twx, c->twz,
                  c->twx_f, c->twz_f, c->ops, c->ws6, c->ws3, c->base64, c->base32, c->U0,
                  c->G0, c->tmp, c->red, c->kry};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->red_host) cudaFreeHost(c->red_host);
  trace_reset(c);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  c->ev_pool.clear();
}

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
  if (c->smem_xz64 == 0) return bail(SP_EINVAL, "grid too large for the FP64 plane kernel");
  const size_t B = (size_t)cfg->max_batch;
  const size_t plane6 = (size_t)6 * c->NY * c->Mm * 16, plane3 = (size_t)3 * c->NY * c->Mm * 16;
  const size_t grid = (size_t)c->NY * c->nx * c->nz;
  c->red_blocks = 2 * c->sm_count;
  bool ok = cudaMalloc(&c->ws6, B * plane6) == cudaSuccess && cudaMalloc(&c->ws3, B * plane3) == cudaSuccess &&
            cudaMalloc((void**)&c->base64, 6 * grid * 8) == cudaSuccess &&
            cudaMalloc((void**)&c->base32, 6 * grid * 4) == cudaSuccess &&
            cudaMalloc((void**)&c->U0, c->state_len * 8) == cudaSuccess &&
            cudaMalloc((void**)&c->G0, c->state_len * 8) == cudaSuccess &&
            cudaMalloc((void**)&c->tmp, B * c->state_len * 8) == cudaSuccess &&
            cudaMalloc((void**)&c->red, (size_t)64 * c->red_blocks * 8 + 4096) == cudaSuccess &&
            cudaMallocHost((void**)&c->red_host, (size_t)64 * c->red_blocks * 8 + 4096) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return bail(SP_ENOMEM, "workspace allocation");
  }
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
    if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_yinv(c, false, u, c->ws6, nb, st); }), "yinv")) != SP_OK) return s;
    if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_xz(c, false, XZ_STEP, c->ws6, c->ws3, nb, st); }), "xz step")) != SP_OK) return s;
    if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_solve(c, false, c->ws3, u, g, nb, st); }), "solve")) != SP_OK) return s;
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
  if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_yinv(c, false, c->U0, c->ws6, 1, st); }), "yinv")) != SP_OK) return s;
  if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_xz(c, false, XZ_BASE, c->ws6, nullptr, 1, st); }), "xz base")) != SP_OK) return s;
  if ((s = sp_cuda(c, traced(c, SP_STAGE_STEP, st, [&] { return launch_base_to_f32(c, st); }), "base f32")) != SP_OK) return s;
  if ((s = step_batch(c, c->U0, c->G0, 1, st)) != SP_OK) return s;
  c->has_base = 1;
  return SP_OK;
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
    if ((s = sp_cuda(c, traced(c, SP_STAGE_YINV, st, [&] { return launch_yinv(c, f32, u, c->ws6, nb, st); }), "yinv")) != SP_OK) return s;
    if ((s = sp_cuda(c, traced(c, SP_STAGE_XZ, st, [&] { return launch_xz(c, f32, XZ_TANGENT, c->ws6, c->ws3, nb, st); }), "xz tangent")) != SP_OK) return s;
    if ((s = sp_cuda(c, traced(c, SP_STAGE_SOLVE, st, [&] { return launch_solve(c, f32, c->ws3, u, g, nb, st); }), "solve")) != SP_OK) return s;
  }
  return SP_OK;
}

static sp_status vjp_impl(sp_ctx* c, const double* r, double* JTr, int n_dir, bool weighted, cudaStream_t st,
                          const char* who) {
  if (!c || !r || !JTr || n_dir < 0 || r == JTr) return sp_fail(c, SP_EINVAL, std::string(who) + ": bad arguments");
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

extern "C" sp_status sp_jvp_fd(sp_ctx* c, const double* du, double* Jdu, int n_dir, void* stream) {
  if (!c || !du || !Jdu || n_dir < 0 || du == Jdu) return sp_fail(c, SP_EINVAL, "sp_jvp_fd: bad arguments");
  if (!c->has_base) return sp_fail(c, SP_EINVAL, "sp_jvp_fd: call sp_set_base first");
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
    if ((s = step_batch(c, c->tmp, g, 1, st)) != SP_OK) return s;
    if ((s = sp_cuda(c, launch_axpby(g, 1.0 / eps, g, -1.0 / eps, c->G0, c->state_len, st), "axpby")) != SP_OK)
      return s;
  }
  return sp_cuda(c, cudaStreamSynchronize(st), "fd sync");
}

extern "C" sp_status sp_seed_state(sp_ctx* c, const double* ra, const double* rb, const double* rc, double amp,
                                   double* U, void* stream) {
  if (!c || !ra || !rb || !rc || !U) return sp_fail(c, SP_EINVAL, "sp_seed_state: bad pointers");
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

// ================================================================= Newton
namespace {

// one-sided Jacobi SVD of the m x n matrix A (column-major, m >= n):
// A = U diag(s) V^T; A is overwritten by U diag(s)
void jacobi_svd(std::vector<double>& A, int m, int n, std::vector<double>& s, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double alpha = 0, beta = 0, gamma = 0;
        for (int i = 0; i < m; ++i) {
          const double ap = A[(size_t)p * m + i], aq = A[(size_t)q * m + i];
          alpha += ap * ap;
          beta += aq * aq;
          gamma += ap * aq;
        }
        if (gamma == 0.0) continue;
        const double rel = std::fabs(gamma) / std::sqrt(alpha * beta);
        if (rel > off) off = rel;
        if (rel < 1e-15) continue;
        const double zeta = (beta - alpha) / (2.0 * gamma);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
        for (int i = 0; i < m; ++i) {
          const double ap = A[(size_t)p * m + i], aq = A[(size_t)q * m + i];
          A[(size_t)p * m + i] = cs * ap - sn * aq;
          A[(size_t)q * m + i] = sn * ap + cs * aq;
        }
        for (int i = 0; i < n; ++i) {
          const double vp = V[(size_t)p * n + i], vq = V[(size_t)q * n + i];
          V[(size_t)p * n + i] = cs * vp - sn * vq;
          V[(size_t)q * n + i] = sn * vp + cs * vq;
        }
      }
    if (off < 1e-15) break;
  }
  s.assign(n, 0.0);
  for (int j = 0; j < n; ++j) {
    double acc = 0;
    for (int i = 0; i < m; ++i) acc += A[(size_t)j * m + i] * A[(size_t)j * m + i];
    s[j] = std::sqrt(acc);
  }
}

// z minimising |p - diag(s) z| with |z| <= delta (hookstep, Sec. 3.2)
std::vector<double> hook(const std::vector<double>& s, const std::vector<double>& p, double delta) {
  const int n = (int)s.size();
  std::vector<double> z(n);
  double nz = 0;
  for (int i = 0; i < n; ++i) {
    z[i] = s[i] > 0 ? p[i] / s[i] : 0.0;
    nz += z[i] * z[i];
  }
  if (std::sqrt(nz) <= delta) return z;
  double smax = 0, spmax = 0;
  for (int i = 0; i < n; ++i) {
    smax = std::max(smax, s[i]);
    spmax = std::max(spmax, s[i] * std::fabs(p[i]));
  }
  double lo = 0, hi = spmax / delta + smax * smax;
  for (int it = 0; it < 200; ++it) {
    const double mu = 0.5 * (lo + hi);
    double acc = 0;
    for (int i = 0; i < n; ++i) {
      const double zi = s[i] * p[i] / (s[i] * s[i] + mu);
      acc += zi * zi;
    }
    if (std::sqrt(acc) > delta) lo = mu;
    else hi = mu;
  }
  for (int i = 0; i < n; ++i) z[i] = s[i] * p[i] / (s[i] * s[i] + hi);
  return z;
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

extern "C" sp_status sp_newton_gmres(sp_ctx* c, double* U, const sp_newton_opts* o, sp_newton_report* rep,
                                     void* stream) {
  if (!c || !U || !o) return sp_fail(c, SP_EINVAL, "sp_newton_gmres: bad arguments");
  const int K = o->max_krylov;
  if (K < 1 || K > 4096 || o->max_newton < 0) return sp_fail(c, SP_EINVAL, "sp_newton_gmres: bad options");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t L = c->state_len;
  if (c->kry_cap < K + 3) {
    if (c->kry) cudaFree(c->kry);
    c->kry = nullptr;
    c->kry_cap = 0;
    if (cudaMalloc((void**)&c->kry, ((size_t)(K + 3) * L + K + 8) * 8) != cudaSuccess) {
      cudaGetLastError();
      return sp_fail(c, SP_ENOMEM, "Krylov basis allocation");
    }
    c->kry_cap = K + 3;
  }
  double* V = c->kry;                       // K+1 basis vectors
  double* F = c->kry + (size_t)(K + 1) * L; // residual
  double* Ut = c->kry + (size_t)(K + 2) * L;// trial state
  double* dh = c->kry + (size_t)(K + 3) * L;  // device copy of h or y (K + 1 doubles)
  sp_newton_report r{};
  const double t0 = now_ms();
  sp_status s;
  auto norm = [&](const double* x, double* out) { return inner_many(c, x, 1, x, out, st); };
  if ((s = step_batch(c, U, F, 1, st)) != SP_OK) return s;
  r.total_steps++;
  double nF;
  if ((s = norm(F, &nF)) != SP_OK) return s;
  nF = std::sqrt(nF);
  r.norm_F0 = nF;
  double nU;
  if ((s = norm(U, &nU)) != SP_OK) return s;
  double delta = o->delta0 > 0 ? o->delta0 : 0.1 * std::max(std::sqrt(nU), 1.0);
  std::vector<double> H((size_t)(K + 1) * K), h(K + 1), h2(K + 1);
  sp_status result = SP_ENOTCONV;
  for (int it = 0; it <= o->max_newton; ++it) {
    if (!std::isfinite(nF)) { result = SP_ENAN; break; }
    if (nF < o->tol) { result = SP_OK; break; }
    if (it == o->max_newton) break;
    if ((s = sp_set_base(c, U, st)) != SP_OK) return s;
    r.total_steps++;
    // GMRES, classical Gram-Schmidt applied twice, basis in V
    std::fill(H.begin(), H.end(), 0.0);
    if ((s = sp_cuda(c, launch_axpby(V, 1.0 / nF, F, 0.0, nullptr, L, st), "v0")) != SP_OK) return s;
    int k = 0;
    for (int j = 0; j < K; ++j) {
      double* vj = V + (size_t)j * L;
      double* w = V + (size_t)(j + 1) * L;
      double ta = now_ms();
      if (o->use_fd) s = sp_jvp_fd(c, vj, w, 1, st);
      else s = sp_jvp(c, vj, w, 1, st);
      if (s != SP_OK) return s;
      if ((s = sp_cuda(c, cudaStreamSynchronize(st), "jvp sync")) != SP_OK) return s;
      double tb = now_ms();
      r.t_action_ms += tb - ta;
      r.total_jvps++;
      for (int pass = 0; pass < 2; ++pass) {
        std::vector<double>& hh = pass == 0 ? h : h2;
        if ((s = inner_many(c, V, j + 1, w, hh.data(), st)) != SP_OK) return s;
        if ((s = sp_cuda(c, cudaMemcpyAsync(dh, hh.data(), (size_t)(j + 1) * 8, cudaMemcpyHostToDevice, st),
                         "h copy")) != SP_OK)
          return s;
        if ((s = sp_cuda(c, launch_multi_axpy(c, V, j + 1, dh, w, st), "axpy")) != SP_OK) return s;
        if ((s = sp_cuda(c, cudaStreamSynchronize(st), "orth sync")) != SP_OK) return s;
      }
      for (int i = 0; i <= j; ++i) H[(size_t)j * (K + 1) + i] = h[i] + h2[i];
      double hn;
      if ((s = norm(w, &hn)) != SP_OK) return s;
      hn = std::sqrt(hn);
      H[(size_t)j * (K + 1) + j + 1] = hn;
      k = j + 1;
      if (hn > 0)
        if ((s = sp_cuda(c, launch_scale(w, 1.0 / hn, L, st), "scale")) != SP_OK) return s;
      r.t_orth_ms += now_ms() - tb;
      // least-squares residual of beta e1 - H_k y via Givens on a copy
      std::vector<double> Hc((size_t)(k + 1) * k), g(k + 1, 0.0);
      for (int cc = 0; cc < k; ++cc)
        for (int i = 0; i <= k; ++i) Hc[(size_t)cc * (k + 1) + i] = H[(size_t)cc * (K + 1) + i];
      g[0] = nF;
      for (int cc = 0; cc < k; ++cc) {
        const double a = Hc[(size_t)cc * (k + 1) + cc], b = Hc[(size_t)cc * (k + 1) + cc + 1];
        const double rr = std::hypot(a, b);
        if (rr == 0) continue;
        const double cs = a / rr, sn = b / rr;
        for (int c2 = cc; c2 < k; ++c2) {
          const double x = Hc[(size_t)c2 * (k + 1) + cc], y = Hc[(size_t)c2 * (k + 1) + cc + 1];
          Hc[(size_t)c2 * (k + 1) + cc] = cs * x + sn * y;
          Hc[(size_t)c2 * (k + 1) + cc + 1] = -sn * x + cs * y;
        }
        const double x = g[cc], y = g[cc + 1];
        g[cc] = cs * x + sn * y;
        g[cc + 1] = -sn * x + cs * y;
      }
      if (std::fabs(g[k]) <= o->eta * nF || hn == 0.0) break;
    }
    // hookstep on the (k+1) x k Hessenberg matrix
    std::vector<double> A((size_t)(k + 1) * k), sv, Vs;
    for (int cc = 0; cc < k; ++cc)
      for (int i = 0; i <= k; ++i) A[(size_t)cc * (k + 1) + i] = H[(size_t)cc * (K + 1) + i];
    std::vector<double> Acopy = A;
    jacobi_svd(A, k + 1, k, sv, Vs);
    std::vector<double> p(k);
    for (int i = 0; i < k; ++i) p[i] = sv[i] > 0 ? nF * A[(size_t)i * (k + 1) + 0] / sv[i] : 0.0;
    bool accepted = false;
    double nT = nF;
    for (int trial = 0; trial < 12; ++trial) {
      std::vector<double> z = hook(sv, p, delta), y(k, 0.0);
      for (int i = 0; i < k; ++i)
        for (int jj = 0; jj < k; ++jj) y[i] += Vs[(size_t)jj * k + i] * z[jj];
      double ylen = 0;
      for (double v : y) ylen += v * v;
      ylen = std::sqrt(ylen);
      // predicted residual |beta e1 - H y|
      double pred = 0;
      for (int i = 0; i <= k; ++i) {
        double acc = i == 0 ? nF : 0.0;
        for (int cc = 0; cc < k; ++cc) acc -= Acopy[(size_t)cc * (k + 1) + i] * y[cc];
        pred += acc * acc;
      }
      pred = std::sqrt(pred);
      // U_trial = U - V y
      std::vector<double> ny(k);
      for (int i = 0; i < k; ++i) ny[i] = y[i];
      if ((s = sp_cuda(c, cudaMemcpyAsync(Ut, U, L * 8, cudaMemcpyDeviceToDevice, st), "copy")) != SP_OK) return s;
      if ((s = sp_cuda(c, cudaMemcpyAsync(dh, ny.data(), (size_t)k * 8, cudaMemcpyHostToDevice, st), "y copy")) != SP_OK)
        return s;
      if ((s = sp_cuda(c, launch_multi_axpy(c, V, k, dh, Ut, st), "update")) != SP_OK) return s;
      if ((s = step_batch(c, Ut, F, 1, st)) != SP_OK) return s;
      r.total_steps++;
      if ((s = norm(F, &nT)) != SP_OK) return s;
      nT = std::sqrt(nT);
      const double denom = nF * nF - pred * pred;
      const double rho = denom > 0 ? (nF * nF - nT * nT) / denom : -1.0;
      if (!(rho >= 0.01) || !std::isfinite(nT)) {
        delta = 0.5 * ylen;
        continue;
      }
      if (rho > 0.75 && ylen >= 0.99 * delta) delta *= 2.0;
      else if (rho < 0.25) delta *= 0.5;
      accepted = true;
      break;
    }
    if (!accepted) {
      // restore F for the report and stop: the trust region collapsed
      if ((s = step_batch(c, U, F, 1, st)) != SP_OK) return s;
      break;
    }
    if ((s = sp_cuda(c, cudaMemcpyAsync(U, Ut, L * 8, cudaMemcpyDeviceToDevice, st), "accept")) != SP_OK) return s;
    nF = nT;
    r.newton_iters++;
  }
  if ((s = sp_cuda(c, cudaStreamSynchronize(st), "newton sync")) != SP_OK) return s;
  r.norm_F = nF;
  r.t_total_ms = now_ms() - t0;
  if (rep) *rep = r;
  if (result == SP_ENOTCONV) c->err = "Newton did not reach the tolerance";
  return result;
}
