// Groups of independent plane Couette problems (sp_group_*): the members of a
// parameter continuation, each with its own grid, box, Reynolds number and dt,
// stepped together. Every stage of the step and of the tangent is ONE launch
// over all members' blocks (kernels.cu, xz_reg.cu); the vector operations of
// GMRES are one launch over all members' slices of a group vector (below).
// Newton-GMRES-hookstep (Sec. 2, Sec. 3.2) runs on all members in lock step:
// Arnoldi step j of every member that is still iterating is one sequence of
// launches (classical Gram-Schmidt with selective reorthogonalisation), optionally
// replayed as a captured CUDA graph. The arithmetic of a
// member is exactly that of its own context.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <new>
#include <numeric>

#include "hookstep.h"
#include "sp_internal.h"

namespace {

constexpr int kVecThreads = 256;
constexpr size_t kAlign = 32;  // member offsets in doubles (256 bytes)

// a member's slice of a group vector and its share of the vector launches
struct GVec {
  size_t off;    // doubles
  size_t ncplx;  // complex values of the state
  int NY, MZ;    // for the weights w(iz) of the inner product
  int nb;        // blocks of the reduction launches (dots, norms)
  int first;     // first of those blocks
  int nb_el;     // blocks of the elementwise launches (axpy, scale)
  int first_el;
};

__device__ __forceinline__ double blk_sum(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? red[lane] : 0.0;
  if (wid == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// partial weighted inner products of rows i0..i0+7 (< k) of V with w, every
// member at once: partials[row][block]. Grid (blocks, ceil(k/8)).
__global__ void __launch_bounds__(kVecThreads) k_gdots(const double* __restrict__ V, size_t vs, int k,
                                                       const double* __restrict__ w, const GVec* __restrict__ recs,
                                                       const int* __restrict__ inst, const int* __restrict__ active,
                                                       double* __restrict__ partials) {
  const int i = inst[blockIdx.x];
  if (active && !active[i]) return;
  const GVec r = recs[i];
  const int b = blockIdx.x - r.first;
  const int i0 = blockIdx.y * 8;
  double acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = 0.0;
  const double2* w2 = reinterpret_cast<const double2*>(w + r.off);
  // the weight of element e depends on iz = (e / NY) mod MZ; follow (iz, e mod NY)
  // incrementally along the stride instead of dividing per element
  const unsigned NY = r.NY, MZ = r.MZ, S = (unsigned)r.nb * blockDim.x;
  const unsigned dq = S / NY, dr = S - dq * NY, dz = dq % MZ;
  unsigned e0 = (unsigned)b * blockDim.x + threadIdx.x;
  unsigned rr = e0 % NY, iz = (e0 / NY) % MZ;
  for (unsigned e = e0; e < r.ncplx; e += S) {
    const double wt = iz == 0 ? 1.0 : 2.0;
    const double2 bv = w2[e];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (i0 + q < k) {
        const double2 a = reinterpret_cast<const double2*>(V + (size_t)(i0 + q) * vs + r.off)[e];
        acc[q] += wt * (a.x * bv.x + a.y * bv.y);
      }
    }
    rr += dr;
    iz += dz;
    if (rr >= NY) {
      rr -= NY;
      ++iz;
    }
    if (iz >= MZ) iz -= MZ;
  }
  // the eight block sums with one barrier: warp shuffles, then one thread per row
  __shared__ double red8[8][kVecThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red8[q][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8 && i0 + (int)threadIdx.x < k) {
    double v = 0.0;
    for (int w8 = 0; w8 < kVecThreads / 32; ++w8) v += red8[threadIdx.x][w8];
    partials[(size_t)(i0 + threadIdx.x) * gridDim.x + blockIdx.x] = v;
  }
}

// h[row * n + i] = sum of member i's partials of that row. Grid (n, k).
__global__ void k_greduce(const double* __restrict__ partials, int ptot, const GVec* __restrict__ recs,
                          const int* __restrict__ active, int n, double* __restrict__ h) {
  const int i = blockIdx.x, row = blockIdx.y;
  if (active && !active[i]) return;
  const GVec r = recs[i];
  double acc = 0.0;
  for (int b = threadIdx.x; b < r.nb; b += blockDim.x) acc += partials[(size_t)row * ptot + r.first + b];
  acc = blk_sum(acc);
  if (threadIdx.x == 0) h[(size_t)row * n + i] = acc;
}

// hn[i] = sqrt(sum of member i's partials of row 0), inv[i] = 1/hn[i] (0 if 0). Grid (n).
__global__ void k_gnorm(const double* __restrict__ partials, const GVec* __restrict__ recs,
                        const int* __restrict__ active, double* __restrict__ hn, double* __restrict__ inv) {
  const int i = blockIdx.x;
  if (active && !active[i]) return;
  const GVec r = recs[i];
  double acc = 0.0;
  for (int b = threadIdx.x; b < r.nb; b += blockDim.x) acc += partials[r.first + b];
  acc = blk_sum(acc);
  if (threadIdx.x == 0) {
    const double s = sqrt(fmax(acc, 0.0));
    hn[i] = s;
    inv[i] = s > 0.0 ? 1.0 / s : 0.0;
  }
}

// Selective reorthogonalisation (Daniel, Gragg, Kaufman & Stewart): after the first
// Gram-Schmidt pass, |w'|^2 = |w|^2 - |h|^2 (V orthonormal); member i needs the second
// pass only if |w'| < |w| / sqrt(2). flag[i] = 1 then; otherwise its second-pass
// coefficients are zeroed. One warp per member.
__global__ void k_greorth_decide(const double* __restrict__ h, int n, int k, const double* __restrict__ wn,
                                 const int* __restrict__ active, int* __restrict__ flag, double* __restrict__ h2) {
  const int i = blockIdx.x;
  if (active && !active[i]) {
    if (threadIdx.x == 0) flag[i] = 0;
    return;
  }
  double acc = 0.0;
  for (int q = threadIdx.x; q < k; q += 32) {
    const double v = h[(size_t)q * n + i];
    acc = fma(v, v, acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  acc = __shfl_sync(0xffffffffu, acc, 0);
  const double w2 = wn[i] * wn[i];
  const int f = (w2 - acc < 0.5 * w2) ? 1 : 0;
  if (threadIdx.x == 0) flag[i] = f;
  if (!f)
    for (int q = threadIdx.x; q < k; q += 32) h2[(size_t)q * n + i] = 0.0;
}

// w_i -= sum_{row < k} h[row * n + i] V_row,i
__global__ void __launch_bounds__(kVecThreads) k_gaxpy(const double* __restrict__ V, size_t vs, int k,
                                                       const double* __restrict__ h, int n, double* __restrict__ w,
                                                       const GVec* __restrict__ recs, const int* __restrict__ inst,
                                                       const int* __restrict__ active) {
  const int i = inst[blockIdx.x];
  if (active && !active[i]) return;
  const GVec r = recs[i];
  const int b = blockIdx.x - r.first_el;
  const size_t len = 2 * r.ncplx;
  double* wi = w + r.off;
  const double* Vi = V + r.off;
  for (size_t e = (size_t)b * blockDim.x + threadIdx.x; e < len; e += (size_t)r.nb_el * blockDim.x) {
    double acc[8] = {wi[e], 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int q = 0;
    for (; q + 8 <= k; q += 8) {
#pragma unroll
      for (int t = 0; t < 8; ++t) acc[t] -= h[(size_t)(q + t) * n + i] * Vi[(size_t)(q + t) * vs + e];
    }
    for (; q < k; ++q) acc[0] -= h[(size_t)q * n + i] * Vi[(size_t)q * vs + e];
    wi[e] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  }
}

// dst_i = s[i] * src_i (s null: plain copy) for the members with mask[i] != 0 (mask null: all)
__global__ void __launch_bounds__(kVecThreads) k_gscale(double* __restrict__ dst, const double* __restrict__ src,
                                                        const double* __restrict__ s, const GVec* __restrict__ recs,
                                                        const int* __restrict__ inst, const int* __restrict__ mask) {
  const int i = inst[blockIdx.x];
  if (mask && !mask[i]) return;
  const GVec r = recs[i];
  const int b = blockIdx.x - r.first_el;
  const size_t len = 2 * r.ncplx;
  const double f = s ? s[i] : 1.0;
  for (size_t e = (size_t)b * blockDim.x + threadIdx.x; e < len; e += (size_t)r.nb_el * blockDim.x)
    dst[r.off + e] = f * src[r.off + e];
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

thread_local std::string g_group_create_error;

}  // namespace

struct sp_group {
  int n = 0;
  int prec = 0;
  std::vector<sp_ctx*> mem;
  std::vector<size_t> off;
  std::vector<int> order;  // members, largest first
  size_t len = 0;          // doubles per group vector
  GrpPlan plan;
  // vector launches
  GVec* vrecs = nullptr;
  int* vinst = nullptr;     // block -> member, reduction launches
  int vblocks = 0;
  int* einst = nullptr;     // block -> member, elementwise launches
  int eblocks = 0;
  std::vector<GVec> vrecs_h;
  // scratch: masks, per-member scalars, partial sums
  int* act = nullptr;       // device [n]
  int* act_h = nullptr;     // pinned [n]
  double* scal = nullptr;   // device [4n]: hn | inv | s | spare
  double* part = nullptr;   // device [8 * vblocks] (norms outside Newton)
  double* host = nullptr;   // pinned [4n]
  double* tmpv = nullptr;   // one group vector
  // Newton: basis and scratch, graphs per Arnoldi step
  double* kry = nullptr;
  int kry_cap = 0;
  double* kry_host = nullptr;  // pinned
  size_t kry_host_len = 0;
  cudaStream_t st = nullptr;
  cudaEvent_t ev_in = nullptr;
  std::vector<cudaEvent_t> ev_step;  // 3 per Arnoldi step (start, after the action, after the orthogonalisation)
  std::map<int, cudaGraphExec_t> graphs;
  std::string err;
};

static sp_status gfail(sp_group* g, sp_status s, const std::string& m) {
  if (g) g->err = m;
  return s;
}

static sp_status gcuda(sp_group* g, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return SP_OK;
  if (g) g->err = std::string(what) + ": " + cudaGetErrorString(e);
  return SP_ECUDA;
}

static void drop_graphs(sp_group* g) {
  for (auto& kv : g->graphs) cudaGraphExecDestroy(kv.second);
  g->graphs.clear();
}

static void free_group(sp_group* g) {
  drop_graphs(g);
  grp_plan_free(&g->plan);
  for (void* p : {(void*)g->vrecs, (void*)g->vinst, (void*)g->einst, (void*)g->act, (void*)g->scal, (void*)g->part, (void*)g->tmpv,
                  (void*)g->kry})
    if (p) cudaFree(p);
  if (g->act_h) cudaFreeHost(g->act_h);
  if (g->host) cudaFreeHost(g->host);
  if (g->kry_host) cudaFreeHost(g->kry_host);
  for (cudaEvent_t e : g->ev_step) cudaEventDestroy(e);
  if (g->ev_in) cudaEventDestroy(g->ev_in);
  if (g->st) cudaStreamDestroy(g->st);
  for (sp_ctx* c : g->mem)
    if (c) sp_destroy(c);
  g->mem.clear();
}

extern "C" sp_status sp_group_create(const sp_config* cfgs, int n, sp_group** out) {
  if (!out) return SP_EINVAL;
  *out = nullptr;
  if (!cfgs || n < 1 || n > 4096) {
    g_group_create_error = "sp_group_create: bad arguments";
    return SP_EINVAL;
  }
  sp_group* g = new (std::nothrow) sp_group();
  if (!g) return SP_ENOMEM;
  auto bail = [&](sp_status s, const std::string& m) {
    g_group_create_error = "sp_group_create: " + m;
    free_group(g);
    delete g;
    return s;
  };
  g->n = n;
  g->prec = cfgs[0].prec;
  g->mem.assign(n, nullptr);
  g->off.assign(n, 0);
  size_t pos = 0;
  for (int i = 0; i < n; ++i) {
    if (cfgs[i].prec != g->prec) return bail(SP_EINVAL, "members differ in precision");
    if (cfgs[i].lam_adv != cfgs[0].lam_adv) return bail(SP_EINVAL, "members differ in lam_adv");
    sp_config c = cfgs[i];
    c.max_batch = 1;
    sp_status s = sp_create(&c, &g->mem[i]);
    if (s != SP_OK) return bail(s, "member " + std::to_string(i) + ": " + sp_last_error(nullptr));
    // the grouped FP64 plane stage is the generic kernel: a member's own calls use it too,
    // so that they compute exactly what the group computes for it
    g->mem[i]->use_xz_reg64 = 0;
    g->mem[i]->use_yinv_tc = 0;
    g->mem[i]->use_rhs_tc = 0;
    g->off[i] = pos;
    pos += (sp_state_len(g->mem[i]) + kAlign - 1) / kAlign * kAlign;
  }
  g->len = pos;
  g->order.resize(n);
  std::iota(g->order.begin(), g->order.end(), 0);
  std::stable_sort(g->order.begin(), g->order.end(),
                   [&](int a, int b) { return g->mem[a]->state_len > g->mem[b]->state_len; });
  cudaError_t e = grp_plan_build(&g->plan, g->mem.data(), n, g->off.data(), g->order.data());
  if (e != cudaSuccess) return bail(SP_ECUDA, std::string("grouped launch tables: ") + cudaGetErrorString(e));
  // reduction launches: 2048-4096 complex values per block; elementwise launches: two
  // doubles per thread
  g->vrecs_h.resize(n);
  std::vector<int> vinst, einst;
  for (int q = 0; q < n; ++q) {
    const int i = g->order[q];
    const sp_ctx* c = g->mem[i];
    GVec& r = g->vrecs_h[i];
    r.off = g->off[i];
    r.ncplx = c->cplx_per_state;
    r.NY = c->NY;
    r.MZ = c->MZ;
    const size_t per = r.ncplx > 65536 ? 4096 : 2048;  // small states: more blocks for parallelism
    r.nb = (int)std::max<size_t>(1, (r.ncplx + per - 1) / per);
    r.first = (int)vinst.size();
    for (int b = 0; b < r.nb; ++b) vinst.push_back(i);
    r.nb_el = (int)std::max<size_t>(1, (2 * r.ncplx + 511) / 512);  // two doubles per thread
    r.first_el = (int)einst.size();
    for (int b = 0; b < r.nb_el; ++b) einst.push_back(i);
  }
  g->vblocks = (int)vinst.size();
  g->eblocks = (int)einst.size();
  if ((e = grp_upload((void**)&g->vrecs, g->vrecs_h.data(), n * sizeof(GVec))) != cudaSuccess ||
      (e = grp_upload((void**)&g->vinst, vinst.data(), vinst.size() * sizeof(int))) != cudaSuccess ||
      (e = grp_upload((void**)&g->einst, einst.data(), einst.size() * sizeof(int))) != cudaSuccess)
    return bail(SP_ECUDA, std::string("vector tables: ") + cudaGetErrorString(e));
  bool ok = cudaMalloc((void**)&g->act, n * sizeof(int)) == cudaSuccess &&
            cudaMallocHost((void**)&g->act_h, n * sizeof(int)) == cudaSuccess &&
            cudaMalloc((void**)&g->scal, 4 * n * sizeof(double)) == cudaSuccess &&
            cudaMallocHost((void**)&g->host, 4 * n * sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&g->part, (size_t)8 * g->vblocks * sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&g->tmpv, g->len * sizeof(double)) == cudaSuccess &&
            cudaStreamCreateWithFlags(&g->st, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreate(&g->ev_in) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return bail(SP_ENOMEM, "group workspaces");
  }
  *out = g;
  return SP_OK;
}

extern "C" sp_status sp_group_destroy(sp_group* g) {
  if (!g) return SP_EINVAL;
  free_group(g);
  delete g;
  return SP_OK;
}

extern "C" const char* sp_group_last_error(const sp_group* g) {
  if (!g) return g_group_create_error.c_str();
  return g->err.c_str();
}

extern "C" int sp_group_size(const sp_group* g) { return g ? g->n : 0; }

extern "C" size_t sp_group_state_len(const sp_group* g) { return g ? g->len : 0; }

extern "C" size_t sp_group_offset(const sp_group* g, int i) {
  if (!g || i < 0 || i >= g->n) return (size_t)-1;
  return g->off[i];
}

extern "C" sp_ctx* sp_group_member(sp_group* g, int i) {
  if (!g || i < 0 || i >= g->n) return nullptr;
  return g->mem[i];
}

// ---------------------------------------------------------------- internals
static sp_status group_step(sp_group* g, const double* U, double* G, const int* act, cudaStream_t st) {
  sp_status s;
  if ((s = gcuda(g, grp_launch_yinv(g->plan, false, U, act, st), "group yinv")) != SP_OK) return s;
  if ((s = gcuda(g, grp_launch_xz(g->plan, false, XZ_STEP, act, st), "group xz step")) != SP_OK) return s;
  return gcuda(g, grp_launch_solve(g->plan, false, U, G, act, st), "group solve");
}

static sp_status group_jvp(sp_group* g, const double* du, double* Jdu, const int* act, cudaStream_t st) {
  const bool f32 = g->prec == SP_MIXED;
  sp_status s;
  if ((s = gcuda(g, grp_launch_yinv(g->plan, f32, du, act, st), "group yinv")) != SP_OK) return s;
  if ((s = gcuda(g, grp_launch_xz(g->plan, f32, XZ_TANGENT, act, st), "group xz tangent")) != SP_OK) return s;
  return gcuda(g, grp_launch_solve(g->plan, f32, du, Jdu, act, st), "group solve");
}

// base fields of every member (FP64 and float copies); with_g0 also stores each
// member's U0 and G(U0) for its finite-difference action
static sp_status group_base(sp_group* g, const double* U, bool with_g0, const int* act, cudaStream_t st) {
  sp_status s;
  if ((s = gcuda(g, grp_launch_yinv(g->plan, false, U, act, st), "group yinv")) != SP_OK) return s;
  if ((s = gcuda(g, grp_launch_xz(g->plan, false, XZ_BASE, act, st), "group xz base")) != SP_OK) return s;
  for (sp_ctx* c : g->mem)
    if ((s = gcuda(g, launch_base_to_f32(c, st), "base f32")) != SP_OK) return s;
  if (with_g0) {
    if ((s = group_step(g, U, g->tmpv, nullptr, st)) != SP_OK) return s;
    for (int i = 0; i < g->n; ++i) {
      sp_ctx* c = g->mem[i];
      const size_t bytes = c->state_len * 8;
      if ((s = gcuda(g, cudaMemcpyAsync(c->U0, U + g->off[i], bytes, cudaMemcpyDeviceToDevice, st), "U0")) != SP_OK)
        return s;
      if ((s = gcuda(g, cudaMemcpyAsync(c->G0, g->tmpv + g->off[i], bytes, cudaMemcpyDeviceToDevice, st), "G0")) !=
          SP_OK)
        return s;
    }
  }
  for (sp_ctx* c : g->mem) c->has_base = 1;
  return SP_OK;
}

// partial sums of <V_row, w> for rows < k into `part` (k <= 8 per pass handled by the grid's y)
static cudaError_t launch_gdots(const sp_group* g, const double* V, size_t vs, int k, const double* w, const int* act,
                                double* part, cudaStream_t st) {
  dim3 grid(g->vblocks, (k + 7) / 8);
  k_gdots<<<grid, kVecThreads, 0, st>>>(V, vs, k, w, g->vrecs, g->vinst, act, part);
  return cudaGetLastError();
}

// h[row * n + i] = <V_row, w>_i for rows < k
static cudaError_t launch_ghdots(const sp_group* g, const double* V, size_t vs, int k, const double* w, const int* act,
                                 double* part, double* h, cudaStream_t st) {
  cudaError_t e = launch_gdots(g, V, vs, k, w, act, part, st);
  if (e != cudaSuccess) return e;
  k_greduce<<<dim3(g->n, k), kVecThreads, 0, st>>>(part, g->vblocks, g->vrecs, act, g->n, h);
  return cudaGetLastError();
}

static cudaError_t launch_gnorm(const sp_group* g, const double* w, const int* act, double* part, double* hn,
                                double* inv, cudaStream_t st) {
  cudaError_t e = launch_gdots(g, w, 0, 1, w, act, part, st);
  if (e != cudaSuccess) return e;
  k_gnorm<<<g->n, kVecThreads, 0, st>>>(part, g->vrecs, act, hn, inv);
  return cudaGetLastError();
}

static cudaError_t launch_gaxpy(const sp_group* g, const double* V, int k, const double* h, double* w, const int* act,
                                cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  k_gaxpy<<<g->eblocks, kVecThreads, 0, st>>>(V, g->len, k, h, g->n, w, g->vrecs, g->einst, act);
  return cudaGetLastError();
}

static cudaError_t launch_gscale(const sp_group* g, double* dst, const double* src, const double* s, const int* mask,
                                 cudaStream_t st) {
  k_gscale<<<g->eblocks, kVecThreads, 0, st>>>(dst, src, s, g->vrecs, g->einst, mask);
  return cudaGetLastError();
}

// per-member norms |x_i| on the host (synchronises st); act may be null
static sp_status group_norms(sp_group* g, const double* x, const int* act, double* out, cudaStream_t st) {
  sp_status s;
  if ((s = gcuda(g, launch_gnorm(g, x, act, g->part, g->scal, g->scal + g->n, st), "norms")) != SP_OK) return s;
  if ((s = gcuda(g, cudaMemcpyAsync(g->host, g->scal, g->n * 8, cudaMemcpyDeviceToHost, st), "norms copy")) != SP_OK)
    return s;
  if ((s = gcuda(g, cudaStreamSynchronize(st), "norms sync")) != SP_OK) return s;
  for (int i = 0; i < g->n; ++i) out[i] = g->host[i];
  return SP_OK;
}

// ---------------------------------------------------------------- entry points
extern "C" sp_status sp_group_step(sp_group* g, const double* U, double* G, void* stream) {
  if (!g || !U || !G || U == G) return gfail(g, SP_EINVAL, "sp_group_step: bad pointers");
  return group_step(g, U, G, nullptr, (cudaStream_t)stream);
}

extern "C" sp_status sp_group_set_base(sp_group* g, const double* U, void* stream) {
  if (!g || !U) return gfail(g, SP_EINVAL, "sp_group_set_base: bad pointers");
  return group_base(g, U, true, nullptr, (cudaStream_t)stream);
}

extern "C" sp_status sp_group_jvp(sp_group* g, const double* du, double* Jdu, void* stream) {
  if (!g || !du || !Jdu || du == Jdu) return gfail(g, SP_EINVAL, "sp_group_jvp: bad pointers");
  for (sp_ctx* c : g->mem)
    if (!c->has_base) return gfail(g, SP_EINVAL, "sp_group_jvp: call sp_group_set_base first");
  return group_jvp(g, du, Jdu, nullptr, (cudaStream_t)stream);
}

extern "C" sp_status sp_group_inner(sp_group* g, const double* a, const double* b, double* out_host, void* stream) {
  if (!g || !a || !b || !out_host) return gfail(g, SP_EINVAL, "sp_group_inner: bad pointers");
  cudaStream_t st = (cudaStream_t)stream;
  sp_status s;
  if ((s = gcuda(g, launch_ghdots(g, a, 0, 1, b, nullptr, g->part, g->scal, st), "inner")) != SP_OK) return s;
  if ((s = gcuda(g, cudaMemcpyAsync(g->host, g->scal, g->n * 8, cudaMemcpyDeviceToHost, st), "inner copy")) != SP_OK)
    return s;
  if ((s = gcuda(g, cudaStreamSynchronize(st), "inner sync")) != SP_OK) return s;
  for (int i = 0; i < g->n; ++i) out_host[i] = g->host[i];
  return SP_OK;
}

// ================================================================= Newton
namespace {

// device scratch of the lock-step Newton iteration, carved from g->kry
struct GNewtonMem {
  double *V, *F, *FT, *Ut;    // K+2 basis vectors, residual, trial residual, trial state
  double *part;               // partial sums [(K+2)][vblocks]
  double *hA, *hB, *y;        // [(K+3)][n] each (row-major over rows, member fastest)
  double *hn, *inv, *s;       // [n] each
  double *wn, *wdummy;        // [n] each: |w| before the first pass
  int* flag;                  // [n]: second Gram-Schmidt pass needed
  // pinned host mirrors
  double *hA_h, *hB_h, *hn_h, *y_h;
};

}  // namespace

static sp_status group_newton_mem(sp_group* g, int K, GNewtonMem* m) {
  const size_t L = g->len, n = (size_t)g->n;
  const size_t vec = (size_t)(K + 5) * L;
  const size_t extra = (size_t)(K + 2) * g->vblocks + 3 * (size_t)(K + 3) * n + 6 * n + 8;
  if (g->kry_cap < K) {
    drop_graphs(g);  // graphs hold pointers into the old basis
    if (g->kry) cudaFree(g->kry);
    g->kry = nullptr;
    g->kry_cap = 0;
    if (cudaMalloc((void**)&g->kry, (vec + extra) * 8) != cudaSuccess) {
      cudaGetLastError();
      return gfail(g, SP_ENOMEM, "group Krylov basis allocation");
    }
    g->kry_cap = K;
  }
  const size_t host_len = 3 * (size_t)(g->kry_cap + 3) * n + n;
  if (g->kry_host_len < host_len) {
    drop_graphs(g);  // graphs copy into the pinned buffers
    if (g->kry_host) cudaFreeHost(g->kry_host);
    g->kry_host = nullptr;
    g->kry_host_len = 0;
    if (cudaMallocHost((void**)&g->kry_host, host_len * 8) != cudaSuccess) {
      cudaGetLastError();
      return gfail(g, SP_ENOMEM, "group pinned scratch");
    }
    g->kry_host_len = host_len;
  }
  // the layout depends on the capacity, not on K, so graphs stay valid for smaller K
  const int Kc = g->kry_cap;
  double* p = g->kry;
  m->V = p;
  m->F = p + (size_t)(Kc + 2) * L;
  m->FT = m->F + L;
  m->Ut = m->FT + L;
  m->part = p + (size_t)(Kc + 5) * L;
  m->hA = m->part + (size_t)(Kc + 2) * g->vblocks;
  m->hB = m->hA + (size_t)(Kc + 3) * n;
  m->y = m->hB + (size_t)(Kc + 3) * n;
  m->hn = m->y + (size_t)(Kc + 3) * n;
  m->inv = m->hn + n;
  m->s = m->inv + n;
  m->wn = m->s + n;
  m->wdummy = m->wn + n;
  m->flag = reinterpret_cast<int*>(m->wdummy + n);
  const size_t hl = (size_t)(Kc + 3) * n;
  m->hA_h = g->kry_host;
  m->hB_h = m->hA_h + hl;
  m->y_h = m->hB_h + hl;
  m->hn_h = m->y_h + hl;
  return SP_OK;
}

// one lock-step Arnoldi step: w = J v_j for the active members, Gram-Schmidt against
// v_0..v_j (second pass where needed), normalisation into v_{j+1}; h columns and
// |w| copied to the host
static sp_status group_arnoldi(sp_group* g, const GNewtonMem& m, int j, bool capturing, cudaStream_t st) {
  const double* vj = m.V + (size_t)j * g->len;
  double* w = m.V + (size_t)(j + 1) * g->len;
  const int n = g->n, k = j + 1;
  cudaEvent_t* ev = g->ev_step.data() + 3 * (size_t)j;
  auto rec = [&](cudaEvent_t e) {
    return capturing ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal) : cudaEventRecord(e, st);
  };
  sp_status s;
  if ((s = gcuda(g, rec(ev[0]), "event")) != SP_OK) return s;
  if ((s = group_jvp(g, vj, w, g->act, st)) != SP_OK) return s;
  if ((s = gcuda(g, rec(ev[1]), "event")) != SP_OK) return s;
  // classical Gram-Schmidt, with the second pass only for the members that need it
  if ((s = gcuda(g, launch_ghdots(g, m.V, g->len, k, w, g->act, m.part, m.hA, st), "dots")) != SP_OK) return s;
  if ((s = gcuda(g, launch_gnorm(g, w, g->act, m.part, m.wn, m.wdummy, st), "norm")) != SP_OK) return s;
  k_greorth_decide<<<n, 32, 0, st>>>(m.hA, n, k, m.wn, g->act, m.flag, m.hB);
  if ((s = gcuda(g, cudaGetLastError(), "decide")) != SP_OK) return s;
  if ((s = gcuda(g, launch_gaxpy(g, m.V, k, m.hA, w, g->act, st), "axpy")) != SP_OK) return s;
  if ((s = gcuda(g, launch_ghdots(g, m.V, g->len, k, w, m.flag, m.part, m.hB, st), "dots")) != SP_OK) return s;
  if ((s = gcuda(g, launch_gaxpy(g, m.V, k, m.hB, w, m.flag, st), "axpy")) != SP_OK) return s;
  if ((s = gcuda(g, launch_gnorm(g, w, g->act, m.part, m.hn, m.inv, st), "norm")) != SP_OK) return s;
  if ((s = gcuda(g, launch_gscale(g, w, w, m.inv, g->act, st), "scale")) != SP_OK) return s;
  const size_t hb = (size_t)k * n * 8;
  if ((s = gcuda(g, cudaMemcpyAsync(m.hA_h, m.hA, hb, cudaMemcpyDeviceToHost, st), "h copy")) != SP_OK) return s;
  if ((s = gcuda(g, cudaMemcpyAsync(m.hB_h, m.hB, hb, cudaMemcpyDeviceToHost, st), "h copy")) != SP_OK) return s;
  if ((s = gcuda(g, cudaMemcpyAsync(m.hn_h, m.hn, n * 8, cudaMemcpyDeviceToHost, st), "h copy")) != SP_OK) return s;
  return gcuda(g, rec(ev[2]), "event");
}

extern "C" sp_status sp_group_newton_gmres(sp_group* g, double* U, const sp_newton_opts* o, int use_graphs,
                                           sp_newton_report* reps, void* stream) {
  if (!g || !U || !o) return gfail(g, SP_EINVAL, "sp_group_newton_gmres: bad arguments");
  if (o->use_fd || o->use_gradient || o->int_steps > 1 || o->krylov != 0)
    return gfail(g, SP_EINVAL, "sp_group_newton_gmres: single-step tangent actions only "
                               "(use_fd = use_gradient = krylov = 0, int_steps <= 1)");
  const int K = o->max_krylov;
  if (K < 1 || K > 4096 || o->max_newton < 0) return gfail(g, SP_EINVAL, "sp_group_newton_gmres: bad options");
  const int n = g->n;
  GNewtonMem m;
  sp_status s = group_newton_mem(g, K, &m);
  if (s != SP_OK) return s;
  while ((int)g->ev_step.size() < 3 * (g->kry_cap + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return gfail(g, SP_ECUDA, "events");
    g->ev_step.push_back(e);
  }
  cudaStream_t ust = (cudaStream_t)stream, st = g->st;
  // the private stream (capturable) starts after the caller's earlier work
  if ((s = gcuda(g, cudaEventRecord(g->ev_in, ust), "event")) != SP_OK) return s;
  if ((s = gcuda(g, cudaStreamWaitEvent(st, g->ev_in, 0), "wait")) != SP_OK) return s;
  const double t0 = now_ms();
  std::vector<sp_newton_report> r(n);
  std::vector<double> nF(n), nT(n), delta(n), pred(n), ylen(n), nU(n);
  // status per member: 0 iterating, 1 converged, 2 stopped (no acceptable step), 3 non-finite
  std::vector<int> stat(n, 0);
  const int LD = K + 2;
  std::vector<std::vector<double>> H(n), R(n), gv(n), cs(n), sn(n);
  std::vector<int> kk(n, 0), run(n, 0), gm(n, 0), tr(n, 0);
  std::vector<Hookstep> hs(n);
  double t_action = 0, t_orth = 0;
  // the mask goes through one pinned buffer: wait until its previous upload has run
  auto upload_act = [&](const std::vector<int>& mask) -> sp_status {
    sp_status q = gcuda(g, cudaStreamSynchronize(st), "mask sync");
    if (q != SP_OK) return q;
    for (int i = 0; i < n; ++i) g->act_h[i] = mask[i];
    return gcuda(g, cudaMemcpyAsync(g->act, g->act_h, n * sizeof(int), cudaMemcpyHostToDevice, st), "mask");
  };
  auto count = [](const std::vector<int>& v) { return std::count_if(v.begin(), v.end(), [](int x) { return x != 0; }); };

  if ((s = group_step(g, U, m.F, nullptr, st)) != SP_OK) return s;
  if ((s = group_norms(g, m.F, nullptr, nF.data(), st)) != SP_OK) return s;
  if ((s = group_norms(g, U, nullptr, nU.data(), st)) != SP_OK) return s;
  for (int i = 0; i < n; ++i) {
    r[i].total_steps = 1;
    r[i].norm_F0 = nF[i];
    delta[i] = o->delta0 > 0 ? o->delta0 : 0.1 * std::max(nU[i], 1.0);
    H[i].assign((size_t)LD * (K + 1), 0.0);
    R[i].assign((size_t)LD * (K + 1), 0.0);
    gv[i].assign(K + 2, 0.0);
    cs[i].assign(K + 1, 0.0);
    sn[i].assign(K + 1, 0.0);
  }
  for (int it = 0; it <= o->max_newton; ++it) {
    for (int i = 0; i < n; ++i) {
      if (stat[i] != 0) continue;
      if (!std::isfinite(nF[i])) stat[i] = 3;
      else if (nF[i] < o->tol) stat[i] = 1;
    }
    for (int i = 0; i < n; ++i) run[i] = stat[i] == 0;
    if (it == o->max_newton || count(run) == 0) break;
    if ((s = upload_act(run)) != SP_OK) return s;
    if ((s = group_base(g, U, false, g->act, st)) != SP_OK) return s;
    // v_0 = F / |F| per member
    for (int i = 0; i < n; ++i) g->host[i] = run[i] ? 1.0 / nF[i] : 0.0;
    if ((s = gcuda(g, cudaMemcpyAsync(m.s, g->host, n * 8, cudaMemcpyHostToDevice, st), "scales")) != SP_OK) return s;
    if ((s = gcuda(g, launch_gscale(g, m.V, m.F, m.s, g->act, st), "v0")) != SP_OK) return s;
    for (int i = 0; i < n; ++i) {
      std::fill(gv[i].begin(), gv[i].end(), 0.0);
      gv[i][0] = nF[i];
      kk[i] = 0;
      gm[i] = run[i];
    }
    // ---- lock-step GMRES
    for (int j = 0; j < K && count(gm) > 0; ++j) {
      if ((s = upload_act(gm)) != SP_OK) return s;
      bool launched = false;
      if (use_graphs) {
        auto itg = g->graphs.find(j);
        if (itg == g->graphs.end()) {
          cudaGraph_t graph = nullptr;
          cudaGraphExec_t exec = nullptr;
          bool ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
          sp_status cs_ = ok ? group_arnoldi(g, m, j, true, st) : SP_ECUDA;
          cudaError_t ce = cudaStreamEndCapture(st, &graph);
          ok = ok && cs_ == SP_OK && ce == cudaSuccess && graph &&
               cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
          if (graph) cudaGraphDestroy(graph);
          if (!ok) {
            cudaGetLastError();
            if (exec) cudaGraphExecDestroy(exec);
            return gfail(g, SP_ECUDA, "sp_group_newton_gmres: graph capture of the Arnoldi step failed");
          }
          itg = g->graphs.emplace(j, exec).first;
        }
        if ((s = gcuda(g, cudaGraphLaunch(itg->second, st), "graph launch")) != SP_OK) return s;
        launched = true;
      }
      if (!launched && (s = group_arnoldi(g, m, j, false, st)) != SP_OK) return s;
      if ((s = gcuda(g, cudaStreamSynchronize(st), "arnoldi sync")) != SP_OK) return s;
      float ta = 0, tb = 0;
      cudaEvent_t* ev = g->ev_step.data() + 3 * (size_t)j;
      if (cudaEventElapsedTime(&ta, ev[0], ev[1]) == cudaSuccess) t_action += ta;
      else cudaGetLastError();  // timing is best effort; keep the error state clean
      if (cudaEventElapsedTime(&tb, ev[1], ev[2]) == cudaSuccess) t_orth += tb;
      else cudaGetLastError();
      for (int i = 0; i < n; ++i) {
        if (!gm[i]) continue;
        double* Hc = H[i].data() + (size_t)j * LD;
        double* Rc = R[i].data() + (size_t)j * LD;
        for (int q = 0; q <= j; ++q) Hc[q] = m.hA_h[(size_t)q * n + i] + m.hB_h[(size_t)q * n + i];
        const double hn = m.hn_h[i];
        Hc[j + 1] = hn;
        givens_column(Hc, Rc, j, cs[i].data(), sn[i].data(), gv[i].data());
        kk[i] = j + 1;
        r[i].total_jvps++;
        if (!std::isfinite(hn)) {
          stat[i] = 3;
          gm[i] = 0;
          run[i] = 0;
          continue;
        }
        if (std::fabs(gv[i][j + 1]) <= o->eta * nF[i] || hn == 0.0) gm[i] = 0;
      }
    }
    // ---- hookstep trials, all members that need one in lock step
    for (int i = 0; i < n; ++i) {
      if (run[i] && kk[i] > 0) r[i].lin_rel = std::fabs(gv[i][kk[i]]) / nF[i];
      tr[i] = run[i] && kk[i] > 0;
      if (tr[i]) {
        hs[i].init(R[i].data(), LD, kk[i], gv[i].data());
        r[i].newton_len = hs[i].ny0;
      }
    }
    for (int trial = 0; trial < 12 && count(tr) > 0; ++trial) {
      std::vector<int> acc(n, 0);
      int kmax = 0;
      std::fill(m.y_h, m.y_h + (size_t)(K + 3) * n, 0.0);
      for (int i = 0; i < n; ++i) {
        if (!tr[i]) continue;
        const std::vector<double> y = hs[i].solve(delta[i], &pred[i], &ylen[i]);
        for (int q = 0; q < kk[i]; ++q) m.y_h[(size_t)q * n + i] = y[q];
        kmax = std::max(kmax, kk[i]);
      }
      if ((s = upload_act(tr)) != SP_OK) return s;
      if ((s = gcuda(g, cudaMemcpyAsync(m.y, m.y_h, (size_t)kmax * n * 8, cudaMemcpyHostToDevice, st), "y")) != SP_OK)
        return s;
      // U_trial = U - sum_q y_q v_q, then its residual
      if ((s = gcuda(g, launch_gscale(g, m.Ut, U, nullptr, g->act, st), "copy")) != SP_OK) return s;
      if ((s = gcuda(g, launch_gaxpy(g, m.V, kmax, m.y, m.Ut, g->act, st), "update")) != SP_OK) return s;
      if ((s = group_step(g, m.Ut, m.FT, g->act, st)) != SP_OK) return s;
      if ((s = group_norms(g, m.FT, g->act, nT.data(), st)) != SP_OK) return s;
      for (int i = 0; i < n; ++i) {
        if (!tr[i]) continue;
        r[i].total_steps++;
        r[i].hook_trials++;
        if (trust_update(nF[i], pred[i], nT[i], ylen[i], &delta[i])) {
          acc[i] = 1;
          tr[i] = 0;
          nF[i] = nT[i];
          r[i].newton_iters++;
        }
      }
      // accepted members take the trial state and its residual now (their slices of
      // Ut and FT are not touched by later trials of the others)
      if (count(acc) > 0) {
        if ((s = upload_act(acc)) != SP_OK) return s;
        if ((s = gcuda(g, launch_gscale(g, U, m.Ut, nullptr, g->act, st), "accept")) != SP_OK) return s;
        if ((s = gcuda(g, launch_gscale(g, m.F, m.FT, nullptr, g->act, st), "accept")) != SP_OK) return s;
      }
    }
    for (int i = 0; i < n; ++i)
      if (tr[i]) stat[i] = 2;  // no acceptable step within the trials: stop this member
  }
  if ((s = gcuda(g, cudaStreamSynchronize(st), "newton sync")) != SP_OK) return s;
  const double ttot = now_ms() - t0;
  sp_status result = SP_OK;
  for (int i = 0; i < n; ++i) {
    if (stat[i] == 0 && nF[i] < o->tol) stat[i] = 1;
    r[i].norm_F = nF[i];
    r[i].delta = delta[i];
    r[i].t_action_ms = t_action;
    r[i].t_orth_ms = t_orth;
    r[i].t_total_ms = ttot;
    if (stat[i] == 3) result = SP_ENAN;
    else if (stat[i] != 1 && result == SP_OK) result = SP_ENOTCONV;
  }
  if (reps)
    for (int i = 0; i < n; ++i) reps[i] = r[i];
  if (result == SP_ENOTCONV) g->err = "Newton did not reach the tolerance on every member";
  if (result == SP_ENAN) g->err = "non-finite residual on a member";
  return result;
}
