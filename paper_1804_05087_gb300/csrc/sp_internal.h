// Internal declarations of the stokesprec library: the context, the complex
// helper type and the kernel launchers shared by the translation units.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <utility>
#include <vector>

#include "stokesprec.h"

// ------------------------------------------------------------------ complex
template <typename T>
struct C2 {
  T x, y;
};

template <typename T>
__host__ __device__ inline C2<T> mk(T a, T b) {
  C2<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T>
__host__ __device__ inline C2<T> operator+(C2<T> a, C2<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T>
__host__ __device__ inline C2<T> operator-(C2<T> a, C2<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T>
__host__ __device__ inline C2<T> operator*(C2<T> a, C2<T> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__host__ __device__ inline C2<T> scl(C2<T> a, T s) { return mk(a.x * s, a.y * s); }
template <typename T>
__host__ __device__ inline C2<T> conj2(C2<T> a) { return mk(a.x, -a.y); }
// multiply by i*s (s = +1 or -1)
template <typename T>
__host__ __device__ inline C2<T> mul_is(C2<T> a, T s) { return mk(-s * a.y, s * a.x); }

// ----------------------------------------------------------------- FFT plan
// Mixed-radix (2, 3, 4) Stockham plan for one transform length.
struct FftPlan {
  int n;
  int nst;
  int radix[12];
};

// contexts whose batches reach this many directions solve the tangent's per-mode
// problems with the O(N) chains (one thread per mode, parity and direction)
constexpr int kChainMinBatch = 32;
constexpr int kChainMaxRows = 512;  // the chains' table of row indices as doubles covers N < 512

// band of the pipe's radial factors: the 9-point stencils reach 6 rows below and 8 above the
// diagonal (wall rows one-sided, axis rows folded onto their mirror points), and the row
// interchanges of partial pivoting widen the upper band to 6 + 8
constexpr int kPipeKL = 6;
constexpr int kPipeKW = 15;

// ------------------------------------------------------------------ context
struct sp_ctx {
  sp_config cfg;
  int geom = 0;                  // 0 plane Couette, 1 pipe (sp_pipe_create)
  sp_pipe_config pcfg{};
  int dev = 0;
  int sm_count = 0;
  int nx = 0, ny = 0, nz = 0;
  int N = 0, NH = 0;             // Chebyshev degree, N/2 + 1
  int Kx = 0, Kz = 0, MX = 0, MZ = 0, NY = 0, Mm = 0;
  int n_unique = 0;              // modes solved: (Kx+1) MZ + Kx (MZ-1)
  double alpha = 0, beta = 0, nu = 0, dt = 0;
  size_t state_len = 0;          // doubles per state
  size_t cplx_per_state = 0;     // complex values per state (pipe: + 1 for the speed)
  size_t field_cplx = 0;         // complex values of the velocity field, 3 Mm NY
  FftPlan px{}, pz{};
  // per-mode solve operators: V0, V1, H0, H1, FP64, column-major (element (row, col) at
  // col * rows + row, so that threads on consecutive rows read consecutive addresses)
  int nv0 = 0, nv1 = 0, cv = 0;  // rows of V0 / V1 (and H0 / H1); cv = N/2: RHS stride
  int rb0 = 0, rb1 = 0;          // columns of V0, H0 / V1, H1: momentum rows of each parity
  int off_v0 = 0, off_v1 = 0, off_h0 = 0, off_h1 = 0, op_stride = 0;
  // laminar advection in L (cfg.lam_adv): complex V' and H' per mode, (N - 1) columns of
  // N + 1 complex rows, column-major (the mean mode keeps H0 / H1)
  int off_vc = 0, off_hc = 0;
  // O(N) per-mode solve of the batched tangent (solve_chain.cu; plan.cpp describes the
  // records): used when cfg.max_batch >= kChainMinBatch and lam_adv = 0
  int use_chain = 0;
  int chain_par = 0, chain_stride = 0;  // doubles per parity record / per mode

  // device tables
  double *Th = nullptr, *TDh = nullptr, *Cfh = nullptr;
  // two-level split of k_yinv (N divisible by 4): Tp, TDp [N/4+1][NY], tq [N/4+1] (kernels.cu)
  double *Tp = nullptr, *TDp = nullptr, *tq = nullptr;
  float *Tp_f = nullptr, *TDp_f = nullptr, *tq_f = nullptr;
  // the same for the forward transform of k_rhs: Cq[n][jq] = 2 / (N cbar_n) cos(pi jq n / N), even
  // rows n <= N-2, jq <= N/4 (solve_chain.cu)
  double* Cq = nullptr;
  float* Cq_f = nullptr;
  // tensor-core inverse transform (41 <= NY <= 72): shared-memory image of T and T' split into
  // TF32 hi and lo parts (yinv_tc.cu)
  float* yinv_tc_mat = nullptr;
  // forward transform on the tensor cores: C_hi, C_lo (yinv_tc.cu)
  float* rhs_tc_mat = nullptr;
  double* yv = nullptr;          // [NY] wall-normal points: cos(pi j / N) (Couette), r_j (pipe)
  double* lam6 = nullptr;        // [NY][6] laminar (U, Omega) per plane: (y,0,0,0,0,-1) / (0,0,1-r^2,0,2r,0)
  float *Th_f = nullptr, *TDh_f = nullptr, *Cfh_f = nullptr;
  double2 *twx = nullptr, *twz = nullptr;
  float2 *twx_f = nullptr, *twz_f = nullptr;
  double* ops = nullptr;
  double* chain = nullptr;       // [n_unique][2 parities][chain_par]
  // pipe: per-mode dense operators (3 NY x 3 NY, column-major), radial FD band (D1) tables
  // pipe: banded LU factors of the per-mode radial problems (plan_pipe.cpp), matrices
  // 0 pressure, 1 u+, 2 u-, 3 u~z (mean mode: 1 u_theta, 2 u_z); one chunk of pb_chunk bytes
  // per (mode, matrix): U [NR][kPipeKW] (entry 0 = 1 / diagonal), L [NR][kPipeKL] multipliers,
  // row interchanges [NR] int32, zero-padded to a multiple of 16 bytes
  unsigned char* pb_fac = nullptr;  // [n_unique][4][pb_chunk]
  size_t pb_chunk = 0;
  double* pb_uh = nullptr;    // [n_unique][3][NR] (u+, u-, u~z) driven by the unit wall pressure
  double* pb_dinv = nullptr;  // [n_unique] 1 / (wall divergence of pb_uh)
  double* fd_w1 = nullptr;       // [2 parities][NY][9] weights of the first derivative
  int* fd_c1 = nullptr;          // [2][NY][9] columns
  double* dzU = nullptr;         // d/dz of the (projected) linearisation point, one state
  // device workspaces
  void* ws6 = nullptr;           // [batch][6][NY][Mm] complex (double-sized)
  void* ws3 = nullptr;           // [batch][3][NY][Mm] complex (double-sized)
  double* base64 = nullptr;      // [6][NY][nx][nz]
  float* base32 = nullptr;
  float* base32t = nullptr;      // [6][NY][nz][nx]: transposed copy for the register-FFT kernel
  double* U0 = nullptr;          // linearisation point
  double* G0 = nullptr;          // G(U0)
  double* tmp = nullptr;         // [batch] states
  double* red = nullptr;         // reduction partials
  double* red_host = nullptr;    // pinned
  double* kry_host = nullptr;    // pinned: two Hessenberg columns of sp_newton_gmres
  int red_blocks = 0;
  int has_base = 0;
  int use_xz_reg = 1;            // float plane stage: register FFT kernel when the size allows
  int use_xz_reg64 = 1;          // FP64 tangent/adjoint plane stage: register FFT kernel (xz_reg64.cu)
  int use_rhs_tc = 0;             // float forward transform of the chains on the tensor cores (yinv_tc.cu)
  int use_yinv_tc = 1;           // float inverse Chebyshev transform on the tensor cores (yinv_tc.cu)
  int solve_shape_tan = 0;       // k_solve tile shape of the tangent (sp_autotune)
  int solve_shape_step = 0;      // k_solve tile shape of the FP64 step
  // sizes of shared memory per kernel (bytes)
  size_t smem_xz64 = 0, smem_xz32 = 0;
  int xz_rp64 = 1, xz_rp32 = 1;
  int xz_cx64 = 1, xz_cx32 = 1;
  int xz_gglob64 = 0, xz_gglob32 = 0;  // plane buffer in global memory (grid too large for chip)
  void* wsG = nullptr;           // [batch][NY][nx * RS] complex, only when a plane does not fit
  std::string err;
  // tracing: event pairs per stage, recorded while `trace` is on
  bool trace = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> trace_ev[SP_NSTAGE];
  std::vector<cudaEvent_t> ev_pool;
  // Newton scratch
  double* kry = nullptr;         // Krylov basis [max_krylov+1] states
  int kry_cap = 0;
  // multi-step map B^n (sp_step_n / sp_set_base_n / sp_jvp_n)
  double* traj = nullptr;        // [traj_cap] states: U_0 .. U_{n-1} of the last sp_set_base_n
  int traj_cap = 0;
  int traj_n = 0;                // steps of the stored trajectory (0: none)
  // base fields of every trajectory step, in the precision the tangent reads (float base32 and
  // base32t in mixed mode, base64 in FP64), so that sp_jvp_n does not recompute them; not
  // kept (traj_base_n = 0) when they would take more than a quarter of the free memory
  unsigned char* traj_base = nullptr;
  size_t traj_base_bytes = 0;
  int traj_base_n = 0;
  double* nbuf = nullptr;        // [2] states: scratch of sp_step_n
  // host-buffer tangent (sp_jvp_host): two copy streams, double-buffered device slots
  cudaStream_t hs_in = nullptr, hs_out = nullptr;
  cudaEvent_t hev_start = nullptr, hev_in[2] = {}, hev_comp[2] = {}, hev_out[2] = {};
  double* hbuf = nullptr;        // [4][hchunk] states: in0, in1, out0, out1
  int hchunk = 0;
  // Newton: captured Arnoldi steps (keyed by step index), their stream and timing events
  std::map<int, cudaGraphExec_t> ngraphs;
  cudaStream_t nstream = nullptr;
  cudaEvent_t nev_in = nullptr;
  std::vector<cudaEvent_t> nev;  // 3 per Arnoldi step
};

// run `launch` (returning cudaError_t) bracketed by trace events when tracing
cudaError_t sp_traced(sp_ctx* c, int stage, cudaStream_t st, cudaError_t (*fn)(void*), void* arg);
template <class F>
cudaError_t traced(sp_ctx* c, int stage, cudaStream_t st, F&& f) {
  return sp_traced(c, stage, st, [](void* p) -> cudaError_t { return (*static_cast<F*>(p))(); }, &f);
}

// status helpers
sp_status sp_fail(sp_ctx* c, sp_status s, const std::string& msg);
sp_status sp_cuda(sp_ctx* c, cudaError_t e, const char* what);

// plan building (plan.cpp, plan_pipe.cpp)
sp_status sp_build_plan(sp_ctx* c);
sp_status sp_build_pipe_plan(sp_ctx* c);
sp_status sp_build_fft_tables(sp_ctx* c);
void sp_unique_mode(const sp_ctx* c, int u, int* pos, int* iz);

// pipe kernels (pipe.cu)
cudaError_t launch_pvals(const sp_ctx* c, bool fp32, const double* in, void* out6, int n_dir, cudaStream_t st);
cudaError_t launch_psolve(const sp_ctx* c, bool fp32, bool tangent, const void* in3, const double* u,
                          double* out, int n_dir, cudaStream_t st);
cudaError_t launch_pipe_dz(const sp_ctx* c, const double* U, double* dzU, cudaStream_t st);
cudaError_t launch_pipe_seed(const sp_ctx* c, const double* streak, const double* pol, int npoly, double* A,
                             double* B, cudaStream_t st);

// shared-memory sizing of k_xz; false if even the FP32 variant cannot fit
bool sp_xz_fits(sp_ctx* c);
size_t sp_xz_global_plane_bytes(const sp_ctx* c);  // per direction, 0 if every plane fits on chip

// ------------------------------------------------------------ grouped launches
// One launch over the blocks of several contexts (the members of an sp_group):
// block b belongs to member inst[b] and is that member's block b - first[inst[b]]
// of its own launch. recs is a device array of per-member launch records.
struct GrpKernel {
  void* recs = nullptr;
  int* inst = nullptr;
  int* first = nullptr;
  int blocks = 0;
  size_t smem = 0;
};
constexpr int kGrpRegClasses = 5;  // register-FFT plane kernels: grids 16, 24, 32, 48, 64
struct GrpPlan {
  int n = 0;
  int lam_adv = 0;                // every member has laminar advection in L (else none has)
  GrpKernel yinv64, yinv32, xz64, solve64, solve32;
  GrpKernel xz32;                 // float plane stage of the members without a register-FFT kernel
  GrpKernel xzr[kGrpRegClasses];  // float plane stage of the others, per grid size class (xz_reg.cu)
};
// members: n contexts; offs: offset (doubles) of each member's state in a group
// vector; order: member indices, largest first (blocks are laid out in this order)
cudaError_t grp_plan_build(GrpPlan* p, sp_ctx* const* members, int n, const size_t* offs, const int* order);
void grp_plan_free(GrpPlan* p);
// active: device int [n] (nonzero = run this member) or null for all
cudaError_t grp_launch_yinv(const GrpPlan& p, bool fp32, const double* in_base, const int* active, cudaStream_t st);
cudaError_t grp_launch_xz(const GrpPlan& p, bool fp32, int mode, const int* active, cudaStream_t st);
cudaError_t grp_launch_solve(const GrpPlan& p, bool fp32, const double* du_base, double* out_base,
                             const int* active, cudaStream_t st);
// register-FFT plane stage over the members with use[m] != 0, one launch per grid
// size class (xz_reg.cu); ks: kGrpRegClasses kernels
cudaError_t grp_build_xz_reg(GrpKernel* ks, sp_ctx* const* members, int n, const int* order,
                             const std::vector<int>& use);
cudaError_t grp_launch_xz_reg(const GrpKernel* ks, const int* active, cudaStream_t st);
// device copy of a host table; frees nothing on failure
cudaError_t grp_upload(void** dst, const void* src, size_t bytes);
void grp_kernel_free(GrpKernel* k);

// kernel launchers (kernels.cu); all asynchronous on `st`
// XZ_STEP_BASE: the step's product and, from the same inverse transforms, the base fields
enum XzMode { XZ_STEP = 0, XZ_TANGENT = 1, XZ_BASE = 2, XZ_ADJOINT = 3, XZ_STEP_BASE = 4 };
cudaError_t launch_yinv(const sp_ctx* c, bool fp32, const double* in, void* out6, int n_dir,
                        cudaStream_t st);
cudaError_t launch_xz(const sp_ctx* c, bool fp32, int mode, const void* in6, void* out3,
                      int n_dir, cudaStream_t st);
// float plane stage with register-resident FFTs (xz_reg.cu), square grids 16..64
bool sp_xz_reg_supported(const sp_ctx* c);
cudaError_t launch_xz_reg(const sp_ctx* c, int mode, const void* in, void* out, int n_dir, cudaStream_t st);
// float inverse Chebyshev transform + curl on the tensor cores (yinv_tc.cu); same inputs and
// outputs as launch_yinv with fp32; yinv_tc_image: the host image of the constant operands from the
// full tables th[j][n] = T_n(y_j), td[j][n] = T_n'(y_j) (NY x NY, row-major)
bool sp_yinv_tc_supported(const sp_ctx* c);
cudaError_t launch_yinv_tc(const sp_ctx* c, const double* in, void* out6, int n_dir, cudaStream_t st);
std::vector<float> yinv_tc_image(const double* th, const double* td, int NY);
// float forward transform + u/dt of the chains' right-hand sides on the tensor cores (yinv_tc.cu):
// same inputs and outputs as launch_chain_rhs with fp32; W strides su, sd, sn
bool sp_rhs_tc_supported(const sp_ctx* c);
cudaError_t launch_rhs_tc(const sp_ctx* c, const void* in3, const double* du, void* work, int n_dir, long long su,
                          long long sd, long long sn, cudaStream_t st);
std::vector<float> rhs_tc_image(const double* cf, int NY, int NR);
size_t yinv_tc_smem(int NY);
// FP64 plane stage with register-resident FFTs (xz_reg64.cu), square grids 16..48
bool sp_xz_reg64_supported(const sp_ctx* c);
cudaError_t launch_xz_reg64(const sp_ctx* c, int mode, const void* in, void* out, int n_dir, cudaStream_t st);
// batched tangent solve by O(N) chains (solve_chain.cu), two launches: k_rhs (values ->
// right-hand sides in work, n_unique x 3 x (N-1) complex per direction), then k_chain
// (one thread per mode, parity and direction); together the same inputs and outputs as
// launch_solve.
cudaError_t launch_chain_rhs(const sp_ctx* c, bool fp32, const void* in3, const double* du, void* work, int n_dir,
                             cudaStream_t st);
cudaError_t launch_chain_solve(const sp_ctx* c, const double* du, double* out, const void* work, void* scratch,
                               int n_dir, cudaStream_t st);
size_t chain_scratch_bytes(const sp_ctx* c, int n_dir);
// the tangent's per-mode solve of one pass (abi.cu): chains or dense operators by the
// context's choice (use_chain); work: scratch of n_unique x 3 x (N-1) complex doubles
// per direction (the chains' right-hand sides; ws6 suffices); vals (vals_bytes long) is
// read by the right-hand-side launch and then serves as the chains' scratch
// (chain_scratch_bytes); if it is too small the dense operators solve instead
sp_status sp_tangent_solve(sp_ctx* c, bool f32, void* vals, size_t vals_bytes, const double* du, double* out,
                           void* work, int nb, cudaStream_t st);
// shape: index into the tile-shape table (sp_solve_shapes); -1 = the context's tangent choice
cudaError_t launch_solve(const sp_ctx* c, bool fp32, const void* in3, const double* du,
                         double* out, int n_dir, cudaStream_t st, int shape = -1);
// the tile shapes of k_solve (modes per block, threads per block); returns their number
int sp_solve_shapes(const sp_ctx* c, int* tm, int* threads);
cudaError_t launch_base_to_f32(const sp_ctx* c, cudaStream_t st);
// adjoint chain (sp_vjp): solve^T + Chebyshev^T, plane stage^T (launch_xz with
// XZ_ADJOINT), values^T + curl^T, then weights and the Hermitian projection
cudaError_t launch_solve_adj(const sp_ctx* c, bool fp32, const double* r, double* out, void* vals3,
                             int n_dir, bool weighted, cudaStream_t st);
cudaError_t launch_yinv_adj(const sp_ctx* c, bool fp32, const void* in6, double* out, int n_dir,
                            cudaStream_t st);
cudaError_t launch_finish_adj(const sp_ctx* c, const double* r, double* out, int n_dir, bool weighted,
                              cudaStream_t st);
cudaError_t launch_seed(const sp_ctx* c, const double* ra, const double* rb, const double* rc,
                        double* U, cudaStream_t st);
cudaError_t launch_scale(double* x, double s, size_t n, cudaStream_t st);
cudaError_t launch_axpby(double* out, double a, const double* x, double b, const double* y,
                         size_t n, cudaStream_t st);
cudaError_t launch_inner_partials(const sp_ctx* c, const double* a, const double* b,
                                  double* partials, int nblocks, cudaStream_t st);
// many inner products <V_i, w> for i < k in one pass: partials [k][nblocks]
cudaError_t launch_multi_inner(const sp_ctx* c, const double* V, int k, const double* w,
                               double* partials, int nblocks, cudaStream_t st);
// device-resident Arnoldi: out[i] = <V_i, w> (+ add[i]); h = |w|, inv = 1/|w|; x *= *s
// gate: device int; when it holds 0 the launches return at once (null: always run)
cudaError_t launch_dev_dots(const sp_ctx* c, const double* V, int k, const double* w, double* partials,
                            int nblocks, double* out, const double* add, cudaStream_t st,
                            const int* gate = nullptr);
cudaError_t launch_dev_norm(const sp_ctx* c, const double* w, double* partials, int nblocks, double* h,
                            double* inv, cudaStream_t st);
cudaError_t launch_scale_dev(const sp_ctx* c, double* x, const double* s, cudaStream_t st);
// w -= sum_i h_i V_i (h on device)
// partial weighted dot products <V[i], w> (i < k) into partials[i][nb] (kernels.cu)
// (gate: if non-null, the launch does nothing unless *gate is set)
cudaError_t launch_partial_dots(const sp_ctx* c, const double* V, int k, const double* w, double* partials, int nb,
                                cudaStream_t st, const int* gate);
// one Arnoldi column (Gram-Schmidt with selective second pass, normalisation) for small states
// (orth.cu); w must be V + k * state_len; normpart holds orth_small_blocks(c) doubles
bool orth_small_applies(const sp_ctx* c, int nb);
int orth_small_blocks(const sp_ctx* c);
cudaError_t launch_orth_small(const sp_ctx* c, const double* V, int k, double* w, double* part, int nb, double* hA,
                              double* hB, double* hn, double* host, int kh, int* flag, double* normpart,
                              cudaStream_t st);
cudaError_t launch_multi_axpy(const sp_ctx* c, const double* V, int k, const double* h,
                              double* w, cudaStream_t st, const int* gate = nullptr);
// second Gram-Schmidt pass needed? *flag = (|w|^2 - |h|^2 < |w|^2 / 2); if not, h2 = 0 (k entries)
cudaError_t launch_reorth_decide(const double* h, int k, const double* wn, int* flag, double* h2, cudaStream_t st);
