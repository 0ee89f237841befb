// Kernels of the pipe-flow step and tangent (the plane stage is k_xz of
// kernels.cu with the pipe's laminar table).
//   k_pvals : per Fourier mode, the six fields u_r, u_theta, u_z and the
//             vorticity at every radial point: omega_r = (i m/r) u_z - i k u_theta,
//             omega_theta = i k u_r - D1 u_z, omega_z = D1 u_theta + u_theta/r - (i m/r) u_r
//             (radial derivatives by the 9-point parity-aware stencils),
//             written plane-major (one radial point per plane).
//   k_psolve: per Fourier mode, the right-hand side u/dt + N + c du/dz (for the
//             tangent + dc dU/dz), rotation to u+- = u_r +- i u_theta and
//             u~_z = -i u_z, the per-mode Stokes problem by banded solves and one
//             influence coefficient (FP64), and G = u_new - u with a Hermitian output.
// Index conventions: position pos over the axial wavenumbers in FFT order
// (k = alpha kz), iz = m' (m = sym m').
#include "dev_util.h"
#include "sp_internal.h"

namespace {

constexpr int kTileP = 8;        // modes per k_pvals block
constexpr int kThreadsP = 256;

struct PArgs {
  const double* r;      // [NR]
  const double* w1;     // [2][NR][9]
  const int* c1;        // [2][NR][9]
  const unsigned char* pb_fac;  // banded factors of the per-mode radial problems (plan_pipe.cpp)
  size_t pb_chunk;
  const double* pb_uh;  // [n_unique][3][NR]
  const double* pb_dinv;
  size_t sstride;       // complex values per state (field + speed)
  int Mm, MX, MZ, Kx, NR, n_unique;
  double alpha, sym, inv_dt;
};

template <typename T>
__device__ __forceinline__ C2<T> cmk(double2 v) { return mk((T)v.x, (T)v.y); }

template <typename T>
__global__ void __launch_bounds__(kThreadsP) k_pvals(const double2* __restrict__ in, C2<T>* __restrict__ out,
                                                     PArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* su = reinterpret_cast<double2*>(smem_raw);  // [3][TM][NR]
  const int TM = kTileP, NR = a.NR, Mm = a.Mm;
  const int m0 = blockIdx.x * TM, dir = blockIdx.y;
  const double2* src = in + (size_t)dir * a.sstride;
  for (int idx = threadIdx.x; idx < 3 * TM * NR; idx += blockDim.x) {
    const int j = idx % NR, t = (idx / NR) % TM, c = idx / (NR * TM);
    const int m = m0 + t;
    su[idx] = m < Mm ? __ldg(src + ((size_t)c * Mm + m) * NR + j) : make_double2(0.0, 0.0);
  }
  __syncthreads();
  C2<T>* o = out + (size_t)dir * 6 * NR * Mm;
  for (int idx = threadIdx.x; idx < TM * NR; idx += blockDim.x) {
    const int t = idx % TM, j = idx / TM;
    const int m = m0 + t;
    if (m >= Mm) continue;
    const int pos = m / a.MZ, iz = m - pos * a.MZ;
    const int kzi = pos <= a.Kx ? pos : pos - a.MX;
    const double k = a.alpha * kzi, mm = a.sym * iz;
    const double rj = a.r[j], ir = 1.0 / rj;
    const double2* ur = su + (0 * TM + t) * NR;
    const double2* ut = su + (1 * TM + t) * NR;
    const double2* uz = su + (2 * TM + t) * NR;
    // D1 of u_z (parity of m) and of u_theta (parity of m + 1)
    const int pz = ((int)mm) & 1, pt = pz ^ 1;
    double2 dz = make_double2(0.0, 0.0), dt = dz;
    for (int q = 0; q < 9; ++q) {
      const double wz = __ldg(a.w1 + ((size_t)pz * NR + j) * 9 + q);
      const int cz = __ldg(a.c1 + ((size_t)pz * NR + j) * 9 + q);
      const double wt = __ldg(a.w1 + ((size_t)pt * NR + j) * 9 + q);
      const int ct = __ldg(a.c1 + ((size_t)pt * NR + j) * 9 + q);
      dz.x += wz * uz[cz].x;
      dz.y += wz * uz[cz].y;
      dt.x += wt * ut[ct].x;
      dt.y += wt * ut[ct].y;
    }
    const double2 vr = ur[j], vt = ut[j], vz = uz[j];
    // i m/r u_z - i k u_theta
    const double2 orr = make_double2(-mm * ir * vz.y + k * vt.y, mm * ir * vz.x - k * vt.x);
    // i k u_r - D1 u_z
    const double2 ot = make_double2(-k * vr.y - dz.x, k * vr.x - dz.y);
    // D1 u_theta + u_theta/r - i m/r u_r
    const double2 oz = make_double2(dt.x + vt.x * ir + mm * ir * vr.y, dt.y + vt.y * ir - mm * ir * vr.x);
    const size_t base = (size_t)j * Mm + m;
    o[0 * (size_t)NR * Mm + base] = cmk<T>(vr);
    o[1 * (size_t)NR * Mm + base] = cmk<T>(vt);
    o[2 * (size_t)NR * Mm + base] = cmk<T>(vz);
    o[3 * (size_t)NR * Mm + base] = cmk<T>(orr);
    o[4 * (size_t)NR * Mm + base] = cmk<T>(ot);
    o[5 * (size_t)NR * Mm + base] = cmk<T>(oz);
  }
}

__device__ __forceinline__ void unique_mode_d(int u, int Kx, int MZ, int* pos, int* iz) {
  const int first = (Kx + 1) * MZ;
  if (u < first) {
    *pos = u / MZ;
    *iz = u - *pos * MZ;
  } else {
    const int v = u - first;
    *pos = Kx + 1 + v / (MZ - 1);
    *iz = 1 + v % (MZ - 1);
  }
}

// Hermitian projection of entry (c, pos, iz, j) of a state
__device__ __forceinline__ double2 sym_load(const double2* s, int c, int pos, int iz, int j, const PArgs& a) {
  double2 v = __ldg(s + ((size_t)c * a.Mm + pos * a.MZ + iz) * a.NR + j);
  if (iz == 0) {
    const int mpos = pos == 0 ? 0 : a.MX - pos;
    const double2 w = __ldg(s + ((size_t)c * a.Mm + mpos * a.MZ) * a.NR + j);
    v = make_double2(0.5 * (v.x + w.x), 0.5 * (v.y - w.y));
  }
  return v;
}

// Banded solve of one real right-hand side in place (b: every second double, the real or the
// imaginary part of a complex vector in shared memory), with one matrix's factors from
// plan_pipe.cpp staged in shared memory: row interchanges and multipliers forward, then the upper
// band backward (two partial sums per row). NR > 0: the vector is held in registers and the loops
// are unrolled (the row interchange of step k is a select among rows k .. k + KL); NR = 0: any
// size, the vector stays in shared memory.
// (the unrolled form is one out-of-line function shared by every kernel that uses it)
template <int NR>
__device__ __noinline__ void band_solve_reg(double* b, const unsigned char* fac) {
  constexpr int KL = kPipeKL, KW = kPipeKW;
  const double* U = reinterpret_cast<const double*>(fac);
  const double* L = U + (size_t)NR * KW;
  const int* piv = reinterpret_cast<const int*>(L + (size_t)NR * KL);
  {
    double x[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) x[i] = b[2 * i];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const int p = piv[k];
      double xk = x[k];
#pragma unroll
      for (int q = 1; q <= KL; ++q) {
        if (k + q < NR) {
          const bool sw = p == k + q;
          const double t = x[k + q];
          x[k + q] = sw ? x[k] : t;
          xk = sw ? t : xk;
        }
      }
      x[k] = xk;
#pragma unroll
      for (int q = 0; q < KL; ++q)
        if (k + 1 + q < NR) x[k + 1 + q] = fma(-L[k * KL + q], xk, x[k + 1 + q]);
    }
#pragma unroll
    for (int i = NR - 1; i >= 0; --i) {
      double s0 = x[i], s1 = 0.0;
#pragma unroll
      for (int q = 1; q < KW; ++q) {
        if (i + q < NR) {
          if (q & 1) s1 = fma(-U[i * KW + q], x[i + q], s1);
          else s0 = fma(-U[i * KW + q], x[i + q], s0);
        }
      }
      x[i] = (s0 + s1) * U[i * KW];
    }
#pragma unroll
    for (int i = 0; i < NR; ++i) b[2 * i] = x[i];
  }
}

template <int NR>
__device__ __forceinline__ void band_solve_d(double* b, const unsigned char* fac, int n) {
  constexpr int KL = kPipeKL, KW = kPipeKW;
  const double* U = reinterpret_cast<const double*>(fac);
  const double* L = U + (size_t)n * KW;
  const int* piv = reinterpret_cast<const int*>(L + (size_t)n * KL);
  if constexpr (NR > 0) {
    band_solve_reg<NR>(b, fac);
  } else {
    for (int k = 0; k < n; ++k) {
      const int p = piv[k];
      double bk = b[2 * k];
      if (p != k) {
        const double t = b[2 * p];
        b[2 * p] = bk;
        bk = t;
        b[2 * k] = bk;
      }
#pragma unroll
      for (int q = 0; q < KL; ++q)
        if (k + 1 + q < n) b[2 * (k + 1 + q)] -= L[k * KL + q] * bk;
    }
    for (int i = n - 1; i >= 0; --i) {
      double s0 = b[2 * i], s1 = 0.0;
#pragma unroll
      for (int q = 1; q < KW; ++q) {
        if (i + q < n) {
          if (q & 1) s1 = fma(-U[i * KW + q], b[2 * (i + q)], s1);
          else s0 = fma(-U[i * KW + q], b[2 * (i + q)], s0);
        }
      }
      b[2 * i] = (s0 + s1) * U[i * KW];
    }
  }
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// bounded wait on an mbarrier phase; false if the limit ran out
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase) {
  for (uint32_t it = 0; it < (1u << 26); ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Shared-memory vectors are NRP >= NR entries apart, NRP = 1 mod 8: the 16 vectors that the 32 lanes
// of a warp walk through (two lanes, real and imaginary part, per vector) then start 4 banks apart
// and a warp's 8-byte accesses take the minimum two wavefronts.
__host__ __device__ __forceinline__ int psolve_nrp(int NR) { return NR + ((9 - (NR & 7)) & 7); }

// threads per block: at least two warps for the parallel phases, one per serial solve
__host__ __device__ constexpr int psolve_threads(int TM, int ND) {
  return 6 * TM * ND <= 64 ? 64 : (6 * TM * ND + 31) / 32 * 32;
}

__host__ __device__ __forceinline__ size_t psolve_smem(int TM, int ND, int NR, size_t chunk) {
  return (size_t)TM * 4 * chunk + (size_t)TM * ND * 4 * psolve_nrp(NR) * 16 + (size_t)2 * NR * 9 * (8 + 4);
}

// in3: [dir][3][NR][Mm] values of N (T); u: the states (step: the state itself, tangent: the
// directions); U0: the base state (tangent only); out: states. One block: TM modes of ND directions.
// Per mode the Stokes problem is solved by banded solves (plan_pipe.cpp): the pressure p_f (Poisson,
// wall value zero), the three velocity components driven by f - grad p_f, and the influence
// coefficient a of the precomputed u_h from the wall continuity row. The stencil work (div_h f,
// grad p) runs over all threads, row by row in parallel; only the banded substitutions are serial,
// one thread per (mode, direction, component, real/imaginary part). The TM modes' factors (4
// matrices each) come into shared memory by bulk TMA copies while the right-hand sides are formed;
// their wait has an iteration limit, past which the block writes NaN into its outputs.
template <typename T, bool TANGENT, int TM, int ND, int NRT>
__global__ void __launch_bounds__(psolve_threads(TM, ND)) k_psolve(const C2<T>* __restrict__ in3,
                                                                   const double2* __restrict__ u,
                                                                   const double2* __restrict__ U0,
                                                                   double2* __restrict__ out, PArgs a, int n_dir) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NR = NRT > 0 ? NRT : a.NR, Mm = a.Mm, NRP = psolve_nrp(NR), n3 = 3 * NRP;
  const size_t chunk = a.pb_chunk;
  unsigned char* sfac = smem_raw;                                             // [TM][4][chunk]
  double2* sf = reinterpret_cast<double2*>(smem_raw + (size_t)TM * 4 * chunk);  // [TM ND][3][NRP]
  double2* sp = sf + TM * ND * n3;                                            // [TM ND][NRP] pressure
  double* sw = reinterpret_cast<double*>(sp + TM * ND * NRP);                 // [2][NR][9] D1 weights
  int* sc = reinterpret_cast<int*>(sw + 2 * NR * 9);                          // [2][NR][9] their columns
  __shared__ int s_pos[TM], s_iz[TM], s_u[TM];
  __shared__ double s_alpha[TM * ND][2];
  __shared__ __align__(8) uint64_t s_bar;
  const int u0 = blockIdx.x * TM, d0 = blockIdx.y * ND;
  const uint32_t bar = smem_addr(&s_bar);
  if (threadIdx.x < TM) {
    const int uu = u0 + threadIdx.x;
    int pos = 0, iz = 0;
    if (uu < a.n_unique) unique_mode_d(uu, a.Kx, a.MZ, &pos, &iz);
    s_pos[threadIdx.x] = pos;
    s_iz[threadIdx.x] = iz;
    s_u[threadIdx.x] = uu;
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int nvalid = min(TM, a.n_unique - u0);
  if (threadIdx.x == 0) {
    // the factors of the block's modes: one bulk copy per (mode, matrix), contiguous in global memory
    const uint32_t bytes = (uint32_t)(nvalid * 4 * chunk);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    for (int q = 0; q < nvalid * 4; ++q)
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_addr(sfac + (size_t)q * chunk)),
                   "l"(a.pb_fac + ((size_t)u0 * 4 + q) * chunk), "r"((uint32_t)chunk), "r"(bar)
                   : "memory");
  }
  for (int i = threadIdx.x; i < 2 * NR * 9; i += blockDim.x) {
    sw[i] = __ldg(a.w1 + i);
    sc[i] = __ldg(a.c1 + i);
  }
  // f = u/dt + N + speed terms, rotated to (f+, f-, f~z) = (f_r + i f_theta, f_r - i f_theta, -i f_z)
  for (int idx = threadIdx.x; idx < TM * ND * NR; idx += blockDim.x) {
    const int tm = idx / NR, j = idx - tm * NR, t = tm / ND, dir = d0 + tm - t * ND;
    if (s_u[t] >= a.n_unique || dir >= n_dir) continue;
    const int pos = s_pos[t], iz = s_iz[t];
    const int kzi = pos <= a.Kx ? pos : pos - a.MX;
    const double k = a.alpha * kzi;
    const double2* us = u + (size_t)dir * a.sstride;
    const C2<T>* vin = in3 + (size_t)dir * 3 * NR * Mm;
    // speed terms: step c du/dz; tangent c0 du/dz + dc dU0/dz
    const double c_eff = TANGENT ? __ldg(U0 + a.sstride - 1).x : __ldg(us + a.sstride - 1).x;
    const double dc = TANGENT ? __ldg(us + a.sstride - 1).x : 0.0;
    double2 f[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double2 v = sym_load(us, c, pos, iz, j, a);
      const C2<T> nv = vin[((size_t)c * NR + j) * Mm + pos * a.MZ + iz];
      f[c] = make_double2(v.x * a.inv_dt + (double)nv.x - c_eff * k * v.y,
                          v.y * a.inv_dt + (double)nv.y + c_eff * k * v.x);
      if (TANGENT) {
        const double2 w = sym_load(U0, c, pos, iz, j, a);
        f[c].x -= dc * k * w.y;
        f[c].y += dc * k * w.x;
      }
      if (pos == 0 && iz == 0) f[c].y = 0.0;
    }
    double2* d = sf + tm * n3;
    if (pos == 0 && iz == 0) {  // the mean mode keeps (f_r, f_theta, f_z)
      d[j] = f[0];
      d[NRP + j] = f[1];
      d[2 * NRP + j] = f[2];
    } else {
      d[j] = make_double2(f[0].x - f[1].y, f[0].y + f[1].x);
      d[NRP + j] = make_double2(f[0].x + f[1].y, f[0].y - f[1].x);
      d[2 * NRP + j] = make_double2(f[2].y, -f[2].x);
    }
  }
  bool ok = mbar_wait_bounded(bar, 0);
  if (!ok) (void)mbar_wait_bounded(bar, 0);  // copies still in flight: a second limit before going on
  ok = __syncthreads_and(ok) != 0;            // the same decision in every thread of the block
  if (ok) {
    // pressure right-hand side: div_h f on the inner rows, wall value 0 (all rows in parallel)
    for (int idx = threadIdx.x; idx < TM * ND * NR; idx += blockDim.x) {
      const int tm = idx / NR, i = idx - tm * NR, t = tm / ND, dir = d0 + tm - t * ND;
      const int pos = s_pos[t], iz = s_iz[t];
      double2 g = make_double2(0.0, 0.0);
      if (s_u[t] < a.n_unique && dir < n_dir && !(pos == 0 && iz == 0) && i > 0) {
        const int kzi = pos <= a.Kx ? pos : pos - a.MX;
        const double k = a.alpha * kzi, mm = a.sym * iz;
        const int pe = (((int)mm) + 1) & 1;
        const double2* fp = sf + tm * n3;
        const double2* fm = fp + NRP;
        const double2* fz = fp + 2 * NRP;
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          const int col = sc[(pe * NR + i) * 9 + q];
          const double w = sw[(pe * NR + i) * 9 + q];
          acc.x = fma(w, fp[col].x + fm[col].x, acc.x);
          acc.y = fma(w, fp[col].y + fm[col].y, acc.y);
        }
        const double ir = 1.0 / __ldg(a.r + i);
        g.x = 0.5 * acc.x + 0.5 * ir * ((1.0 + mm) * fp[i].x + (1.0 - mm) * fm[i].x) - k * fz[i].x;
        g.y = 0.5 * acc.y + 0.5 * ir * ((1.0 + mm) * fp[i].y + (1.0 - mm) * fm[i].y) - k * fz[i].y;
      }
      sp[tm * NRP + i] = g;
    }
    __syncthreads();
    // serial tasks go round-robin over the warps (task = lane * warps + warp), so that every warp
    // of the block, on its own scheduler, runs some of the chains
    constexpr int kWarps = psolve_threads(TM, ND) / 32;
    const int task = (threadIdx.x & 31) * kWarps + (threadIdx.x >> 5);
    // pressure solve: one task per (mode, direction, part)
    if (task < 2 * TM * ND) {
      const int tm = task >> 1, part = task & 1, t = tm / ND, dir = d0 + tm - t * ND;
      if (s_u[t] < a.n_unique && dir < n_dir && !(s_pos[t] == 0 && s_iz[t] == 0))
        band_solve_d<NRT>(reinterpret_cast<double*>(sp + tm * NRP) + part, sfac + (size_t)t * 4 * chunk, NR);
    }
    __syncthreads();
    // velocity right-hand sides f - grad p on the inner rows, no slip at the wall (parallel)
    for (int idx = threadIdx.x; idx < TM * ND * 3 * NR; idx += blockDim.x) {
      const int tm = idx / (3 * NR), rem = idx - tm * 3 * NR, comp = rem / NR, i = rem - comp * NR;
      const int t = tm / ND, dir = d0 + tm - t * ND;
      if (s_u[t] >= a.n_unique || dir >= n_dir) continue;
      const int pos = s_pos[t], iz = s_iz[t];
      double2& x = sf[tm * n3 + comp * NRP + i];
      if (pos == 0 && iz == 0) {  // mean flow: u_r = 0, wall rows zero
        if (comp == 0 || i == 0) x = make_double2(0.0, 0.0);
        continue;
      }
      if (i == 0) {
        x = make_double2(0.0, 0.0);
        continue;
      }
      const int kzi = pos <= a.Kx ? pos : pos - a.MX;
      const double k = a.alpha * kzi, mm = a.sym * iz;
      const double2* p = sp + tm * NRP;
      double2 gp;
      if (comp == 2) {
        gp = make_double2(k * p[i].x, k * p[i].y);
      } else {
        const int pz = ((int)mm) & 1;
        double2 d1 = make_double2(0.0, 0.0);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          const int col = sc[(pz * NR + i) * 9 + q];
          const double w = sw[(pz * NR + i) * 9 + q];
          d1.x = fma(w, p[col].x, d1.x);
          d1.y = fma(w, p[col].y, d1.y);
        }
        const double mr = mm / __ldg(a.r + i);
        gp = comp == 0 ? make_double2(d1.x - mr * p[i].x, d1.y - mr * p[i].y)
                       : make_double2(d1.x + mr * p[i].x, d1.y + mr * p[i].y);
      }
      x.x -= gp.x;
      x.y -= gp.y;
    }
    __syncthreads();
    // velocity solves: one task per (mode, direction, component, part)
    if (task < 6 * TM * ND) {
      const int tm = task / 6, rem = task - 6 * tm, comp = rem >> 1, part = rem & 1;
      const int t = tm / ND, dir = d0 + tm - t * ND;
      const bool mean = s_pos[t] == 0 && s_iz[t] == 0;
      if (s_u[t] < a.n_unique && dir < n_dir && !(mean && comp == 0)) {
        const int slot = mean ? comp : comp + 1;
        band_solve_d<NRT>(reinterpret_cast<double*>(sf + tm * n3 + comp * NRP) + part,
                          sfac + ((size_t)t * 4 + slot) * chunk, NR);
      }
    }
    __syncthreads();
    // influence coefficient from the wall continuity row: 0.5 D1 (u+ + u-) at r = 1 vanishes
    if (threadIdx.x < 2 * TM * ND) {
      const int tm = threadIdx.x >> 1, part = threadIdx.x & 1, t = tm / ND;
      const int uu = s_u[t], pos = s_pos[t], iz = s_iz[t];
      double al = 0.0;
      if (uu < a.n_unique && !(pos == 0 && iz == 0)) {
        const int pe = (((int)(a.sym * iz)) + 1) & 1;
        const double* up = reinterpret_cast<const double*>(sf + tm * n3) + part;
        const double* um = up + 2 * NRP;
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          const int col = sc[pe * NR * 9 + q];
          s += sw[pe * NR * 9 + q] * (up[2 * col] + um[2 * col]);
        }
        al = -0.5 * s * __ldg(a.pb_dinv + uu);
      }
      s_alpha[tm][part] = al;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < TM * ND * 3 * NR; idx += blockDim.x) {
      const int tm = idx / (3 * NR), rem = idx - tm * 3 * NR, comp = rem / NR, j = rem - comp * NR;
      const int t = tm / ND, uu = s_u[t];
      if (uu >= a.n_unique || (s_pos[t] == 0 && s_iz[t] == 0)) continue;
      const double h = __ldg(a.pb_uh + (size_t)uu * 3 * NR + rem);
      double2& x = sf[tm * n3 + comp * NRP + j];
      x.x += s_alpha[tm][0] * h;
      x.y += s_alpha[tm][1] * h;
    }
    __syncthreads();
  }
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  for (int idx = threadIdx.x; idx < TM * ND * NR; idx += blockDim.x) {
    const int tm = idx / NR, j = idx - tm * NR, t = tm / ND, dir = d0 + tm - t * ND;
    if (s_u[t] >= a.n_unique || dir >= n_dir) continue;
    const int pos = s_pos[t], iz = s_iz[t];
    const double2* us = u + (size_t)dir * a.sstride;
    double2* dst = out + (size_t)dir * a.sstride;
    const double2* x = sf + tm * n3;
    double2 vr, vt, vz;
    if (!ok) {
      vr = vt = vz = make_double2(nan, nan);
    } else if (pos == 0 && iz == 0) {
      vr = make_double2(0.0, 0.0);
      vt = make_double2(x[NRP + j].x, 0.0);
      vz = make_double2(x[2 * NRP + j].x, 0.0);
    } else {
      const double2 up = x[j], um = x[NRP + j], uzt = x[2 * NRP + j];
      vr = make_double2(0.5 * (up.x + um.x), 0.5 * (up.y + um.y));
      vt = make_double2(0.5 * (up.y - um.y), -0.5 * (up.x - um.x));  // (u+ - u-)/(2i)
      vz = make_double2(-uzt.y, uzt.x);                                // i u~z
    }
    const double2 res[3] = {vr, vt, vz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double2 d = sym_load(us, c, pos, iz, j, a);
      double2 g = make_double2(res[c].x - d.x, res[c].y - d.y);
      if (pos == 0 && iz == 0) g.y = 0.0;
      dst[((size_t)c * Mm + pos * a.MZ + iz) * NR + j] = g;
      if (iz == 0 && pos != 0) dst[((size_t)c * Mm + (a.MX - pos) * a.MZ) * NR + j] = make_double2(g.x, -g.y);
    }
  }
  // the speed slot of a step is zero (no equation of its own); the tangent's
  // phase condition is written afterwards
  if (blockIdx.x == 0 && threadIdx.x < ND && d0 + (int)threadIdx.x < n_dir)
    out[(size_t)(d0 + threadIdx.x) * a.sstride + a.sstride - 1] = make_double2(0.0, 0.0);
}

// dzU = i k P(U) (P: Hermitian projection), speed slot zero
__global__ void k_pipe_dz(const double2* U, double2* dzU, PArgs a) {
  const size_t n = (size_t)3 * a.Mm * a.NR;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % a.NR);
    const int m = (int)((e / a.NR) % a.Mm);
    const int c = (int)(e / ((size_t)a.NR * a.Mm));
    const int pos = m / a.MZ, iz = m - pos * a.MZ;
    const int kzi = pos <= a.Kx ? pos : pos - a.MX;
    const double k = a.alpha * kzi;
    const double2 v = sym_load(U, c, pos, iz, j, a);
    dzU[e] = make_double2(-k * v.y, k * v.x);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) dzU[n] = make_double2(0.0, 0.0);
}

// seeded pipe state: A = streak part, B = poloidal part (both unscaled)
__global__ void k_pipe_seed(const double* streak, const double2* pol, int npoly, double2* A, double2* B, PArgs a) {
  const int m = blockIdx.x;  // stored mode index
  if (m >= a.Mm) return;
  const int pos = m / a.MZ, iz = m - pos * a.MZ;
  const int kzi = pos <= a.Kx ? pos : pos - a.MX;
  const double k = a.alpha * kzi;
  const int mm = (int)lround(a.sym) * iz;
  for (int j = threadIdx.x; j < a.NR; j += blockDim.x) {
    const double r = a.r[j], x = 1.0 - r * r;
    double2 zr = make_double2(0.0, 0.0), zt = zr, zz = zr, sz = zr;
    if (kzi == 0 && iz >= 1 && iz <= 3) {
      double rm = 1.0;
      for (int q = 0; q < mm; ++q) rm *= r;
      sz = make_double2(streak[iz] * x * rm, 0.0);
    }
    if (kzi != 0) {
      // phi = (1 - r^2)^3 r^m s(r), s = sum_n p_n r^(2n): phi', phi'' by the product rule
      double2 s = make_double2(0.0, 0.0), s1 = s, s2 = s;
      double rp = 1.0;  // r^(2n)
      for (int n = 0; n < npoly; ++n) {
        const double2 p = pol[((size_t)pos * a.MZ + iz) * npoly + n];
        const double e = 2.0 * n;
        const double d1 = n > 0 ? e * rp / r : 0.0;                  // d/dr r^(2n)
        const double d2 = n > 0 ? e * (e - 1.0) * rp / (r * r) : 0.0;  // d2/dr2 r^(2n)
        s.x += p.x * rp; s.y += p.y * rp;
        s1.x += p.x * d1; s1.y += p.y * d1;
        s2.x += p.x * d2; s2.y += p.y * d2;
        rp *= r * r;
      }
      double rm = 1.0;
      for (int q = 0; q < mm; ++q) rm *= r;
      // g = (1 - r^2)^3 r^m
      const double g = x * x * x * rm;
      const double g1 = -6.0 * r * x * x * rm + (mm > 0 ? mm * x * x * x * rm / r : 0.0);
      const double g2 = 24.0 * r * r * x * rm - 6.0 * x * x * rm - (mm > 0 ? 12.0 * mm * x * x * rm : 0.0) +
                        (mm > 1 ? mm * (mm - 1.0) * x * x * x * rm / (r * r) : 0.0);
      const double2 ph = make_double2(g * s.x, g * s.y);
      const double2 p1 = make_double2(g1 * s.x + g * s1.x, g1 * s.y + g * s1.y);
      const double2 p2 = make_double2(g2 * s.x + 2.0 * g1 * s1.x + g * s2.x, g2 * s.y + 2.0 * g1 * s1.y + g * s2.y);
      zr = make_double2(-k * p1.y, k * p1.x);                   // i k phi'
      zt = make_double2(-mm * k / r * ph.x, -mm * k / r * ph.y);  // -(m k / r) phi
      zz = make_double2(-(p2.x + p1.x / r - mm * mm * ph.x / (r * r)), -(p2.y + p1.y / r - mm * mm * ph.y / (r * r)));
    }
    const size_t e = (size_t)m * a.NR + j;
    A[0 * (size_t)a.Mm * a.NR + e] = make_double2(0.0, 0.0);
    A[1 * (size_t)a.Mm * a.NR + e] = make_double2(0.0, 0.0);
    A[2 * (size_t)a.Mm * a.NR + e] = sz;
    B[0 * (size_t)a.Mm * a.NR + e] = zr;
    B[1 * (size_t)a.Mm * a.NR + e] = zt;
    B[2 * (size_t)a.Mm * a.NR + e] = zz;
  }
  if (m == 0 && threadIdx.x == 0) {
    A[(size_t)3 * a.Mm * a.NR] = make_double2(0.0, 0.0);
    B[(size_t)3 * a.Mm * a.NR] = make_double2(0.0, 0.0);
  }
}

PArgs pargs(const sp_ctx* c) {
  PArgs a;
  a.r = c->yv;
  a.w1 = c->fd_w1;
  a.c1 = c->fd_c1;
  a.pb_fac = c->pb_fac;
  a.pb_chunk = c->pb_chunk;
  a.pb_uh = c->pb_uh;
  a.pb_dinv = c->pb_dinv;
  a.sstride = c->cplx_per_state;
  a.Mm = c->Mm; a.MX = c->MX; a.MZ = c->MZ; a.Kx = c->Kx; a.NR = c->NY; a.n_unique = c->n_unique;
  a.alpha = c->alpha; a.sym = c->beta; a.inv_dt = 1.0 / c->dt;
  return a;
}

}  // namespace

cudaError_t launch_pvals(const sp_ctx* c, bool fp32, const double* in, void* out6, int n_dir, cudaStream_t st) {
  PArgs a = pargs(c);
  dim3 grid((c->Mm + kTileP - 1) / kTileP, n_dir);
  const size_t sm = (size_t)3 * kTileP * c->NY * sizeof(double2);
  if (fp32) {
    cudaFuncSetAttribute(k_pvals<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_pvals<float><<<grid, kThreadsP, sm, st>>>(reinterpret_cast<const double2*>(in),
                                                reinterpret_cast<C2<float>*>(out6), a);
  } else {
    cudaFuncSetAttribute(k_pvals<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_pvals<double><<<grid, kThreadsP, sm, st>>>(reinterpret_cast<const double2*>(in),
                                                 reinterpret_cast<C2<double>*>(out6), a);
  }
  return cudaGetLastError();
}

template <typename T, bool TG, int TM, int ND, int NRT>
static cudaError_t psolve_t(const sp_ctx* c, const PArgs& a, const void* in3, const double2* uu, const double2* U0,
                            double2* o, int n_dir, cudaStream_t st) {
  const size_t sm = psolve_smem(TM, ND, c->NY, c->pb_chunk);
  auto kern = k_psolve<T, TG, TM, ND, NRT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid((c->n_unique + TM - 1) / TM, (n_dir + ND - 1) / ND);
  kern<<<grid, psolve_threads(TM, ND), sm, st>>>(reinterpret_cast<const C2<T>*>(in3), uu, U0, o, a, n_dir);
  return cudaGetLastError();
}

// The radial size of the pipe workload (Nr = 64) has register-resident solves; other sizes use
// the shared-memory solve. The widest block whose staged factors and vectors fit is taken.
template <typename T, bool TG>
static cudaError_t psolve_tm(const sp_ctx* c, const PArgs& a, const void* in3, const double2* uu, const double2* U0,
                             double2* o, int n_dir, cudaStream_t st) {
  constexpr size_t kMax = 225 * 1024;
  auto fits = [&](int tm, int nd) { return psolve_smem(tm, nd, c->NY, c->pb_chunk) <= kMax; };
  const bool wide = n_dir >= 8 && fits(2, 8);
  if (c->NY == 64) {
    return wide ? psolve_t<T, TG, 2, 8, 64>(c, a, in3, uu, U0, o, n_dir, st)
                : psolve_t<T, TG, 2, 1, 64>(c, a, in3, uu, U0, o, n_dir, st);
  }
  if (wide) return psolve_t<T, TG, 2, 8, 0>(c, a, in3, uu, U0, o, n_dir, st);
  if (fits(2, 1)) return psolve_t<T, TG, 2, 1, 0>(c, a, in3, uu, U0, o, n_dir, st);
  if (fits(1, 1)) return psolve_t<T, TG, 1, 1, 0>(c, a, in3, uu, U0, o, n_dir, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_psolve(const sp_ctx* c, bool fp32, bool tangent, const void* in3, const double* u, double* out,
                          int n_dir, cudaStream_t st) {
  PArgs a = pargs(c);
  const double2* uu = reinterpret_cast<const double2*>(u);
  const double2* U0 = reinterpret_cast<const double2*>(c->U0);
  double2* o = reinterpret_cast<double2*>(out);
  if (fp32) return tangent ? psolve_tm<float, true>(c, a, in3, uu, U0, o, n_dir, st)
                           : psolve_tm<float, false>(c, a, in3, uu, U0, o, n_dir, st);
  return tangent ? psolve_tm<double, true>(c, a, in3, uu, U0, o, n_dir, st)
                 : psolve_tm<double, false>(c, a, in3, uu, U0, o, n_dir, st);
}

cudaError_t launch_pipe_dz(const sp_ctx* c, const double* U, double* dzU, cudaStream_t st) {
  PArgs a = pargs(c);
  k_pipe_dz<<<256, 256, 0, st>>>(reinterpret_cast<const double2*>(U), reinterpret_cast<double2*>(dzU), a);
  return cudaGetLastError();
}

cudaError_t launch_pipe_seed(const sp_ctx* c, const double* streak, const double* pol, int npoly, double* A,
                             double* B, cudaStream_t st) {
  PArgs a = pargs(c);
  k_pipe_seed<<<c->Mm, 64, 0, st>>>(streak, reinterpret_cast<const double2*>(pol), npoly,
                                    reinterpret_cast<double2*>(A), reinterpret_cast<double2*>(B), a);
  return cudaGetLastError();
}
