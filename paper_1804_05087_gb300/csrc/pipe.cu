// Kernels of the pipe-flow step and tangent (the plane stage is k_xz of
// kernels.cu with the pipe's laminar table).
//   k_pvals : per Fourier mode, the six fields u_r, u_theta, u_z and the
//             vorticity at every radial point: omega_r = (i m/r) u_z - i k u_theta,
//             omega_theta = i k u_r - D1 u_z, omega_z = D1 u_theta + u_theta/r - (i m/r) u_r
//             (radial derivatives by the 9-point parity-aware stencils),
//             written plane-major (one radial point per plane).
//   k_psolve: per Fourier mode, the right-hand side u/dt + N + c du/dz (for the
//             tangent + dc dU/dz), rotation to u+- = u_r +- i u_theta and
//             u~_z = -i u_z, the dense per-mode Stokes operator (FP64), and
//             G = u_new - u with a Hermitian output.
// Index conventions: position pos over the axial wavenumbers in FFT order
// (k = alpha kz), iz = m' (m = sym m').
#include "dev_util.h"
#include "sp_internal.h"

namespace {

constexpr int kTileP = 8;        // modes per k_pvals block
constexpr int kThreadsP = 256;
constexpr int kTilePS = 2;       // modes per k_psolve block
constexpr int kThreadsPS = 256;

struct PArgs {
  const double* r;      // [NR]
  const double* w1;     // [2][NR][9]
  const int* c1;        // [2][NR][9]
  const double* pops;   // [n_unique][3NR][3NR], column-major
  size_t pop_stride;
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

// in3: [dir][3][NR][Mm] values of N (T); u: the states (step: the state itself,
// tangent: the directions); U0: the base state (tangent only); out: states.
template <typename T, bool TANGENT>
__global__ void __launch_bounds__(kThreadsPS) k_psolve(const C2<T>* __restrict__ in3, const double2* __restrict__ u,
                                                       const double2* __restrict__ U0, double2* __restrict__ out,
                                                       PArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TM = kTilePS, NR = a.NR, Mm = a.Mm, n3 = 3 * NR;
  double2* su = reinterpret_cast<double2*>(smem_raw);  // [TM][3NR] projected input u
  double2* sf = su + TM * n3;                          // [TM][3NR] (f+, f-, f~z)
  double2* sx = sf + TM * n3;                          // [TM][3NR] (u+, u-, u~z)
  __shared__ int s_pos[kTilePS], s_iz[kTilePS], s_u[kTilePS];
  const int u0 = blockIdx.x * TM, dir = blockIdx.y;
  if (threadIdx.x < TM) {
    const int uu = u0 + threadIdx.x;
    int pos = 0, iz = 0;
    if (uu < a.n_unique) unique_mode_d(uu, a.Kx, a.MZ, &pos, &iz);
    s_pos[threadIdx.x] = pos;
    s_iz[threadIdx.x] = iz;
    s_u[threadIdx.x] = uu;
  }
  __syncthreads();
  const double2* us = u + (size_t)dir * a.sstride;
  const C2<T>* vin = in3 + (size_t)dir * 3 * NR * Mm;
  // speed terms: step c du/dz; tangent c0 du/dz + dc dU0/dz
  double c_eff, dc = 0.0;
  if (TANGENT) {
    c_eff = __ldg(U0 + a.sstride - 1).x;
    dc = __ldg(us + a.sstride - 1).x;
  } else {
    c_eff = __ldg(us + a.sstride - 1).x;
  }
  for (int idx = threadIdx.x; idx < TM * n3; idx += blockDim.x) {
    const int t = idx / n3, rem = idx - t * n3, c = rem / NR, j = rem - c * NR;
    if (s_u[t] >= a.n_unique) continue;
    const int pos = s_pos[t], iz = s_iz[t];
    const double2 v = sym_load(us, c, pos, iz, j, a);
    su[idx] = v;
    const C2<T> nv = vin[((size_t)c * NR + j) * Mm + pos * a.MZ + iz];
    const int kzi = pos <= a.Kx ? pos : pos - a.MX;
    const double k = a.alpha * kzi;
    double2 f = make_double2(v.x * a.inv_dt + (double)nv.x - c_eff * k * v.y,
                             v.y * a.inv_dt + (double)nv.y + c_eff * k * v.x);
    if (TANGENT) {
      const double2 w = sym_load(U0, c, pos, iz, j, a);
      f.x -= dc * k * w.y;
      f.y += dc * k * w.x;
    }
    if (pos == 0 && iz == 0) f.y = 0.0;
    sf[idx] = f;  // (f_r, f_theta, f_z) for now
  }
  __syncthreads();
  // rotate to (f+, f-, f~z) = (f_r + i f_theta, f_r - i f_theta, -i f_z)
  for (int idx = threadIdx.x; idx < TM * NR; idx += blockDim.x) {
    const int t = idx / NR, j = idx - t * NR;
    double2* f = sf + t * n3;
    const double2 fr = f[j], ft = f[NR + j], fz = f[2 * NR + j];
    if (s_pos[t] == 0 && s_iz[t] == 0) continue;  // mean mode keeps (f_r, f_theta, f_z)
    f[j] = make_double2(fr.x - ft.y, fr.y + ft.x);
    f[NR + j] = make_double2(fr.x + ft.y, fr.y - ft.x);
    f[2 * NR + j] = make_double2(fz.y, -fz.x);
  }
  __syncthreads();
  // dense per-mode operator (FP64)
  for (int idx = threadIdx.x; idx < TM * n3; idx += blockDim.x) {
    const int t = idx / n3, row = idx - t * n3;
    if (s_u[t] >= a.n_unique) continue;
    const double* S = a.pops + (size_t)s_u[t] * a.pop_stride;
    const double2* f = sf + t * n3;
    double2 acc = make_double2(0.0, 0.0);
    if (s_pos[t] == 0 && s_iz[t] == 0) {
      // rows NR..2NR-1: u_theta = H1 f_theta; rows 2NR..3NR-1: u_z = H0 f_z; u_r = 0
      if (row >= NR) {
        const int blk = row < 2 * NR ? 0 : 1, i = row - (blk + 1) * NR;
        // column-major blocks: row i of block blk
        acc = dot4(S + (size_t)blk * NR * NR + i, NR, f + (blk + 1) * NR, 1, NR);
      }
    } else {
      acc = dot4(S + row, n3, f, 1, n3);  // row `row` of the column-major operator
    }
    sx[idx] = acc;
  }
  __syncthreads();
  double2* dst = out + (size_t)dir * a.sstride;
  for (int idx = threadIdx.x; idx < TM * NR; idx += blockDim.x) {
    const int t = idx / NR, j = idx - t * NR;
    if (s_u[t] >= a.n_unique) continue;
    const int pos = s_pos[t], iz = s_iz[t];
    const double2* x = sx + t * n3;
    double2 vr, vt, vz;
    if (pos == 0 && iz == 0) {
      vr = make_double2(0.0, 0.0);
      vt = make_double2(x[NR + j].x, 0.0);
      vz = make_double2(x[2 * NR + j].x, 0.0);
    } else {
      const double2 up = x[j], um = x[NR + j], uzt = x[2 * NR + j];
      vr = make_double2(0.5 * (up.x + um.x), 0.5 * (up.y + um.y));
      vt = make_double2(0.5 * (up.y - um.y), -0.5 * (up.x - um.x));  // (u+ - u-)/(2i)
      vz = make_double2(-uzt.y, uzt.x);                                // i u~z
    }
    const double2 res[3] = {vr, vt, vz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double2 d = su[t * n3 + c * NR + j];
      double2 g = make_double2(res[c].x - d.x, res[c].y - d.y);
      if (pos == 0 && iz == 0) g.y = 0.0;
      dst[((size_t)c * Mm + pos * a.MZ + iz) * NR + j] = g;
      if (iz == 0 && pos != 0) dst[((size_t)c * Mm + (a.MX - pos) * a.MZ) * NR + j] = make_double2(g.x, -g.y);
    }
  }
  // the speed slot of a step is zero (no equation of its own); the tangent's
  // phase condition is written afterwards
  if (blockIdx.x == 0 && threadIdx.x == 0) dst[a.sstride - 1] = make_double2(0.0, 0.0);
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
  a.pops = c->pops;
  a.pop_stride = c->pop_stride;
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

cudaError_t launch_psolve(const sp_ctx* c, bool fp32, bool tangent, const void* in3, const double* u, double* out,
                          int n_dir, cudaStream_t st) {
  PArgs a = pargs(c);
  dim3 grid((c->n_unique + kTilePS - 1) / kTilePS, n_dir);
  const size_t sm = (size_t)3 * kTilePS * 3 * c->NY * sizeof(double2);
  const double2* uu = reinterpret_cast<const double2*>(u);
  const double2* U0 = reinterpret_cast<const double2*>(c->U0);
  double2* o = reinterpret_cast<double2*>(out);
#define SP_PSOLVE(T, TG)                                                                                     \
  do {                                                                                                       \
    cudaFuncSetAttribute(k_psolve<T, TG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);              \
    k_psolve<T, TG><<<grid, kThreadsPS, sm, st>>>(reinterpret_cast<const C2<T>*>(in3), uu, U0, o, a);        \
  } while (0)
  if (fp32) {
    if (tangent) SP_PSOLVE(float, true);
    else SP_PSOLVE(float, false);
  } else {
    if (tangent) SP_PSOLVE(double, true);
    else SP_PSOLVE(double, false);
  }
#undef SP_PSOLVE
  return cudaGetLastError();
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
