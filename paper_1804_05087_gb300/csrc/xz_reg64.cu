// Plane stage of the step, the tangent and the adjoint in FP64 with register-resident FFTs
// (the FP64 counterpart of xz_reg.cu; same mathematics as k_xz in kernels.cu):
// per y-plane, inverse FFT along x of every (field, kz) column, packed c2r along
// z of pairs of x-rows, the pointwise product, packed r2c along z, forward FFT
// along x truncated to the 2/3-rule modes (pseudospectral products, Sec. 3.2).
//
// On this GPU the FP64 pipe is the limit, so the kernel is laid out to issue as
// few FP64 instructions as the transforms need, on full warps:
//  * two threads per transform. The first decimation-in-frequency level of a
//    length-N transform (N = 2M) is a radix-2 butterfly; half h = 0 keeps the
//    sums x_m + x_{m+M} (whose length-M transform gives the even outputs X_2k),
//    half h = 1 the twiddled differences (x_m - x_{m+M}) w_N^m (odd outputs
//    X_2k+1). Each half then runs the in-register transform of length M on its
//    own M values, so a thread holds N/2 complex doubles;
//  * the halves are warp-uniform (warp w takes half w & 1), so no warp diverges;
//  * zero inputs of the padded inverse transforms are skipped at compile time,
//    and outputs that are never stored (the truncated modes) are dead code.
// Square grids of 16, 24, 32 and 48 points; others use k_xz<double>.
#include <algorithm>
#include <utility>

#include "fft_reg.h"
#include "sp_internal.h"

namespace {

using namespace fftreg;
using cd = C2<double>;

struct Xz64Args {
  const cd* in;         // [dir][NIN][NY][Mm]
  cd* out;              // [dir][NOUT][NY][Mm]
  double* base;         // [6][NY][NX][NZ] FP64 base fields (U_tot, Omega_tot): read by the tangent and
                        // the adjoint, written by XZ_STEP_BASE
  const double* lam;    // [NY][6] laminar U and Omega of each plane (XZ_STEP, XZ_STEP_BASE)
  int NY, Mm;
};

// threads: two halves per transform, 32 transforms per warp pair, enough warps
// for the largest phase (the packed z transforms of the NIN input fields)
template <int NX, int NZ, int NIN>
constexpr int threads64() {
  constexpr int MZ = (NZ - 1) / 3 + 1, NQ = NX / 2;
  constexpr int big = NIN * (MZ > NQ ? MZ : NQ);
  return 64 * ((big + 31) / 32);
}

// one input of the split level: v = x_m + x_{m+M} (H = 0) or (x_m - x_{m+M}) w_N^{SGN m} (H = 1),
// with the compile-time zero pattern of the source
template <int N, int SGN, int H, int m, class Src>
__device__ __forceinline__ void split_one(cd (&y)[N / 2], const Src& src) {
  constexpr int M = N / 2;
  constexpr bool za = Src::zero(m), zb = Src::zero(m + M);
  cd v;
  if constexpr (za && zb) {
    v = mk(0.0, 0.0);
  } else if constexpr (H == 0) {
    if constexpr (za) v = src(m + M);
    else if constexpr (zb) v = src(m);
    else v = src(m) + src(m + M);
  } else {
    if constexpr (za) {
      const cd b = src(m + M);
      v = mk(-b.x, -b.y);
    } else if constexpr (zb) {
      v = src(m);
    } else {
      v = src(m) - src(m + M);
    }
    v = twiddle<double, N, SGN, m>(v);
  }
  y[m] = v;
}

template <int N, int SGN, int H, class Src, int... Ms>
__device__ __forceinline__ void split_all(cd (&y)[N / 2], const Src& src, std::integer_sequence<int, Ms...>) {
  (split_one<N, SGN, H, Ms>(y, src), ...);
}

// half H of a length-N transform: y[out_pos<N/2>(k)] = X_{2k+H}
template <int N, int SGN, int H, class Src>
__device__ __forceinline__ void half_fft(cd (&y)[N / 2], const Src& src) {
  split_all<N, SGN, H>(y, src, std::make_integer_sequence<int, N / 2>{});
  fft_reg<N / 2, SGN>(y);
}

// ----------------------------------------------------------------- sources
// phase 1: column (field, kz) of the retained x-modes, zero-padded to NX
template <int NX>
struct SrcX {
  static constexpr int KX = (NX - 1) / 3, MX = 2 * KX + 1;
  const cd* p;  // element e at p[e * MZ] (e <= KX) or p[(e - NX + MX) * MZ]
  int MZ;
  double sc;
  __host__ __device__ static constexpr bool zero(int e) { return e > KX && e < NX - KX; }
  __device__ __forceinline__ cd operator()(int e) const {
    const int r = e <= KX ? e : e - NX + MX;
    const double2 v = __ldg(reinterpret_cast<const double2*>(p + (size_t)r * MZ));
    return mk(v.x * sc, v.y * sc);
  }
};

// phase 2a: two real x-rows packed as real + i imag; phase 1 stored the packed z-spectrum
// (kz = 0..KZ in the first row's slots, the mirrored frequencies NZ - kz in the second's)
template <int NZ>
struct SrcZP {
  static constexpr int KZ = (NZ - 1) / 3;
  const cd* g0;  // first row of the pair
  const cd* g1;  // second row of the pair
  __host__ __device__ static constexpr bool zero(int e) { return e > KZ && e < NZ - KZ; }
  __device__ __forceinline__ cd operator()(int e) const { return e <= KZ ? g0[e] : g1[NZ - e]; }
};

// row pair q of the z transforms: rows 4 (q >> 1) + (q & 1) and that + 2, both held by one
// half of a phase-1 transform (half h holds the rows 2k + h)
__device__ __forceinline__ int pair_row(int q) { return 4 * (q >> 1) + (q & 1); }

// phases 2c and 3: a dense row of shared memory with a stride
struct SrcDense {
  const cd* p;
  int stride;
  __host__ __device__ static constexpr bool zero(int) { return false; }
  __device__ __forceinline__ cd operator()(int e) const { return p[e * stride]; }
};

// run half h (warp-uniform) of a transform
template <int N, int SGN, class Src>
__device__ __forceinline__ void half_fft_rt(int h, cd (&y)[N / 2], const Src& src) {
  if (h == 0) half_fft<N, SGN, 0>(y, src);
  else half_fft<N, SGN, 1>(y, src);
}

template <int NZ, int H, int... Ks>
__device__ __forceinline__ void sep_store(const cd (&y)[NZ / 2], cd* g0, cd* g1, std::integer_sequence<int, Ks...>) {
  constexpr int MZH = NZ / 2;
  (
      [&] {
        constexpr int iz = 2 * Ks + H;
        constexpr int km = ((NZ - iz) % NZ - H) / 2;
        const cd X = y[out_pos<MZH>(Ks)];
        const cd Xm = y[out_pos<MZH>(km)];
        g0[iz] = mk(0.5 * (X.x + Xm.x), 0.5 * (X.y - Xm.y));
        g1[iz] = mk(0.5 * (X.y + Xm.y), -0.5 * (X.x - Xm.x));
      }(),
      ...);
}

// r2c half H of a packed row pair and its separation: rows g0 (real part) and g1
// (imaginary part) receive the modes kz = 2k + H <= KZ. X_{NZ - kz} has the
// parity of kz, so both factors of the separation come from the same half.
template <int NZ, int H>
__device__ __forceinline__ void sep_half(const SrcDense& src, cd* g0, cd* g1) {
  constexpr int KZ = (NZ - 1) / 3, MZH = NZ / 2;
  cd y[MZH];
  half_fft<NZ, -1, H>(y, src);
  sep_store<NZ, H>(y, g0, g1, std::make_integer_sequence<int, (KZ - H) / 2 + 1>{});
}

// (bx, by): Gauss-Lobatto plane, direction
template <int NX, int NZ, int MODE>
__device__ __forceinline__ void xz64_body(const Xz64Args& a, int bx, int by) {
  constexpr int NIN = MODE == XZ_ADJOINT ? 3 : 6;
  constexpr int NOUT = MODE == XZ_ADJOINT ? 6 : 3;
  constexpr int KX = (NX - 1) / 3, KZ = (NZ - 1) / 3;
  constexpr int MX = 2 * KX + 1, MZ = KZ + 1;
  constexpr int FS = MZ + 1, RS = 6 * FS + 1;  // G: [NX rows][6 fields][FS], row stride RS
  constexpr int NQ = NX / 2, NZP = NZ + 1;      // Ph: [6][NQ][NZP], z fastest
  static_assert(NX % 4 == 0, "row pairs (pair_row) need NX divisible by 4");
  constexpr int MXH = NX / 2, MZH = NZ / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cd* G = reinterpret_cast<cd*>(smem_raw);
  cd* Ph = G + NX * RS;
  const int j = bx, dir = by;
  const size_t planeMm = (size_t)a.NY * a.Mm;
  const cd* in = a.in + (size_t)dir * NIN * planeMm + (size_t)j * a.Mm;
  const double inv = 1.0 / ((double)NX * (double)NZ);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

  // phase 1: inverse FFT along x, transform (field, kz), output rows 2k + h
  {
    constexpr int ntr = NIN * MZ, ngrp = (ntr + 31) / 32;
    for (int w2 = warp; w2 < 2 * ngrp; w2 += nwarps) {
      const int h = w2 & 1, tr = (w2 >> 1) * 32 + lane;
      if (tr >= ntr) continue;
      const int f = tr / MZ, iz = tr - f * MZ;
      double sc = 1.0;
      if constexpr (MODE == XZ_ADJOINT) sc = iz == 0 ? inv : 0.5 * inv;
      SrcX<NX> src{in + (size_t)f * planeMm + iz, MZ, sc};
      cd y[MXH];
      half_fft_rt<NX, 1>(h, y, src);
      // rows 2k + h in pairs (k = 2p, 2p + 1), stored as the packed z-spectrum of phase 2a:
      // A + iB at kz (the real parts only at kz = 0) and conj(A) + i conj(B) at NZ - kz
      cd* g = G + f * FS + iz;
#pragma unroll
      for (int p = 0; p < MXH / 2; ++p) {
        const cd A = y[out_pos<MXH>(2 * p)], B = y[out_pos<MXH>(2 * p + 1)];
        cd* g1 = g + (4 * p + h) * RS;
        if (iz == 0) {
          g1[0] = mk(A.x, B.x);
        } else {
          g1[0] = mk(A.x - B.y, A.y + B.x);
          g1[2 * RS] = mk(A.x + B.y, B.x - A.y);
        }
      }
    }
  }
  __syncthreads();

  // phase 2a: c2r along z of row pairs (pair_row(q), pair_row(q) + 2), output z-points 2k + h
  {
    constexpr int ntr = NIN * NQ, ngrp = (ntr + 31) / 32;
    for (int w2 = warp; w2 < 2 * ngrp; w2 += nwarps) {
      const int h = w2 & 1, tr = (w2 >> 1) * 32 + lane;
      if (tr >= ntr) continue;
      const int f = tr / NQ, q = tr - f * NQ;
      const cd* g0 = G + pair_row(q) * RS + f * FS;
      SrcZP<NZ> src{g0, g0 + 2 * RS};
      cd y[MZH];
      half_fft_rt<NZ, 1>(h, y, src);
      cd* dst = Ph + (f * NQ + q) * NZP;
#pragma unroll
      for (int k = 0; k < MZH; ++k) dst[2 * k + h] = y[out_pos<MZH>(k)];
    }
  }
  __syncthreads();

  // phase 2b: pointwise products (in place: each point reads its NIN fields first);
  // consecutive threads take consecutive z: coalesced base reads, conflict-free Ph
  {
    const size_t nxz = (size_t)NX * NZ;
    const double* bj = a.base + (size_t)j * nxz;
    double lamj[6] = {0, 0, 0, 0, 0, 0};
    if constexpr (MODE == XZ_STEP || MODE == XZ_STEP_BASE) {
#pragma unroll
      for (int f = 0; f < 6; ++f) lamj[f] = a.lam[(size_t)j * 6 + f];
    }
    for (int it = threadIdx.x; it < NQ * NZ; it += blockDim.x) {
      const int q = it / NZ, k = it - q * NZ;
      const int r0 = pair_row(q);
      cd fv[NIN];
#pragma unroll
      for (int f = 0; f < NIN; ++f) fv[f] = Ph[(f * NQ + q) * NZP + k];
      double res[2][NOUT];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        double F[NIN], B[6];
#pragma unroll
        for (int f = 0; f < NIN; ++f) F[f] = r ? fv[f].y : fv[f].x;
        if constexpr (MODE == XZ_TANGENT || MODE == XZ_ADJOINT) {
          const size_t gi = (size_t)(r0 + 2 * r) * NZ + k;
#pragma unroll
          for (int f = 0; f < 6; ++f) B[f] = __ldg(bj + (size_t)f * a.NY * nxz + gi);
        }
        if constexpr (MODE == XZ_STEP || MODE == XZ_STEP_BASE) {
          // the step: U_tot x Omega_tot of the state plus laminar flow (B unused)
          double Tt[6];
#pragma unroll
          for (int f = 0; f < 6; ++f) Tt[f] = F[f] + lamj[f];
          if constexpr (MODE == XZ_STEP_BASE) {
            const size_t gi = (size_t)(r0 + 2 * r) * NZ + k;
#pragma unroll
            for (int f = 0; f < 6; ++f) a.base[(size_t)f * a.NY * nxz + (size_t)j * nxz + gi] = Tt[f];
          }
          res[r][0] = Tt[1] * Tt[5] - Tt[2] * Tt[4];
          res[r][1] = Tt[2] * Tt[3] - Tt[0] * Tt[5];
          res[r][2] = Tt[0] * Tt[4] - Tt[1] * Tt[3];
        } else if constexpr (MODE == XZ_TANGENT) {
          res[r][0] = (B[1] * F[5] - B[2] * F[4]) + (F[1] * B[5] - F[2] * B[4]);
          res[r][1] = (B[2] * F[3] - B[0] * F[5]) + (F[2] * B[3] - F[0] * B[5]);
          res[r][2] = (B[0] * F[4] - B[1] * F[3]) + (F[0] * B[4] - F[1] * B[3]);
        } else {
          res[r][0] = B[4] * F[2] - B[5] * F[1];
          res[r][1] = B[5] * F[0] - B[3] * F[2];
          res[r][2] = B[3] * F[1] - B[4] * F[0];
          res[r][3] = F[1] * B[2] - F[2] * B[1];
          res[r][4] = F[2] * B[0] - F[0] * B[2];
          res[r][5] = F[0] * B[1] - F[1] * B[0];
        }
      }
#pragma unroll
      for (int c = 0; c < NOUT; ++c) Ph[(c * NQ + q) * NZP + k] = mk(res[0][c], res[1][c]);
    }
  }
  __syncthreads();

  // phase 2c: r2c along z and separation of the two rows into G (kz = 2k + h only)
  {
    constexpr int ntr = NOUT * NQ, ngrp = (ntr + 31) / 32;
    for (int w2 = warp; w2 < 2 * ngrp; w2 += nwarps) {
      const int h = w2 & 1, tr = (w2 >> 1) * 32 + lane;
      if (tr >= ntr) continue;
      const int c = tr / NQ, q = tr - c * NQ;
      SrcDense src{Ph + (c * NQ + q) * NZP, 1};
      cd* g0 = G + pair_row(q) * RS + c * FS;
      if (h == 0) sep_half<NZ, 0>(src, g0, g0 + 2 * RS);
      else sep_half<NZ, 1>(src, g0, g0 + 2 * RS);
    }
  }
  __syncthreads();

  // phase 3: forward FFT along x, keep the 2/3-rule modes (outputs 2k + h)
  {
    cd* out = a.out + (size_t)dir * NOUT * planeMm + (size_t)j * a.Mm;
    constexpr int ntr = NOUT * MZ, ngrp = (ntr + 31) / 32;
    for (int w2 = warp; w2 < 2 * ngrp; w2 += nwarps) {
      const int h = w2 & 1, tr = (w2 >> 1) * 32 + lane;
      if (tr >= ntr) continue;
      const int c = tr / MZ, iz = tr - c * MZ;
      SrcDense src{G + c * FS + iz, RS};
      cd y[MXH];
      half_fft_rt<NX, -1>(h, y, src);
      double sc = inv;
      if constexpr (MODE == XZ_ADJOINT) sc = iz == 0 ? 1.0 : 2.0;
      cd* dst = out + (size_t)c * planeMm + iz;
#pragma unroll
      for (int k = 0; k < MXH; ++k) {
        const int e = 2 * k + h;
        const cd v = y[out_pos<MXH>(k)];
        if (e <= KX) dst[e * MZ] = mk(v.x * sc, v.y * sc);
        else if (e >= NX - KX) dst[(e - NX + MX) * MZ] = mk(v.x * sc, v.y * sc);
      }
    }
  }
}

template <int NX, int NZ, int MODE>
__global__ void __launch_bounds__(threads64<NX, NZ, (MODE == XZ_ADJOINT ? 3 : 6)>())
    k_xz_reg64(Xz64Args a) {
  xz64_body<NX, NZ, MODE>(a, blockIdx.x, blockIdx.y);
}

template <int NX, int NZ>
constexpr size_t smem64() {
  constexpr int MZ = (NZ - 1) / 3 + 1, FS = MZ + 1, RS = 6 * FS + 1;
  return sizeof(cd) * ((size_t)NX * RS + (size_t)6 * (NX / 2) * (NZ + 1));
}

template <int NX, int NZ, int MODE>
cudaError_t launch64(const sp_ctx* c, const void* in, void* out, int n_dir, cudaStream_t st) {
  constexpr size_t smem = smem64<NX, NZ>();
  static_assert(smem <= 227 * 1024, "FP64 plane does not fit in shared memory");
  constexpr int thr = threads64<NX, NZ, (MODE == XZ_ADJOINT ? 3 : 6)>();
  Xz64Args a;
  a.in = reinterpret_cast<const cd*>(in);
  a.out = reinterpret_cast<cd*>(out);
  a.base = c->base64;
  a.lam = c->lam6;
  a.NY = c->NY;
  a.Mm = c->Mm;
  cudaError_t e = cudaFuncSetAttribute(k_xz_reg64<NX, NZ, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(c->NY, n_dir);
  k_xz_reg64<NX, NZ, MODE><<<grid, thr, smem, st>>>(a);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t dispatch64(const sp_ctx* c, const void* in, void* out, int n_dir, cudaStream_t st) {
  switch (c->nx) {
    case 16: return launch64<16, 16, MODE>(c, in, out, n_dir, st);
    case 24: return launch64<24, 24, MODE>(c, in, out, n_dir, st);
    case 32: return launch64<32, 32, MODE>(c, in, out, n_dir, st);
    case 48: return launch64<48, 48, MODE>(c, in, out, n_dir, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace

bool sp_xz_reg64_supported(const sp_ctx* c) {
  return c->nx == c->nz && (c->nx == 16 || c->nx == 24 || c->nx == 32 || c->nx == 48);
}

cudaError_t launch_xz_reg64(const sp_ctx* c, int mode, const void* in, void* out, int n_dir, cudaStream_t st) {
  if (!sp_xz_reg64_supported(c)) return cudaErrorNotSupported;
  if (mode == XZ_TANGENT) return dispatch64<XZ_TANGENT>(c, in, out, n_dir, st);
  if (mode == XZ_ADJOINT) return dispatch64<XZ_ADJOINT>(c, in, out, n_dir, st);
  if (mode == XZ_STEP) return dispatch64<XZ_STEP>(c, in, out, n_dir, st);
  if (mode == XZ_STEP_BASE) return dispatch64<XZ_STEP_BASE>(c, in, out, n_dir, st);
  return cudaErrorNotSupported;
}
