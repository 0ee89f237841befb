// Plane stage of the tangent and the adjoint in float, with register-resident
// FFTs: one thread owns a whole transform (length <= 64), so each phase of
// the plane needs a single barrier instead of one per FFT stage.
//
// Same mathematics as k_xz (kernels.cu): per y-plane, inverse FFT along x of
// every (field, kz) column, packed c2r along z of pairs of x-rows, the
// pointwise product, packed r2c along z, forward FFT along x truncated to the
// 2/3-rule modes (pseudospectral products, Sec. 3.2).
//
// The FFTs are the compile-time register transforms of fft_reg.h.
#include <algorithm>
#include <utility>
#include <vector>

#include "fft_reg.h"
#include "sp_internal.h"

namespace {

using namespace fftreg;

struct XzRegArgs {
  const C2<float>* in;  // [dir][NIN][NY][Mm]
  C2<float>* out;       // [dir][NOUT][NY][Mm]
  const float* base;    // [6][NY][NZ][NX] (transposed float copy of the base fields)
  const double* yv;
  int NY, Mm;
};

constexpr int kThreadsReg = 256;

// (bx, by): Gauss-Lobatto plane, direction
template <int NX, int NZ, int MODE>
__device__ __forceinline__ void xz_reg_body(const XzRegArgs& a, int bx, int by) {
  constexpr int NIN = MODE == XZ_ADJOINT ? 3 : 6;
  constexpr int NOUT = MODE == XZ_ADJOINT ? 6 : 3;
  constexpr int KX = (NX - 1) / 3, KZ = (NZ - 1) / 3;
  constexpr int MX = 2 * KX + 1, MZ = KZ + 1;
  // row stride = 1 (mod 8): neighbouring row pairs start 4 banks apart
  constexpr int FS = MZ + 1, RS = ((6 * FS + 7) / 8) * 8 + 1;
  constexpr int NQ = NX / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<float>* G = reinterpret_cast<C2<float>*>(smem_raw);  // [NX][6][FS] (row stride RS)
  C2<float>* Ph = G + NX * RS;                              // [6][NZ][NQ] packed row pairs, pair fastest
  const int j = bx, dir = by;
  const size_t planeMm = (size_t)a.NY * a.Mm;
  const C2<float>* in = a.in + (size_t)dir * NIN * planeMm + (size_t)j * a.Mm;
  const float inv = (float)(1.0 / ((double)NX * (double)NZ));

  // phase 1: inverse FFT along x, one thread per (field, kz) column
  for (int col = threadIdx.x; col < NIN * MZ; col += blockDim.x) {
    const int f = col / MZ, iz = col - f * MZ;
    const C2<float>* src = in + (size_t)f * planeMm + iz;
    float sc = 1.0f;
    if constexpr (MODE == XZ_ADJOINT) sc = iz == 0 ? inv : 0.5f * inv;
    C2<float> x[NX];
#pragma unroll
    for (int e = 0; e < NX; ++e) {
      if (e <= KX) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(src + e * MZ));
        x[e] = mk(v.x * sc, v.y * sc);
      } else if (e >= NX - KX) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(src + (e - NX + MX) * MZ));
        x[e] = mk(v.x * sc, v.y * sc);
      } else {
        x[e] = mk(0.f, 0.f);
      }
    }
    fft_reg<NX, 1>(x);
#pragma unroll
    for (int p = 0; p < NX; ++p) G[p * RS + f * FS + iz] = x[out_pos<NX>(p)];
  }
  __syncthreads();

  // phase 2a: c2r along z of row pairs (2q, 2q+1) packed as real + i imag
  for (int it = threadIdx.x; it < NIN * NQ; it += blockDim.x) {
    const int f = it / NQ, q = it - f * NQ;  // consecutive threads: consecutive row pairs
    const C2<float>* g0 = G + (2 * q) * RS + f * FS;
    const C2<float>* g1 = g0 + RS;
    C2<float> z[NZ];
#pragma unroll
    for (int e = 0; e < NZ; ++e) {
      if (e == 0) {
        z[e] = mk(g0[0].x, g1[0].x);
      } else if (e <= KZ) {
        const C2<float> A = g0[e], B = g1[e];
        z[e] = mk(A.x - B.y, A.y + B.x);
      } else if (e >= NZ - KZ) {
        const C2<float> A = g0[NZ - e], B = g1[NZ - e];
        z[e] = mk(A.x + B.y, B.x - A.y);
      } else {
        z[e] = mk(0.f, 0.f);
      }
    }
    fft_reg<NZ, 1>(z);
    C2<float>* dst = Ph + f * NZ * NQ + q;
#pragma unroll
    for (int k = 0; k < NZ; ++k) dst[k * NQ] = z[out_pos<NZ>(k)];
  }
  __syncthreads();

  // phase 2b: pointwise products (in place: each point reads its NIN fields first)
  const size_t nxz = (size_t)NX * NZ;
  for (int it = threadIdx.x; it < NQ * NZ; it += blockDim.x) {
    const int k = it / NQ, q = it - k * NQ;  // pair fastest: conflict-free Ph, coalesced base
    C2<float> fv[NIN];
#pragma unroll
    for (int f = 0; f < NIN; ++f) fv[f] = Ph[(f * NZ + k) * NQ + q];
    // base fields in the transposed layout [6][NY][NZ][NX]: rows 2q and 2q+1 are adjacent
    float2 bp[6];
    const size_t gidx = (size_t)j * nxz + (size_t)k * NX + 2 * q;
#pragma unroll
    for (int f = 0; f < 6; ++f) bp[f] = __ldg(reinterpret_cast<const float2*>(a.base + (size_t)f * a.NY * nxz + gidx));
    float res[2][NOUT];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      float F[NIN], B[6];
#pragma unroll
      for (int f = 0; f < NIN; ++f) F[f] = r ? fv[f].y : fv[f].x;
#pragma unroll
      for (int f = 0; f < 6; ++f) B[f] = r ? bp[f].y : bp[f].x;
      if constexpr (MODE == XZ_TANGENT) {
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
    for (int c = 0; c < NOUT; ++c) Ph[(c * NZ + k) * NQ + q] = mk(res[0][c], res[1][c]);
  }
  __syncthreads();

  // phase 2c: r2c along z and separation of the two rows; result into G rows
  for (int it = threadIdx.x; it < NOUT * NQ; it += blockDim.x) {
    const int c = it / NQ, q = it - c * NQ;
    C2<float> z[NZ];
    const C2<float>* src = Ph + c * NZ * NQ + q;
#pragma unroll
    for (int k = 0; k < NZ; ++k) z[k] = src[k * NQ];
    fft_reg<NZ, -1>(z);
    C2<float>* g0 = G + (2 * q) * RS + c * FS;
    C2<float>* g1 = g0 + RS;
#pragma unroll
    for (int iz = 0; iz <= KZ; ++iz) {
      const C2<float> X = z[out_pos<NZ>(iz)];
      const C2<float> Xm = z[out_pos<NZ>((NZ - iz) % NZ)];
      const C2<float> Aa = scl(X + conj2(Xm), 0.5f);
      const C2<float> D = X - conj2(Xm);
      g0[iz] = Aa;
      g1[iz] = mk(D.y * 0.5f, -D.x * 0.5f);
    }
  }
  __syncthreads();

  // phase 3: forward FFT along x, keep the 2/3-rule modes
  C2<float>* out = a.out + (size_t)dir * NOUT * planeMm + (size_t)j * a.Mm;
  for (int col = threadIdx.x; col < NOUT * MZ; col += blockDim.x) {
    const int c = col / MZ, iz = col - c * MZ;
    C2<float> x[NX];
#pragma unroll
    for (int p = 0; p < NX; ++p) x[p] = G[p * RS + c * FS + iz];
    fft_reg<NX, -1>(x);
    float sc = inv;
    if constexpr (MODE == XZ_ADJOINT) sc = iz == 0 ? 1.0f : 2.0f;
    C2<float>* dst = out + (size_t)c * planeMm + iz;
#pragma unroll
    for (int e = 0; e < NX; ++e) {
      if (e <= KX) dst[e * MZ] = scl(x[out_pos<NX>(e)], sc);
      else if (e >= NX - KX) dst[(e - NX + MX) * MZ] = scl(x[out_pos<NX>(e)], sc);
    }
  }
}

template <int NX, int NZ, int MODE>
__global__ void __launch_bounds__(kThreadsReg) k_xz_reg(XzRegArgs a) {
  xz_reg_body<NX, NZ, MODE>(a, blockIdx.x, blockIdx.y);
}

// one launch over the members of a group that share the grid size NX = NZ
// (one such launch per size class keeps each class at its own register count)
struct GXzReg {
  XzRegArgs a;
};

template <int NX, int NZ, int MODE>
__global__ void __launch_bounds__(kThreadsReg) k_xz_reg_grp(const GXzReg* __restrict__ recs,
                                                           const int* __restrict__ inst,
                                                           const int* __restrict__ first,
                                                           const int* __restrict__ active) {
  const int i = inst[blockIdx.x];
  if (active && !active[i]) return;
  __shared__ GXzReg r;
  if (threadIdx.x == 0) r = recs[i];
  __syncthreads();
  xz_reg_body<NX, NZ, MODE>(r.a, blockIdx.x - first[i], 0);
}

constexpr int kRegSizes[5] = {16, 24, 32, 48, 64};

constexpr size_t reg_smem(int n) {
  return sizeof(C2<float>) * ((size_t)n * ((6 * ((n - 1) / 3 + 2) + 7) / 8 * 8 + 1) + (size_t)6 * (n / 2) * n);
}

template <int NX, int NZ, int MODE>
cudaError_t launch_reg(const sp_ctx* c, const void* in, void* out, int n_dir, cudaStream_t st) {
  constexpr int KZ = (NZ - 1) / 3, MZ = KZ + 1, FS = MZ + 1, RS = ((6 * FS + 7) / 8) * 8 + 1;
  const size_t smem = sizeof(C2<float>) * ((size_t)NX * RS + (size_t)6 * (NX / 2) * NZ);
  if (smem > 227 * 1024) return cudaErrorNotSupported;
  XzRegArgs a;
  a.in = reinterpret_cast<const C2<float>*>(in);
  a.out = reinterpret_cast<C2<float>*>(out);
  a.base = c->base32t;
  a.yv = c->yv;
  a.NY = c->NY;
  a.Mm = c->Mm;
  cudaFuncSetAttribute(k_xz_reg<NX, NZ, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid(c->NY, n_dir);
  k_xz_reg<NX, NZ, MODE><<<grid, kThreadsReg, smem, st>>>(a);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t dispatch_reg(const sp_ctx* c, const void* in, void* out, int n_dir, cudaStream_t st) {
  if (c->nx != c->nz) return cudaErrorNotSupported;
  switch (c->nx) {
    case 16: return launch_reg<16, 16, MODE>(c, in, out, n_dir, st);
    case 24: return launch_reg<24, 24, MODE>(c, in, out, n_dir, st);
    case 32: return launch_reg<32, 32, MODE>(c, in, out, n_dir, st);
    case 48: return launch_reg<48, 48, MODE>(c, in, out, n_dir, st);
    case 64: return launch_reg<64, 64, MODE>(c, in, out, n_dir, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace

template <int NX>
static cudaError_t reg_grp_attr(size_t smem) {
  return cudaFuncSetAttribute(k_xz_reg_grp<NX, NX, XZ_TANGENT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t grp_build_xz_reg(GrpKernel* ks, sp_ctx* const* mem, int n, const int* order,
                             const std::vector<int>& use) {
  std::vector<GXzReg> recs(n);
  for (int m = 0; m < n; ++m) {
    const sp_ctx* c = mem[m];
    recs[m] = GXzReg{};
    if (!use[m]) continue;
    if (!sp_xz_reg_supported(c)) return cudaErrorNotSupported;
    recs[m].a.in = reinterpret_cast<const C2<float>*>(c->ws6);
    recs[m].a.out = reinterpret_cast<C2<float>*>(c->ws3);
    recs[m].a.base = c->base32t;
    recs[m].a.yv = c->yv;
    recs[m].a.NY = c->NY;
    recs[m].a.Mm = c->Mm;
  }
  for (int cls = 0; cls < kGrpRegClasses; ++cls) {
    const int nx = kRegSizes[cls];
    std::vector<int> inst, first(n, 0);
    for (int q = 0; q < n; ++q) {
      const int m = order[q];
      if (!use[m] || mem[m]->nx != nx) continue;
      first[m] = (int)inst.size();
      for (int b = 0; b < mem[m]->NY; ++b) inst.push_back(m);
    }
    GrpKernel* k = ks + cls;
    if (inst.empty()) continue;
    const size_t smem = reg_smem(nx);
    cudaError_t e;
    switch (nx) {
      case 16: e = reg_grp_attr<16>(smem); break;
      case 24: e = reg_grp_attr<24>(smem); break;
      case 32: e = reg_grp_attr<32>(smem); break;
      case 48: e = reg_grp_attr<48>(smem); break;
      default: e = reg_grp_attr<64>(smem); break;
    }
    if (e != cudaSuccess) return e;
    k->blocks = (int)inst.size();
    k->smem = smem;
    if ((e = grp_upload(&k->recs, recs.data(), recs.size() * sizeof(GXzReg))) != cudaSuccess) return e;
    if ((e = grp_upload((void**)&k->inst, inst.data(), inst.size() * sizeof(int))) != cudaSuccess) return e;
    if ((e = grp_upload((void**)&k->first, first.data(), first.size() * sizeof(int))) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t grp_launch_xz_reg(const GrpKernel* ks, const int* active, cudaStream_t st) {
  // largest grids first
  for (int cls = kGrpRegClasses - 1; cls >= 0; --cls) {
    const GrpKernel& k = ks[cls];
    if (k.blocks == 0) continue;
    const GXzReg* r = static_cast<const GXzReg*>(k.recs);
    switch (kRegSizes[cls]) {
      case 16: k_xz_reg_grp<16, 16, XZ_TANGENT><<<k.blocks, kThreadsReg, k.smem, st>>>(r, k.inst, k.first, active); break;
      case 24: k_xz_reg_grp<24, 24, XZ_TANGENT><<<k.blocks, kThreadsReg, k.smem, st>>>(r, k.inst, k.first, active); break;
      case 32: k_xz_reg_grp<32, 32, XZ_TANGENT><<<k.blocks, kThreadsReg, k.smem, st>>>(r, k.inst, k.first, active); break;
      case 48: k_xz_reg_grp<48, 48, XZ_TANGENT><<<k.blocks, kThreadsReg, k.smem, st>>>(r, k.inst, k.first, active); break;
      default: k_xz_reg_grp<64, 64, XZ_TANGENT><<<k.blocks, kThreadsReg, k.smem, st>>>(r, k.inst, k.first, active); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

bool sp_xz_reg_supported(const sp_ctx* c) {
  if (c->nx != c->nz) return false;
  return c->nx == 16 || c->nx == 24 || c->nx == 32 || c->nx == 48 || c->nx == 64;
}

cudaError_t launch_xz_reg(const sp_ctx* c, int mode, const void* in, void* out, int n_dir, cudaStream_t st) {
  if (mode == XZ_TANGENT) return dispatch_reg<XZ_TANGENT>(c, in, out, n_dir, st);
  if (mode == XZ_ADJOINT) return dispatch_reg<XZ_ADJOINT>(c, in, out, n_dir, st);
  return cudaErrorNotSupported;
}
