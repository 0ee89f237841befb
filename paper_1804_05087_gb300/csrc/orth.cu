// One Arnoldi column for small states in a single launch (GMRES, Sec. 2 and Sec. 3.3: the second
// term of the cost model is the orthogonalisation of each new Krylov vector against the basis).
//
// Classical Gram-Schmidt applied twice, then the normalisation, on a new vector w against the k basis
// vectors V[0..k):
//   hA = <V, w>,  w' = w - V hA,  hB = <V, w'>,  w'' = w' - V hB,  hn = |w''|,  w <- w'' / hn,
// with the inner product <a, b> = sum_e wt(e) Re(conj(a_e) b_e) of the stored coefficients (wt = 1 on
// the kz = 0 plane, 2 elsewhere). The Hessenberg column is hA + hB with hn below the diagonal.
//
// For states of a few hundred kilobytes the basis sits in L2 and the separate launches of this
// sequence (two dot products with their reductions, two updates, the norm, the scaling, three copies)
// cost more in launch latency than in data movement. Here one cooperative launch does all of it:
// block b owns a contiguous slice of the entries, keeps its slice of w in registers through every
// phase, and the five grid-wide dependencies (each dot product needs every block's partial sums) are
// barriers between phases. Partial sums are reduced in a fixed order, so the result does not depend
// on timing. Block 0 writes hA, hB and hn straight into pinned host memory.
//
// Every barrier wait has an iteration limit; a block whose wait runs out writes NaN into its slice of
// w and into hn and returns, so the caller sees a non-finite column instead of a hang.
#include <algorithm>
#include <cstdint>

#include "sp_internal.h"

namespace {

constexpr int kOrthThreads = 256;  // 8 warps
constexpr int kOrthWarps = kOrthThreads / 32;
constexpr int kOrthEpl = 8;        // entries per lane: a block's slice is at most 256 entries
constexpr uint32_t kSpinLimit = 1u << 24;

struct OrthArgs {
  const double2* V;  // basis: vector i at V + i * n
  double2* w;        // new vector, orthogonalised and normalised in place
  int k, n, chunk;   // basis size, complex entries per state, entries per block
  int NY, MZ;        // entry e lies on the plane iz = (e / NY) mod MZ
  double* part;      // partial sums: [k][G] for the dot products, then [G] for the norm
  double* hA;        // [k] first pass
  double* hB;        // [k] second pass
  double* hn;        // [0] = |w''|, [1] = 1/|w''| (0 if |w''| = 0)
  double* host;      // pinned: hA at [0, k), hB at [kh, kh + k), hn at [2 kh]
  int kh;
  unsigned* bar;     // [0] arrivals, [1] generation
};

// Grid-wide barrier for a cooperative launch: arrive, then wait until the last block to arrive
// advances the generation. Returns false if the wait ran out.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();  // this block's writes before its arrival
    int ok = 1;
    if (atomicAdd(bar, 1u) == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      uint32_t it = 0;
      while (*gen == g) {
        if (++it > kSpinLimit) {
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();  // the other blocks' writes after the release
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partial dot products of the block's slice x (weights folded in) with every basis vector: warp q
// takes the vectors i = q mod 8
__device__ __forceinline__ void slice_dots(const OrthArgs& a, const double2 (&xw)[kOrthEpl], int e0, int cnt,
                                           int nr, int warp, int lane) {
  const int G = gridDim.x;
#pragma unroll 2
  for (int i = warp; i < a.k; i += kOrthWarps) {
    const double2* vi = a.V + (size_t)i * a.n + e0;
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < kOrthEpl; ++r) {
      const int e = lane + 32 * r;
      if (r < nr && e < cnt) {
        const double2 v = __ldg(vi + e);
        s += v.x * xw[r].x + v.y * xw[r].y;
      }
    }
    s = warp_sum(s);
    if (lane == 0) a.part[(size_t)i * G + blockIdx.x] = s;
  }
}

// h[i] = sum over blocks of part[i][.] in block order; one warp per i over the whole grid
__device__ __forceinline__ void reduce_parts(const OrthArgs& a, double* h, int warp, int lane) {
  const int G = gridDim.x;
  for (int i = blockIdx.x * kOrthWarps + warp; i < a.k; i += G * kOrthWarps) {
    double s = 0.0;
    for (int b = lane; b < G; b += 32) s += a.part[(size_t)i * G + b];
    s = warp_sum(s);
    if (lane == 0) h[i] = s;
  }
}

// x <- x - sum_i h[i] V[i] on the block's slice: warp q sums the vectors i = q mod 8, the eight
// partial sums meet in shared memory, and every warp keeps the updated slice in registers
__device__ __forceinline__ void slice_update(const OrthArgs& a, const double* h_glob, double* sh,
                                             double2* red, double2 (&x)[kOrthEpl], int e0, int cnt, int nr,
                                             int warp, int lane) {
  for (int i = threadIdx.x; i < a.k; i += kOrthThreads) sh[i] = h_glob[i];
  __syncthreads();
  double2 acc[kOrthEpl];
#pragma unroll
  for (int r = 0; r < kOrthEpl; ++r) acc[r] = make_double2(0.0, 0.0);
#pragma unroll 2
  for (int i = warp; i < a.k; i += kOrthWarps) {
    const double2* vi = a.V + (size_t)i * a.n + e0;
    const double hi = sh[i];
#pragma unroll
    for (int r = 0; r < kOrthEpl; ++r) {
      const int e = lane + 32 * r;
      if (r < nr && e < cnt) {
        const double2 v = __ldg(vi + e);
        acc[r].x = fma(hi, v.x, acc[r].x);
        acc[r].y = fma(hi, v.y, acc[r].y);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kOrthEpl; ++r)
    if (r < nr) red[warp * (32 * kOrthEpl) + lane + 32 * r] = acc[r];
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kOrthEpl; ++r) {
    if (r < nr) {
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int q = 0; q < kOrthWarps; ++q) {
        const double2 p = red[q * (32 * kOrthEpl) + lane + 32 * r];
        s.x += p.x;
        s.y += p.y;
      }
      x[r].x -= s.x;
      x[r].y -= s.y;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kOrthThreads, 1) k_orth_cgs2(OrthArgs a) {
  extern __shared__ __align__(16) double osh[];  // h [k], then the cross-warp sums [8][256] double2
  double* sh = osh;
  double2* red = reinterpret_cast<double2*>(osh + ((a.k + 1) & ~1));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned G = gridDim.x;
  const int e0 = blockIdx.x * a.chunk;
  const int cnt = max(0, min(a.n - e0, a.chunk));
  const int nr = (cnt + 31) / 32;
  double2 x[kOrthEpl];
  double wt[kOrthEpl];
#pragma unroll
  for (int r = 0; r < kOrthEpl; ++r) {
    const int e = lane + 32 * r;
    x[r] = make_double2(0.0, 0.0);
    wt[r] = 0.0;
    if (r < nr && e < cnt) {
      x[r] = a.w[e0 + e];
      wt[r] = (((unsigned)(e0 + e) / (unsigned)a.NY) % (unsigned)a.MZ) == 0 ? 1.0 : 2.0;
    }
  }
  double2 xw[kOrthEpl];
  bool ok = true;
  // pass A: hA = <V, w>
#pragma unroll
  for (int r = 0; r < kOrthEpl; ++r) xw[r] = make_double2(wt[r] * x[r].x, wt[r] * x[r].y);
  slice_dots(a, xw, e0, cnt, nr, warp, lane);
  ok = grid_barrier(a.bar, G);
  if (ok) {
    reduce_parts(a, a.hA, warp, lane);
    ok = grid_barrier(a.bar, G);
  }
  // w' = w - V hA, pass B: hB = <V, w'>
  if (ok) {
    slice_update(a, a.hA, sh, red, x, e0, cnt, nr, warp, lane);
#pragma unroll
    for (int r = 0; r < kOrthEpl; ++r) xw[r] = make_double2(wt[r] * x[r].x, wt[r] * x[r].y);
    slice_dots(a, xw, e0, cnt, nr, warp, lane);
    ok = grid_barrier(a.bar, G);
  }
  if (ok) {
    reduce_parts(a, a.hB, warp, lane);
    ok = grid_barrier(a.bar, G);
  }
  // w'' = w' - V hB and its squared norm
  double* pn = a.part + (size_t)a.k * G;
  if (ok) {
    slice_update(a, a.hB, sh, red, x, e0, cnt, nr, warp, lane);
    if (warp == 0) {
      double s = 0.0;
#pragma unroll
      for (int r = 0; r < kOrthEpl; ++r) s += wt[r] * (x[r].x * x[r].x + x[r].y * x[r].y);
      s = warp_sum(s);
      if (lane == 0) pn[blockIdx.x] = s;
    }
    ok = grid_barrier(a.bar, G);
  }
  if (!ok) {
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    if (warp == 0) {
#pragma unroll
      for (int r = 0; r < kOrthEpl; ++r) {
        const int e = lane + 32 * r;
        if (r < nr && e < cnt) a.w[e0 + e] = make_double2(nan, nan);
      }
      if (lane == 0) {
        a.hn[0] = nan;
        a.hn[1] = nan;
        a.host[2 * a.kh] = nan;
      }
    }
    return;
  }
  // normalisation: every block sums the norm's partials in the same order
  if (warp == 0) {
    double s = 0.0;
    for (int b = lane; b < (int)G; b += 32) s += pn[b];
    s = warp_sum(s);
    const double h = sqrt(s);
    const double inv = h > 0.0 ? 1.0 / h : 0.0;
#pragma unroll
    for (int r = 0; r < kOrthEpl; ++r) {
      const int e = lane + 32 * r;
      if (r < nr && e < cnt) a.w[e0 + e] = make_double2(x[r].x * inv, x[r].y * inv);
    }
    if (blockIdx.x == 0 && lane == 0) {
      a.hn[0] = h;
      a.hn[1] = inv;
      a.host[2 * a.kh] = h;
    }
  }
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < a.k; i += kOrthThreads) {
      a.host[i] = a.hA[i];
      a.host[a.kh + i] = a.hB[i];
    }
  }
}

}  // namespace

// blocks of the fused launch for this context (0: the state is too large for it)
int orth_fused_blocks(const sp_ctx* c) {
  const size_t n = c->cplx_per_state;
  if (n == 0 || c->state_len >= 65536 || !c->coop) return 0;
  const int G = (int)std::min<size_t>((size_t)c->sm_count, (n + 63) / 64);
  if ((n + G - 1) / G > (size_t)32 * kOrthEpl) return 0;
  return G;
}

size_t orth_fused_smem(int k) {
  return (size_t)((k + 1) & ~1) * 8 + (size_t)kOrthWarps * 32 * kOrthEpl * 16;
}

cudaError_t launch_orth_fused(const sp_ctx* c, const double* V, int k, double* w, double* part, int G, double* hA,
                              double* hB, double* hn, double* host, int kh, unsigned* bar, cudaStream_t st) {
  OrthArgs a;
  a.V = reinterpret_cast<const double2*>(V);
  a.w = reinterpret_cast<double2*>(w);
  a.k = k;
  a.n = (int)c->cplx_per_state;
  a.chunk = (a.n + G - 1) / G;
  a.NY = c->NY;
  a.MZ = c->MZ;
  a.part = part;
  a.hA = hA;
  a.hB = hB;
  a.hn = hn;
  a.host = host;
  a.kh = kh;
  a.bar = bar;
  const size_t sm = orth_fused_smem(k);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_orth_cgs2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kOrthThreads);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_orth_cgs2, a);
}
