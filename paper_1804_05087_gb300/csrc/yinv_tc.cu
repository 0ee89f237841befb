// Inverse Chebyshev transform of the mixed-precision tangent on the tensor cores.
//
// Row a2 of the step (Sec. 3.2: Chebyshev in y, products at the collocation points): per Fourier
// mode the values at the Gauss-Lobatto points y_j of u, v, w and of du/dy, dw/dy are
//   V[j][col] = sum_n T[j][n] a_n(col),   D[j][col] = sum_n T'[j][n] a_n(col),
// a dense contraction of the fixed matrices T = (T_n(y_j)) and T' = (T_n'(y_j)) with the columns of
// Chebyshev coefficients of every (field, mode, re/im) of a batch. It runs on the 5th-generation
// tensor cores: tcgen05.mma kind::tf32 with FP32 accumulators in tensor memory, the constant matrices
// brought into shared memory once per block by a bulk TMA copy. TF32 keeps 10 mantissa bits, so each
// operand is split into hi + lo parts (hi = the value rounded to TF32, lo = the rest) and the product
// is hi*hi + hi*lo + lo*hi (three passes; the dropped lo*lo term is below FP32 rounding), which keeps
// the mixed path's accuracy of float arithmetic.
//
// One block (8 warps) handles tiles of 16 modes of one direction: the 96 columns (u, w, v) x 16 modes
// x (re, im), split and stored in the canonical K-major layout of the MMA (8-row x 16-byte core
// matrices, no swizzle); one thread issues the MMAs (M = 128 rows y_j, N = 96 columns with T and
// N = 64 columns (u, w) with T', K = NY rounded up to 8); the tcgen05.commit arrives on an mbarrier;
// each warp then reads 32 rows of the accumulators for 8 of the modes (tcgen05.ld), forms the curl and
// stages the six fields for coalesced stores. Every wait on an mbarrier has an iteration limit: past it the block writes NaN into its
// outputs (a caller sees a non-finite result), frees its tensor memory and returns.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "sp_internal.h"

namespace {

constexpr int kTcModes = 16;       // modes per tile
constexpr int kTcM = 128;          // MMA rows (Gauss-Lobatto points; rows >= NY are zero)
constexpr int kTcCols = 96;        // B columns: (u, w, v) x 16 modes x (re, im)
constexpr int kTcThreads = 256;    // 8 warps: two per TMEM sub-partition
constexpr int kTmemCols = 256;     // accumulators: V in columns [0, 96), D in [96, 160)
constexpr uint32_t kWaitLimit = 1u << 26;
// K-direction stride of the B tiles: 12 core matrices of 128 B plus 16 B, so that the 32 lanes of a
// warp writing 32 consecutive K of one column hit 32 different banks
constexpr uint32_t kLboB = (kTcCols / 8) * 128 + 16;
constexpr uint32_t kLboA = (kTcM / 8) * 128;
// Shared memory is laid out B_hi, B_lo, T_hi, T_lo, T'_hi, T'_lo, padding. Every byte an MMA can
// address stays inside this allocation for 48 <= K <= 72, even if the hardware read the two strides
// of the descriptor the other way round (the padding covers the last tile's reach).
constexpr uint32_t kTcPad = 26880;
constexpr uint32_t kSbo = 128;  // stride between the 8-row core-matrix groups of a K-major tile

// End (exclusive, counted from the descriptor's start address) of what one MMA with K = 8 can
// address in a K-major operand of `rows` rows: two core matrices of 128 bytes along K and rows / 8
// along the rows, with the two strides read as written (lbo along K, sbo along the rows) or swapped.
__host__ __device__ constexpr uint32_t mma_reach(int rows, uint32_t lbo, uint32_t sbo) {
  const uint32_t as_written = lbo + (uint32_t)(rows / 8 - 1) * sbo + 128;
  const uint32_t swapped = sbo + (uint32_t)(rows / 8 - 1) * lbo + 128;
  return as_written > swapped ? as_written : swapped;
}

struct TcArgs {
  const double2* in;     // [dir][3][Mm][NY] complex double (the state layout)
  float2* out;           // [dir][6][NY][Mm] float complex
  const float* amat;     // host-built shared-memory image of T_hi, T_lo, T'_hi, T'_lo
  int NY, Mm, MX, MZ, Kx, ntiles, mtiles;
  double alpha, beta;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: canonical K-major layout without swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture
  return d;                // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
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

// TF32 split: hi keeps the 10 mantissa bits the tensor core reads (rounded), lo the remainder
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  lo = x - hi;
}

// Byte offset of element (row, k) in a K-major canonical tile: 8-row x 16-byte core matrices, rows
// fastest (stride 128 B between 8-row groups), then K (stride lbo between 4-element K groups). With
// either reading of the two descriptor strides every access of an MMA stays inside the allocation.
__host__ __device__ __forceinline__ uint32_t kmajor_off(int row, int k, uint32_t lbo) {
  return (uint32_t)((k >> 2) * lbo + (row >> 3) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

template <int KP>
__global__ void __launch_bounds__(kTcThreads, 1) k_yinv_tc(TcArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_mma, bar_load;
  __shared__ uint32_t tmem_base;
  __shared__ float skx[kTcModes], skz[kTcModes];
  const int NY = a.NY;
  constexpr uint32_t abytes = (uint32_t)kTcM * KP * 4;   // one A matrix
  constexpr uint32_t bbytes = (uint32_t)(KP / 4) * kLboB;  // one B matrix
  // the last MMA on the last A matrix and on the second B matrix stays inside the allocation
  static_assert(3 * abytes + (KP / 8 - 1) * 2 * kLboA + mma_reach(kTcM, kLboA, kSbo) <= 4 * abytes + kTcPad,
                "an MMA on T'_lo could address past the shared-memory allocation");
  static_assert(bbytes + (KP / 8 - 1) * 2 * kLboB + mma_reach(kTcCols, kLboB, kSbo) <= 2 * bbytes + 4 * abytes + kTcPad,
                "an MMA on B_lo could address past the shared-memory allocation");
  unsigned char* sB = smem;                  // B_hi, B_lo
  unsigned char* sA = smem + 2 * bbytes;     // T_hi, T_lo, T'_hi, T'_lo, then kTcPad bytes
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ub_mma = smem_u32(&bar_mma), ub_load = smem_u32(&bar_load);

  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ub_mma));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ub_load));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  bool ok = true;

  // the constant matrices: one bulk copy into shared memory
  if (threadIdx.x == 0) {
    const uint32_t bytes = 4 * abytes;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ub_load), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(sA)),
                 "l"(a.amat), "r"(bytes), "r"(ub_load)
                 : "memory");
  }
  ok = mbar_wait(ub_load, 0);

  constexpr uint32_t sbo = kSbo;
  constexpr uint32_t id_v = idesc_tf32(kTcM, kTcCols), id_d = idesc_tf32(kTcM, 64);
  const size_t planeMm = (size_t)NY * a.Mm;
  uint32_t phase = 0;
  // The B columns of a tile (column c = slot * 32 + 2 * ml + re/im; slot 0 u, 1 w, 2 v; K rows >= NY
  // zero) come from kItems coefficient pairs per thread, consecutive threads taking consecutive K.
  // They are loaded into registers one tile ahead, so that the loads are in flight while the
  // previous tile's MMAs and epilogue run.
  constexpr int kItems = (3 * kTcModes * KP + kTcThreads - 1) / kTcThreads;
  double2 pre[kItems];
  auto prefetch = [&](int tile) {
    const int dir = tile / a.mtiles, m0 = (tile - dir * a.mtiles) * kTcModes;
    const double2* src = a.in + (size_t)dir * 3 * a.Mm * NY;
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const int it = threadIdx.x + r * kTcThreads;
      const int k = it % KP, ml = (it / KP) % kTcModes, slot = it / (KP * kTcModes);
      const int comp = slot == 0 ? 0 : (slot == 1 ? 2 : 1);
      const int m = m0 + ml;
      pre[r] = make_double2(0.0, 0.0);
      if (slot < 3 && k < NY && m < a.Mm) pre[r] = __ldg(src + ((size_t)comp * a.Mm + m) * NY + k);
    }
  };
  float2* stage = reinterpret_cast<float2*>(sB);  // [6][NY][16] output tile, XOR-swizzled columns
  int tile = blockIdx.x;
  if (tile < a.ntiles) prefetch(tile);
  while (tile < a.ntiles && ok) {
    const int dir = tile / a.mtiles, m0 = (tile - dir * a.mtiles) * kTcModes;
    if (threadIdx.x < kTcModes) {
      const int m = min(m0 + threadIdx.x, a.Mm - 1);
      const int pos = m / a.MZ, iz = m - pos * a.MZ;
      const int ix = pos <= a.Kx ? pos : pos - a.MX;
      skx[threadIdx.x] = (float)(a.alpha * ix);
      skz[threadIdx.x] = (float)(a.beta * iz);
    }
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const int it = threadIdx.x + r * kTcThreads;
      const int k = it % KP, ml = (it / KP) % kTcModes, slot = it / (KP * kTcModes);
      if (slot >= 3) continue;
      float h0, l0, h1, l1;
      tf32_split((float)pre[r].x, h0, l0);
      tf32_split((float)pre[r].y, h1, l1);
      const uint32_t off = kmajor_off(slot * 32 + 2 * ml, k, kLboB);
      *reinterpret_cast<float*>(sB + off) = h0;
      *reinterpret_cast<float*>(sB + off + 16) = h1;
      *reinterpret_cast<float*>(sB + bbytes + off) = l0;
      *reinterpret_cast<float*>(sB + bbytes + off + 16) = l1;
    }
    // generic-proxy writes -> visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (threadIdx.x == 0) {
      const uint32_t aT = smem_u32(sA), aTl = aT + abytes, aD = aT + 2 * abytes, aDl = aT + 3 * abytes;
      const uint32_t bh = smem_u32(sB), bl = bh + bbytes;
      const uint32_t pa[3] = {aT, aT, aTl}, pb[3] = {bh, bl, bh};       // hi*hi, hi*lo, lo*hi (T)
      const uint32_t qa[3] = {aD, aD, aDl};                             // the same with T'
#pragma unroll
      for (int pass = 0; pass < 3; ++pass) {
#pragma unroll
        for (int ks = 0; ks < KP / 8; ++ks) {  // 8 TF32 elements of K = two core matrices
          const uint32_t ka = (uint32_t)ks * 2 * kLboA, kb = (uint32_t)ks * 2 * kLboB;
          const uint32_t acc = (pass > 0 || ks > 0) ? 1u : 0u;
          const uint64_t bd = smem_desc(pb[pass] + kb, kLboB, sbo);
          mma_tf32(tmem, smem_desc(pa[pass] + ka, kLboA, sbo), bd, id_v, acc);
          mma_tf32(tmem + kTcCols, smem_desc(qa[pass] + ka, kLboA, sbo), bd, id_d, acc);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(ub_mma)
                   : "memory");
    }
    const int next = tile + gridDim.x;
    if (next < a.ntiles) prefetch(next);
    ok = mbar_wait(ub_mma, phase);
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // epilogue: warp w reads the rows 32 (w mod 4) .. + 31 of its TMEM sub-partition (lane = row j)
    // for the modes 8 (w / 4) .. + 7, 4 at a time, and stages the six fields in shared memory (the B
    // operands are no longer needed)
    const int sub = warp & 3, j = sub * 32 + lane;
    for (int quarter = 2 * (warp >> 2); quarter < 2 * (warp >> 2) + 2 && ok; ++quarter) {
      uint32_t r[5][8];
      const uint32_t base = tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(quarter * 8);
      const uint32_t cols[5] = {0u, 32u, 64u, 96u, 128u};  // u, w, v, Du, Dw
#pragma unroll
      for (int f = 0; f < 5; ++f) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[f][0]), "=r"(r[f][1]), "=r"(r[f][2]), "=r"(r[f][3]), "=r"(r[f][4]), "=r"(r[f][5]),
                       "=r"(r[f][6]), "=r"(r[f][7])
                     : "r"(base + cols[f]));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (j < NY) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int ml = quarter * 4 + q;
          const float kx = skx[ml], kz = skz[ml];
          const float ur = __uint_as_float(r[0][2 * q]), ui = __uint_as_float(r[0][2 * q + 1]);
          const float wr = __uint_as_float(r[1][2 * q]), wi = __uint_as_float(r[1][2 * q + 1]);
          const float vr = __uint_as_float(r[2][2 * q]), vi = __uint_as_float(r[2][2 * q + 1]);
          const float dur = __uint_as_float(r[3][2 * q]), dui = __uint_as_float(r[3][2 * q + 1]);
          const float dwr = __uint_as_float(r[4][2 * q]), dwi = __uint_as_float(r[4][2 * q + 1]);
          // curl: wx = Dw - i kz v, wy = i kz u - i kx w, wz = i kx v - Du
          float2* st = stage + (size_t)j * kTcModes + (ml ^ (j & 15));
          const size_t fs = (size_t)NY * kTcModes;
          st[0 * fs] = make_float2(ur, ui);
          st[1 * fs] = make_float2(vr, vi);
          st[2 * fs] = make_float2(wr, wi);
          st[3 * fs] = make_float2(dwr + kz * vi, dwi - kz * vr);
          st[4 * fs] = make_float2(-kz * ui + kx * wi, kz * ur - kx * wr);
          st[5 * fs] = make_float2(-kx * vi - dur, kx * vr - dui);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    // coalesced stores: 16 consecutive modes of one (field, point) are 128 contiguous bytes
    {
      float2* o = a.out + (size_t)dir * 6 * planeMm;
      const int ml = threadIdx.x & (kTcModes - 1), j0 = threadIdx.x / kTcModes;
      constexpr int rows = kTcThreads / kTcModes;
      if (m0 + ml < a.Mm) {
        for (int f = 0; f < 6; ++f)
          for (int jj = j0; jj < NY; jj += rows)
            o[(size_t)f * planeMm + (size_t)jj * a.Mm + m0 + ml] =
                stage[((size_t)f * NY + jj) * kTcModes + (ml ^ (jj & 15))];
      }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    tile = next;
  }
  if (!ok) {
    // a wait ran out: poison this block's tiles so that the caller sees non-finite values
    const float nan = __int_as_float(0x7fc00000);
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
      const int dir = tile / a.mtiles, m0 = (tile - dir * a.mtiles) * kTcModes;
      for (int it = threadIdx.x; it < 6 * NY * kTcModes; it += blockDim.x) {
        const int ml = it % kTcModes, jj = (it / kTcModes) % NY, f = it / (kTcModes * NY);
        if (m0 + ml < a.Mm) a.out[(size_t)dir * 6 * planeMm + f * planeMm + (size_t)jj * a.Mm + m0 + ml] = make_float2(nan, nan);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

template <int KP>
cudaError_t launch_tc(const TcArgs& a, int grid, size_t sm, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_yinv_tc<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_yinv_tc<KP><<<grid, kTcThreads, sm, st>>>(a);
  return cudaGetLastError();
}

// Forward Chebyshev transform of the mixed tangent on the tensor cores (row a6 of the step, Sec. 3.2):
// the right-hand sides of the per-mode tau rows n <= N-2,
//   W[n][col] = sum_j C[n][j] f_j(col) + u_n(col) / dt,   C[n][j] = 2 T_n(y_j) / (N cbar_n cbar_j),
// for the columns (field, direction, mode, re/im) of a tile of 4 unique modes x 4 directions. The same
// split-TF32 MMAs as the inverse transform (M = 128 rows n, zero past N-2; N = 96 columns; K = NY
// rounded up to 8), the constants C_hi, C_lo brought in by one bulk TMA copy. The epilogue adds the
// FP64 state u/dt (Hermitian-projected on the kz = 0 plane) and writes the chains' right-hand sides.
struct RhsTcArgs {
  const float2* in;       // [dir][3][NY][Mm] float complex values
  const double2* du;      // [dir][3][Mm][NY] the directions (FP64)
  double2* W;             // right-hand sides (u, d, row c NR + n) at u su + d sd + row sn
  long long su, sd, sn;
  const float* amat;      // shared-memory image of C_hi, C_lo
  int NY, Mm, MX, MZ, Kx, NR, n_unique, n_dir, mtiles, ntiles;  // tiles: 4 modes x 4 directions
  double inv_dt;
};

__device__ __forceinline__ void unique_mode_tc(int u, int Kx, int MZ, int* pos, int* iz) {
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

template <int KP>
__global__ void __launch_bounds__(kTcThreads, 1) k_rhs_tc(RhsTcArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_mma, bar_load;
  __shared__ uint32_t tmem_base;
  __shared__ int s_m[4], s_pos[4], s_iz[4];
  const int NY = a.NY;
  constexpr uint32_t abytes = (uint32_t)kTcM * KP * 4;     // one A matrix
  constexpr uint32_t bbytes = (uint32_t)(KP / 4) * kLboB;  // one B matrix
  static_assert(abytes + (KP / 8 - 1) * 2 * kLboA + mma_reach(kTcM, kLboA, kSbo) <= 2 * abytes + kTcPad,
                "an MMA on C_lo could address past the shared-memory allocation");
  static_assert(bbytes + (KP / 8 - 1) * 2 * kLboB + mma_reach(kTcCols, kLboB, kSbo) <= 2 * bbytes + 2 * abytes + kTcPad,
                "an MMA on B_lo could address past the shared-memory allocation");
  constexpr int kCols = 128;                               // tensor-memory columns (96 used)
  unsigned char* sB = smem;                  // B_hi, B_lo
  unsigned char* sA = smem + 2 * bbytes;     // C_hi, C_lo, then kTcPad bytes
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ub_mma = smem_u32(&bar_mma), ub_load = smem_u32(&bar_load);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ub_mma));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ub_load));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  bool ok = true;
  if (threadIdx.x == 0) {
    const uint32_t bytes = 2 * abytes;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ub_load), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(sA)),
                 "l"(a.amat), "r"(bytes), "r"(ub_load)
                 : "memory");
  }
  ok = mbar_wait(ub_load, 0);
  constexpr uint32_t sbo = kSbo;
  constexpr uint32_t id_w = idesc_tf32(kTcM, kTcCols);
  uint32_t phase = 0;
  // A tile is 4 unique modes x 4 directions. B columns: c 32 + 2 (4 dl + ml) + re/im for field c,
  // direction dl, mode ml; K rows >= NY zero. Loaded into registers one tile ahead; a warp takes the 4
  // modes of one direction (one 32-byte sector of the values) at 8 consecutive K, which the padded K
  // stride spreads over the 32 banks.
  constexpr int kItems = (3 * kTcModes * KP + kTcThreads - 1) / kTcThreads;
  float2 pre[kItems];
  auto prefetch = [&](int tile) {
    const int dg = tile / a.mtiles, u0 = (tile - dg * a.mtiles) * 4;
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const int it = threadIdx.x + r * kTcThreads;
      const int ml = it & 3, kr = it >> 2, k = kr % KP, rest = kr / KP, dl = rest & 3, c = rest >> 2;
      pre[r] = make_float2(0.0f, 0.0f);
      const int u = u0 + ml, dir = dg * 4 + dl;
      if (c < 3 && k < NY && u < a.n_unique && dir < a.n_dir) {
        int pos, iz;
        unique_mode_tc(u, a.Kx, a.MZ, &pos, &iz);
        pre[r] = __ldg(a.in + (size_t)dir * 3 * NY * a.Mm + ((size_t)c * NY + k) * a.Mm + pos * a.MZ + iz);
      }
    }
  };
  int tile = blockIdx.x;
  if (tile < a.ntiles) prefetch(tile);
  while (tile < a.ntiles && ok) {
    const int dg = tile / a.mtiles, u0 = (tile - dg * a.mtiles) * 4;
    if (threadIdx.x < 4) {
      const int u = u0 + threadIdx.x;
      int pos = 0, iz = 0;
      if (u < a.n_unique) unique_mode_tc(u, a.Kx, a.MZ, &pos, &iz);
      s_m[threadIdx.x] = u;
      s_pos[threadIdx.x] = pos;
      s_iz[threadIdx.x] = iz;
    }
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const int it = threadIdx.x + r * kTcThreads;
      const int ml = it & 3, kr = it >> 2, k = kr % KP, rest = kr / KP, dl = rest & 3, c = rest >> 2;
      if (c >= 3) continue;
      float h0, l0, h1, l1;
      tf32_split(pre[r].x, h0, l0);
      tf32_split(pre[r].y, h1, l1);
      const uint32_t off = kmajor_off(c * 32 + 2 * (4 * dl + ml), k, kLboB);
      *reinterpret_cast<float*>(sB + off) = h0;
      *reinterpret_cast<float*>(sB + off + 16) = h1;
      *reinterpret_cast<float*>(sB + bbytes + off) = l0;
      *reinterpret_cast<float*>(sB + bbytes + off + 16) = l1;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (threadIdx.x == 0) {
      const uint32_t aC = smem_u32(sA), aCl = aC + abytes;
      const uint32_t bh = smem_u32(sB), bl = bh + bbytes;
      const uint32_t pa[3] = {aC, aC, aCl}, pb[3] = {bh, bl, bh};  // hi*hi, hi*lo, lo*hi
#pragma unroll
      for (int pass = 0; pass < 3; ++pass) {
#pragma unroll
        for (int ks = 0; ks < KP / 8; ++ks) {
          const uint32_t ka = (uint32_t)ks * 2 * kLboA, kb = (uint32_t)ks * 2 * kLboB;
          const uint32_t acc = (pass > 0 || ks > 0) ? 1u : 0u;
          mma_tf32(tmem, smem_desc(pa[pass] + ka, kLboA, sbo), smem_desc(pb[pass] + kb, kLboB, sbo), id_w, acc);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(ub_mma)
                   : "memory");
    }
    const int next = tile + gridDim.x;
    if (next < a.ntiles) prefetch(next);
    ok = mbar_wait(ub_mma, phase);
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // epilogue: warp w reads rows n = 32 (w mod 4) .. + 31 (lane = n) for the directions 2 (w / 4) and
    // 2 (w / 4) + 1 (quarter = direction), adds u_n / dt and writes the right-hand sides of the rows
    // n <= N - 2: a thread writes two adjacent directions of each (mode, field, row)
    const int sub = warp & 3, n = sub * 32 + lane;
    for (int quarter = 2 * (warp >> 2); quarter < 2 * (warp >> 2) + 2 && ok; ++quarter) {
      const int dir = dg * 4 + quarter;
      const double2* dsrc = a.du + (size_t)dir * 3 * a.Mm * NY;
      uint32_t r[3][8];
      const uint32_t base = tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(quarter * 8);
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[f][0]), "=r"(r[f][1]), "=r"(r[f][2]), "=r"(r[f][3]), "=r"(r[f][4]), "=r"(r[f][5]),
                       "=r"(r[f][6]), "=r"(r[f][7])
                     : "r"(base + (uint32_t)(32 * f)));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (n < a.NR && dir < a.n_dir) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int ml = q, u = s_m[ml];
          if (u >= a.n_unique) continue;
          const int pos = s_pos[ml], iz = s_iz[ml];
          const int mpos = pos == 0 ? 0 : a.MX - pos;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            double2 d = __ldg(dsrc + ((size_t)c * a.Mm + pos * a.MZ + iz) * NY + n);
            if (iz == 0) {
              const double2 w = __ldg(dsrc + ((size_t)c * a.Mm + mpos * a.MZ) * NY + n);
              d = make_double2(0.5 * (d.x + w.x), 0.5 * (d.y - w.y));
            }
            double2 fo = make_double2((double)__uint_as_float(r[c][2 * q]) + d.x * a.inv_dt,
                                      (double)__uint_as_float(r[c][2 * q + 1]) + d.y * a.inv_dt);
            if (pos == 0 && iz == 0) fo.y = 0.0;
            a.W[u * a.su + dir * a.sd + (long long)(c * a.NR + n) * a.sn] = fo;
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    tile = next;
  }
  if (!ok) {
    // a wait ran out: poison this block's right-hand sides so that the caller sees non-finite values
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
      const int dg = t / a.mtiles, u0 = (t - dg * a.mtiles) * 4;
      for (int it = threadIdx.x; it < 16 * 3 * a.NR; it += blockDim.x) {
        const int ml = it & 3, dl = (it >> 2) & 3, row = it >> 4, u = u0 + ml, dir = dg * 4 + dl;
        if (u < a.n_unique && dir < a.n_dir)
          a.W[u * a.su + dir * a.sd + (long long)row * a.sn] = make_double2(nan, nan);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
  }
}

template <int KP>
cudaError_t launch_rtc(const RhsTcArgs& a, int grid, size_t sm, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_rhs_tc<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_rhs_tc<KP><<<grid, kTcThreads, sm, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t rhs_tc_smem(int NY) {
  const int Kp = (NY + 7) / 8 * 8;
  return (size_t)2 * kTcM * Kp * 4 + (size_t)2 * (Kp / 4) * kLboB + kTcPad;
}

size_t yinv_tc_smem(int NY) {
  const int Kp = (NY + 7) / 8 * 8;
  return (size_t)4 * kTcM * Kp * 4 + (size_t)2 * (Kp / 4) * kLboB + kTcPad;
}

// 41 <= NY <= 72: the operands fit in shared memory (K <= 72), and K >= 48 keeps every byte an MMA can
// address inside the block's shared memory whichever way the two descriptor strides are read
bool sp_yinv_tc_supported(const sp_ctx* c) {
  return c->geom == 0 && c->yinv_tc_mat != nullptr && c->NY >= 41 && c->NY <= 72;
}

// Host image of the four constant matrices in the kernel's shared-memory layout: T_hi, T_lo,
// T'_hi, T'_lo, each 128 rows x Kp (K-major canonical), rows >= NY and columns >= NY zero.
// th[j][n] = T_n(y_j), td[j][n] = T_n'(y_j) for j, n < NY (row-major, FP64).
std::vector<float> yinv_tc_image(const double* th, const double* td, int NY) {
  const int Kp = (NY + 7) / 8 * 8;
  const size_t one = (size_t)kTcM * Kp;
  std::vector<float> img(4 * one, 0.0f);
  auto put = [&](int which, int row, int k, float v) { img[which * one + kmajor_off(row, k, kLboA) / 4] = v; };
  for (int j = 0; j < NY; ++j)
    for (int n = 0; n < NY; ++n) {
      for (int mat = 0; mat < 2; ++mat) {
        const double x = mat == 0 ? th[(size_t)j * NY + n] : td[(size_t)j * NY + n];
        const float xf = (float)x;
        // round to TF32 (10 mantissa bits, nearest, ties away) as cvt.rna.tf32.f32 does
        uint32_t u;
        std::memcpy(&u, &xf, 4);
        const uint32_t hiu = (u + 0x1000u) & 0xFFFFE000u;
        float hi;
        std::memcpy(&hi, &hiu, 4);
        put(2 * mat, j, n, hi);
        put(2 * mat + 1, j, n, xf - hi);
      }
    }
  return img;
}

cudaError_t launch_yinv_tc(const sp_ctx* c, const double* in, void* out6, int n_dir, cudaStream_t st) {
  if (n_dir <= 0) return cudaSuccess;
  TcArgs a;
  a.in = reinterpret_cast<const double2*>(in);
  a.out = reinterpret_cast<float2*>(out6);
  a.amat = c->yinv_tc_mat;
  a.NY = c->NY;
  a.Mm = c->Mm;
  a.MX = c->MX;
  a.MZ = c->MZ;
  a.Kx = c->Kx;
  a.mtiles = (c->Mm + kTcModes - 1) / kTcModes;
  a.ntiles = a.mtiles * n_dir;
  a.alpha = c->alpha;
  a.beta = c->beta;
  const size_t sm = yinv_tc_smem(c->NY);
  const int grid = std::min(a.ntiles, c->sm_count);
  switch ((c->NY + 7) / 8 * 8) {
    case 48: return launch_tc<48>(a, grid, sm, st);
    case 56: return launch_tc<56>(a, grid, sm, st);
    case 64: return launch_tc<64>(a, grid, sm, st);
    case 72: return launch_tc<72>(a, grid, sm, st);
    default: return cudaErrorInvalidValue;
  }
}

// Host image of C_hi, C_lo for the forward transform: 128 rows n (the tau rows n < NR, then zero) x Kp
// (K-major canonical), cf[n][j] = C[n][j] for n < NR, j < NY (row-major, FP64).
std::vector<float> rhs_tc_image(const double* cf, int NY, int NR) {
  const int Kp = (NY + 7) / 8 * 8;
  const size_t one = (size_t)kTcM * Kp;
  std::vector<float> img(2 * one, 0.0f);
  for (int n = 0; n < NR; ++n)
    for (int j = 0; j < NY; ++j) {
      const float xf = (float)cf[(size_t)n * NY + j];
      uint32_t u;
      std::memcpy(&u, &xf, 4);
      const uint32_t hiu = (u + 0x1000u) & 0xFFFFE000u;  // round to TF32 as cvt.rna.tf32.f32 does
      float hi;
      std::memcpy(&hi, &hiu, 4);
      img[kmajor_off(n, j, kLboA) / 4] = hi;
      img[one + kmajor_off(n, j, kLboA) / 4] = xf - hi;
    }
  return img;
}

bool sp_rhs_tc_supported(const sp_ctx* c) {
  return c->geom == 0 && c->rhs_tc_mat != nullptr && c->NY >= 41 && c->NY <= 72 && c->N - 1 <= kTcM;
}

cudaError_t launch_rhs_tc(const sp_ctx* c, const void* in3, const double* du, void* work, int n_dir, long long su,
                          long long sd, long long sn, cudaStream_t st) {
  if (n_dir <= 0) return cudaSuccess;
  RhsTcArgs a;
  a.in = static_cast<const float2*>(in3);
  a.du = reinterpret_cast<const double2*>(du);
  a.W = static_cast<double2*>(work);
  a.su = su;
  a.sd = sd;
  a.sn = sn;
  a.amat = c->rhs_tc_mat;
  a.NY = c->NY;
  a.Mm = c->Mm;
  a.MX = c->MX;
  a.MZ = c->MZ;
  a.Kx = c->Kx;
  a.NR = c->N - 1;
  a.n_unique = c->n_unique;
  a.n_dir = n_dir;
  a.mtiles = (c->n_unique + 3) / 4;
  a.ntiles = a.mtiles * ((n_dir + 3) / 4);
  a.inv_dt = 1.0 / c->dt;
  const size_t sm = rhs_tc_smem(c->NY);
  const int grid = std::min(a.ntiles, c->sm_count);
  switch ((c->NY + 7) / 8 * 8) {
    case 48: return launch_rtc<48>(a, grid, sm, st);
    case 56: return launch_rtc<56>(a, grid, sm, st);
    case 64: return launch_rtc<64>(a, grid, sm, st);
    case 72: return launch_rtc<72>(a, grid, sm, st);
    default: return cudaErrorInvalidValue;
  }
}
