// One Arnoldi column for small states (GMRES, Sec. 2 and Sec. 3.3: the second term of the cost model
// is the orthogonalisation of each new Krylov vector against the basis).
//
// Classical Gram-Schmidt with selective reorthogonalisation (Daniel, Gragg, Kaufman and Stewart), then
// the normalisation, of a new vector w against the k basis vectors V[0..k):
//   hA = <V, w>,  w' = w - V hA;
//   if |w'|^2 = |w|^2 - |hA|^2 < |w|^2 / 2:  hB = <V, w'>,  w'' = w' - V hB   (else hB = 0, w'' = w');
//   hn = |w''|,  w <- w'' / hn,
// with the inner product <a, b> = sum_e wt(e) Re(conj(a_e) b_e) of the stored coefficients (wt = 1 on
// the kz = 0 plane, 2 elsewhere). The Hessenberg column is hA + hB with hn below the diagonal.
//
// On GB300 the FP64 rate, not memory, bounds this column once the basis sits in L2, so the launches
// are arranged to do the least FP64 work in the fewest dependent steps:
//  * w is stored right after the basis (w = V[k]), so the first dot-product launch over k + 1 rows
//    also gives |w|^2 for the decision;
//  * every block of an update sums the nb partial sums of every coefficient itself (nb <= 32), so no
//    reduction launch sits between a dot product and its update;
//  * the first update takes the decision (every block the same, from the same sums); the second pass
//    runs only when it is needed (its launches return at once otherwise);
//  * the update that produces the final vector also leaves the partial sums of its norm, and the
//    last launch sums them and scales;
//  * the coefficients and the norm go from the kernels straight into pinned host memory.
#include <algorithm>
#include <cstdint>

#include "sp_internal.h"

namespace {

constexpr int kAxTile = 32;   // consecutive entries per row of a block
constexpr int kAxSub = 4;     // tiles per block: 128 entries
constexpr int kAxRows = 8;    // warps: the basis vectors split over them
constexpr int kAxEntries = kAxTile * kAxSub;

struct AxArgs {
  const double* V;   // basis: vector i at V + i * n
  double* w;         // updated in place
  int k;             // basis vectors
  size_t n;          // real entries per state (2 per stored coefficient)
  int NY, MZ;        // coefficient c lies on the plane iz = (c / NY) mod MZ
  const double* part;  // [k (+1)][nb] partial dot products
  int nb;
  double* hdev;      // [k] coefficients (device)
  double* hhost;     // [k] coefficients (pinned host)
  double* hhost2;    // pass 1: the second pass's host coefficients, zeroed if it is skipped
  int* flag;         // pass 1: writes the decision (1: second pass); pass 2: runs only if set
  int pass;          // 1 or 2
  double* normpart;  // [blocks] partial |w_out|^2 of the final vector
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// w -= sum_i h_i V_i on 128 consecutive entries per block, h_i = sum_b part[i][b] summed by the block
// in a fixed order (every block holds the same h)
__global__ void __launch_bounds__(kAxTile * kAxRows) k_axpy_reduce(AxArgs a) {
  extern __shared__ double sh[];  // [k]
  __shared__ double red[kAxRows][kAxTile + 1];
  __shared__ int s_run;
  const int tid = threadIdx.y * kAxTile + threadIdx.x;
  if (a.pass == 2 && !*a.flag) return;  // the first pass kept enough: no second pass
  for (int i = tid; i < a.k; i += kAxTile * kAxRows) {
    double s = 0.0;
    for (int b = 0; b < a.nb; ++b) s += a.part[(size_t)i * a.nb + b];
    sh[i] = s;
    if (blockIdx.x == 0) {
      a.hdev[i] = s;
      a.hhost[i] = s;
    }
  }
  __syncthreads();
  if (a.pass == 1) {
    // decision from |w|^2 (row k of the dot products) and |hA|^2, the same in every block
    if (threadIdx.y == 0) {
      double h2 = 0.0, w2 = 0.0;
      for (int i = threadIdx.x; i < a.k; i += kAxTile) h2 = fma(sh[i], sh[i], h2);
      for (int b = threadIdx.x; b < a.nb; b += kAxTile) w2 += a.part[(size_t)a.k * a.nb + b];
      h2 = warp_sum(h2);
      w2 = warp_sum(w2);
      if (threadIdx.x == 0) {
        s_run = (w2 - h2 < 0.5 * w2) ? 1 : 0;
        if (blockIdx.x == 0) *a.flag = s_run;
      }
    }
    __syncthreads();
    if (!s_run && blockIdx.x == 0)
      for (int i = tid; i < a.k; i += kAxTile * kAxRows) a.hhost2[i] = 0.0;
  }
  const bool final_vec = a.pass == 2 || !s_run;
  double nrm = 0.0;
  for (int t = 0; t < kAxSub; ++t) {
    const size_t e = ((size_t)blockIdx.x * kAxSub + t) * kAxTile + threadIdx.x;
    double acc = 0.0;
    if (e < a.n)
      for (int r = threadIdx.y; r < a.k; r += kAxRows) acc = fma(sh[r], a.V[(size_t)r * a.n + e], acc);
    red[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && e < a.n) {
      double sum = 0.0;
#pragma unroll
      for (int q = 0; q < kAxRows; ++q) sum += red[q][threadIdx.x];
      const double v = a.w[e] - sum;
      a.w[e] = v;
      const unsigned c = (unsigned)(e >> 1);
      const double wt = ((c / (unsigned)a.NY) % (unsigned)a.MZ) == 0 ? 1.0 : 2.0;
      nrm = fma(wt * v, v, nrm);
    }
    __syncthreads();
  }
  if (final_vec && threadIdx.y == 0) {
    nrm = warp_sum(nrm);
    if (threadIdx.x == 0) a.normpart[blockIdx.x] = nrm;
  }
}

// hn = sqrt(sum_b normpart[b]), x <- x / hn (x <- 0 if hn = 0); every block sums the partials itself
// (one warp, fixed order), block 0 stores hn, 1/hn to hdev and hn to hhost
__global__ void k_scale_reduce(double* __restrict__ x, size_t n, const double* part, int np, double* hdev,
                               double* hhost) {
  __shared__ double s_inv;
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int b = threadIdx.x; b < np; b += 32) s += part[b];
    s = warp_sum(s);
    if (threadIdx.x == 0) {
      const double h = sqrt(fmax(s, 0.0));
      const double inv = h > 0.0 ? 1.0 / h : 0.0;
      s_inv = inv;
      if (blockIdx.x == 0) {
        hdev[0] = h;
        hdev[1] = inv;
        hhost[0] = h;
      }
    }
  }
  __syncthreads();
  const double f = s_inv;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] *= f;
}

}  // namespace

int orth_small_blocks(const sp_ctx* c) {
  return (int)((c->state_len + kAxEntries - 1) / kAxEntries);
}

bool orth_small_applies(const sp_ctx* c, int nb) { return c->state_len < 65536 && nb <= 32; }

cudaError_t launch_orth_small(const sp_ctx* c, const double* V, int k, double* w, double* part, int nb, double* hA,
                              double* hB, double* hn, double* host, int kh, int* flag, double* normpart,
                              cudaStream_t st) {
  if (w != V + (size_t)k * c->state_len) return cudaErrorInvalidValue;  // |w|^2 comes from row k
  const size_t n = c->state_len;
  const unsigned blocks = (unsigned)orth_small_blocks(c);
  const size_t sm = (size_t)k * 8;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_axpy_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  AxArgs a;
  a.V = V;
  a.w = w;
  a.k = k;
  a.n = n;
  a.NY = c->NY;
  a.MZ = c->MZ;
  a.part = part;
  a.nb = nb;
  a.hdev = hA;
  a.hhost = host;
  a.hhost2 = host + kh;
  a.flag = flag;
  a.pass = 1;
  a.normpart = normpart;
  cudaError_t e;
  // pass 1 over k + 1 rows: the last is <w, w>
  if ((e = launch_partial_dots(c, V, k + 1, w, part, nb, st, nullptr)) != cudaSuccess) return e;
  k_axpy_reduce<<<blocks, dim3(kAxTile, kAxRows), sm, st>>>(a);
  // pass 2, gated by the decision of pass 1
  if ((e = launch_partial_dots(c, V, k, w, part, nb, st, flag)) != cudaSuccess) return e;
  a.hdev = hB;
  a.hhost = host + kh;
  a.pass = 2;
  k_axpy_reduce<<<blocks, dim3(kAxTile, kAxRows), sm, st>>>(a);
  k_scale_reduce<<<std::max(1u, std::min(blocks, (unsigned)c->sm_count)), 256, 0, st>>>(w, n, normpart, (int)blocks,
                                                                                      hn, host + 2 * kh);
  return cudaGetLastError();
}
