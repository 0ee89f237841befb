// CUDA kernels of the BEFE step, its tangent and the vector operations.
//
// One step (Sec. 2, Eq. befe) in Fourier x,z / Chebyshev y is three kernels:
//   k_yinv : per Fourier mode, Chebyshev coefficients -> values at the
//            Gauss-Lobatto points of u, v, w and of the vorticity (curl taken
//            in spectral space: i kx, i kz and the coefficient derivative),
//            written plane-major so that each y-plane is contiguous.
//   k_xz   : per y-plane, the inverse x/z FFTs of the six fields, the
//            pointwise product (U_tot x Omega_tot for the step,
//            U_tot x omega + u x Omega_tot for the tangent), and the forward
//            FFTs truncated to the 2/3-rule modes (pseudospectral products,
//            Sec. 3.2).
//   k_solve: per Fourier mode, values -> Chebyshev coefficients, the
//            right-hand side u/dt + N, the Chebyshev-tau Stokes solve through
//            the precomputed per-mode operators, and G = u_new - u.
//            With laminar advection in L (Sec. 3.6) the right-hand side gains
//            M u = y du/dx + v e_x and the operators are the complex ones of
//            that system (template flag LA).
// T is the real type of the transforms and the product (double or float);
// the solve and everything after it are double.
#include <algorithm>
#include <cstdio>

#include "dev_util.h"
#include "sp_internal.h"

namespace {

constexpr int kThreadsXZ = 256;
constexpr int kThreadsYinv = 256;
constexpr int kThreadsSolve = 128;
constexpr int kThreadsSolveGrp = 192;  // grouped solve (4 modes per block)
constexpr int kTileYinv = 16;   // modes per k_yinv block
constexpr int kTileSolve = 4;   // modes per k_solve block

// ------------------------------------------------------------------ FFT
// Batched complex FFT of length pl.n in shared memory, Stockham
// decimation-in-time with radices 2, 3 and 4. Stage s combines p = radix[s]
// sub-transforms of length L (product of the earlier radices):
//   out[(t0 + L d) R' + b'] = sum_c (w_n^{c t0 R'} in[t0 R + b' + R' c]) w_p^{c d}
// with R = n/L, R' = R/p, w_m = exp(sgn 2 pi i / m). The first stage reads its
// input through `load(b, e)` (element e of transform b), the last stage hands
// its outputs to `store(b, e, v)`; the stages in between ping-pong between s0
// and s1 (layout [element][batch]). Ends with __syncthreads().
template <typename T, class LoadF, class StoreF>
__device__ void fft_batch(const FftPlan& pl, int nb, const C2<T>* __restrict__ tw, T sgn,
                          C2<T>* s0, C2<T>* s1, LoadF load, StoreF store) {
  const int n = pl.n;
  const T h3 = (T)0.86602540378443864676;  // sqrt(3)/2
  int L = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const int p = pl.radix[s];
    const int R = n / L, Rp = R / p;
    const int nbf = n / p;
    const C2<T>* src = (s & 1) ? s0 : s1;
    C2<T>* dst = (s & 1) ? s1 : s0;
    const bool first = (s == 0), last = (s == pl.nst - 1);
    for (int idx = threadIdx.x; idx < nb * nbf; idx += blockDim.x) {
      const int b = idx % nb;
      const int bf = idx / nb;
      const int t0 = bf / Rp, bp = bf - t0 * Rp;
      C2<T> x[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (c < p) {
          const int e = t0 * R + bp + Rp * c;
          x[c] = first ? load(b, e) : src[e * nb + b];
        }
      }
      if (t0 != 0) {
#pragma unroll
        for (int c = 1; c < 4; ++c) {
          if (c < p) {
            C2<T> w = tw[(c * t0 * Rp) % n];
            if (sgn > (T)0) w.y = -w.y;
            x[c] = x[c] * w;
          }
        }
      }
      C2<T> y[4];
      if (p == 2) {
        y[0] = x[0] + x[1];
        y[1] = x[0] - x[1];
      } else if (p == 3) {
        C2<T> t1 = x[1] + x[2];
        C2<T> t2 = mul_is(x[1] - x[2], sgn * h3);
        C2<T> m = x[0] - scl(t1, (T)0.5);
        y[0] = x[0] + t1;
        y[1] = m + t2;
        y[2] = m - t2;
      } else {
        C2<T> a = x[0] + x[2], bb = x[0] - x[2];
        C2<T> c = x[1] + x[3], d = mul_is(x[1] - x[3], sgn);
        y[0] = a + c;
        y[2] = a - c;
        y[1] = bb + d;
        y[3] = bb - d;
      }
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        if (d < p) {
          const int e = (t0 + L * d) * Rp + bp;
          if (last) store(b, e, y[d]);
          else dst[e * nb + b] = y[d];
        }
      }
    }
    __syncthreads();
    L *= p;
  }
}

template <typename T>
__device__ __forceinline__ C2<T> ld_c2(const C2<T>* p) { return *p; }
__device__ __forceinline__ C2<double> ld_c2(const C2<double>* p) {
  double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return mk(v.x, v.y);
}
__device__ __forceinline__ C2<float> ld_c2(const C2<float>* p) {
  float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return mk(v.x, v.y);
}

// ------------------------------------------------------------ k_yinv
struct YinvArgs {
  int Mm, MZ, MX, Kx, NY, N, NH, jchunk;
  int q2, NQ;  // two-level split (N divisible by 4): quarter grid jq = 0..N/4
  double alpha, beta;
};

// Chebyshev tables of k_yinv (T = double or float): Th[j][n] = T_n(y_j), TDh[j][n] = T_n'(y_j)
// on the half grid j <= N/2; for the two-level split also, on the quarter grid jq <= N/4 and
// odd n = 2m+1, Tp[jq][n] = T_n(y_{N/2-jq}) = (-1)^m sin(pi jq n / N) and
// TDp[jq][n] = T_n'(y_{N/2-jq}) = (-1)^m n cos(pi jq n / N) / cos(pi jq / N), and
// tq[jq] = tan(pi jq / N) (the even-degree derivatives at y_{N/2-jq} are tq times the
// alternating sums at y_jq)
template <typename T>
struct YinvTabs {
  const T* Th;
  const T* TDh;
  const T* Tp;
  const T* TDp;
  const T* tq;
};

// in : [dir][3][Mm][NY] complex double (the boundary state layout)
// out: [dir][6][NY][Mm] complex T, fields u, v, w, wx, wy, wz
// (bx, by, bz): mode tile, Gauss-Lobatto chunk, direction
// curl and stores at the Gauss-Lobatto point j: fields u, v, w, wx, wy, wz of mode m
template <typename T>
__device__ __forceinline__ void yinv_store(C2<T>* o, size_t NYMm, size_t base, T kx, T kz, C2<T> u, C2<T> v,
                                           C2<T> w, C2<T> Du, C2<T> Dw) {
  const C2<T> ox = Dw - mul_is(v, kz);
  const C2<T> oy = mul_is(u, kz) - mul_is(w, kx);
  const C2<T> oz = mul_is(v, kx) - Du;
  o[0 * NYMm + base] = u;
  o[1 * NYMm + base] = v;
  o[2 * NYMm + base] = w;
  o[3 * NYMm + base] = ox;
  o[4 * NYMm + base] = oy;
  o[5 * NYMm + base] = oz;
}

// Two-level even/odd split: per quarter-grid point jq the sums over degrees n = 0 and
// n = 2 (mod 4) and over odd n give the values at the four points jq, N - jq, N/2 - jq,
// N/2 + jq (T_n(y_{N-j}) = (-1)^n T_n(y_j); T_n(y_{N/2-j}) = +-T_n(y_j) for n = 0, 2 mod 4),
// a quarter less work than the one-level split.
template <typename T>
__device__ __forceinline__ void yinv_q2(const C2<T>* sc, C2<T>* o, const YinvTabs<T>& tb, const YinvArgs& a, int m0,
                                        int by) {
  const int TM = kTileYinv;
  const int NY = a.NY, Mm = a.Mm, N = a.N;
  const int j_lo = by * a.jchunk;
  const int j_hi = min(a.NQ, j_lo + a.jchunk);
  const int items = TM * (j_hi - j_lo);
  const size_t NYMm = (size_t)NY * Mm;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int t = it % TM;
    const int jq = j_lo + it / TM;
    const int m = m0 + t;
    if (m >= Mm) continue;
    const C2<T> z = mk((T)0, (T)0);
    // [field][0 EE, 1 EO, 2 O, 3 O'] for u, v, w; the same with the derivative tables for u, w
    C2<T> A[3][4] = {{z, z, z, z}, {z, z, z, z}, {z, z, z, z}};
    C2<T> Dd[2][4] = {{z, z, z, z}, {z, z, z, z}};
    const T* trow = tb.Th + (size_t)jq * NY;
    const T* drow = tb.TDh + (size_t)jq * NY;
    const T* prow = tb.Tp + (size_t)jq * NY;
    const T* qrow = tb.TDp + (size_t)jq * NY;
    for (int n = 0; n < NY; ++n) {
      const int r = n & 3;
      const C2<T> u = sc[(0 * NY + n) * TM + t], v = sc[(1 * NY + n) * TM + t], w = sc[(2 * NY + n) * TM + t];
      const T tc = trow[n], td = drow[n];
      if (r == 0) {
        A[0][0] = A[0][0] + scl(u, tc);
        A[1][0] = A[1][0] + scl(v, tc);
        A[2][0] = A[2][0] + scl(w, tc);
        Dd[0][0] = Dd[0][0] + scl(u, td);
        Dd[1][0] = Dd[1][0] + scl(w, td);
      } else if (r == 2) {
        A[0][1] = A[0][1] + scl(u, tc);
        A[1][1] = A[1][1] + scl(v, tc);
        A[2][1] = A[2][1] + scl(w, tc);
        Dd[0][1] = Dd[0][1] + scl(u, td);
        Dd[1][1] = Dd[1][1] + scl(w, td);
      } else {
        const T tp = prow[n], tdp = qrow[n];
        A[0][2] = A[0][2] + scl(u, tc);
        A[1][2] = A[1][2] + scl(v, tc);
        A[2][2] = A[2][2] + scl(w, tc);
        A[0][3] = A[0][3] + scl(u, tp);
        A[1][3] = A[1][3] + scl(v, tp);
        A[2][3] = A[2][3] + scl(w, tp);
        Dd[0][2] = Dd[0][2] + scl(u, td);
        Dd[1][2] = Dd[1][2] + scl(w, td);
        Dd[0][3] = Dd[0][3] + scl(u, tdp);
        Dd[1][3] = Dd[1][3] + scl(w, tdp);
      }
    }
    const int pos = m / a.MZ, iz = m - pos * a.MZ;
    const int ix = pos <= a.Kx ? pos : pos - a.MX;
    const T kx = (T)(a.alpha * ix), kz = (T)(a.beta * iz);
    const T tqv = tb.tq[jq];
    // E at jq and at N/2 - jq; derivatives: even part at N/2 - jq is tq (EO' - EE')
    C2<T> E1[3], E2[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      E1[f] = A[f][0] + A[f][1];
      E2[f] = A[f][0] - A[f][1];
    }
    const C2<T> DE1u = Dd[0][0] + Dd[0][1], DE1w = Dd[1][0] + Dd[1][1];
    const C2<T> DE2u = scl(Dd[0][1] - Dd[0][0], tqv), DE2w = scl(Dd[1][1] - Dd[1][0], tqv);
    const int jl[4] = {jq, N - jq, N / 2 - jq, N / 2 + jq};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = jl[q];
      if (q == 1 && j == jq) continue;                         // jq = N/2 would coincide (never, N >= 4)
      if (q >= 2 && 4 * jq == N) continue;                     // N/2 - jq = jq: already written
      if (q == 3 && jq == 0) continue;                         // N/2 + 0 = N/2 - 0
      const bool hi = (q & 1) != 0;                            // the mirrored point N - j'
      const T sg = hi ? (T)-1 : (T)1;
      const int s2 = q >= 2;
      const C2<T> uu = (s2 ? E2[0] : E1[0]) + scl(A[0][s2 ? 3 : 2], sg);
      const C2<T> vv = (s2 ? E2[1] : E1[1]) + scl(A[1][s2 ? 3 : 2], sg);
      const C2<T> ww = (s2 ? E2[2] : E1[2]) + scl(A[2][s2 ? 3 : 2], sg);
      const C2<T> Du = scl(s2 ? DE2u : DE1u, sg) + Dd[0][s2 ? 3 : 2];
      const C2<T> Dw = scl(s2 ? DE2w : DE1w, sg) + Dd[1][s2 ? 3 : 2];
      yinv_store(o, NYMm, (size_t)j * Mm + m, kx, kz, uu, vv, ww, Du, Dw);
    }
  }
}

template <typename T>
__device__ __forceinline__ void yinv_body(const double2* __restrict__ in, C2<T>* __restrict__ out,
                                          const YinvTabs<T>& tb, const YinvArgs& a, int bx, int by, int bz) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* sc = reinterpret_cast<C2<T>*>(smem_raw);  // [3][NY][TM]
  const int TM = kTileYinv;
  const int m0 = bx * TM;
  const int dir = bz;
  const int NY = a.NY, Mm = a.Mm;
  const double2* src = in + (size_t)dir * 3 * Mm * NY;
  for (int idx = threadIdx.x; idx < 3 * TM * NY; idx += blockDim.x) {
    const int c = idx / (TM * NY);
    const int rem = idx - c * TM * NY;
    const int t = rem / NY, n = rem - t * NY;
    const int m = m0 + t;
    C2<T> v = mk((T)0, (T)0);
    if (m < Mm) {
      double2 d = __ldg(src + ((size_t)c * Mm + m) * NY + n);
      v = mk((T)d.x, (T)d.y);
    }
    sc[(c * NY + n) * TM + t] = v;
  }
  __syncthreads();
  if (sizeof(T) == 8 && a.q2) {  // FP64 only: the float kernel is bound by memory, not arithmetic
    yinv_q2<T>(sc, out + (size_t)dir * 6 * NY * Mm, tb, a, m0, by);
    return;
  }
  const T* Th = tb.Th;
  const T* TDh = tb.TDh;
  const int j_lo = by * a.jchunk;
  const int j_hi = min(a.NH, j_lo + a.jchunk);
  const int items = TM * (j_hi - j_lo);
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int t = it % TM;
    const int jh = j_lo + it / TM;
    const int m = m0 + t;
    if (m >= Mm) continue;
    C2<T> Eu = mk((T)0, (T)0), Ou = Eu, Ev = Eu, Ov = Eu, Ew = Eu, Ow = Eu;
    C2<T> EDu = Eu, ODu = Eu, EDw = Eu, ODw = Eu;
    const T* trow = Th + (size_t)jh * NY;
    const T* drow = TDh + (size_t)jh * NY;
    int n = 0;
    for (; n + 1 < NY; n += 2) {
      const T t0 = trow[n], t1 = trow[n + 1];
      const T d0 = drow[n], d1 = drow[n + 1];
      const C2<T> u0 = sc[(0 * NY + n) * TM + t], u1 = sc[(0 * NY + n + 1) * TM + t];
      const C2<T> v0 = sc[(1 * NY + n) * TM + t], v1 = sc[(1 * NY + n + 1) * TM + t];
      const C2<T> w0 = sc[(2 * NY + n) * TM + t], w1 = sc[(2 * NY + n + 1) * TM + t];
      Eu = Eu + scl(u0, t0); Ou = Ou + scl(u1, t1);
      Ev = Ev + scl(v0, t0); Ov = Ov + scl(v1, t1);
      Ew = Ew + scl(w0, t0); Ow = Ow + scl(w1, t1);
      EDu = EDu + scl(u0, d0); ODu = ODu + scl(u1, d1);
      EDw = EDw + scl(w0, d0); ODw = ODw + scl(w1, d1);
    }
    if (n < NY) {  // NY odd: last (even) degree
      const T t0 = trow[n], d0 = drow[n];
      const C2<T> u0 = sc[(0 * NY + n) * TM + t];
      const C2<T> v0 = sc[(1 * NY + n) * TM + t];
      const C2<T> w0 = sc[(2 * NY + n) * TM + t];
      Eu = Eu + scl(u0, t0); Ev = Ev + scl(v0, t0); Ew = Ew + scl(w0, t0);
      EDu = EDu + scl(u0, d0); EDw = EDw + scl(w0, d0);
    }
    const int pos = m / a.MZ, iz = m - pos * a.MZ;
    const int ix = pos <= a.Kx ? pos : pos - a.MX;
    const T kx = (T)(a.alpha * ix), kz = (T)(a.beta * iz);
    C2<T>* o = out + (size_t)dir * 6 * NY * Mm;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int j = side == 0 ? jh : a.N - jh;
      if (side == 1 && j == jh) break;
      const T sg = side == 0 ? (T)1 : (T)-1;
      // T_n(-y) = (-1)^n T_n(y); T_n'(-y) = (-1)^(n+1) T_n'(y)
      const C2<T> u = Eu + scl(Ou, sg), v = Ev + scl(Ov, sg), w = Ew + scl(Ow, sg);
      const C2<T> Du = scl(EDu, sg) + ODu, Dw = scl(EDw, sg) + ODw;
      const C2<T> ox = Dw - mul_is(v, kz);
      const C2<T> oy = mul_is(u, kz) - mul_is(w, kx);
      const C2<T> oz = mul_is(v, kx) - Du;
      const size_t base = (size_t)j * Mm + m;
      o[0 * (size_t)NY * Mm + base] = u;
      o[1 * (size_t)NY * Mm + base] = v;
      o[2 * (size_t)NY * Mm + base] = w;
      o[3 * (size_t)NY * Mm + base] = ox;
      o[4 * (size_t)NY * Mm + base] = oy;
      o[5 * (size_t)NY * Mm + base] = oz;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreadsYinv) k_yinv(const double2* __restrict__ in,
                                                      C2<T>* __restrict__ out, YinvTabs<T> tb, YinvArgs a) {
  yinv_body<T>(in, out, tb, a, blockIdx.x, blockIdx.y, blockIdx.z);
}

// -------------------------------------------------------------- k_xz
template <typename T>
struct XzArgs {
  const C2<T>* in6;   // [dir][NIN][NY][Mm]  (NIN = 6, or 3 for the adjoint)
  C2<T>* out3;        // [dir][NOUT][NY][Mm] (NOUT = 3, or 6 for the adjoint)
  T* base;            // [6][NY][nx][nz] (read for the tangent, written for BASE)
  const C2<T>* twx;   // [nx] exp(-2 pi i k/nx)
  const C2<T>* twz;
  const double* lam;  // [NY][6] laminar U and Omega added on each plane (step and base)
  FftPlan px, pz;
  int nx, nz, NY, Mm, MX, MZ, Kx, Kz;
  int rp, cx;         // row pairs per z chunk, columns per x chunk
  int FS, RS;         // field and row strides of the plane buffer G
  C2<T>* Gg;          // if non-null, the plane buffers live here, [dir][NY][nx * RS] (large grids)
};

// MODE XZ_ADJOINT runs the transpose of the tangent's plane stage: the
// transpose of the truncated forward FFT (an inverse FFT with the iz > 0 terms
// halved and the 1/(Nx Nz) factor), the transposed product
// (u* = Omega_tot x a, omega* = a x U_tot) and the transpose of the inverse
// FFT (a forward FFT weighted by 1 for iz = 0 and 2 for iz > 0).
// (bx, by): Gauss-Lobatto plane, direction
template <typename T, int MODE>
__device__ __forceinline__ void xz_body(const XzArgs<T>& a, int bx, int by) {
  constexpr int NIN = MODE == XZ_ADJOINT ? 3 : 6;
  constexpr int NOUT = MODE == XZ_ADJOINT ? 6 : 3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<T>* stwx = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* stwz = stwx + a.nx;
  // plane buffer G [nx][6][FS] (row stride RS): in shared memory, or in global
  // memory (L2-resident) for grids whose plane does not fit on chip
  C2<T>* G = a.Gg ? a.Gg + ((size_t)by * a.NY + bx) * a.nx * a.RS : stwz + a.nz;
  C2<T>* S = a.Gg ? stwz + a.nz : G + (size_t)a.nx * a.RS;  // scratch
  const int j = bx;
  const int dir = by;
  const int nx = a.nx, nz = a.nz, MZ = a.MZ, Kx = a.Kx, Kz = a.Kz;
  const int FS = a.FS, RS = a.RS;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) stwx[i] = ld_c2(a.twx + i);
  for (int i = threadIdx.x; i < nz; i += blockDim.x) stwz[i] = ld_c2(a.twz + i);
  __syncthreads();
  const C2<T> zero = mk((T)0, (T)0);
  const size_t planeMm = (size_t)a.NY * a.Mm;
  const C2<T>* in6 = a.in6 + (size_t)dir * NIN * planeMm + (size_t)j * a.Mm;
  const T inv_nxnz = (T)(1.0 / ((double)nx * (double)nz));

  // ---- phase 1: inverse FFT along x of every (field, iz) column
  {
    const int ncol = NIN * MZ;
    for (int c0 = 0; c0 < ncol; c0 += a.cx) {
      const int nb = min(a.cx, ncol - c0);
      auto load = [&](int b, int e) -> C2<T> {
        const int col = c0 + b;
        const int f = col / MZ, iz = col - f * MZ;
        int pos;
        if (e <= Kx) pos = e;
        else if (e >= nx - Kx) pos = e - nx + a.MX;
        else return zero;
        const C2<T> v = ld_c2(in6 + (size_t)f * planeMm + pos * MZ + iz);
        if (MODE == XZ_ADJOINT) return scl(v, iz == 0 ? inv_nxnz : (T)0.5 * inv_nxnz);
        return v;
      };
      auto store = [&](int b, int e, C2<T> v) {
        const int col = c0 + b;
        const int f = col / MZ, iz = col - f * MZ;
        G[e * RS + f * FS + iz] = v;
      };
      fft_batch<T>(a.px, nb, stwx, (T)1, S, S + (size_t)a.cx * nx, load, store);
    }
  }

  // ---- phase 2: per pair of x-rows, c2r along z, product, r2c along z
  T lam[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) lam[f] = (T)a.lam[(size_t)j * 6 + f];
  const int rp = a.rp;
  C2<T>* P0 = S;
  C2<T>* P1 = S + (size_t)6 * rp * nz;
  C2<T>* Q = S + (size_t)12 * rp * nz;
  C2<T>* R = S + (size_t)18 * rp * nz;  // 6 rp nz (the adjoint writes six fields)
  const size_t nxz = (size_t)nx * nz;
  for (int q0 = 0; q0 < nx / 2; q0 += rp) {
    const int nq = min(rp, nx / 2 - q0);
    {
      const int nb = NIN * nq;
      auto load = [&](int b, int e) -> C2<T> {
        const int qq = b / NIN, f = b - qq * NIN;
        const int x0 = 2 * (q0 + qq);
        const C2<T>* g0 = G + x0 * RS + f * FS;
        const C2<T>* g1 = g0 + RS;
        if (e == 0) return mk(g0[0].x, g1[0].x);
        if (e <= Kz) {
          const C2<T> A = g0[e], B = g1[e];
          return mk(A.x - B.y, A.y + B.x);
        }
        if (e >= nz - Kz) {
          const C2<T> A = g0[nz - e], B = g1[nz - e];
          return mk(A.x + B.y, B.x - A.y);
        }
        return zero;
      };
      auto store = [&](int b, int e, C2<T> v) { Q[e * nb + b] = v; };
      fft_batch<T>(a.pz, nb, stwz, (T)1, P0, P1, load, store);
    }
    // pointwise products on the two rows of each pair
    {
      const int nbi = NIN * nq, nbo = NOUT * nq;
      for (int it = threadIdx.x; it < nq * nz; it += blockDim.x) {
        const int qq = it / nz, k = it - qq * nz;
        const int x0 = 2 * (q0 + qq);
        C2<T> fv[NIN];
#pragma unroll
        for (int f = 0; f < NIN; ++f) fv[f] = Q[k * nbi + qq * NIN + f];
        T res[2][NOUT];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          T F[6];
#pragma unroll
          for (int f = 0; f < NIN; ++f) F[f] = r ? fv[f].y : fv[f].x;
          const size_t gidx = (size_t)j * nxz + (size_t)(x0 + r) * nz + k;
          if constexpr (MODE == XZ_BASE) {
#pragma unroll
            for (int f = 0; f < 6; ++f) a.base[(size_t)f * a.NY * nxz + gidx] = F[f] + lam[f];
          } else if constexpr (MODE == XZ_STEP || MODE == XZ_STEP_BASE) {
            const T U0 = F[0] + lam[0], U1 = F[1] + lam[1], U2 = F[2] + lam[2];
            const T O0 = F[3] + lam[3], O1 = F[4] + lam[4], O2 = F[5] + lam[5];
            if constexpr (MODE == XZ_STEP_BASE) {
              const T tot[6] = {U0, U1, U2, O0, O1, O2};
#pragma unroll
              for (int f = 0; f < 6; ++f) a.base[(size_t)f * a.NY * nxz + gidx] = tot[f];
            }
            res[r][0] = U1 * O2 - U2 * O1;
            res[r][1] = U2 * O0 - U0 * O2;
            res[r][2] = U0 * O1 - U1 * O0;
          } else if constexpr (MODE == XZ_TANGENT) {
            T B[6];
#pragma unroll
            for (int f = 0; f < 6; ++f) B[f] = a.base[(size_t)f * a.NY * nxz + gidx];
            // U_tot x omega + u x Omega_tot
            res[r][0] = (B[1] * F[5] - B[2] * F[4]) + (F[1] * B[5] - F[2] * B[4]);
            res[r][1] = (B[2] * F[3] - B[0] * F[5]) + (F[2] * B[3] - F[0] * B[5]);
            res[r][2] = (B[0] * F[4] - B[1] * F[3]) + (F[0] * B[4] - F[1] * B[3]);
          } else {
            T B[6];
#pragma unroll
            for (int f = 0; f < 6; ++f) B[f] = a.base[(size_t)f * a.NY * nxz + gidx];
            // transposed product: u* = Omega_tot x a, omega* = a x U_tot
            res[r][0] = B[4] * F[2] - B[5] * F[1];
            res[r][1] = B[5] * F[0] - B[3] * F[2];
            res[r][2] = B[3] * F[1] - B[4] * F[0];
            res[r][3] = F[1] * B[2] - F[2] * B[1];
            res[r][4] = F[2] * B[0] - F[0] * B[2];
            res[r][5] = F[0] * B[1] - F[1] * B[0];
          }
        }
        if constexpr (MODE != XZ_BASE) {
#pragma unroll
          for (int cc = 0; cc < NOUT; ++cc) R[k * nbo + qq * NOUT + cc] = mk(res[0][cc], res[1][cc]);
        }
      }
      __syncthreads();
    }
    if (MODE != XZ_BASE) {
      const int nb = NOUT * nq;
      auto load = [&](int b, int e) -> C2<T> { return R[e * nb + b]; };
      auto store = [&](int b, int e, C2<T> v) { Q[e * nb + b] = v; };
      fft_batch<T>(a.pz, nb, stwz, (T)-1, P0, P1, load, store);
      // separate the two real rows: A(k) = (X(k) + conj X(-k))/2, B(k) = (X(k) - conj X(-k))/(2i)
      for (int it = threadIdx.x; it < nb * MZ; it += blockDim.x) {
        const int iz = it / nb, b = it - iz * nb;
        const int qq = b / NOUT, cc = b - qq * NOUT;
        const int x0 = 2 * (q0 + qq);
        const C2<T> X = Q[iz * nb + b];
        const C2<T> Xm = Q[((nz - iz) % nz) * nb + b];
        const C2<T> A = scl(X + conj2(Xm), (T)0.5);
        const C2<T> D = X - conj2(Xm);
        G[x0 * RS + cc * FS + iz] = A;
        G[(x0 + 1) * RS + cc * FS + iz] = mk(D.y * (T)0.5, -D.x * (T)0.5);
      }
      __syncthreads();
    }
  }
  if (MODE == XZ_BASE) return;

  // ---- phase 3: forward FFT along x, keep the 2/3-rule modes
  {
    C2<T>* out = a.out3 + (size_t)dir * NOUT * planeMm + (size_t)j * a.Mm;
    const int ncol = NOUT * MZ;
    for (int c0 = 0; c0 < ncol; c0 += a.cx) {
      const int nb = min(a.cx, ncol - c0);
      auto load = [&](int b, int e) -> C2<T> {
        const int col = c0 + b;
        const int cc = col / MZ, iz = col - cc * MZ;
        return G[e * RS + cc * FS + iz];
      };
      auto store = [&](int b, int e, C2<T> v) {
        int pos;
        if (e <= Kx) pos = e;
        else if (e >= nx - Kx) pos = e - nx + a.MX;
        else return;
        const int col = c0 + b;
        const int cc = col / MZ, iz = col - cc * MZ;
        const T sc = MODE == XZ_ADJOINT ? (iz == 0 ? (T)1 : (T)2) : inv_nxnz;
        out[(size_t)cc * planeMm + pos * MZ + iz] = scl(v, sc);
      };
      fft_batch<T>(a.px, nb, stwx, (T)-1, S, S + (size_t)a.cx * nx, load, store);
    }
  }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreadsXZ) k_xz(XzArgs<T> a) {
  xz_body<T, MODE>(a, blockIdx.x, blockIdx.y);
}

// ------------------------------------------------------------ k_solve
struct SolveArgs {
  const double* ops;
  const double* Cfh_d;
  const float* Cfh_f;
  int n_unique, Mm, MX, MZ, Kx, NY, N, NH;
  int cv, rb0, rb1, off_v0, off_v1, off_h0, off_h1, op_stride;
  int off_vc, off_hc;  // complex operators of the laminar-advection variant
  double alpha, beta, inv_dt;
};

__device__ __forceinline__ void unique_to_mode(int u, int Kx, int MZ, int* pos, int* iz) {
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

// in3: [dir][3][NY][Mm] complex T (values of N at the Gauss-Lobatto points)
// du : [dir][3][Mm][NY] complex double; out: same layout (G = u_new - u)
// (bx, by): tile of solved modes, direction
// TM: solved modes per block (any block size works; every mode's arithmetic is the same)
// LA: laminar advection in L (right-hand side + M du, complex operators)
template <typename T, int TM, bool LA>
__device__ __forceinline__ void solve_body(const C2<T>* __restrict__ in3, const double2* __restrict__ du,
                                           double2* __restrict__ out, const SolveArgs& a, int bx, int by) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NY = a.NY, N = a.N, NH = a.NH, Mm = a.Mm, MZ = a.MZ;
  const int NR = N - 1;  // tau rows 0..N-2
  C2<T>* svals = reinterpret_cast<C2<T>*>(smem_raw);                    // [3][NY][TM]
  double2* sdu = reinterpret_cast<double2*>(svals + 3 * NY * TM + (3 * NY * TM) % 2);  // [3][TM][NY]
  double2* sf = sdu + 3 * TM * NY;            // [3][TM][NR]
  double2* srv = sf + 3 * TM * NR;            // [TM][2][cv]
  double2* sfb = srv + TM * 2 * a.cv;         // [TM][NR]
  double2* sfw = sfb + TM * NR;               // [TM][NR] (mean mode w)
  double2* sv = sfw + TM * NR;                // [TM][NY]
  double2* sb = sv + TM * NY;                 // [TM][NY]
  __shared__ int s_pos[TM], s_iz[TM], s_u[TM];
  __shared__ double s_kx[TM], s_kz[TM], s_ik[TM];
  const int u0 = bx * TM;
  const int dir = by;
  if (threadIdx.x < TM) {
    const int u = u0 + threadIdx.x;
    int pos = 0, iz = 0;
    if (u < a.n_unique) unique_to_mode(u, a.Kx, MZ, &pos, &iz);
    s_pos[threadIdx.x] = pos;
    s_iz[threadIdx.x] = iz;
    s_u[threadIdx.x] = u;
    // wavenumbers once per mode: no division or square root in the loops below
    const int ix = pos <= a.Kx ? pos : pos - a.MX;
    const double kx = a.alpha * ix, kz = a.beta * iz;
    const double kk = sqrt(kx * kx + kz * kz);
    s_kx[threadIdx.x] = kx;
    s_kz[threadIdx.x] = kz;
    s_ik[threadIdx.x] = kk > 0 ? 1.0 / kk : 0.0;
  }
  __syncthreads();
  const C2<T>* vin = in3 + (size_t)dir * 3 * NY * Mm;
  const double2* dsrc = du + (size_t)dir * 3 * Mm * NY;
  // phase A: load values and the (Hermitian-projected) input state
  for (int idx = threadIdx.x; idx < 3 * NY * TM; idx += blockDim.x) {
    const int t = idx % TM;
    const int jc = idx / TM;  // c*NY + j
    const int c = jc / NY, jj = jc - c * NY;
    C2<T> v = mk((T)0, (T)0);
    if (s_u[t] < a.n_unique) v = ld_c2(vin + ((size_t)c * NY + jj) * Mm + s_pos[t] * MZ + s_iz[t]);
    svals[idx] = v;
  }
  for (int idx = threadIdx.x; idx < 3 * TM * NY; idx += blockDim.x) {
    const int n = idx % NY;
    const int t = (idx / NY) % TM;
    const int c = idx / (NY * TM);
    double2 v = make_double2(0.0, 0.0);
    if (s_u[t] < a.n_unique) {
      const int pos = s_pos[t], iz = s_iz[t];
      v = __ldg(dsrc + ((size_t)c * Mm + pos * MZ + iz) * NY + n);
      if (iz == 0) {
        const int mpos = pos == 0 ? 0 : a.MX - pos;
        const double2 w = __ldg(dsrc + ((size_t)c * Mm + mpos * MZ) * NY + n);
        v = make_double2(0.5 * (v.x + w.x), 0.5 * (v.y - w.y));
      }
    }
    sdu[(c * TM + t) * NY + n] = v;
  }
  __syncthreads();
  // phase A2: even/odd pairs of the values, once per (component, mode, point pair):
  // s_j = f(y_j) + f(y_N-j) replaces f(y_j), d_j = f(y_j) - f(y_N-j) replaces f(y_N-j)
  // (T_n(y_N-j) = (-1)^n T_n(y_j), so even rows read s and odd rows read d)
  for (int idx = threadIdx.x; idx < 3 * TM * (NH - 1); idx += blockDim.x) {
    const int t = idx % TM;
    const int jj = (idx / TM) % (NH - 1);
    const int c = idx / (TM * (NH - 1));
    C2<T>* col = svals + (c * NY) * TM + t;
    const C2<T> p = col[jj * TM], q = col[(N - jj) * TM];
    col[jj * TM] = p + q;
    col[(N - jj) * TM] = p - q;
  }
  __syncthreads();
  // phase B: forward Chebyshev transform of N (rows 0..N-2) and the RHS u/dt + N; the even and
  // the odd rows in separate loops, so that no warp mixes the two trip counts
  for (int par = 0; par < 2; ++par)
  for (int idx = threadIdx.x, cnt = par ? NR / 2 : (NR + 1) / 2; idx < 3 * TM * cnt; idx += blockDim.x) {
    const int t = idx % TM;
    const int n = 2 * ((idx / TM) % cnt) + par;
    const int c = idx / (TM * cnt);
    C2<T> acc = mk((T)0, (T)0);
    const C2<T>* col = svals + (c * NY) * TM + t;
    if (sizeof(T) == 8) {
      const double* cf = a.Cfh_d + (size_t)n * NH;
      if ((n & 1) == 0) {
        for (int jj = 0; jj < NH - 1; ++jj) acc = acc + scl(col[jj * TM], (T)cf[jj]);
        acc = acc + scl(col[(NH - 1) * TM], (T)cf[NH - 1]);
      } else {
        for (int jj = 0; jj < NH - 1; ++jj) acc = acc + scl(col[(N - jj) * TM], (T)cf[jj]);
      }
    } else {
      const float* cf = a.Cfh_f + (size_t)n * NH;
      if ((n & 1) == 0) {
        for (int jj = 0; jj < NH - 1; ++jj) acc = acc + scl(col[jj * TM], (T)cf[jj]);
        acc = acc + scl(col[(NH - 1) * TM], (T)cf[NH - 1]);
      } else {
        for (int jj = 0; jj < NH - 1; ++jj) acc = acc + scl(col[(N - jj) * TM], (T)cf[jj]);
      }
    }
    const double2 d = sdu[(c * TM + t) * NY + n];
    double2 f = make_double2((double)acc.x + d.x * a.inv_dt, (double)acc.y + d.y * a.inv_dt);
    if constexpr (LA) {
      // + M du on the momentum rows: i kx (Y du)_n, and dv_n in the x-momentum rows
      const double2* dc = sdu + (c * TM + t) * NY;
      double2 yv;
      if (n == 0) yv = make_double2(0.5 * dc[1].x, 0.5 * dc[1].y);
      else if (n == 1) yv = make_double2(dc[0].x + 0.5 * dc[2].x, dc[0].y + 0.5 * dc[2].y);
      else yv = make_double2(0.5 * (dc[n - 1].x + dc[n + 1].x), 0.5 * (dc[n - 1].y + dc[n + 1].y));
      const double kx = s_kx[t];
      f.x = fma(-kx, yv.y, f.x);
      f.y = fma(kx, yv.x, f.y);
      if (c == 0) {
        const double2 dv = sdu[(TM + t) * NY + n];
        f.x += dv.x;
        f.y += dv.y;
      }
    }
    if (s_pos[t] == 0 && s_iz[t] == 0) f.y = 0.0;
    sf[(c * TM + t) * NR + n] = f;
  }
  __syncthreads();
  // phase C: rotate to the components along / across the wavevector; f_v goes to
  // srv (per parity), f~_a = -i f_a replaces f_x in sf (same thread, same slot)
  double2* sfa = sf;  // [TM][NR]: component 0 of sf after this phase
  for (int idx = threadIdx.x; idx < TM * NR; idx += blockDim.x) {
    const int t = idx / NR, n = idx - t * NR;
    const int pos = s_pos[t], iz = s_iz[t];
    const double kx = s_kx[t], kz = s_kz[t], ik = s_ik[t];
    const double2 fx = sf[(0 * TM + t) * NR + n];
    const double2 fy = sf[(1 * TM + t) * NR + n];
    const double2 fz = sf[(2 * TM + t) * NR + n];
    if (pos == 0 && iz == 0) {
      sfb[t * NR + n] = fx;
      sfw[t * NR + n] = fz;
      continue;
    }
    const double2 fa = make_double2((kx * fx.x + kz * fz.x) * ik, (kx * fx.y + kz * fz.y) * ik);
    const double2 fb = make_double2((-kz * fx.x + kx * fz.x) * ik, (-kz * fx.y + kx * fz.y) * ik);
    sfb[t * NR + n] = fb;
    srv[(t * 2 + (n & 1)) * a.cv + n / 2] = fy;         // f_v row n -> parity n & 1
    sfa[t * NR + n] = make_double2(fa.y, -fa.x);        // f~_a = -i f_a
  }
  __syncthreads();
  // phase C2: reduced right-hand side g_n = f_v,n - (2 / (c_n k)) sum_{m > n, m + n odd,
  // m <= N-2} m f~_a,m for each parity P. With x_n = (n+1) f~_a,n+1 the sum is the inclusive
  // suffix sum of x over the rows of parity P: one warp per (mode, parity), a shuffle scan over
  // chunks of 32 rows from the top, carrying the total of the chunks above.
  {
    const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int pair = threadIdx.x >> 5; pair < 2 * TM; pair += nwarps) {
      const int t = pair >> 1, P = pair & 1;
      if (s_u[t] >= a.n_unique || (s_pos[t] == 0 && s_iz[t] == 0)) continue;  // whole warp
      const double ik = s_ik[t];
      double2* g = srv + (t * 2 + P) * a.cv;
      const int cnt = P == 0 ? a.rb0 : a.rb1;  // rows n = 2i + P <= N-2
      double2 carry = make_double2(0.0, 0.0);
      for (int c0 = ((cnt - 1) >> 5) << 5; c0 >= 0; c0 -= 32) {
        const int i = c0 + lane, n = 2 * i + P;
        double2 x = make_double2(0.0, 0.0);
        if (i < cnt && n + 1 <= N - 2) {
          const double2 fa = sfa[t * NR + n + 1];
          x = make_double2((double)(n + 1) * fa.x, (double)(n + 1) * fa.y);
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const double yx = __shfl_down_sync(0xffffffffu, x.x, o);
          const double yy = __shfl_down_sync(0xffffffffu, x.y, o);
          if (lane + o < 32) {
            x.x += yx;
            x.y += yy;
          }
        }
        x.x += carry.x;
        x.y += carry.y;
        if (i < cnt) {
          const double f = (n == 0 ? 1.0 : 2.0) * ik;
          const double2 v = g[i];
          g[i] = make_double2(v.x - f * x.x, v.y - f * x.y);
        }
        carry = make_double2(__shfl_sync(0xffffffffu, x.x, 0), __shfl_sync(0xffffffffu, x.y, 0));
      }
    }
  }
  __syncthreads();
  // phase D: apply the per-mode operators (FP64). Threads take the even unknowns of a
  // mode first, then the odd ones, so that a warp reads consecutive rows of one
  // column-major operator (coalesced). The mean-mode test is hoisted out of the
  // loops so that no predicated-off double FMA occupies the FP64 pipe.
  const int nv0 = N / 2 + 1;  // even unknowns
  if constexpr (LA) {
    // D1: v = V' g, one complex row per thread (consecutive rows: coalesced columns)
    for (int idx = threadIdx.x; idx < TM * NY; idx += blockDim.x) {
      const int t = idx / NY, n = idx - t * NY;
      if (s_u[t] >= a.n_unique || (s_pos[t] == 0 && s_iz[t] == 0)) continue;
      const double2* V = reinterpret_cast<const double2*>(a.ops + (size_t)s_u[t] * a.op_stride + a.off_vc) + n;
      sv[t * NY + n] = cdot4(V, NY, srv + t * 2 * a.cv, NR);
    }
    __syncthreads();
    // D1b: right-hand side of b, f_b + (kz/k) v on the momentum rows
    for (int idx = threadIdx.x; idx < TM * NR; idx += blockDim.x) {
      const int t = idx / NR, n = idx - t * NR;
      if (s_u[t] >= a.n_unique || (s_pos[t] == 0 && s_iz[t] == 0)) continue;
      const double s = s_kz[t] * s_ik[t];
      const double2 v = sv[t * NY + n];
      double2 fb = sfb[t * NR + n];
      fb.x = fma(s, v.x, fb.x);
      fb.y = fma(s, v.y, fb.y);
      sfb[t * NR + n] = fb;
    }
    __syncthreads();
    // D2: b = H' (f_b + (kz/k) v); the mean mode uses the real Helmholtz operators
    for (int idx = threadIdx.x; idx < TM * NY; idx += blockDim.x) {
      const int t = idx / NY, k = idx - t * NY;
      if (s_u[t] >= a.n_unique) continue;
      const double* op = a.ops + (size_t)s_u[t] * a.op_stride;
      if (s_pos[t] == 0 && s_iz[t] == 0) {
        const int Q = k < nv0 ? 0 : 1, row = Q == 0 ? k : k - nv0, n = 2 * row + Q;
        const int nrow = Q == 0 ? nv0 : NY - nv0;
        const int rb = Q == 0 ? a.rb0 : a.rb1;
        const double* H = op + (Q == 0 ? a.off_h0 : a.off_h1) + row;
        sb[t * NY + n] = dot4(H, nrow, sfb + t * NR + Q, 2, rb);
        sv[t * NY + n] = dot4(H, nrow, sfw + t * NR + Q, 2, rb);
        continue;
      }
      const double2* H = reinterpret_cast<const double2*>(op + a.off_hc) + k;
      sb[t * NY + k] = cdot4(H, NY, sfb + t * NR, NR);
    }
    __syncthreads();
  } else {
  for (int idx = threadIdx.x; idx < TM * NY; idx += blockDim.x) {
    const int t = idx / NY, k = idx - t * NY;
    if (s_u[t] >= a.n_unique) continue;
    const double* op = a.ops + (size_t)s_u[t] * a.op_stride;
    const int Q = k < nv0 ? 0 : 1, row = Q == 0 ? k : k - nv0, n = 2 * row + Q;
    const int nrow = Q == 0 ? nv0 : NY - nv0;
    const int rb = Q == 0 ? a.rb0 : a.rb1;
    const double* H = op + (Q == 0 ? a.off_h0 : a.off_h1) + row;
    const double2* fbq = sfb + t * NR + Q;
    if (s_pos[t] == 0 && s_iz[t] == 0) {
      // mean flow: u and w from the Helmholtz operator, v = 0
      const double2* fwq = sfw + t * NR + Q;
      sb[t * NY + n] = dot4(H, nrow, fbq, 2, rb);
      sv[t * NY + n] = dot4(H, nrow, fwq, 2, rb);
      continue;
    }
    sb[t * NY + n] = dot4(H, nrow, fbq, 2, rb);
    const double* V = op + (Q == 0 ? a.off_v0 : a.off_v1) + row;
    sv[t * NY + n] = dot4(V, nrow, srv + (t * 2 + Q) * a.cv, 1, rb);
  }
  __syncthreads();
  }
  // (D v)_n = (2/c_n) sum_{p > n, p + n odd} p v_p: one suffix sum per (mode, parity),
  // kept in sfb (free after phase D) as S_n = sum_{p >= n, p = n mod 2} p v_p
  double2* ssum = sfb;
  if (threadIdx.x < 2 * TM) {
    const int t = threadIdx.x >> 1, par = threadIdx.x & 1;
    double2 acc = make_double2(0.0, 0.0);
    const int top = ((NY - 1 - par) & 1) ? NY - 2 : NY - 1;  // largest index of this parity
    for (int p = top; p >= 0; p -= 2) {
      const double2 vp = sv[t * NY + p];
      acc.x += p * vp.x;
      acc.y += p * vp.y;
      ssum[t * NY + p] = acc;
    }
  }
  __syncthreads();
  // phase E: a = (i/k) D v, back-rotation, G = u_new - u, Hermitian output
  double2* dst = out + (size_t)dir * 3 * Mm * NY;
  for (int idx = threadIdx.x; idx < TM * NY; idx += blockDim.x) {
    const int t = idx / NY, n = idx - t * NY;
    if (s_u[t] >= a.n_unique) continue;
    const int pos = s_pos[t], iz = s_iz[t];
    double2 un, vn, wn;
    if (pos == 0 && iz == 0) {
      un = make_double2(sb[t * NY + n].x, 0.0);
      wn = make_double2(sv[t * NY + n].x, 0.0);
      vn = make_double2(0.0, 0.0);
    } else {
      const double kx = s_kx[t], kz = s_kz[t], ik = s_ik[t];
      double2 dv = make_double2(0.0, 0.0);
      if (n + 1 < NY) {
        const double2 sp = ssum[t * NY + n + 1];
        const double f = n == 0 ? 1.0 : 2.0;
        dv = make_double2(f * sp.x, f * sp.y);
      }
      const double2 an = make_double2(-dv.y * ik, dv.x * ik);  // (i/k) Dv
      const double2 bn = sb[t * NY + n];
      un = make_double2((kx * an.x - kz * bn.x) * ik, (kx * an.y - kz * bn.y) * ik);
      wn = make_double2((kz * an.x + kx * bn.x) * ik, (kz * an.y + kx * bn.y) * ik);
      vn = sv[t * NY + n];
    }
    const double2 res[3] = {un, vn, wn};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double2 d = sdu[(c * TM + t) * NY + n];
      double2 g = make_double2(res[c].x - d.x, res[c].y - d.y);
      if (pos == 0 && iz == 0) g.y = 0.0;
      dst[((size_t)c * Mm + pos * MZ + iz) * NY + n] = g;
      if (iz == 0 && pos != 0) {
        dst[((size_t)c * Mm + (a.MX - pos) * MZ) * NY + n] = make_double2(g.x, -g.y);
      }
    }
  }
}

template <typename T, int TM, int THREADS, bool LA>
__global__ void __launch_bounds__(THREADS) k_solve(const C2<T>* __restrict__ in3, const double2* __restrict__ du,
                                                   double2* __restrict__ out, SolveArgs a) {
  // with laminar advection in L the grid runs directions fastest: blocks that run together share a
  // mode tile, so its complex operators (133 KB per mode) are read from DRAM once and from L2 after
  if constexpr (LA) solve_body<T, TM, LA>(in3, du, out, a, blockIdx.y, blockIdx.x);
  else solve_body<T, TM, LA>(in3, du, out, a, blockIdx.x, blockIdx.y);
}


// ------------------------------------------------------------ adjoint
// The adjoint of the tangent in the weighted inner product <a,b> =
// sum w(iz) Re(conj a b) is J* = W^-1 J^T W with J^T the plain transpose.
// The tangent is J = P S (1/dt + M) P - P (P: Hermitian projection, S: the
// per-mode solve, M: curl, values, plane stage, Chebyshev coefficients), so
// J^T r' = P (1/dt + M^T) S^T P r' - P r' with r' = W r. The chain below
// evaluates it stage by stage in reverse order.

// k_solve_adj: r' = P W r, f* = S^T r' (transposed per-mode operators),
// out = f*/dt (boundary layout) and vals = Cf^T f* (values at the
// Gauss-Lobatto points, plane-major) for every stored mode.
template <typename T>
__global__ void __launch_bounds__(kThreadsSolve) k_solve_adj(const double2* __restrict__ r,
                                                             double2* __restrict__ out,
                                                             C2<T>* __restrict__ vals, SolveArgs a,
                                                             int weighted) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TM = kTileSolve;
  const int NY = a.NY, N = a.N, NH = a.NH, Mm = a.Mm, MZ = a.MZ;
  const int NR = N - 1;
  double2* sg = reinterpret_cast<double2*>(smem_raw);  // [3][TM][NY] r' (u, v, w)
  double2* sga = sg + 3 * TM * NY;                     // [TM][NY] along-k part
  double2* sgb = sga + TM * NY;                        // [TM][NY] across-k part
  double2* sva = sgb + TM * NY;                        // [TM][NY] v* = gv + D^T(-i ga/k)
  double2* srv = sva + TM * NY;                        // [TM][2][cv] V_P^T v*
  double2* sfb = srv + TM * 2 * a.cv;                  // [TM][NR] H^T gb (or H^T gu)
  double2* sfw = sfb + TM * NR;                        // [TM][NR] H^T gw (mean mode)
  double2* sf = sfw + TM * NR;                         // [3][TM][NR] f*
  __shared__ int s_pos[kTileSolve], s_iz[kTileSolve], s_u[kTileSolve];
  __shared__ double s_kx[kTileSolve], s_kz[kTileSolve], s_ik[kTileSolve];
  const int u0 = blockIdx.x * TM;
  const int dir = blockIdx.y;
  if (threadIdx.x < TM) {
    const int u = u0 + threadIdx.x;
    int pos = 0, iz = 0;
    if (u < a.n_unique) unique_to_mode(u, a.Kx, MZ, &pos, &iz);
    s_pos[threadIdx.x] = pos;
    s_iz[threadIdx.x] = iz;
    s_u[threadIdx.x] = u;
    const int ix = pos <= a.Kx ? pos : pos - a.MX;
    const double kx = a.alpha * ix, kz = a.beta * iz;
    const double k = sqrt(kx * kx + kz * kz);
    s_kx[threadIdx.x] = kx;
    s_kz[threadIdx.x] = kz;
    s_ik[threadIdx.x] = k > 0 ? 1.0 / k : 0.0;
  }
  __syncthreads();
  const double2* rsrc = r + (size_t)dir * 3 * Mm * NY;
  // r' = P W r
  for (int idx = threadIdx.x; idx < 3 * TM * NY; idx += blockDim.x) {
    const int n = idx % NY;
    const int t = (idx / NY) % TM;
    const int c = idx / (NY * TM);
    double2 v = make_double2(0.0, 0.0);
    if (s_u[t] < a.n_unique) {
      const int pos = s_pos[t], iz = s_iz[t];
      v = __ldg(rsrc + ((size_t)c * Mm + pos * MZ + iz) * NY + n);
      if (iz == 0) {
        const int mpos = pos == 0 ? 0 : a.MX - pos;
        const double2 w = __ldg(rsrc + ((size_t)c * Mm + mpos * MZ) * NY + n);
        v = make_double2(0.5 * (v.x + w.x), 0.5 * (v.y - w.y));
      } else if (weighted) {
        v = make_double2(2.0 * v.x, 2.0 * v.y);
      }
    }
    sg[(c * TM + t) * NY + n] = v;
  }
  __syncthreads();
  // rotation^T: ga = (kx gu + kz gw)/k, gb = (-kz gu + kx gw)/k
  for (int idx = threadIdx.x; idx < TM * NY; idx += blockDim.x) {
    const int t = idx / NY, n = idx - t * NY;
    const double2 gu = sg[(0 * TM + t) * NY + n], gw = sg[(2 * TM + t) * NY + n];
    if (s_pos[t] == 0 && s_iz[t] == 0) {
      sga[idx] = gu;
      sgb[idx] = gw;
      continue;
    }
    const double kx = s_kx[t], kz = s_kz[t], ik = s_ik[t];
    sga[idx] = make_double2((kx * gu.x + kz * gw.x) * ik, (kx * gu.y + kz * gw.y) * ik);
    sgb[idx] = make_double2((-kz * gu.x + kx * gw.x) * ik, (-kz * gu.y + kx * gw.y) * ik);
  }
  __syncthreads();
  // a = (i/k) D v  =>  v* = gv + D^T (-i ga / k); (D^T x)_n = sum_{m<n, m+n odd} (2n/c_m) x_m
  for (int idx = threadIdx.x; idx < TM * NY; idx += blockDim.x) {
    const int t = idx / NY, n = idx - t * NY;
    const double2 gv = sg[(1 * TM + t) * NY + n];
    if (s_pos[t] == 0 && s_iz[t] == 0) {
      sva[idx] = make_double2(0.0, 0.0);
      continue;
    }
    double2 acc = make_double2(0.0, 0.0);
    for (int m = (n & 1) ? 0 : 1; m < n; m += 2) {
      const double2 x = sga[t * NY + m];
      const double cm = m == 0 ? 0.5 : 1.0;
      acc.x += cm * x.x;
      acc.y += cm * x.y;
    }
    const double s = 2.0 * n * s_ik[t];
    // -i ga / k: (x + i y) * (-i) = y - i x
    sva[idx] = make_double2(gv.x + s * acc.y, gv.y - s * acc.x);
  }
  __syncthreads();
  // V_P^T v* (columns of V_P: the adjoint of g) and H_Q^T gb
  for (int idx = threadIdx.x; idx < TM * 2 * a.cv; idx += blockDim.x) {
    const int t = idx / (2 * a.cv), rem = idx - t * 2 * a.cv;
    const int P = rem / a.cv, col = rem - P * a.cv;
    if (s_u[t] >= a.n_unique || (s_pos[t] == 0 && s_iz[t] == 0) || col >= (P == 0 ? a.rb0 : a.rb1)) {
      srv[idx] = make_double2(0.0, 0.0);
      continue;
    }
    const double* V = a.ops + (size_t)s_u[t] * a.op_stride + (P == 0 ? a.off_v0 : a.off_v1);
    const int nv = P == 0 ? N / 2 + 1 : N / 2;
    srv[idx] = dot4(V + (size_t)col * nv, 1, sva + t * NY + P, 2, nv);  // column col of V_P
  }
  for (int idx = threadIdx.x; idx < TM * NR; idx += blockDim.x) {
    const int t = idx / NR, n = idx - t * NR;  // momentum row n
    if (s_u[t] >= a.n_unique) continue;
    const int Q = n & 1, col = n >> 1;
    const int nrow = Q == 0 ? N / 2 + 1 : N / 2;
    const double* H = a.ops + (size_t)s_u[t] * a.op_stride + (Q == 0 ? a.off_h0 : a.off_h1);
    const bool mean = s_pos[t] == 0 && s_iz[t] == 0;
    const double* Hc = H + (size_t)col * nrow;  // column col of H_Q
    sfb[idx] = dot4(Hc, 1, sgb + t * NY + Q, 2, nrow);
    // sga holds gu and sgb holds gw for the mean mode
    sfw[idx] = mean ? dot4(Hc, 1, sga + t * NY + Q, 2, nrow) : make_double2(0.0, 0.0);
  }
  __syncthreads();
  // g = f_v - (1/k) D f~_a  =>  f_v* = g*, f~_a*,m = -(2m/k) sum_{n < m, n + m odd} g*_n / c_n
  // (prefix sums over the f_v rows of the other parity), kept in component 0 of sf
  double2* sfa = sf;
  if (threadIdx.x < 2 * TM) {
    const int t = threadIdx.x >> 1, q = threadIdx.x & 1;  // parity of the f~_a rows
    if (s_u[t] < a.n_unique && !(s_pos[t] == 0 && s_iz[t] == 0)) {
      const double2* gs = srv + (t * 2 + (1 - q)) * a.cv;  // g* of parity 1 - q
      const double ik = s_ik[t];
      double2 S = make_double2(0.0, 0.0);
      for (int m = q; m <= N - 2; m += 2) {
        if (m >= 1) {
          const int n = m - 1;
          const double w = n == 0 ? 0.5 : 1.0;
          const double2 x = gs[n >> 1];
          S.x = fma(w, x.x, S.x);
          S.y = fma(w, x.y, S.y);
        }
        const double f = -2.0 * m * ik;
        sfa[t * NR + m] = make_double2(f * S.x, f * S.y);
      }
    }
  }
  __syncthreads();
  // f* per component, rows 0..N-2 (each thread reads its f~_a* slot before overwriting it)
  for (int idx = threadIdx.x; idx < TM * NR; idx += blockDim.x) {
    const int t = idx / NR, n = idx - t * NR;
    double2 fx, fy, fz;
    if (s_pos[t] == 0 && s_iz[t] == 0) {
      fx = make_double2(sfw[idx].x, 0.0);  // H^T gu
      fz = make_double2(sfb[idx].x, 0.0);  // H^T gw
      fy = make_double2(0.0, 0.0);
    } else {
      const int P = n & 1;
      fy = srv[(t * 2 + P) * a.cv + (n >> 1)];
      const double2 fta = sfa[t * NR + n];
      const double2 fa = make_double2(-fta.y, fta.x);  // f_a* = i f~_a*
      const double2 fb = sfb[idx];
      const double kx = s_kx[t], kz = s_kz[t], ik = s_ik[t];
      fx = make_double2((kx * fa.x - kz * fb.x) * ik, (kx * fa.y - kz * fb.y) * ik);
      fz = make_double2((kz * fa.x + kx * fb.x) * ik, (kz * fa.y + kx * fb.y) * ik);
    }
    sf[(0 * TM + t) * NR + n] = fx;
    sf[(1 * TM + t) * NR + n] = fy;
    sf[(2 * TM + t) * NR + n] = fz;
  }
  __syncthreads();
  // out = f*/dt (boundary layout, rows N-1, N zero), mirrored for iz = 0
  double2* dst = out + (size_t)dir * 3 * Mm * NY;
  for (int idx = threadIdx.x; idx < 3 * TM * NY; idx += blockDim.x) {
    const int n = idx % NY;
    const int t = (idx / NY) % TM;
    const int c = idx / (NY * TM);
    if (s_u[t] >= a.n_unique) continue;
    const int pos = s_pos[t], iz = s_iz[t];
    double2 v = make_double2(0.0, 0.0);
    if (n < NR) {
      const double2 f = sf[(c * TM + t) * NR + n];
      v = make_double2(f.x * a.inv_dt, f.y * a.inv_dt);
    }
    dst[((size_t)c * Mm + pos * MZ + iz) * NY + n] = v;
    if (iz == 0 && pos != 0) dst[((size_t)c * Mm + (a.MX - pos) * MZ) * NY + n] = make_double2(v.x, -v.y);
  }
  // vals = Cf^T f*: sum_n Cf[n][j] f*_n with Cf[n][N-j] = (-1)^n Cf[n][j]
  C2<T>* vdst = vals + (size_t)dir * 3 * NY * Mm;
  for (int idx = threadIdx.x; idx < 3 * TM * NH; idx += blockDim.x) {
    const int t = idx % TM;
    const int jh = (idx / TM) % NH;
    const int c = idx / (TM * NH);
    if (s_u[t] >= a.n_unique) continue;
    C2<T> E = mk((T)0, (T)0), O = E;
    const double2* f = sf + (c * TM + t) * NR;
    for (int n = 0; n < NR; ++n) {
      const T cf = sizeof(T) == 8 ? (T)a.Cfh_d[(size_t)n * NH + jh] : (T)a.Cfh_f[(size_t)n * NH + jh];
      const C2<T> fv = mk((T)f[n].x, (T)f[n].y);
      if (n & 1) O = O + scl(fv, cf);
      else E = E + scl(fv, cf);
    }
    const int pos = s_pos[t], iz = s_iz[t];
    const int m = pos * MZ + iz, mm = (a.MX - pos) * MZ;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int j = side == 0 ? jh : N - jh;
      if (side == 1 && j == jh) break;
      const C2<T> v = side == 0 ? E + O : E - O;
      vdst[((size_t)c * NY + j) * Mm + m] = v;
      if (iz == 0 && pos != 0) vdst[((size_t)c * NY + j) * Mm + mm] = conj2(v);
    }
  }
}

// k_yinv_adj: the transpose of k_yinv. In value space the curl gives
//   u* += gu - i kz gy, v* += gv + i kz gx - i kx gz, w* += gw + i kx gy,
//   (Du)* = -gz, (Dw)* = gx;
// then coefficients: x*_n = sum_j T_n(y_j) x*_j + sum_j T_n'(y_j) (Dx)*_j,
// added to `out` (which already holds f*/dt).
template <typename T>
__global__ void __launch_bounds__(kThreadsYinv) k_yinv_adj(const C2<T>* __restrict__ in,
                                                          double2* __restrict__ out,
                                                          const T* __restrict__ Th,
                                                          const T* __restrict__ TDh, YinvArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TM = kTileYinv;
  const int NY = a.NY, Mm = a.Mm, N = a.N, NH = a.NH;
  C2<T>* s5 = reinterpret_cast<C2<T>*>(smem_raw);  // [5][NY][TM]: u*, v*, w*, Du*, Dw* values
  const int m0 = blockIdx.x * TM;
  const int dir = blockIdx.z;
  const C2<T>* src = in + (size_t)dir * 6 * NY * Mm;
  for (int idx = threadIdx.x; idx < TM * NY; idx += blockDim.x) {
    const int t = idx % TM, j = idx / TM;
    const int m = m0 + t;
    C2<T> g[6];
    if (m < Mm) {
#pragma unroll
      for (int f = 0; f < 6; ++f) g[f] = ld_c2(src + ((size_t)f * NY + j) * Mm + m);
    } else {
#pragma unroll
      for (int f = 0; f < 6; ++f) g[f] = mk((T)0, (T)0);
    }
    const int pos = m / a.MZ, iz = m - pos * a.MZ;
    const int ix = pos <= a.Kx ? pos : pos - a.MX;
    const T kx = (T)(a.alpha * ix), kz = (T)(a.beta * iz);
    s5[(0 * NY + j) * TM + t] = g[0] - mul_is(g[4], kz);
    s5[(1 * NY + j) * TM + t] = g[1] + mul_is(g[3], kz) - mul_is(g[5], kx);
    s5[(2 * NY + j) * TM + t] = g[2] + mul_is(g[4], kx);
    s5[(3 * NY + j) * TM + t] = mk(-g[5].x, -g[5].y);
    s5[(4 * NY + j) * TM + t] = g[3];
  }
  __syncthreads();
  double2* dst = out + (size_t)dir * 3 * Mm * NY;
  for (int idx = threadIdx.x; idx < TM * NY; idx += blockDim.x) {
    const int t = idx % TM, n = idx / TM;
    const int m = m0 + t;
    if (m >= Mm) continue;
    const T sgT = (n & 1) ? (T)-1 : (T)1;  // T_n(y_{N-j}) = (-1)^n T_n(y_j)
    const T sgD = -sgT;                    // T_n'(y_{N-j}) = (-1)^(n+1) T_n'(y_j)
    C2<T> au = mk((T)0, (T)0), av = au, aw = au;
    for (int jh = 0; jh < NH; ++jh) {
      const T tv = Th[(size_t)jh * NY + n], dv = TDh[(size_t)jh * NY + n];
      const int j2 = N - jh;
      const bool mid = (j2 == jh);
      C2<T> xu = s5[(0 * NY + jh) * TM + t], xv = s5[(1 * NY + jh) * TM + t], xw = s5[(2 * NY + jh) * TM + t];
      C2<T> xdu = s5[(3 * NY + jh) * TM + t], xdw = s5[(4 * NY + jh) * TM + t];
      if (!mid) {
        xu = xu + scl(s5[(0 * NY + j2) * TM + t], sgT);
        xv = xv + scl(s5[(1 * NY + j2) * TM + t], sgT);
        xw = xw + scl(s5[(2 * NY + j2) * TM + t], sgT);
        xdu = xdu + scl(s5[(3 * NY + j2) * TM + t], sgD);
        xdw = xdw + scl(s5[(4 * NY + j2) * TM + t], sgD);
      }
      au = au + scl(xu, tv) + scl(xdu, dv);
      av = av + scl(xv, tv);
      aw = aw + scl(xw, tv) + scl(xdw, dv);
    }
    const C2<T> res[3] = {au, av, aw};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double2* p = dst + ((size_t)c * Mm + m) * NY + n;
      const double2 o = *p;
      *p = make_double2(o.x + (double)res[c].x, o.y + (double)res[c].y);
    }
  }
}

// weighted: out = W^-1 (P out - P W r), i.e. iz > 0: out/2 - r; iz = 0: P out - P r.
// plain (Euclidean transpose): out = P out - P r.
__global__ void k_finish_adj(const double2* __restrict__ r, double2* __restrict__ out, int Mm, int MX, int MZ,
                             int Kx, int NY, int n_dir, int weighted) {
  const size_t per = (size_t)3 * Mm * NY;
  const size_t total = per * n_dir;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t rem = e % per;
    const int n = (int)(rem % NY);
    const int m = (int)((rem / NY) % Mm);
    const size_t cbase = e - rem + (rem / ((size_t)Mm * NY)) * Mm * NY;  // start of this component
    const int pos = m / MZ, iz = m - pos * MZ;
    if (iz > 0) {
      const double2 o = out[e], rr = r[e];
      const double h = weighted ? 0.5 : 1.0;
      out[e] = make_double2(h * o.x - rr.x, h * o.y - rr.y);
      continue;
    }
    if (pos > Kx) continue;  // handled with its mirror
    const int mpos = pos == 0 ? 0 : MX - pos;
    const size_t em = cbase + (size_t)(mpos * MZ) * NY + n;
    const double2 o = out[e], om = out[em], rr = r[e], rm = r[em];
    const double2 res = make_double2(0.5 * (o.x + om.x) - 0.5 * (rr.x + rm.x),
                                     0.5 * (o.y - om.y) - 0.5 * (rr.y - rm.y));
    if (pos == 0) {
      out[e] = make_double2(res.x, 0.0);
    } else {
      out[e] = res;
      out[em] = make_double2(res.x, -res.y);
    }
  }
}

// ------------------------------------------------------------ seeding
struct SeedArgs {
  int Mm, MX, MZ, Kx, NY;
  double alpha, beta;
};

// (1 - y^2) T_n = T_n/2 - T_{n+2}/4 - T_{|n-2|}/4, applied in coefficient space
__device__ void mul_bump(const double2* in, double2* out, int NY) {
  for (int m = 0; m < NY; ++m) out[m] = make_double2(0.0, 0.0);
  for (int n = 0; n < NY; ++n) {
    const double2 a = in[n];
    out[n].x += 0.5 * a.x; out[n].y += 0.5 * a.y;
    if (n + 2 < NY) { out[n + 2].x -= 0.25 * a.x; out[n + 2].y -= 0.25 * a.y; }
    const int q = n >= 2 ? n - 2 : 2 - n;
    if (q < NY) { out[q].x -= 0.25 * a.x; out[q].y -= 0.25 * a.y; }
  }
}

// one block per mode; the series are short, so one thread does the arithmetic
// on shared-memory copies (3 NY complex values)
__global__ void k_seed(const double2* ra, const double2* rb, const double2* rc, double2* U,
                       SeedArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = blockIdx.x;
  if (m >= a.Mm || threadIdx.x != 0) return;
  const int NY = a.NY;
  double2* t1 = reinterpret_cast<double2*>(smem_raw);
  double2* v = t1 + NY;
  double2* eta = v + NY;
  const int pos = m / a.MZ, iz = m - pos * a.MZ;
  const int ix = pos <= a.Kx ? pos : pos - a.MX;
  const double kx = a.alpha * ix, kz = a.beta * iz, k2 = kx * kx + kz * kz;
  double2* Uu = U + (size_t)(0 * a.Mm + m) * NY;
  double2* Uv = U + (size_t)(1 * a.Mm + m) * NY;
  double2* Uw = U + (size_t)(2 * a.Mm + m) * NY;
  if (pos == 0 && iz == 0) {
    mul_bump(rb + (size_t)m * NY, v, NY);
    mul_bump(rc + (size_t)m * NY, eta, NY);
    for (int n = 0; n < NY; ++n) {
      Uu[n] = make_double2(v[n].x, 0.0);
      Uv[n] = make_double2(0.0, 0.0);
      Uw[n] = make_double2(eta[n].x, 0.0);
    }
    return;
  }
  mul_bump(ra + (size_t)m * NY, t1, NY);
  mul_bump(t1, v, NY);
  mul_bump(rb + (size_t)m * NY, eta, NY);
  // Dv by the backward recurrence c_n b_n = b_{n+2} + 2 (n+1) v_{n+1}
  double2 bnext = make_double2(0.0, 0.0), bnext2 = make_double2(0.0, 0.0);  // b_{n+1}, b_{n+2}
  for (int n = NY - 1; n >= 0; --n) {
    double2 bn = make_double2(0.0, 0.0);
    if (n + 1 < NY) {
      bn.x = bnext2.x + 2.0 * (n + 1) * v[n + 1].x;
      bn.y = bnext2.y + 2.0 * (n + 1) * v[n + 1].y;
    }
    if (n == 0) { bn.x *= 0.5; bn.y *= 0.5; }
    t1[n] = bn;  // t1 now holds Dv
    bnext2 = bnext;
    bnext = bn;
  }
  const double ik2 = 1.0 / k2;
  for (int n = 0; n < NY; ++n) {
    const double2 dv = t1[n], e = eta[n];
    // u = i (kx Dv - kz eta)/k^2, w = i (kz Dv + kx eta)/k^2
    const double ur = kx * dv.x - kz * e.x, ui = kx * dv.y - kz * e.y;
    const double wr = kz * dv.x + kx * e.x, wi = kz * dv.y + kx * e.y;
    Uu[n] = make_double2(-ui * ik2, ur * ik2);
    Uv[n] = v[n];
    Uw[n] = make_double2(-wi * ik2, wr * ik2);
  }
}

// ------------------------------------------------------------ vectors
__global__ void k_axpby(double* out, double a, const double* x, double b, const double* y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

__global__ void k_scale(double* x, double s, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] *= s;
}

__device__ __forceinline__ double block_sum(double v) {
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

// weighted inner products of rows of V (k states) with w; partials [k][gridDim.x]
__global__ void k_multi_inner(const double2* V, int k, size_t ncplx, const double2* w, int NY, int MZ,
                              double* partials) {
  const int i = blockIdx.y;
  const double2* vi = V + (size_t)i * ncplx;
  double acc = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < ncplx; e += (size_t)gridDim.x * blockDim.x) {
    const int iz = (int)((e / NY) % MZ);
    const double2 a = vi[e], b = w[e];
    const double d = a.x * b.x + a.y * b.y;
    acc += iz == 0 ? d : 2.0 * d;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[(size_t)i * gridDim.x + blockIdx.x] = acc;
}

// partial weighted inner products of 8 rows of V with w per block row: grid (nb, ceil(k/8))
__global__ void k_multi_inner8(const double2* V, int k, size_t ncplx, const double2* w, int NY, int MZ,
                               double* partials, const int* gate) {
  if (gate && !*gate) return;  // device-side switch (selective reorthogonalisation)
  const int i0 = blockIdx.y * 8;
  double acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = 0.0;
  // weight of element e: iz = (e / NY) mod MZ, followed incrementally along the stride
  const unsigned S = gridDim.x * blockDim.x, dq = S / (unsigned)NY, dr = S - dq * (unsigned)NY,
                 dz = dq % (unsigned)MZ;
  const unsigned e0 = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned rr = e0 % (unsigned)NY, iz = (e0 / (unsigned)NY) % (unsigned)MZ;
  for (size_t e = e0; e < ncplx; e += S) {
    const double wt = iz == 0 ? 1.0 : 2.0;
    const double2 b0 = w[e];
    const double2 b = make_double2(wt * b0.x, wt * b0.y);  // the weight once per entry
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (i0 + q < k) {
        const double2 a = V[(size_t)(i0 + q) * ncplx + e];
        acc[q] = fma(a.y, b.y, fma(a.x, b.x, acc[q]));
      }
    }
    rr += dr;
    iz += dz;
    if (rr >= (unsigned)NY) {
      rr -= NY;
      ++iz;
    }
    if (iz >= (unsigned)MZ) iz -= MZ;
  }
  // the eight block sums with one barrier: warp shuffles, then one thread per row
  __shared__ double red8[8][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red8[q][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8 && i0 + (int)threadIdx.x < k) {
    double v = 0.0;
    for (int w8 = 0; w8 < nw; ++w8) v += red8[threadIdx.x][w8];
    partials[(size_t)(i0 + threadIdx.x) * gridDim.x + blockIdx.x] = v;
  }
}

// out[i] = sum_b partials[i][b] (+ add[i] if add != null); one block per i
__global__ void k_reduce_rows(const double* partials, int nb, double* out, const double* add, const int* gate) {
  if (gate && !*gate) return;
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += partials[(size_t)i * nb + b];
  acc = block_sum(acc);
  if (threadIdx.x == 0) out[i] = acc + (add ? add[i] : 0.0);
}

// h = sqrt(sum of partials); inv = 1/h (0 if h == 0)
__global__ void k_norm_finish(const double* partials, int nb, double* h, double* inv) {
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += partials[b];
  acc = block_sum(acc);
  if (threadIdx.x == 0) {
    const double s = sqrt(fmax(acc, 0.0));
    *h = s;
    *inv = s > 0.0 ? 1.0 / s : 0.0;
  }
}

__global__ void k_scale_dev(double* x, size_t n, const double* s) {
  const double f = *s;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] *= f;
}

// Selective reorthogonalisation (Daniel, Gragg, Kaufman & Stewart): after the first
// Gram-Schmidt pass |w'|^2 = |w|^2 - |h|^2; the second pass runs only if
// |w'| < |w| / sqrt(2) (flag = 1), otherwise its coefficients are zeroed. One warp.
__global__ void k_reorth_decide(const double* __restrict__ h, int k, const double* __restrict__ wn,
                                int* __restrict__ flag, double* __restrict__ h2) {
  double acc = 0.0;
  for (int q = threadIdx.x; q < k; q += 32) acc = fma(h[q], h[q], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  acc = __shfl_sync(0xffffffffu, acc, 0);
  const double w2 = wn[0] * wn[0];
  const int f = (w2 - acc < 0.5 * w2) ? 1 : 0;
  if (threadIdx.x == 0) *flag = f;
  if (!f)
    for (int q = threadIdx.x; q < k; q += 32) h2[q] = 0.0;
}

// w -= sum_i h_i V_i with the rows split over the 8 warps of a block: each block owns 32
// consecutive elements (coalesced row reads), each warp a slice of the rows, then a
// shared-memory sum; short dependent chains for small states with many rows
__global__ void __launch_bounds__(256) k_multi_axpy_tiled(const double* __restrict__ V, int k, size_t n,
                                                         const double* __restrict__ h, double* __restrict__ w,
                                                         const int* __restrict__ gate) {
  if (gate && !*gate) return;
  __shared__ double part[8][33];
  const size_t e = (size_t)blockIdx.x * 32 + threadIdx.x;
  double acc = 0.0;
  if (e < n)
    for (int r = threadIdx.y; r < k; r += 8) acc = fma(h[r], V[(size_t)r * n + e], acc);
  part[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && e < n) {
    double sum = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) sum += part[q][threadIdx.x];
    w[e] -= sum;
  }
}

__global__ void k_multi_axpy(const double* V, int k, size_t n, const double* h, double* w, const int* gate) {
  if (gate && !*gate) return;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    // eight independent partial sums keep eight loads in flight
    double acc[8] = {w[e], 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int i = 0;
    for (; i + 8 <= k; i += 8) {
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] -= h[i + q] * V[(size_t)(i + q) * n + e];
    }
    for (; i < k; ++i) acc[0] -= h[i] * V[(size_t)i * n + e];
    w[e] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  }
}

// float copies of the base fields: b in the layout [6][NY][NX][NZ] of a, bt transposed to
// [6][NY][NZ][NX] for the register-FFT plane kernel
__global__ void k_f64_to_f32(const double* a, float* b, float* bt, size_t n, int nx, int nz) {
  const size_t plane = (size_t)nx * nz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float v = (float)a[i];
    b[i] = v;
    const size_t p = i / plane, r = i - p * plane;
    const size_t x = r / nz, z = r - x * nz;
    bt[p * plane + z * nx + x] = v;
  }
}

static YinvArgs yinv_args(const sp_ctx* c) {
  YinvArgs a;
  a.Mm = c->Mm; a.MZ = c->MZ; a.MX = c->MX; a.Kx = c->Kx; a.NY = c->NY; a.N = c->N; a.NH = c->NH;
  a.alpha = c->alpha; a.beta = c->beta;
  a.q2 = (c->N % 4 == 0 && c->Tp != nullptr) ? 1 : 0;
  a.NQ = c->N / 4 + 1;
  a.jchunk = 1;
  return a;
}

template <typename T>
static YinvTabs<T> yinv_tabs(const sp_ctx* c) {
  YinvTabs<T> t;
  if constexpr (sizeof(T) == 8) {
    t = {c->Th, c->TDh, c->Tp, c->TDp, c->tq};
  } else {
    t = {c->Th_f, c->TDh_f, c->Tp_f, c->TDp_f, c->tq_f};
  }
  return t;
}

// ------------------------------------------------------------ grouped kernels
// One launch over several independent problems: block b runs block
// b - first[inst[b]] of member inst[b]'s own launch (with a single direction),
// reading that member's launch record. The stage bodies are the ones above.
template <typename T>
struct GYinv {
  size_t off;  // offset (doubles) of the member's state in a group vector
  C2<T>* out;
  YinvTabs<T> tb;
  YinvArgs a;
  int gx;      // mode tiles of the member's launch
};

template <typename T>
__global__ void __launch_bounds__(kThreadsYinv) k_yinv_grp(const double* __restrict__ in_base,
                                                          const GYinv<T>* __restrict__ recs,
                                                          const int* __restrict__ inst,
                                                          const int* __restrict__ first,
                                                          const int* __restrict__ active) {
  const int i = inst[blockIdx.x];
  if (active && !active[i]) return;
  __shared__ GYinv<T> r;
  if (threadIdx.x == 0) r = recs[i];
  __syncthreads();
  const int b = blockIdx.x - first[i];
  yinv_body<T>(reinterpret_cast<const double2*>(in_base + r.off), r.out, r.tb, r.a, b % r.gx, b / r.gx, 0);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kThreadsXZ) k_xz_grp(const XzArgs<T>* __restrict__ recs,
                                                      const int* __restrict__ inst,
                                                      const int* __restrict__ first,
                                                      const int* __restrict__ active) {
  const int i = inst[blockIdx.x];
  if (active && !active[i]) return;
  __shared__ XzArgs<T> r;
  if (threadIdx.x == 0) r = recs[i];
  __syncthreads();
  xz_body<T, MODE>(r, blockIdx.x - first[i], 0);
}

struct GSolve {
  size_t off;
  const void* in3;  // the member's product values
  SolveArgs a;
};

template <typename T, bool LA>
__global__ void __launch_bounds__(kThreadsSolveGrp) k_solve_grp(const double* __restrict__ du_base,
                                                            double* __restrict__ out_base,
                                                            const GSolve* __restrict__ recs,
                                                            const int* __restrict__ inst,
                                                            const int* __restrict__ first,
                                                            const int* __restrict__ active) {
  const int i = inst[blockIdx.x];
  if (active && !active[i]) return;
  __shared__ GSolve r;
  if (threadIdx.x == 0) r = recs[i];
  __syncthreads();
  solve_body<T, kTileSolve, LA>(reinterpret_cast<const C2<T>*>(r.in3), reinterpret_cast<const double2*>(du_base + r.off),
                reinterpret_cast<double2*>(out_base + r.off), r.a, blockIdx.x - first[i], 0);
}

int grid_for(size_t n, int threads, int sms) {
  size_t g = (n + threads - 1) / threads;
  size_t cap = (size_t)sms * 8;
  return (int)(g < cap ? (g == 0 ? 1 : g) : cap);
}

}  // namespace

// ================================================================ launchers
static size_t xz_smem_bytes(const sp_ctx* c, int esize, int rp, int cx, bool g_on_chip) {
  const int FS = c->MZ + 1, RS = 6 * FS;
  size_t scr = (size_t)2 * cx * c->nx;
  size_t zs = (size_t)24 * rp * c->nz;
  if (zs > scr) scr = zs;
  return (size_t)esize * 2 * ((size_t)c->nx + c->nz + (g_on_chip ? (size_t)c->nx * RS : 0) + scr);
}

// pick the largest chunking that fits the shared-memory budget; the plane buffer
// moves to global memory only when it cannot fit on chip
static bool xz_config(const sp_ctx* c, int esize, int* rp, int* cx, size_t* bytes, int* g_glob) {
  for (int glob = 0; glob <= 1; ++glob) {
    // prefer two resident blocks per SM (about 113 KB each), else one (up to 220 KB)
    for (size_t budget : {(size_t)113 * 1024, (size_t)220 * 1024}) {
      for (int r = 4; r >= 1; --r) {
        int scr_c = 24 * r * c->nz;
        int x = scr_c / (2 * c->nx);
        if (x < 1) x = 1;
        if (x > 6 * c->MZ) x = 6 * c->MZ;
        size_t b = xz_smem_bytes(c, esize, r, x, glob == 0);
        if (b <= budget) {
          *rp = r;
          *cx = x;
          *bytes = b;
          *g_glob = glob;
          return true;
        }
      }
    }
  }
  return false;
}

bool sp_xz_fits(sp_ctx* c) {
  bool ok64 = xz_config(c, 8, &c->xz_rp64, &c->xz_cx64, &c->smem_xz64, &c->xz_gglob64);
  bool ok32 = xz_config(c, 4, &c->xz_rp32, &c->xz_cx32, &c->smem_xz32, &c->xz_gglob32);
  if (!ok64) c->smem_xz64 = 0;
  return ok32 && ok64;
}

size_t sp_xz_global_plane_bytes(const sp_ctx* c) {
  const size_t RS = 6 * (size_t)(c->MZ + 1);
  const size_t per = (size_t)c->NY * c->nx * RS;  // complex values per direction
  size_t b = 0;
  if (c->xz_gglob64) b = per * 16;
  if (c->xz_gglob32 && per * 8 > b) b = per * 8;
  return b;
}

cudaError_t launch_yinv(const sp_ctx* c, bool fp32, const double* in, void* out6, int n_dir,
                        cudaStream_t st) {
  if (fp32 && c->use_yinv_tc && sp_yinv_tc_supported(c)) return launch_yinv_tc(c, in, out6, n_dir, st);
  YinvArgs a = yinv_args(c);
  if (fp32) a.q2 = 0;
  const int nj = a.q2 ? a.NQ : c->NH;
  const int tiles = (c->Mm + kTileYinv - 1) / kTileYinv;
  int jsplit = 1;
  while (tiles * jsplit * n_dir < c->sm_count && jsplit < nj) ++jsplit;
  a.jchunk = (nj + jsplit - 1) / jsplit;
  dim3 grid(tiles, (nj + a.jchunk - 1) / a.jchunk, n_dir);
  if (fp32) {
    size_t sm = (size_t)3 * c->NY * kTileYinv * sizeof(C2<float>);
    cudaFuncSetAttribute(k_yinv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_yinv<float><<<grid, kThreadsYinv, sm, st>>>(reinterpret_cast<const double2*>(in),
                                                  reinterpret_cast<C2<float>*>(out6), yinv_tabs<float>(c), a);
  } else {
    size_t sm = (size_t)3 * c->NY * kTileYinv * sizeof(C2<double>);
    cudaFuncSetAttribute(k_yinv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_yinv<double><<<grid, kThreadsYinv, sm, st>>>(reinterpret_cast<const double2*>(in),
                                                   reinterpret_cast<C2<double>*>(out6), yinv_tabs<double>(c), a);
  }
  return cudaGetLastError();
}

template <typename T>
static XzArgs<T> make_xz_args(const sp_ctx* c, const void* in6, void* out3, T* base, const C2<T>* twx,
                              const C2<T>* twz, int rp, int cx) {
  XzArgs<T> a;
  a.in6 = reinterpret_cast<const C2<T>*>(in6);
  a.out3 = reinterpret_cast<C2<T>*>(out3);
  a.base = base;
  a.twx = twx;
  a.twz = twz;
  a.lam = c->lam6;
  a.px = c->px;
  a.pz = c->pz;
  a.nx = c->nx; a.nz = c->nz; a.NY = c->NY; a.Mm = c->Mm; a.MX = c->MX; a.MZ = c->MZ;
  a.Kx = c->Kx; a.Kz = c->Kz;
  a.rp = rp; a.cx = cx;
  a.FS = c->MZ + 1;
  a.RS = 6 * a.FS;
  const bool glob = sizeof(T) == 8 ? c->xz_gglob64 : c->xz_gglob32;
  a.Gg = glob ? reinterpret_cast<C2<T>*>(c->wsG) : nullptr;
  return a;
}

template <typename T, int MODE>
static cudaError_t launch_xz_t(const sp_ctx* c, const void* in6, void* out3, T* base, const C2<T>* twx,
                               const C2<T>* twz, int rp, int cx, size_t smem, int n_dir, cudaStream_t st) {
  XzArgs<T> a = make_xz_args<T>(c, in6, out3, base, twx, twz, rp, cx);
  if (a.Gg && n_dir > c->cfg.max_batch) return cudaErrorInvalidValue;
  cudaFuncSetAttribute(k_xz<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid(c->NY, n_dir);
  k_xz<T, MODE><<<grid, kThreadsXZ, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_xz(const sp_ctx* c, bool fp32, int mode, const void* in6, void* out3, int n_dir,
                      cudaStream_t st) {
  if (fp32 && c->use_xz_reg && sp_xz_reg_supported(c) && (mode == XZ_TANGENT || mode == XZ_ADJOINT))
    return launch_xz_reg(c, mode, in6, out3, n_dir, st);
  if (!fp32 && c->use_xz_reg64 && sp_xz_reg64_supported(c) &&
      (mode == XZ_TANGENT || mode == XZ_ADJOINT || mode == XZ_STEP || mode == XZ_STEP_BASE))
    return launch_xz_reg64(c, mode, in6, out3, n_dir, st);
  if (fp32) {
    const C2<float>* tx = reinterpret_cast<const C2<float>*>(c->twx_f);
    const C2<float>* tz = reinterpret_cast<const C2<float>*>(c->twz_f);
    if (mode == XZ_TANGENT)
      return launch_xz_t<float, XZ_TANGENT>(c, in6, out3, c->base32, tx, tz, c->xz_rp32, c->xz_cx32,
                                            c->smem_xz32, n_dir, st);
    if (mode == XZ_ADJOINT)
      return launch_xz_t<float, XZ_ADJOINT>(c, in6, out3, c->base32, tx, tz, c->xz_rp32, c->xz_cx32,
                                            c->smem_xz32, n_dir, st);
    return cudaErrorInvalidValue;  // the step and the base are always FP64
  }
  if (c->smem_xz64 == 0) return cudaErrorInvalidConfiguration;
  const C2<double>* tx = reinterpret_cast<const C2<double>*>(c->twx);
  const C2<double>* tz = reinterpret_cast<const C2<double>*>(c->twz);
  switch (mode) {
    case XZ_STEP:
      return launch_xz_t<double, XZ_STEP>(c, in6, out3, nullptr, tx, tz, c->xz_rp64, c->xz_cx64,
                                          c->smem_xz64, n_dir, st);
    case XZ_STEP_BASE:
      if (n_dir != 1) return cudaErrorInvalidValue;  // one base state
      return launch_xz_t<double, XZ_STEP_BASE>(c, in6, out3, c->base64, tx, tz, c->xz_rp64, c->xz_cx64,
                                               c->smem_xz64, n_dir, st);
    case XZ_TANGENT:
      return launch_xz_t<double, XZ_TANGENT>(c, in6, out3, c->base64, tx, tz, c->xz_rp64, c->xz_cx64,
                                             c->smem_xz64, n_dir, st);
    case XZ_ADJOINT:
      return launch_xz_t<double, XZ_ADJOINT>(c, in6, out3, c->base64, tx, tz, c->xz_rp64, c->xz_cx64,
                                             c->smem_xz64, n_dir, st);
    default:
      return launch_xz_t<double, XZ_BASE>(c, in6, out3, c->base64, tx, tz, c->xz_rp64, c->xz_cx64,
                                          c->smem_xz64, n_dir, st);
  }
}

static size_t solve_smem(const sp_ctx* c, int esize, int TM = kTileSolve) {
  const int NY = c->NY, NR = c->N - 1;
  size_t vals = (size_t)3 * NY * TM * 2 * esize;
  vals = (vals + 15) / 16 * 16;
  size_t d = (size_t)16 * (3 * TM * NY + 3 * TM * NR + TM * 2 * c->cv + 2 * TM * NR + 2 * TM * NY);
  return vals + d + 16;
}

static SolveArgs solve_args(const sp_ctx* c) {
  SolveArgs a;
  a.ops = c->ops;
  a.Cfh_d = c->Cfh;
  a.Cfh_f = c->Cfh_f;
  a.n_unique = c->n_unique; a.Mm = c->Mm; a.MX = c->MX; a.MZ = c->MZ; a.Kx = c->Kx;
  a.NY = c->NY; a.N = c->N; a.NH = c->NH;
  a.cv = c->cv; a.rb0 = c->rb0; a.rb1 = c->rb1;
  a.off_v0 = c->off_v0; a.off_v1 = c->off_v1; a.off_h0 = c->off_h0; a.off_h1 = c->off_h1;
  a.op_stride = c->op_stride;
  a.off_vc = c->off_vc; a.off_hc = c->off_hc;
  a.alpha = c->alpha; a.beta = c->beta; a.inv_dt = 1.0 / c->dt;
  return a;
}

// tile shapes of k_solve: (modes per block, threads per block); the autotuner picks one.
// threads = 0: one thread per solved row, TM * NY rounded up to a whole warp.
struct SolveShape {
  int tm, threads;
};
constexpr SolveShape kSolveShapes[SP_TUNE_MAX] = {{4, 128}, {2, 64}, {8, 256}, {4, 192},
                                                  {16, 512}, {2, 0}, {4, 0}, {8, 0}};
constexpr int kNumSolveShapes = 8;

static int shape_threads(const sp_ctx* c, int shape) {
  const SolveShape sh = kSolveShapes[shape];
  return sh.threads > 0 ? sh.threads : (sh.tm * c->NY + 31) / 32 * 32;
}

template <typename T, int TM, int MAXT>
static cudaError_t launch_solve_t(const sp_ctx* c, const SolveArgs& a, const void* in3, const double* du, double* out,
                                  int n_dir, int threads, cudaStream_t st) {
  const size_t sm = solve_smem(c, (int)sizeof(T), TM);
  if (sm + 40 * TM + 64 > (size_t)232448 || threads > MAXT) return cudaErrorInvalidConfiguration;  // does not fit
  auto kern = c->cfg.lam_adv ? k_solve<T, TM, MAXT, true> : k_solve<T, TM, MAXT, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const unsigned tiles = (c->n_unique + TM - 1) / TM;
  const dim3 grid = c->cfg.lam_adv ? dim3(n_dir, tiles) : dim3(tiles, n_dir);
  kern<<<grid, threads, sm, st>>>(reinterpret_cast<const C2<T>*>(in3), reinterpret_cast<const double2*>(du),
                                  reinterpret_cast<double2*>(out), a);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_solve_shape(const sp_ctx* c, int shape, const SolveArgs& a, const void* in3,
                                      const double* du, double* out, int n_dir, cudaStream_t st) {
  const int th = shape_threads(c, shape);
  switch (shape) {
    case 0: return launch_solve_t<T, 4, 128>(c, a, in3, du, out, n_dir, th, st);
    case 1: return launch_solve_t<T, 2, 64>(c, a, in3, du, out, n_dir, th, st);
    case 2: return launch_solve_t<T, 8, 256>(c, a, in3, du, out, n_dir, th, st);
    case 3: return launch_solve_t<T, 4, 192>(c, a, in3, du, out, n_dir, th, st);
    case 4: return launch_solve_t<T, 16, 512>(c, a, in3, du, out, n_dir, th, st);
    case 5: return launch_solve_t<T, 2, 1024>(c, a, in3, du, out, n_dir, th, st);
    case 6: return launch_solve_t<T, 4, 1024>(c, a, in3, du, out, n_dir, th, st);
    case 7: return launch_solve_t<T, 8, 1024>(c, a, in3, du, out, n_dir, th, st);
    default: return cudaErrorInvalidValue;
  }
}

int sp_solve_shapes(const sp_ctx* c, int* tm, int* threads) {
  for (int i = 0; i < kNumSolveShapes; ++i) {
    if (tm) tm[i] = kSolveShapes[i].tm;
    if (threads) threads[i] = shape_threads(c, i);
  }
  return kNumSolveShapes;
}

cudaError_t launch_solve(const sp_ctx* c, bool fp32, const void* in3, const double* du, double* out,
                         int n_dir, cudaStream_t st, int shape) {
  const SolveArgs a = solve_args(c);
  if (shape < 0) shape = c->solve_shape_tan;
  if (fp32) return launch_solve_shape<float>(c, shape, a, in3, du, out, n_dir, st);
  return launch_solve_shape<double>(c, shape, a, in3, du, out, n_dir, st);
}

static size_t solve_adj_smem(const sp_ctx* c) {
  const int TM = kTileSolve, NY = c->NY, NR = c->N - 1;
  return (size_t)16 * (3 * TM * NY + 3 * TM * NY + TM * 2 * c->cv + 2 * TM * NR + 3 * TM * NR) + 16;
}


cudaError_t launch_solve_adj(const sp_ctx* c, bool fp32, const double* r, double* out, void* vals3, int n_dir,
                             bool weighted, cudaStream_t st) {
  SolveArgs a = solve_args(c);
  dim3 grid((c->n_unique + kTileSolve - 1) / kTileSolve, n_dir);
  size_t sm = solve_adj_smem(c);
  if (fp32) {
    cudaFuncSetAttribute(k_solve_adj<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_solve_adj<float><<<grid, kThreadsSolve, sm, st>>>(reinterpret_cast<const double2*>(r),
                                                        reinterpret_cast<double2*>(out),
                                                        reinterpret_cast<C2<float>*>(vals3), a, weighted ? 1 : 0);
  } else {
    cudaFuncSetAttribute(k_solve_adj<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_solve_adj<double><<<grid, kThreadsSolve, sm, st>>>(reinterpret_cast<const double2*>(r),
                                                         reinterpret_cast<double2*>(out),
                                                         reinterpret_cast<C2<double>*>(vals3), a, weighted ? 1 : 0);
  }
  return cudaGetLastError();
}

cudaError_t launch_yinv_adj(const sp_ctx* c, bool fp32, const void* in6, double* out, int n_dir,
                            cudaStream_t st) {
  YinvArgs a;
  a.Mm = c->Mm; a.MZ = c->MZ; a.MX = c->MX; a.Kx = c->Kx; a.NY = c->NY; a.N = c->N; a.NH = c->NH;
  a.alpha = c->alpha; a.beta = c->beta;
  a.jchunk = c->NH;
  const int tiles = (c->Mm + kTileYinv - 1) / kTileYinv;
  dim3 grid(tiles, 1, n_dir);
  if (fp32) {
    size_t sm = (size_t)5 * c->NY * kTileYinv * sizeof(C2<float>);
    cudaFuncSetAttribute(k_yinv_adj<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_yinv_adj<float><<<grid, kThreadsYinv, sm, st>>>(reinterpret_cast<const C2<float>*>(in6),
                                                      reinterpret_cast<double2*>(out), c->Th_f, c->TDh_f, a);
  } else {
    size_t sm = (size_t)5 * c->NY * kTileYinv * sizeof(C2<double>);
    cudaFuncSetAttribute(k_yinv_adj<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_yinv_adj<double><<<grid, kThreadsYinv, sm, st>>>(reinterpret_cast<const C2<double>*>(in6),
                                                       reinterpret_cast<double2*>(out), c->Th, c->TDh, a);
  }
  return cudaGetLastError();
}

cudaError_t launch_finish_adj(const sp_ctx* c, const double* r, double* out, int n_dir, bool weighted,
                              cudaStream_t st) {
  size_t n = (size_t)3 * c->Mm * c->NY * n_dir;
  k_finish_adj<<<grid_for(n, 256, c->sm_count), 256, 0, st>>>(reinterpret_cast<const double2*>(r),
                                                             reinterpret_cast<double2*>(out), c->Mm, c->MX,
                                                             c->MZ, c->Kx, c->NY, n_dir, weighted ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_base_to_f32(const sp_ctx* c, cudaStream_t st) {
  size_t n = (size_t)6 * c->NY * c->nx * c->nz;
  k_f64_to_f32<<<grid_for(n, 256, c->sm_count), 256, 0, st>>>(c->base64, c->base32, c->base32t, n, c->nx, c->nz);
  return cudaGetLastError();
}

cudaError_t launch_seed(const sp_ctx* c, const double* ra, const double* rb, const double* rc, double* U,
                        cudaStream_t st) {
  SeedArgs a;
  a.Mm = c->Mm; a.MX = c->MX; a.MZ = c->MZ; a.Kx = c->Kx; a.NY = c->NY;
  a.alpha = c->alpha; a.beta = c->beta;
  k_seed<<<c->Mm, 32, (size_t)3 * c->NY * sizeof(double2), st>>>(reinterpret_cast<const double2*>(ra),
                                           reinterpret_cast<const double2*>(rb),
                                           reinterpret_cast<const double2*>(rc),
                                           reinterpret_cast<double2*>(U), a);
  return cudaGetLastError();
}

cudaError_t launch_scale(double* x, double s, size_t n, cudaStream_t st) {
  k_scale<<<grid_for(n, 256, 152), 256, 0, st>>>(x, s, n);
  return cudaGetLastError();
}

cudaError_t launch_axpby(double* out, double a, const double* x, double b, const double* y, size_t n,
                         cudaStream_t st) {
  k_axpby<<<grid_for(n, 256, 152), 256, 0, st>>>(out, a, x, b, y, n);
  return cudaGetLastError();
}

cudaError_t launch_multi_inner(const sp_ctx* c, const double* V, int k, const double* w, double* partials,
                               int nblocks, cudaStream_t st) {
  dim3 grid(nblocks, k);
  k_multi_inner<<<grid, 256, 0, st>>>(reinterpret_cast<const double2*>(V), k, c->cplx_per_state,
                                      reinterpret_cast<const double2*>(w), c->NY, c->MZ, partials);
  return cudaGetLastError();
}

cudaError_t launch_inner_partials(const sp_ctx* c, const double* a, const double* b, double* partials,
                                  int nblocks, cudaStream_t st) {
  return launch_multi_inner(c, a, 1, b, partials, nblocks, st);
}

// device-resident Arnoldi helpers (no host round trip)
cudaError_t launch_reorth_decide(const double* h, int k, const double* wn, int* flag, double* h2, cudaStream_t st) {
  k_reorth_decide<<<1, 32, 0, st>>>(h, k, wn, flag, h2);
  return cudaGetLastError();
}

cudaError_t launch_dev_dots(const sp_ctx* c, const double* V, int k, const double* w, double* partials,
                            int nblocks, double* out, const double* add, cudaStream_t st, const int* gate) {
  dim3 grid(nblocks, (k + 7) / 8);
  k_multi_inner8<<<grid, 256, 0, st>>>(reinterpret_cast<const double2*>(V), k, c->cplx_per_state,
                                       reinterpret_cast<const double2*>(w), c->NY, c->MZ, partials, gate);
  k_reduce_rows<<<k, 256, 0, st>>>(partials, nblocks, out, add, gate);
  return cudaGetLastError();
}

cudaError_t launch_partial_dots(const sp_ctx* c, const double* V, int k, const double* w, double* partials, int nb,
                                cudaStream_t st, const int* gate) {
  dim3 grid(nb, (k + 7) / 8);
  k_multi_inner8<<<grid, 256, 0, st>>>(reinterpret_cast<const double2*>(V), k, c->cplx_per_state,
                                       reinterpret_cast<const double2*>(w), c->NY, c->MZ, partials, gate);
  return cudaGetLastError();
}

cudaError_t launch_dev_norm(const sp_ctx* c, const double* w, double* partials, int nblocks, double* h,
                            double* inv, cudaStream_t st) {
  dim3 grid(nblocks, 1);
  k_multi_inner8<<<grid, 256, 0, st>>>(reinterpret_cast<const double2*>(w), 1, c->cplx_per_state,
                                       reinterpret_cast<const double2*>(w), c->NY, c->MZ, partials, nullptr);
  k_norm_finish<<<1, 256, 0, st>>>(partials, nblocks, h, inv);
  return cudaGetLastError();
}

cudaError_t launch_scale_dev(const sp_ctx* c, double* x, const double* s, cudaStream_t st) {
  k_scale_dev<<<grid_for(c->state_len, 256, c->sm_count), 256, 0, st>>>(x, c->state_len, s);
  return cudaGetLastError();
}

cudaError_t launch_multi_axpy(const sp_ctx* c, const double* V, int k, const double* h, double* w,
                              cudaStream_t st, const int* gate) {
  if (k <= 0) return cudaSuccess;
  if (k >= 16) {  // many rows: split them over warps
    const unsigned blocks = (unsigned)((c->state_len + 31) / 32);
    k_multi_axpy_tiled<<<blocks, dim3(32, 8), 0, st>>>(V, k, c->state_len, h, w, gate);
  } else {
    k_multi_axpy<<<grid_for(c->state_len, 256, c->sm_count), 256, 0, st>>>(V, k, c->state_len, h, w, gate);
  }
  return cudaGetLastError();
}


// ================================================================ grouped launches
cudaError_t grp_upload(void** dst, const void* src, size_t bytes) {
  *dst = nullptr;
  if (bytes == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(dst, bytes);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
}

void grp_kernel_free(GrpKernel* k) {
  if (k->recs) cudaFree(k->recs);
  if (k->inst) cudaFree(k->inst);
  if (k->first) cudaFree(k->first);
  *k = GrpKernel{};
}

void grp_plan_free(GrpPlan* p) {
  for (GrpKernel* k : {&p->yinv64, &p->yinv32, &p->xz64, &p->xz32, &p->solve64, &p->solve32}) grp_kernel_free(k);
  for (GrpKernel& k : p->xzr) grp_kernel_free(&k);
  p->n = 0;
}

// lay the members' blocks out in `order`, upload the records and the block maps
template <typename R>
static cudaError_t grp_make(GrpKernel* k, const std::vector<R>& recs, const std::vector<int>& nblk, const int* order,
                            int n, size_t smem) {
  std::vector<int> inst, first(n, 0);
  for (int q = 0; q < n; ++q) {
    const int m = order[q];
    first[m] = (int)inst.size();
    for (int b = 0; b < nblk[m]; ++b) inst.push_back(m);
  }
  k->blocks = (int)inst.size();
  k->smem = smem;
  cudaError_t e;
  if ((e = grp_upload(&k->recs, recs.data(), recs.size() * sizeof(R))) != cudaSuccess) return e;
  if ((e = grp_upload((void**)&k->inst, inst.data(), inst.size() * sizeof(int))) != cudaSuccess) return e;
  return grp_upload((void**)&k->first, first.data(), first.size() * sizeof(int));
}

template <typename T>
static cudaError_t grp_build_yinv(GrpKernel* k, sp_ctx* const* mem, int n, const size_t* offs, const int* order,
                                  int jsplit) {
  std::vector<GYinv<T>> recs(n);
  std::vector<int> nblk(n);
  size_t smem = 0;
  for (int m = 0; m < n; ++m) {
    const sp_ctx* c = mem[m];
    GYinv<T>& r = recs[m];
    r.off = offs[m];
    r.out = reinterpret_cast<C2<T>*>(c->ws6);
    r.tb = yinv_tabs<T>(c);
    YinvArgs& a = r.a;
    a = yinv_args(c);
    if (sizeof(T) == 4) a.q2 = 0;
    const int nj = a.q2 ? a.NQ : c->NH;
    a.jchunk = (nj + jsplit - 1) / jsplit;
    r.gx = (c->Mm + kTileYinv - 1) / kTileYinv;
    nblk[m] = r.gx * ((nj + a.jchunk - 1) / a.jchunk);
    smem = std::max(smem, (size_t)3 * c->NY * kTileYinv * sizeof(C2<T>));
  }
  cudaError_t e = cudaFuncSetAttribute(k_yinv_grp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return grp_make(k, recs, nblk, order, n, smem);
}

// skip[m] != 0 leaves member m out of this launch (its plane stage runs elsewhere)
template <typename T>
static cudaError_t grp_build_xz(GrpKernel* k, sp_ctx* const* mem, int n, const int* order,
                                const std::vector<int>* skip = nullptr) {
  std::vector<XzArgs<T>> recs(n);
  std::vector<int> nblk(n);
  size_t smem = 0;
  for (int m = 0; m < n; ++m) {
    const sp_ctx* c = mem[m];
    if constexpr (sizeof(T) == 8) {
      recs[m] = make_xz_args<double>(c, c->ws6, c->ws3, c->base64, reinterpret_cast<const C2<double>*>(c->twx),
                                     reinterpret_cast<const C2<double>*>(c->twz), c->xz_rp64, c->xz_cx64);
      smem = std::max(smem, c->smem_xz64);
    } else {
      recs[m] = make_xz_args<float>(c, c->ws6, c->ws3, c->base32, reinterpret_cast<const C2<float>*>(c->twx_f),
                                    reinterpret_cast<const C2<float>*>(c->twz_f), c->xz_rp32, c->xz_cx32);
      smem = std::max(smem, c->smem_xz32);
    }
    nblk[m] = skip && (*skip)[m] ? 0 : c->NY;
  }
  for (auto fn : {k_xz_grp<T, XZ_STEP>, k_xz_grp<T, XZ_BASE>, k_xz_grp<T, XZ_TANGENT>}) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return grp_make(k, recs, nblk, order, n, smem);
}

static cudaError_t grp_build_solve(GrpKernel* k, sp_ctx* const* mem, int n, const size_t* offs, const int* order,
                                   int esize) {
  std::vector<GSolve> recs(n);
  std::vector<int> nblk(n);
  size_t smem = 0;
  for (int m = 0; m < n; ++m) {
    const sp_ctx* c = mem[m];
    recs[m].off = offs[m];
    recs[m].in3 = c->ws3;
    recs[m].a = solve_args(c);
    nblk[m] = (c->n_unique + kTileSolve - 1) / kTileSolve;
    smem = std::max(smem, solve_smem(c, esize));
  }
  const bool la = mem[0]->cfg.lam_adv != 0;
  const void* kern = esize == 8 ? (la ? (const void*)k_solve_grp<double, true> : (const void*)k_solve_grp<double, false>)
                                : (la ? (const void*)k_solve_grp<float, true> : (const void*)k_solve_grp<float, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return grp_make(k, recs, nblk, order, n, smem);
}

cudaError_t grp_plan_build(GrpPlan* p, sp_ctx* const* mem, int n, const size_t* offs, const int* order) {
  p->n = n;
  p->lam_adv = mem[0]->cfg.lam_adv != 0;
  // split the Gauss-Lobatto points of k_yinv only when the whole group has too few mode tiles
  int tiles = 0, nh_min = 1 << 30;
  for (int m = 0; m < n; ++m) {
    tiles += (mem[m]->Mm + kTileYinv - 1) / kTileYinv;
    nh_min = std::min(nh_min, mem[m]->NH);
  }
  int jsplit = 1;
  while (tiles * jsplit < 2 * mem[0]->sm_count && jsplit < nh_min) ++jsplit;
  cudaError_t e;
  if ((e = grp_build_yinv<double>(&p->yinv64, mem, n, offs, order, jsplit)) != cudaSuccess) return e;
  if ((e = grp_build_yinv<float>(&p->yinv32, mem, n, offs, order, jsplit)) != cudaSuccess) return e;
  if ((e = grp_build_xz<double>(&p->xz64, mem, n, order)) != cudaSuccess) return e;
  // float plane stage: the register-FFT kernel for the members whose own context uses it,
  // the generic kernel for the others (so every member computes exactly as on its own)
  std::vector<int> reg(n);
  for (int m = 0; m < n; ++m) reg[m] = mem[m]->use_xz_reg && sp_xz_reg_supported(mem[m]);
  if ((e = grp_build_xz_reg(p->xzr, mem, n, order, reg)) != cudaSuccess) return e;
  if ((e = grp_build_xz<float>(&p->xz32, mem, n, order, &reg)) != cudaSuccess) return e;
  if ((e = grp_build_solve(&p->solve64, mem, n, offs, order, 8)) != cudaSuccess) return e;
  return grp_build_solve(&p->solve32, mem, n, offs, order, 4);
}

cudaError_t grp_launch_yinv(const GrpPlan& p, bool fp32, const double* in_base, const int* active, cudaStream_t st) {
  const GrpKernel& k = fp32 ? p.yinv32 : p.yinv64;
  if (k.blocks == 0) return cudaSuccess;
  if (fp32)
    k_yinv_grp<float><<<k.blocks, kThreadsYinv, k.smem, st>>>(in_base, static_cast<const GYinv<float>*>(k.recs),
                                                               k.inst, k.first, active);
  else
    k_yinv_grp<double><<<k.blocks, kThreadsYinv, k.smem, st>>>(in_base, static_cast<const GYinv<double>*>(k.recs),
                                                                k.inst, k.first, active);
  return cudaGetLastError();
}

cudaError_t grp_launch_xz(const GrpPlan& p, bool fp32, int mode, const int* active, cudaStream_t st) {
  if (fp32) {
    if (mode != XZ_TANGENT) return cudaErrorInvalidValue;  // the step and the base are always FP64
    cudaError_t e = grp_launch_xz_reg(p.xzr, active, st);
    if (e != cudaSuccess) return e;
    const GrpKernel& k = p.xz32;
    if (k.blocks == 0) return cudaSuccess;
    k_xz_grp<float, XZ_TANGENT><<<k.blocks, kThreadsXZ, k.smem, st>>>(static_cast<const XzArgs<float>*>(k.recs),
                                                                       k.inst, k.first, active);
    return cudaGetLastError();
  }
  const GrpKernel& k = p.xz64;
  if (k.blocks == 0) return cudaSuccess;
  const XzArgs<double>* r = static_cast<const XzArgs<double>*>(k.recs);
  switch (mode) {
    case XZ_STEP: k_xz_grp<double, XZ_STEP><<<k.blocks, kThreadsXZ, k.smem, st>>>(r, k.inst, k.first, active); break;
    case XZ_BASE: k_xz_grp<double, XZ_BASE><<<k.blocks, kThreadsXZ, k.smem, st>>>(r, k.inst, k.first, active); break;
    case XZ_TANGENT:
      k_xz_grp<double, XZ_TANGENT><<<k.blocks, kThreadsXZ, k.smem, st>>>(r, k.inst, k.first, active);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t grp_launch_solve(const GrpPlan& p, bool fp32, const double* du_base, double* out_base, const int* active,
                             cudaStream_t st) {
  const GrpKernel& k = fp32 ? p.solve32 : p.solve64;
  if (k.blocks == 0) return cudaSuccess;
  const GSolve* r = static_cast<const GSolve*>(k.recs);
  auto kern = p.lam_adv ? k_solve_grp<float, true> : k_solve_grp<float, false>;
  auto kern64 = p.lam_adv ? k_solve_grp<double, true> : k_solve_grp<double, false>;
  if (fp32)
    kern<<<k.blocks, kThreadsSolveGrp, k.smem, st>>>(du_base, out_base, r, k.inst, k.first, active);
  else
    kern64<<<k.blocks, kThreadsSolveGrp, k.smem, st>>>(du_base, out_base, r, k.inst, k.first, active);
  return cudaGetLastError();
}
