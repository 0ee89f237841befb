// Per-mode Stokes solve of the batched tangent in O(N) per right-hand side.
//
// Same problem and result as k_solve (kernels.cu): per Fourier mode, the forward
// Chebyshev transform of the product, the right-hand side u/dt + N, the
// Chebyshev-tau Stokes problem (Sec. 2, Eq. befe; Sec. 3.2: exact per-mode
// inversion, divergence-free to machine accuracy) and G = u_new - u. k_solve
// applies precomputed dense solution operators (O(N^2) FP64 work per mode and
// right-hand side, spread over the rows of one right-hand side); here each
// problem is solved by tridiagonal sweeps (plan.cpp states the reformulation and
// the records): O(N) FP64 work, one thread per (mode, parity, direction), lanes
// over directions so that a warp reads each record entry once (a broadcast).
//
//   k_rhs  : values at the Gauss-Lobatto points -> Chebyshev coefficients of rows
//            0..N-2, plus du/dt, for the three components (threads over rows).
//   k_chain: thread (mode, P, direction) solves the (v, a, p) problem of parity P
//            (two Helmholtz sweeps and the 2 x 2 influence correction) and the
//            Helmholtz problem of b of parity 1-P, then writes G_v on the rows of
//            parity P and G_u, G_w on the rows of parity 1-P. Every row it writes
//            depends only on its own sweeps, so threads never wait on each other.
// The mean mode (0,0) solves the two Dirichlet Helmholtz problems of u and w.
#include <algorithm>

#include "sp_internal.h"

namespace {

// ------------------------------------------------------------------ k_rhs
struct RhsArgs {
  const double* Cfh_d;
  const float* Cfh_f;
  const double* Cq_d;      // second-level split (N divisible by 4), null otherwise: see k_rhs
  const float* Cq_f;
  int NQ;
  double2* W;              // right-hand sides: (u, d, row c (N-1) + n) at u su + d sd + row sn
  long long su, sd, sn;    // complex strides of W: unique mode, direction, row (c (N-1) + n)
  int n_unique, Mm, MX, MZ, Kx, NY, N, NH;
  double inv_dt;
};

constexpr int kRhsTM = 4;
constexpr int kRhsThreads = 256;

__device__ __forceinline__ void mode_of(int u, int Kx, int MZ, int* pos, int* iz) {
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

template <typename T>
__device__ __forceinline__ C2<T> ldv(const C2<T>* p) { return *p; }
template <>
__device__ __forceinline__ C2<double> ldv(const C2<double>* p) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return mk(v.x, v.y);
}
template <>
__device__ __forceinline__ C2<float> ldv(const C2<float>* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return mk(v.x, v.y);
}

// in3: [dir][3][NY][Mm] complex T; du: [dir][3][Mm][NY] complex double
template <typename T>
__global__ void __launch_bounds__(kRhsThreads) k_rhs(const C2<T>* __restrict__ in3, const double2* __restrict__ du,
                                                    RhsArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int TM = kRhsTM;
  const int NY = a.NY, N = a.N, NH = a.NH, Mm = a.Mm, MZ = a.MZ, NR = N - 1;
  C2<T>* sv = reinterpret_cast<C2<T>*>(smem_raw);  // [3][NY][TM]
  __shared__ int s_pos[TM], s_iz[TM], s_u[TM];
  const int u0 = blockIdx.x * TM, dir = blockIdx.y;
  if (threadIdx.x < TM) {
    const int u = u0 + threadIdx.x;
    int pos = 0, iz = 0;
    if (u < a.n_unique) mode_of(u, a.Kx, MZ, &pos, &iz);
    s_pos[threadIdx.x] = pos;
    s_iz[threadIdx.x] = iz;
    s_u[threadIdx.x] = u;
  }
  __syncthreads();
  const C2<T>* vin = in3 + (size_t)dir * 3 * NY * Mm;
  for (int idx = threadIdx.x; idx < 3 * NY * TM; idx += blockDim.x) {
    const int t = idx % TM, jc = idx / TM;  // jc = c NY + j
    const int c = jc / NY, j = jc - c * NY;
    C2<T> v = mk((T)0, (T)0);
    if (s_u[t] < a.n_unique) v = ldv(vin + ((size_t)c * NY + j) * Mm + s_pos[t] * MZ + s_iz[t]);
    sv[idx] = v;
  }
  __syncthreads();
  // even/odd pairs: s_j = f(y_j) + f(y_N-j) at j, d_j = f(y_j) - f(y_N-j) at N - j
  for (int idx = threadIdx.x; idx < 3 * TM * (NH - 1); idx += blockDim.x) {
    const int t = idx % TM, jj = (idx / TM) % (NH - 1), c = idx / (TM * (NH - 1));
    C2<T>* col = sv + (c * NY) * TM + t;
    const C2<T> p = col[jj * TM], q = col[(N - jj) * TM];
    col[jj * TM] = p + q;
    col[(N - jj) * TM] = p - q;
  }
  __syncthreads();
  // second level for the even degrees (N divisible by 4): with s'_j = s_j / cbar_j (cbar_0 = 2),
  // T_2m(y_{N/2-j}) = (-1)^m T_2m(y_j) pairs j with N/2 - j: slot j < N/4 receives
  // s'_j + s'_{N/2-j} (degrees 0 mod 4), slot N/2 - j receives s'_j - s'_{N/2-j} (2 mod 4)
  const bool q2 = a.Cq_d != nullptr;
  const int NQ = a.NQ, NQ1 = NQ - 1;  // NQ1 = N/4
  if (q2) {
    for (int idx = threadIdx.x; idx < 3 * TM * NQ1; idx += blockDim.x) {
      const int t = idx % TM, jj = (idx / TM) % NQ1, c = idx / (TM * NQ1);
      C2<T>* col = sv + (c * NY) * TM + t;
      C2<T> p = col[jj * TM];
      if (jj == 0) p = scl(p, (T)0.5);
      const C2<T> q = col[(N / 2 - jj) * TM];
      col[jj * TM] = p + q;
      col[(N / 2 - jj) * TM] = p - q;
    }
    __syncthreads();
  }
  // rows in three classes, each its own loop so that every warp runs one trip count:
  // odd n (half-length sums over d), n = 0 mod 4 and n = 2 mod 4 (quarter-length sums over the
  // second-level pairs; without that level, every even n: half-length sums over s)
  const double2* dsrc = du + (size_t)dir * 3 * Mm * NY;
  const int nodd = (NR - 1 + 1) / 2;             // odd rows 1, 3, .., <= N-2
  const int nev0 = q2 ? (NR + 3) / 4 : (NR + 1) / 2;  // rows 0, 4, .. (q2) or 0, 2, .. (one level)
  const int nev2 = q2 ? (NR + 1) / 4 : 0;        // rows 2, 6, .. <= N-2
  for (int cls = 0; cls < 3; ++cls) {
    const int cnt = cls == 0 ? nodd : (cls == 1 ? nev0 : nev2);
    for (int idx = threadIdx.x; idx < 3 * TM * cnt; idx += blockDim.x) {
      const int t = idx % TM, r = (idx / TM) % cnt, c = idx / (TM * cnt);
      const int n = cls == 0 ? 2 * r + 1 : (cls == 1 ? (q2 ? 4 * r : 2 * r) : 4 * r + 2);
      const int u = s_u[t];
      if (u >= a.n_unique) continue;
      const C2<T>* col = sv + (c * NY) * TM + t;
      C2<T> acc = mk((T)0, (T)0);
      const T* cf;
      const T* cq;
      if constexpr (sizeof(T) == 8) {
        cf = a.Cfh_d + (size_t)n * NH;
        cq = a.Cq_d + (size_t)n * NQ;
      } else {
        cf = a.Cfh_f + (size_t)n * NH;
        cq = a.Cq_f + (size_t)n * NQ;
      }
      if (cls == 0) {
        for (int jj = 0; jj < NH - 1; ++jj) acc = acc + scl(col[(N - jj) * TM], cf[jj]);
      } else if (!q2) {
        for (int jj = 0; jj < NH - 1; ++jj) acc = acc + scl(col[jj * TM], cf[jj]);
        acc = acc + scl(col[(NH - 1) * TM], cf[NH - 1]);
      } else if (cls == 1) {
        for (int jj = 0; jj < NQ; ++jj) acc = acc + scl(col[jj * TM], cq[jj]);
      } else {  // degrees 2 mod 4: the j = N/4 term vanishes
        for (int jj = 0; jj < NQ1; ++jj) acc = acc + scl(col[(N / 2 - jj) * TM], cq[jj]);
      }
      // du (Hermitian-projected on the kz = 0 plane)
      const int pos = s_pos[t], iz = s_iz[t];
      double2 d = __ldg(dsrc + ((size_t)c * Mm + pos * MZ + iz) * NY + n);
      if (iz == 0) {
        const int mpos = pos == 0 ? 0 : a.MX - pos;
        const double2 w = __ldg(dsrc + ((size_t)c * Mm + mpos * MZ) * NY + n);
        d = make_double2(0.5 * (d.x + w.x), 0.5 * (d.y - w.y));
      }
      double2 f = make_double2((double)acc.x + d.x * a.inv_dt, (double)acc.y + d.y * a.inv_dt);
      if (pos == 0 && iz == 0) f.y = 0.0;
      a.W[u * a.su + dir * a.sd + (long long)(c * NR + n) * a.sn] = f;
    }
  }
}

// ---------------------------------------------------------------- k_chain
struct ChainArgs {
  const double2* W;
  const double2* du;       // [dir][3][Mm][NY]
  double2* out;            // same layout
  const double* rec;       // [n_unique][2][par]
  long long su, sd, sn;
  int n_unique, n_dir, dirs_fast;
  int Mm, MX, MZ, Kx, NY, N, NH, par, stride;
  double alpha, beta;
  double2* Sg;             // work vectors of every thread: entry i of thread t at Sg[i * T + t] (the
                           // second vector) and Sg[(NH + i) * T + t] (the first), T threads in all
};

constexpr int kChainWarps = 2;  // threads per block = 32 kChainWarps (warp pairs: parity 0, 1)
constexpr int kChainBlocksPerSM = 12;  // register budget: 24 warps per SM (80 registers a thread)
constexpr int kDirsFastMin = 16;  // batches of this many directions put lanes over directions

__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscl(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// a s + b t (real s, t)
__device__ __forceinline__ double2 cmix(double2 a, double s, double2 b, double t) {
  return make_double2(fma(a.x, s, b.x * t), fma(a.y, s, b.y * t));
}
// a + b s
__device__ __forceinline__ double2 caxpy(double2 a, double2 b, double s) {
  return make_double2(fma(b.x, s, a.x), fma(b.y, s, a.y));
}

// The row indices n and n^2 as doubles: a warp-uniform table read instead of an
// integer-to-FP64 conversion, which would take the FP64 pipe.
struct RowTable {
  double n[kChainMaxRows];
  double n2[kChainMaxRows];
};
constexpr RowTable make_row_table() {
  RowTable t{};
  for (int i = 0; i < kChainMaxRows; ++i) {
    t.n[i] = (double)i;
    t.n2[i] = (double)i * (double)i;
  }
  return t;
}
__constant__ RowTable kRow = make_row_table();

// One Dirichlet Helmholtz tau solve of parity Q in the tridiagonal form (records of
// plan.cpp: per unknown i, (q w_0, q w_1, q w_2, p, psi, alpha)): rhs(n) gives the
// right-hand side of tau row n (zero above N-2), bc the boundary value; X (stride st)
// receives x_i, i = 0..m; the return value is x_m.
template <class Rhs>
__device__ __forceinline__ double2 tri_sweep(const double* __restrict__ r6, double g, int N, int Q, Rhs rhs,
                                             double2 bc, double2* X, int st) {
  const int m = (N - Q) / 2;
  double2 Rhi = make_double2(0.0, 0.0);              // R_{n+2}
  double2 Rmid = rhs(2 * m + Q);                     // R_n (zero when n > N-2)
  double2 Rlo = rhs(2 * m + Q - 2);                  // R_{n-2}, fetched one step ahead
  double2 bnext = make_double2(0.0, 0.0), acc = make_double2(0.0, 0.0);
  for (int i = m; i >= 1; --i) {
    const int n = 2 * i + Q;
    // the next step's right-hand side (same descending order of calls): its loads are in flight
    // while this step's dependent arithmetic runs
    const double2 Rnext = i >= 2 ? rhs(n - 4) : make_double2(0.0, 0.0);
    const double* t = r6 + 6 * i;
    double2 b;
    b.x = fma(-t[3], bnext.x, fma(t[2], Rhi.x, fma(t[1], Rmid.x, t[0] * Rlo.x)));
    b.y = fma(-t[3], bnext.y, fma(t[2], Rhi.y, fma(t[1], Rmid.y, t[0] * Rlo.y)));
    acc = caxpy(acc, b, t[4]);
    X[i * st] = b;
    bnext = b;
    Rhi = Rmid;
    Rmid = Rlo;
    Rlo = Rnext;
  }
  double2 x = cscl(csub(bc, acc), g);
  X[0] = x;
  for (int i = 1; i <= m; ++i) {
    x = caxpy(X[i * st], x, r6[6 * i + 5]);
    X[i * st] = x;
  }
  return x;
}

__global__ void __launch_bounds__(32 * kChainWarps, kChainBlocksPerSM) k_chain(ChainArgs a) {
  // two work vectors of NH entries per thread, both in global scratch (one thread per column,
  // consecutive threads adjacent: coalesced, mostly L2-resident). Without shared memory the
  // registers alone bound the warps an SM holds for the dependent sweeps.
  const int st2 = gridDim.x * blockDim.x, st = st2;
  double2* S2 = a.Sg + (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double2* S1 = S2 + (size_t)a.NH * st2;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int P = gw & 1, Q = 1 - P;
  const int item = (gw >> 1) * 32 + (threadIdx.x & 31);
  if (item >= a.n_unique * a.n_dir) return;  // no barrier follows
  int u, d;
  if (a.dirs_fast) {
    u = item / a.n_dir;
    d = item - u * a.n_dir;
  } else {
    d = item / a.n_unique;
    u = item - d * a.n_unique;
  }
  int pos, iz;
  mode_of(u, a.Kx, a.MZ, &pos, &iz);
  const int N = a.N, NY = a.NY, Mm = a.Mm, MZ = a.MZ, NR = N - 1;
  const double2* Wb = a.W + u * a.su + d * a.sd;
  auto fval = [&](int c, int n) -> double2 {  // right-hand side row n of component c (0 above N-2)
    return (n >= 0 && n <= N - 2) ? Wb[(long long)(c * NR + n) * a.sn] : make_double2(0.0, 0.0);
  };
  const double2* dsrc = a.du + (size_t)d * 3 * Mm * NY;
  double2* dst = a.out + (size_t)d * 3 * Mm * NY;
  const int mpos = pos == 0 ? 0 : a.MX - pos;
  auto duv = [&](int c, int n) -> double2 {  // Hermitian-projected input
    double2 v = __ldg(dsrc + ((size_t)c * Mm + pos * MZ + iz) * NY + n);
    if (iz == 0) {
      const double2 w = __ldg(dsrc + ((size_t)c * Mm + mpos * MZ) * NY + n);
      v = make_double2(0.5 * (v.x + w.x), 0.5 * (v.y - w.y));
    }
    return v;
  };
  auto put = [&](int c, int n, double2 g) {
    if (pos == 0 && iz == 0) g.y = 0.0;
    dst[((size_t)c * Mm + pos * MZ + iz) * NY + n] = g;
    if (iz == 0 && pos != 0) dst[((size_t)c * Mm + mpos * MZ) * NY + n] = make_double2(g.x, -g.y);
  };
  const double* rec = a.rec + (size_t)u * a.stride;
  const int NH = a.NH;
  const double2 zero = make_double2(0.0, 0.0);

  if (u == 0) {
    // mean flow: (1/dt - nu D^2) u_00 = f_x, the same for w_00, v_00 = 0 (parity P rows)
    const double* rP = rec + P * a.par;
    const double gH = rP[14 * NH];
    tri_sweep(rP, gH, N, P, [&](int n) { return fval(0, n); }, zero, S1, st);
    tri_sweep(rP, gH, N, P, [&](int n) { return fval(2, n); }, zero, S2, st2);
    const int m = (N - P) / 2;
    for (int i = 0; i <= m; ++i) {
      const int n = 2 * i + P;
      put(0, n, csub(S1[i * st], duv(0, n)));
      put(1, n, csub(zero, duv(1, n)));
      put(2, n, csub(S2[i * st2], duv(2, n)));
    }
    return;
  }

  const double kx = a.alpha * (pos <= a.Kx ? pos : pos - a.MX), kz = a.beta * iz;
  const double k2 = kx * kx + kz * kz, k = sqrt(k2), ik = 1.0 / k;
  const double cx = kx * ik, cz = kz * ik;
  const double ik2 = 2.0 * ik;  // (2 / c_n) / k for n >= 1
  const double* rP = rec + P * a.par;
  const double* rQ = rec + Q * a.par;
  const int m = (N - P) / 2;

  // (1) w_A: (lam - nu D^2) w = -k^2 g on the rows of parity P, w(+-1) = 0, with the
  // reduced right-hand side g_n = f_v,n - (2 / (c_n k)) S_n, S_n = sum over rows
  // m' > n of parity Q of m' f~_a,m' (f~_a = -i f_a), built while the sweep descends
  double2 S = zero;
  int next_add = 2 * m + P - 1;  // the next row m' of parity Q to add to S
  auto gneg = [&](int n) -> double2 {  // -k^2 g_n, called for n = top, then descending
    if (n > N - 2) return zero;
    while (next_add > n) {
      if (next_add <= N - 2) {
        const double2 fx = fval(0, next_add), fz = fval(2, next_add);
        const double2 fa = cmix(fx, cx, fz, cz);
        S = caxpy(S, make_double2(fa.y, -fa.x), kRow.n[next_add]);
      }
      next_add -= 2;
    }
    const double2 fv = fval(1, n);
    const double2 g = caxpy(fv, S, n == 0 ? -ik : -ik2);
    return cscl(g, -k2);
  };
  const double2 wtop = tri_sweep(rP, rP[14 * NH], N, P, gneg, zero, S1, st);
  // (2) v_A: (D^2 - k^2) v = w_A on the rows <= N-2 of parity P, v(+-1) = 0
  const double2 vtop = tri_sweep(rP + 6 * NH, rP[14 * NH + 1], N, P,
                                 [&](int n) { return n <= N - 2 ? S1[((n - P) >> 1) * st] : zero; }, zero, S2, st2);
  // (3) influence correction: sigma psi + tau h fixes w_top = -k^2 v_top and Dv(+-1) = 0
  double2 e2 = zero;
  for (int i = 0; i <= m; ++i) e2 = caxpy(e2, S2[i * st2], kRow.n2[2 * i + P]);
  const double2 e1 = caxpy(wtop, vtop, k2);
  const double* sc = rP + 14 * NH;
  const double2 sig = cmix(e1, -sc[2], e2, -sc[3]);
  const double2 tau = cmix(e1, -sc[4], e2, -sc[5]);
  // (4) v = v_A + sigma v_psi + tau v_h, G_v on the rows of parity P; a = (i/k) D v on the
  // rows of parity Q by a suffix sum, stored in S2 (slot i holds a_{2i+P-1})
  const double* v2 = rP + 12 * NH;
  double2 Sa = zero;
  for (int i = m; i >= 0; --i) {
    const int n = 2 * i + P;
    double2 v = S2[i * st2];
    v = caxpy(v, sig, v2[2 * i]);
    v = caxpy(v, tau, v2[2 * i + 1]);
    put(1, n, csub(v, duv(1, n)));
    Sa = caxpy(Sa, v, kRow.n[n]);
    if (n >= 1) {
      const double f = n - 1 == 0 ? ik : ik2;  // (i/k)(2/c_{n-1}) Sa
      S2[i * st2] = make_double2(-Sa.y * f, Sa.x * f);
    }
  }
  // (5) b of parity Q: (lam - nu D^2) b = f_b, b(+-1) = 0; then u = cx a - cz b,
  // w = cz a + cx b and G_u, G_w on the rows of parity Q
  tri_sweep(rQ, rQ[14 * NH], N, Q,
            [&](int n) { return cmix(fval(0, n), -cz, fval(2, n), cx); }, zero, S1, st);
  const int mq = (N - Q) / 2;
  for (int i = 0; i <= mq; ++i) {
    const int n = 2 * i + Q;
    const int ia = P == 0 ? i + 1 : i;  // slot of a_n in S2
    const double2 an = (ia <= m) ? S2[ia * st2] : zero;
    const double2 bn = S1[i * st];
    put(0, n, csub(cmix(an, cx, bn, -cz), duv(0, n)));
    put(2, n, csub(cmix(an, cz, bn, cx), duv(2, n)));
  }
}

}  // namespace

static void chain_strides(const sp_ctx* c, int n_dir, long long* su, long long* sd, long long* sn) {
  const long long NR = c->N - 1;
  if (n_dir >= kDirsFastMin) {  // lanes over directions: coalesced right-hand sides
    *sd = 1;
    *sn = n_dir;
    *su = 3 * NR * n_dir;
  } else {  // lanes over modes
    *su = 1;
    *sn = c->n_unique;
    *sd = 3 * NR * c->n_unique;
  }
}

cudaError_t launch_chain_rhs(const sp_ctx* c, bool fp32, const void* in3, const double* du, void* work, int n_dir,
                             cudaStream_t st) {
  if (n_dir <= 0) return cudaSuccess;
  RhsArgs r;
  chain_strides(c, n_dir, &r.su, &r.sd, &r.sn);
  if (fp32 && c->use_rhs_tc && sp_rhs_tc_supported(c))  // forward transform on the tensor cores
    return launch_rhs_tc(c, in3, du, work, n_dir, r.su, r.sd, r.sn, st);
  r.Cfh_d = c->Cfh;
  r.Cfh_f = c->Cfh_f;
  r.Cq_d = c->Cq;
  r.Cq_f = c->Cq_f;
  r.NQ = c->N / 4 + 1;
  r.W = static_cast<double2*>(work);
  r.n_unique = c->n_unique;
  r.Mm = c->Mm;
  r.MX = c->MX;
  r.MZ = c->MZ;
  r.Kx = c->Kx;
  r.NY = c->NY;
  r.N = c->N;
  r.NH = c->NH;
  r.inv_dt = 1.0 / c->dt;
  const dim3 grid((c->n_unique + kRhsTM - 1) / kRhsTM, n_dir);
  if (fp32) {
    const size_t sm = sizeof(C2<float>) * 3 * c->NY * kRhsTM;
    k_rhs<float><<<grid, kRhsThreads, sm, st>>>(static_cast<const C2<float>*>(in3),
                                                reinterpret_cast<const double2*>(du), r);
  } else {
    const size_t sm = sizeof(C2<double>) * 3 * c->NY * kRhsTM;
    k_rhs<double><<<grid, kRhsThreads, sm, st>>>(static_cast<const C2<double>*>(in3),
                                                 reinterpret_cast<const double2*>(du), r);
  }
  return cudaGetLastError();
}

// global scratch of k_chain for n_dir directions (the two work vectors of every thread)
size_t chain_scratch_bytes(const sp_ctx* c, int n_dir) {
  const long long items = (long long)c->n_unique * n_dir;
  const long long warps = 2 * ((items + 31) / 32);
  const long long blocks = (warps + kChainWarps - 1) / kChainWarps;
  return 2 * sizeof(double2) * (size_t)c->NH * (size_t)(blocks * 32 * kChainWarps);
}

cudaError_t launch_chain_solve(const sp_ctx* c, const double* du, double* out, const void* work, void* scratch,
                               int n_dir, cudaStream_t st) {
  if (n_dir <= 0) return cudaSuccess;
  ChainArgs a;
  a.Sg = static_cast<double2*>(scratch);
  chain_strides(c, n_dir, &a.su, &a.sd, &a.sn);
  a.W = static_cast<const double2*>(work);
  a.du = reinterpret_cast<const double2*>(du);
  a.out = reinterpret_cast<double2*>(out);
  a.rec = c->chain;
  a.n_unique = c->n_unique;
  a.n_dir = n_dir;
  a.dirs_fast = n_dir >= kDirsFastMin ? 1 : 0;
  a.Mm = c->Mm;
  a.MX = c->MX;
  a.MZ = c->MZ;
  a.Kx = c->Kx;
  a.NY = c->NY;
  a.N = c->N;
  a.NH = c->NH;
  a.par = c->chain_par;
  a.stride = c->chain_stride;
  a.alpha = c->alpha;
  a.beta = c->beta;
  const long long items = (long long)c->n_unique * n_dir;
  const long long warps = 2 * ((items + 31) / 32);
  const long long blocks = (warps + kChainWarps - 1) / kChainWarps;
  k_chain<<<(unsigned)blocks, 32 * kChainWarps, 0, st>>>(a);
  return cudaGetLastError();
}
