// Plan of a pipe-flow context: radial finite-difference tables and the per-mode
// Stokes solution operators (built once on the host, used by the kernels in
// pipe.cu).
//
// Radial grid r_j = cos(pi j / (2 Nr - 1)), j = 0..Nr-1: r_0 = 1 is the wall, the
// axis is not a grid point. A field of azimuthal number m has the parity
// f(-r) = (-1)^q f(r) (q = m for u_z and p, m +- 1 for u+- = u_r +- i u_theta), so
// derivatives near the axis use the mirrored points -r_j with that sign; each row
// uses the 9 nearest points and Fornberg's recursion for the weights
// (B. Fornberg, Math. Comp. 51 (1988) 699-706).
//
// Per Fourier mode (m, k) the BEFE step solves (Sec. 2, Eq. befe) the Stokes
// problem (lam - nu lap) u + grad p = f with lam = 1/dt. With u+-, u~_z = -i u_z
// and f~_z = -i f_z the system is real:
//   (lam - nu L_{m+-1}) u+- + (D1 -+ m/r) p = f+-     interior points
//   (lam - nu L_m) u~_z + k p = f~_z                   interior points
//   u+-(1) = u~_z(1) = 0                               wall
//   L_m p = div_h f                                    interior points
//   div_h u = 0                                        wall
// with L_q = D2 + D1/r - q^2/r^2 - k^2 and
// div_h u = (1/2)[(D1 + (1+m)/r) u+ + (D1 + (1-m)/r) u-] - k u~_z.
// The system is solved by banded solves and one influence coefficient (the
// pressure boundary value that the Poisson rows leave free):
//   p = p_f + a p_h, with L_m p_f = div_h f inside, p_f(1) = 0, and L_m p_h = 0
//   inside, p_h(1) = 1; u = u_f + a u_h, with u_f the Helmholtz solutions driven by
//   f - grad p_f and u_h (precomputed) those driven by -grad p_h; a from the wall
//   continuity row div_h u(1) = 0. Every row of the 4Nr system then holds, so this is
//   its solution. Per mode the plan stores the banded LU factors (partial pivoting) of
//   the four Nr x Nr matrices (Poisson for p, Helmholtz for u+, u-, u~_z), u_h and
//   1 / div_h u_h(1).
// Mode (0,0): u_r = 0 and two Helmholtz problems (u_theta with L_1, u_z with L_0).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

#include "sp_internal.h"

namespace {

// Fornberg's recursion: weights w[i * (mmax+1) + d] of f(x_i) in the derivative of
// order d at x0
void fornberg(double x0, const double* x, int n, int mmax, std::vector<double>& w) {
  w.assign((size_t)n * (mmax + 1), 0.0);
  auto W = [&](int i, int d) -> double& { return w[(size_t)i * (mmax + 1) + d]; };
  double c1 = 1.0, c4 = x[0] - x0;
  W(0, 0) = 1.0;
  for (int i = 1; i < n; ++i) {
    const int mn = std::min(i, mmax);
    double c2 = 1.0;
    const double c5 = c4;
    c4 = x[i] - x0;
    for (int j = 0; j < i; ++j) {
      const double c3 = x[i] - x[j];
      c2 *= c3;
      if (j == i - 1) {
        for (int d = mn; d >= 1; --d) W(i, d) = c1 * (d * W(i - 1, d - 1) - c5 * W(i - 1, d)) / c2;
        W(i, 0) = -c1 * c5 * W(i - 1, 0) / c2;
      }
      for (int d = mn; d >= 1; --d) W(j, d) = (c4 * W(j, d) - d * W(j, d - 1)) / c3;
      W(j, 0) = c4 * W(j, 0) / c3;
    }
    c1 = c2;
  }
}

// Banded LU with partial pivoting of a dense n x n matrix A (row-major) whose nonzeros lie within kl
// sub-diagonals and ku super-diagonals. Row k is exchanged with the row of largest |A[i][k]|,
// k <= i <= k + kl; after the exchanges the upper factor has kl + ku super-diagonals. Stored as the
// interchanges piv[k], the multipliers L[k][q] of rows k + 1 + q, and the rows of the upper factor
// U[i][q] = U(i, i + q), with U[i][0] replaced by its reciprocal. Forward and back substitution in
// band_solve (here) and k_psolve (pipe.cu) apply them in the same order.
struct Band {
  std::vector<int> piv;
  std::vector<double> L, U;
};

bool band_factor(std::vector<double> A, int n, int kl, int kw, Band& B) {
  B.piv.assign(n, 0);
  B.L.assign((size_t)n * kl, 0.0);
  B.U.assign((size_t)n * kw, 0.0);
  for (int k = 0; k < n; ++k) {
    const int last = std::min(n - 1, k + kl);
    int p = k;
    double best = std::fabs(A[(size_t)k * n + k]);
    for (int i = k + 1; i <= last; ++i) {
      const double v = std::fabs(A[(size_t)i * n + k]);
      if (v > best) { best = v; p = i; }
    }
    if (best == 0.0) return false;
    B.piv[k] = p;
    if (p != k)
      for (int j = k; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
    const double d = A[(size_t)k * n + k];
    for (int i = k + 1; i <= last; ++i) {
      const double l = A[(size_t)i * n + k] / d;
      B.L[(size_t)k * kl + (i - k - 1)] = l;
      if (l != 0.0)
        for (int j = k + 1; j < std::min(n, k + kw); ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
    }
    B.U[(size_t)k * kw] = 1.0 / d;
    for (int q = 1; q < kw && k + q < n; ++q) B.U[(size_t)k * kw + q] = A[(size_t)k * n + k + q];
    for (int j = k + kw; j < n; ++j)
      if (A[(size_t)k * n + j] != 0.0) return false;  // outside the assumed band
  }
  return true;
}

void band_solve(const Band& B, int n, int kl, int kw, double* b) {
  for (int k = 0; k < n; ++k) {
    const int p = B.piv[k];
    if (p != k) std::swap(b[k], b[p]);
    const double bk = b[k];
    for (int q = 0; q < kl && k + 1 + q < n; ++q) b[k + 1 + q] -= B.L[(size_t)k * kl + q] * bk;
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int q = 1; q < kw && i + q < n; ++q) s -= B.U[(size_t)i * kw + q] * b[i + q];
    b[i] = s * B.U[(size_t)i * kw];
  }
}

}  // namespace

sp_status sp_build_pipe_plan(sp_ctx* c) {
  const int nr = c->NY;
  std::vector<double> r(nr);
  for (int j = 0; j < nr; ++j) r[j] = std::cos(M_PI * j / (2.0 * nr - 1.0));
  const int st = 9;
  // dense derivative matrices D[par][order-1] and the band table of D1
  std::vector<double> D[2][2];
  std::vector<double> w1((size_t)2 * nr * st);
  std::vector<int> c1((size_t)2 * nr * st);
  for (int par = 0; par < 2; ++par) {
    D[par][0].assign((size_t)nr * nr, 0.0);
    D[par][1].assign((size_t)nr * nr, 0.0);
    const double sg = par ? -1.0 : 1.0;
    std::vector<double> pts(2 * nr);
    for (int i = 0; i < nr; ++i) {
      pts[i] = r[i];
      pts[nr + i] = -r[i];
    }
    for (int j = 0; j < nr; ++j) {
      std::vector<int> idx(2 * nr);
      std::iota(idx.begin(), idx.end(), 0);
      std::stable_sort(idx.begin(), idx.end(),
                       [&](int a, int b) { return std::fabs(pts[a] - r[j]) < std::fabs(pts[b] - r[j]); });
      double xs[st];
      for (int q = 0; q < st; ++q) xs[q] = pts[idx[q]];
      std::vector<double> w;
      fornberg(r[j], xs, st, 2, w);
      for (int q = 0; q < st; ++q) {
        const int col = idx[q] % nr;
        const double s = idx[q] < nr ? 1.0 : sg;
        D[par][0][(size_t)j * nr + col] += s * w[(size_t)q * 3 + 1];
        D[par][1][(size_t)j * nr + col] += s * w[(size_t)q * 3 + 2];
        w1[((size_t)par * nr + j) * st + q] = s * w[(size_t)q * 3 + 1];
        c1[((size_t)par * nr + j) * st + q] = col;
      }
    }
  }
  const double nu = c->nu, lam = 1.0 / c->dt;
  // band of the 9-point stencils (both parities): kl below, ku above the diagonal
  int kl = 0, ku = 0;
  for (int par = 0; par < 2; ++par)
    for (int j = 0; j < nr; ++j)
      for (int q = 0; q < st; ++q) {
        const int col = c1[((size_t)par * nr + j) * st + q];
        kl = std::max(kl, j - col);
        ku = std::max(ku, col - j);
      }
  if (kl > kPipeKL || kl + ku + 1 > kPipeKW) return sp_fail(c, SP_EINVAL, "radial stencil band wider than supported");
  kl = kPipeKL;               // the factors are stored with the fixed widths the kernel is built for
  const int kw = kPipeKW;     // upper factor after the row interchanges
  const size_t chunk = (size_t)nr * (kw + kl) * 8 + ((size_t)nr * 4 + 15) / 16 * 16;
  c->pb_chunk = chunk;
  const size_t nu4 = (size_t)c->n_unique * 4;
  std::vector<unsigned char> fac(nu4 * chunk, 0);
  std::vector<double> uh_all((size_t)c->n_unique * 3 * nr, 0.0), dinv_all(c->n_unique, 0.0);
  auto lapl = [&](int q, int par, double k, std::vector<double>& L) {
    L.assign((size_t)nr * nr, 0.0);
    for (int i = 0; i < nr; ++i) {
      for (int j = 0; j < nr; ++j)
        L[(size_t)i * nr + j] = D[par][1][(size_t)i * nr + j] + D[par][0][(size_t)i * nr + j] / r[i];
      L[(size_t)i * nr + i] -= (double)q * q / (r[i] * r[i]) + k * k;
    }
  };
  int nthreads = (int)std::thread::hardware_concurrency();
  nthreads = std::max(1, std::min(nthreads, 32));
  std::vector<int> bad(nthreads, 0);
  auto work = [&](int tid) {
    std::vector<double> Lq, M;
    Band B[4];
    auto put = [&](int u, int slot, const Band& b) {
      unsigned char* o = fac.data() + ((size_t)u * 4 + slot) * chunk;
      std::memcpy(o, b.U.data(), (size_t)nr * kw * 8);
      std::memcpy(o + (size_t)nr * kw * 8, b.L.data(), (size_t)nr * kl * 8);
      std::memcpy(o + (size_t)nr * (kw + kl) * 8, b.piv.data(), (size_t)nr * 4);
    };
    // row 0: the wall condition (value 0); rows i >= 1: lam - nu L_q (Helmholtz) or L_q (Poisson)
    auto build = [&](int q, int par, double k, bool helm, Band& b) -> bool {
      lapl(q, par, k, Lq);
      M.assign((size_t)nr * nr, 0.0);
      M[0] = 1.0;
      for (int i = 1; i < nr; ++i)
        for (int j = 0; j < nr; ++j)
          M[(size_t)i * nr + j] = helm ? (i == j ? lam : 0.0) - nu * Lq[(size_t)i * nr + j] : Lq[(size_t)i * nr + j];
      return band_factor(M, nr, kl, kw, b);
    };
    auto ident = [&](Band& b) {
      b.piv.resize(nr);
      std::iota(b.piv.begin(), b.piv.end(), 0);
      b.L.assign((size_t)nr * kl, 0.0);
      b.U.assign((size_t)nr * kw, 0.0);
      for (int i = 0; i < nr; ++i) b.U[(size_t)i * kw] = 1.0;
    };
    for (int u = tid; u < c->n_unique; u += nthreads) {
      int pos, iz;
      sp_unique_mode(c, u, &pos, &iz);
      const int kzi = pos <= c->Kx ? pos : pos - c->MX;
      const double k = c->alpha * kzi;
      const int m = (int)std::lround(c->beta) * iz;
      if (pos == 0 && iz == 0) {
        // mean flow: u_theta (L_1, odd parity) and u_z (L_0, even parity); no pressure
        ident(B[0]);
        ident(B[3]);
        if (!build(1, 1, 0.0, true, B[1]) || !build(0, 0, 0.0, true, B[2])) { bad[tid] = 1; continue; }
        for (int s = 0; s < 4; ++s) put(u, s, B[s]);
        continue;
      }
      const int pe = (m + 1) & 1, pz = m & 1;
      if (!build(m, pz, k, false, B[0]) || !build(m + 1, pe, k, true, B[1]) || !build(m - 1, pe, k, true, B[2]) ||
          !build(m, pz, k, true, B[3])) {
        bad[tid] = 1;
        continue;
      }
      for (int s = 0; s < 4; ++s) put(u, s, B[s]);
      // p_h: interior Laplacian zero, unit wall value; u_h: the velocity it drives
      std::vector<double> ph(nr, 0.0);
      ph[0] = 1.0;
      band_solve(B[0], nr, kl, kw, ph.data());
      const std::vector<double>& Dp = D[pz][0];
      const std::vector<double>& Du = D[pe][0];
      double* uh = uh_all.data() + (size_t)u * 3 * nr;
      for (int comp = 0; comp < 3; ++comp) {
        std::vector<double> b(nr, 0.0);
        for (int i = 1; i < nr; ++i) {
          double g = 0.0;
          for (int j = 0; j < nr; ++j) g += Dp[(size_t)i * nr + j] * ph[j];
          const double gp = comp == 0 ? g - m / r[i] * ph[i] : comp == 1 ? g + m / r[i] * ph[i] : k * ph[i];
          b[i] = -gp;
        }
        band_solve(B[comp + 1], nr, kl, kw, b.data());
        std::copy(b.begin(), b.end(), uh + (size_t)comp * nr);
      }
      // wall divergence of u_h (its wall values are zero, so only D1 of u+ + u- remains)
      double den = 0.0;
      for (int j = 0; j < nr; ++j) den += 0.5 * Du[j] * (uh[j] + uh[nr + j]);
      if (den == 0.0 || !std::isfinite(den)) { bad[tid] = 1; continue; }
      dinv_all[u] = 1.0 / den;
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t) th.emplace_back(work, t);
  for (auto& t : th) t.join();
  for (int b : bad)
    if (b) return sp_fail(c, SP_EINVAL, "singular per-mode pipe system");
  // per-plane laminar fields: U = (1 - r^2) e_z, curl U = 2 r e_theta
  std::vector<double> lam6((size_t)nr * 6, 0.0);
  for (int j = 0; j < nr; ++j) {
    lam6[(size_t)j * 6 + 2] = 1.0 - r[j] * r[j];
    lam6[(size_t)j * 6 + 4] = 2.0 * r[j];
  }
  auto up = [&](void** dst, const void* src, size_t bytes) -> bool {
    if (cudaMalloc(dst, bytes) != cudaSuccess) return false;
    return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  const bool ok = up((void**)&c->pb_fac, fac.data(), fac.size()) &&
                  up((void**)&c->pb_uh, uh_all.data(), uh_all.size() * 8) &&
                  up((void**)&c->pb_dinv, dinv_all.data(), dinv_all.size() * 8) && up((void**)&c->yv, r.data(), r.size() * 8) &&
                  up((void**)&c->lam6, lam6.data(), lam6.size() * 8) &&
                  up((void**)&c->fd_w1, w1.data(), w1.size() * 8) && up((void**)&c->fd_c1, c1.data(), c1.size() * 4);
  if (!ok) return sp_fail(c, SP_ENOMEM, "device allocation of the pipe plan failed");
  return sp_build_fft_tables(c);
}
