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
// The operator stored per mode maps (f+, f-, f~_z) at all radial points to
// (u+, u-, u~_z): a dense real 3Nr x 3Nr matrix (stored column-major), the
// restriction of the inverse of the 4Nr x 4Nr system composed with its
// right-hand-side map.
// Mode (0,0): u_r = 0 and two Helmholtz problems (u_theta with L_1, u_z with L_0).
#include <algorithm>
#include <cmath>
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

bool lu_factor(std::vector<double>& A, int n, std::vector<int>& piv) {
  piv.resize(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(A[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      const double v = std::fabs(A[(size_t)i * n + k]);
      if (v > best) { best = v; p = i; }
    }
    if (best == 0.0) return false;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
    const double inv = 1.0 / A[(size_t)k * n + k];
    for (int i = k + 1; i < n; ++i) {
      const double l = A[(size_t)i * n + k] * inv;
      A[(size_t)i * n + k] = l;
      if (l != 0.0)
        for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
    }
  }
  return true;
}

void lu_solve(const std::vector<double>& LU, int n, const std::vector<int>& piv, double* b) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k) std::swap(b[k], b[piv[k]]);
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int j = 0; j < i; ++j) s -= LU[(size_t)i * n + j] * b[j];
    b[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= LU[(size_t)i * n + j] * b[j];
    b[i] = s / LU[(size_t)i * n + i];
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
  const int n3 = 3 * nr, n4 = 4 * nr;
  c->pop_stride = (size_t)n3 * n3;
  std::vector<double> ops((size_t)c->n_unique * c->pop_stride, 0.0);
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
    std::vector<double> L1, L2, L3, A, X;
    std::vector<int> piv;
    for (int u = tid; u < c->n_unique; u += nthreads) {
      int pos, iz;
      sp_unique_mode(c, u, &pos, &iz);
      const int kzi = pos <= c->Kx ? pos : pos - c->MX;
      const double k = c->alpha * kzi;
      const int m = (int)std::lround(c->beta) * iz;
      double* out = ops.data() + (size_t)u * c->pop_stride;
      if (pos == 0 && iz == 0) {
        // mean flow: u_theta (L_1, odd parity) and u_z (L_0, even parity)
        for (int blk = 0; blk < 2; ++blk) {
          const int q = blk == 0 ? 1 : 0, par = blk == 0 ? 1 : 0;
          lapl(q, par, 0.0, L1);
          A.assign((size_t)nr * nr, 0.0);
          for (int i = 1; i < nr; ++i)
            for (int j = 0; j < nr; ++j) A[(size_t)i * nr + j] = (i == j ? lam : 0.0) - nu * L1[(size_t)i * nr + j];
          A[0] = 1.0;
          if (!lu_factor(A, nr, piv)) { bad[tid] = 1; continue; }
          std::vector<double> b(nr);
          for (int col = 1; col < nr; ++col) {
            std::fill(b.begin(), b.end(), 0.0);
            b[col] = 1.0;
            lu_solve(A, nr, piv, b.data());
            for (int i = 0; i < nr; ++i) out[(size_t)blk * nr * nr + (size_t)col * nr + i] = b[i];
          }
        }
        continue;
      }
      const int pe = (m + 1) & 1, pz = m & 1;
      lapl(m + 1, pe, k, L1);
      lapl(m - 1, pe, k, L2);
      lapl(m, pz, k, L3);
      const std::vector<double>& Dp = D[pz][0];
      const std::vector<double>& Du = D[pe][0];
      A.assign((size_t)n4 * n4, 0.0);
      std::vector<double> B((size_t)n4 * n3, 0.0);
      auto a = [&](int row, int col) -> double& { return A[(size_t)row * n4 + col]; };
      auto bb = [&](int row, int col) -> double& { return B[(size_t)row * n3 + col]; };
      const int U1 = 0, U2 = nr, U3 = 2 * nr, PP = 3 * nr;
      for (int blk = 0; blk < 3; ++blk) {
        const std::vector<double>& L = blk == 0 ? L1 : blk == 1 ? L2 : L3;
        const int base = blk * nr;
        a(base, base) = 1.0;  // no-slip
        for (int i = 1; i < nr; ++i) {
          for (int j = 0; j < nr; ++j) a(base + i, base + j) = (i == j ? lam : 0.0) - nu * L[(size_t)i * nr + j];
          if (blk < 2) {
            for (int j = 0; j < nr; ++j) a(base + i, PP + j) = Dp[(size_t)i * nr + j];
            a(base + i, PP + i) += (blk == 0 ? -1.0 : 1.0) * m / r[i];
          } else {
            a(base + i, PP + i) = k;
          }
          bb(base + i, base + i) = 1.0;
        }
      }
      // divergence rows: continuity at the wall, Poisson right-hand side inside
      for (int i = 0; i < nr; ++i) {
        const int row = PP + i;
        if (i == 0) {
          for (int j = 0; j < nr; ++j) {
            a(row, U1 + j) = 0.5 * Du[j];
            a(row, U2 + j) = 0.5 * Du[j];
          }
          a(row, U1) += 0.5 * (1 + m) / r[0];
          a(row, U2) += 0.5 * (1 - m) / r[0];
          a(row, U3) = -k;
        } else {
          for (int j = 0; j < nr; ++j) a(row, PP + j) = L3[(size_t)i * nr + j];
          for (int j = 0; j < nr; ++j) {
            bb(row, U1 + j) = 0.5 * Du[(size_t)i * nr + j];
            bb(row, U2 + j) = 0.5 * Du[(size_t)i * nr + j];
          }
          bb(row, U1 + i) += 0.5 * (1 + m) / r[i];
          bb(row, U2 + i) += 0.5 * (1 - m) / r[i];
          bb(row, U3 + i) = -k;
        }
      }
      if (!lu_factor(A, n4, piv)) { bad[tid] = 1; continue; }
      std::vector<double> col(n4);
      for (int cc = 0; cc < n3; ++cc) {
        bool any = false;
        for (int i = 0; i < n4; ++i) {
          col[i] = B[(size_t)i * n3 + cc];
          any = any || col[i] != 0.0;
        }
        if (!any) continue;  // wall entries of f do not enter
        lu_solve(A, n4, piv, col.data());
        for (int i = 0; i < n3; ++i) out[(size_t)cc * n3 + i] = col[i];
      }
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
  const bool ok = up((void**)&c->pops, ops.data(), ops.size() * 8) && up((void**)&c->yv, r.data(), r.size() * 8) &&
                  up((void**)&c->lam6, lam6.data(), lam6.size() * 8) &&
                  up((void**)&c->fd_w1, w1.data(), w1.size() * 8) && up((void**)&c->fd_c1, c1.data(), c1.size() * 4);
  if (!ok) return sp_fail(c, SP_ENOMEM, "device allocation of the pipe plan failed");
  return sp_build_fft_tables(c);
}
