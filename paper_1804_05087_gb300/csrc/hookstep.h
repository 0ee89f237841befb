// Host-side pieces of Newton-GMRES-hookstep shared by sp_newton_gmres (one
// problem) and sp_group_newton_gmres (many problems in lock step): the Givens
// update of one Arnoldi column, the hookstep (trust-region) solve in the Krylov
// space, and the trust-radius update (Sec. 3.2).
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

// Trust-region subproblem min |g - R y| s.t. |y| <= delta in the Krylov space (the hookstep,
// Sec. 3.2): R^T R = Q T Q^T by Householder tridiagonalisation (once per Newton step), then
// for each radius a safeguarded Newton iteration on 1/|z(mu)| - 1/delta with
// z(mu) = (T + mu I)^-1 Q^T R^T g (two tridiagonal solves per iteration), y = Q z.
struct TrustRegion {
  int k = 0;
  std::vector<double> d, e, c, V;  // diagonal, off-diagonal, Q^T b, Householder vectors (k x k)
  std::vector<double> beta;        // reflector scalars

  void setup(const double* R, int ld, int k_, const double* g) {
    k = k_;
    // M = R^T R, stored in full (row-major, symmetric), and b = R^T g. Every O(k^3) loop below is
    // an axpy over a contiguous row (no reductions), which the compiler vectorises without
    // reassociating sums: M accumulates the rank-one terms of the rows of R, and the product
    // M v of the tridiagonalisation is the sum of the rows of M weighted by v.
    std::vector<double> M((size_t)k * k, 0.0), b(k, 0.0), row(k);
    for (int l = 0; l < k; ++l) {
      for (int i = l; i < k; ++i) row[i] = R[(size_t)i * ld + l];  // row l of R: entries i >= l
      for (int i = l; i < k; ++i) {
        double* Mi = M.data() + (size_t)i * k;
        const double ri = row[i];
        for (int j = l; j < k; ++j) Mi[j] += ri * row[j];
      }
    }
    for (int i = 0; i < k; ++i) {
      double acc = 0;
      for (int l = 0; l <= i; ++l) acc += R[(size_t)i * ld + l] * g[l];
      b[i] = acc;
    }
    V.assign((size_t)k * k, 0.0);
    beta.assign(k, 0.0);
    d.assign(k, 0.0);
    e.assign(k, 0.0);
    std::vector<double> p(k), wv(k);
    // Householder reflector of step col from row col of M (= its column below the diagonal):
    // H = I - bt v v^T, H M[col+1.., col] = s e_1; returns false when the column is already reduced
    auto reflector = [&](int col) -> bool {
      const int c1 = col + 1;
      const double* x = M.data() + (size_t)col * k;
      double alpha = 0;
      for (int i = c1; i < k; ++i) alpha += x[i] * x[i];
      alpha = std::sqrt(alpha);
      const double x0 = x[c1];
      e[col] = x0;
      if (alpha == 0.0) return false;
      const double s = x0 >= 0 ? -alpha : alpha;
      double* v = V.data() + (size_t)col * k;
      v[c1] = x0 - s;
      for (int i = c1 + 1; i < k; ++i) v[i] = x[i];
      double vv = 0;
      for (int i = c1; i < k; ++i) vv += v[i] * v[i];
      if (vv == 0.0) return false;
      beta[col] = 2.0 / vv;
      e[col] = s;
      return true;
    };
    // p = bt A v on the trailing block A = M[c1.., c1..] of step col (rows weighted by v)
    auto product = [&](int col) {
      const int c1 = col + 1;
      const double* v = V.data() + (size_t)col * k;
      for (int j = c1; j < k; ++j) p[j] = 0.0;
      for (int i = c1; i < k; ++i) {
        const double* Mi = M.data() + (size_t)i * k;
        const double vi = beta[col] * v[i];
        for (int j = c1; j < k; ++j) p[j] += vi * Mi[j];
      }
    };
    // Step col: A <- H A H = A - v w^T - w v^T with w = p - (bt v.p / 2) v. The product of the
    // next step is accumulated in the same pass over the rows: row c1 is updated first, which
    // gives the next reflector, and every later row, once updated, adds its share of the next p.
    bool have = k >= 3 && reflector(0);
    if (have) product(0);
    for (int col = 0; col + 2 < k; ++col) {
      const int c1 = col + 1;
      const bool next = c1 + 2 < k;
      if (!have) {  // nothing to apply at this step; set up the next one
        have = next && reflector(c1);
        if (have) product(c1);
        continue;
      }
      const double* v = V.data() + (size_t)col * k;
      const double bt = beta[col];
      double vp = 0;
      for (int i = c1; i < k; ++i) vp += v[i] * p[i];
      const double kk = 0.5 * bt * vp;
      for (int i = c1; i < k; ++i) wv[i] = p[i] - kk * v[i];
      {
        double* Mi = M.data() + (size_t)c1 * k;
        const double vi = v[c1], wi = wv[c1];
        for (int j = c1; j < k; ++j) Mi[j] -= vi * wv[j] + wi * v[j];
      }
      const bool have_next = next && reflector(c1);
      const int c2 = c1 + 1;
      if (have_next) {
        const double* vn = V.data() + (size_t)c1 * k;
        const double btn = beta[c1];
        for (int j = c2; j < k; ++j) p[j] = 0.0;
        for (int i = c2; i < k; ++i) {
          double* Mi = M.data() + (size_t)i * k;
          const double vi = v[i], wi = wv[i], ui = btn * vn[i];
          Mi[c1] -= vi * wv[c1] + wi * v[c1];
          for (int j = c2; j < k; ++j) {
            const double m = Mi[j] - (vi * wv[j] + wi * v[j]);
            Mi[j] = m;
            p[j] += ui * m;
          }
        }
      } else {
        for (int i = c2; i < k; ++i) {
          double* Mi = M.data() + (size_t)i * k;
          const double vi = v[i], wi = wv[i];
          for (int j = c1; j < k; ++j) Mi[j] -= vi * wv[j] + wi * v[j];
        }
      }
      have = have_next;
    }
    for (int i = 0; i < k; ++i) d[i] = M[(size_t)i * k + i];
    if (k >= 2) e[k - 2] = M[(size_t)(k - 1) * k + (k - 2)];
    // c = Q^T b, Q = H_0 H_1 ... (apply H_0 first)
    c = b;
    for (int col = 0; col + 2 < k; ++col) apply(col, c);
  }

  void apply(int col, std::vector<double>& x) const {
    if (beta[col] == 0.0) return;
    const double* v = V.data() + (size_t)col * k;
    double acc = 0;
    for (int i = col + 1; i < k; ++i) acc += v[i] * x[i];
    acc *= beta[col];
    for (int i = col + 1; i < k; ++i) x[i] -= acc * v[i];
  }

  // (T + mu I) z = rhs by the Thomas algorithm (T + mu I is positive definite for mu > 0)
  void tri_solve(double mu, const std::vector<double>& rhs, std::vector<double>& z) const {
    std::vector<double> cp(k), dp(k);
    double den = d[0] + mu;
    cp[0] = k > 1 ? e[0] / den : 0.0;
    dp[0] = rhs[0] / den;
    for (int i = 1; i < k; ++i) {
      den = d[i] + mu - e[i - 1] * cp[i - 1];
      cp[i] = i + 1 < k ? e[i] / den : 0.0;
      dp[i] = (rhs[i] - e[i - 1] * dp[i - 1]) / den;
    }
    z.assign(k, 0.0);
    z[k - 1] = dp[k - 1];
    for (int i = k - 2; i >= 0; --i) z[i] = dp[i] - cp[i] * z[i + 1];
  }

  std::vector<double> solve(double delta) const {
    double tmax = 0;
    for (int i = 0; i < k; ++i)
      tmax = std::max(tmax, std::fabs(d[i]) + (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(e[i]) : 0.0));
    double cn = 0;
    for (double v : c) cn += v * v;
    cn = std::sqrt(cn);
    double lo = 0.0, hi = cn / delta + tmax;   // |z(hi)| <= delta
    double mu = std::max(1e-12 * tmax, 1e-300);
    std::vector<double> z, z2;
    for (int it = 0; it < 100; ++it) {
      tri_solve(mu, c, z);
      double nz = 0;
      for (double v : z) nz += v * v;
      nz = std::sqrt(nz);
      if (!std::isfinite(nz)) {  // mu too close to the spectrum's bottom
        lo = mu;
        mu = 0.5 * (lo + hi);
        continue;
      }
      if (std::fabs(nz - delta) <= 1e-10 * delta) break;
      if (nz > delta) lo = mu;
      else hi = mu;
      tri_solve(mu, z, z2);
      double zz2 = 0;
      for (int i = 0; i < k; ++i) zz2 += z[i] * z2[i];
      // Newton step on phi(mu) = 1/|z| - 1/delta, phi' = (z . z2)/|z|^3
      double step = (1.0 / nz - 1.0 / delta) * nz * nz * nz / std::max(zz2, 1e-300);
      double next = mu - step;
      if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
      if (hi - lo <= 1e-15 * hi) { mu = hi; tri_solve(mu, c, z); break; }
      mu = next;
    }
    // y = Q z: apply the reflectors in reverse order
    std::vector<double> y = z;
    for (int col = k - 3; col >= 0; --col) apply(col, y);
    return y;
  }
};

// Column j of the Hessenberg matrix (Hc, entries 0..j+1, already filled) is
// copied to Rc and reduced by the earlier rotations and a new one for rows
// (j, j+1); g (the rotated right-hand side beta e_1) is updated. Afterwards
// |g[j+1]| is the GMRES residual norm.
inline void givens_column(const double* Hc, double* Rc, int j, double* cs, double* sn, double* g) {
  for (int i = 0; i <= j + 1; ++i) Rc[i] = Hc[i];
  for (int i = 0; i < j; ++i) {
    const double x = Rc[i], y = Rc[i + 1];
    Rc[i] = cs[i] * x + sn[i] * y;
    Rc[i + 1] = -sn[i] * x + cs[i] * y;
  }
  const double rr = std::hypot(Rc[j], Rc[j + 1]);
  cs[j] = rr > 0 ? Rc[j] / rr : 1.0;
  sn[j] = rr > 0 ? Rc[j + 1] / rr : 0.0;
  Rc[j] = rr;
  Rc[j + 1] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
}

// The Krylov-space correction of one Newton step: y0 = R^-1 g (plain GMRES)
// when it lies inside the trust region, else the hookstep y(mu) with
// |y| = delta. R: k x k upper triangle (column-major, leading dimension LD).
struct Hookstep {
  const double* R = nullptr;
  const double* g = nullptr;
  int LD = 0, k = 0;
  std::vector<double> y0;
  double ny0 = 0;
  TrustRegion tr;
  bool have_tr = false;

  void init(const double* R_, int LD_, int k_, const double* g_) {
    R = R_;
    LD = LD_;
    k = k_;
    g = g_;
    have_tr = false;
    y0.assign(k, 0.0);
    for (int i = k - 1; i >= 0; --i) {
      double acc = g[i];
      for (int jj = i + 1; jj < k; ++jj) acc -= R[(size_t)jj * LD + i] * y0[jj];
      y0[i] = R[(size_t)i * LD + i] != 0.0 ? acc / R[(size_t)i * LD + i] : 0.0;
    }
    ny0 = 0;
    for (double v : y0) ny0 += v * v;
    ny0 = std::sqrt(ny0);
  }

  // y for radius delta; pred = predicted |G| after the step, ylen = |y|
  std::vector<double> solve(double delta, double* pred, double* ylen) {
    std::vector<double> y;
    if (ny0 <= delta) {
      y = y0;
    } else {
      if (!have_tr) {
        tr.setup(R, LD, k, g);
        have_tr = true;
      }
      y = tr.solve(delta);
    }
    double pred2 = g[k] * g[k];
    for (int i = 0; i < k; ++i) {
      double acc = g[i];
      for (int jj = i; jj < k; ++jj) acc -= R[(size_t)jj * LD + i] * y[jj];
      pred2 += acc * acc;
    }
    double yl = 0;
    for (double v : y) yl += v * v;
    *ylen = std::sqrt(yl);
    *pred = std::sqrt(pred2);
    return y;
  }
};

// Ratio test of a trial step: returns true if accepted; updates delta.
inline bool trust_update(double nF, double pred, double nT, double ylen, double* delta) {
  const double denom = nF * nF - pred * pred;
  const double rho = denom > 0 ? (nF * nF - nT * nT) / denom : -1.0;
  if (!(rho >= 0.01) || !std::isfinite(nT)) {
    *delta = 0.5 * ylen;
    return false;
  }
  if (rho > 0.75 && ylen >= 0.99 * *delta) *delta *= 2.0;
  else if (rho < 0.25) *delta *= 0.5;
  return true;
}
