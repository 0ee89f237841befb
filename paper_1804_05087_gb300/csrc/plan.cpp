// Plan building: transform tables and the per-mode Stokes solution operators.
//
// Everything here runs once per context on the host and is uploaded to the
// device; no step of the BEFE map itself runs on the host.
//
// The per-mode operators restate the Chebyshev-tau Stokes problem that one
// BEFE step solves for every Fourier mode (Sec. 2, Eq. befe; Sec. 3.2: exact
// direct inversions per mode, pressure through incompressibility satisfied to
// machine accuracy). Rotating the wall-parallel velocity into the component
// along the wavevector (a = (kx u + kz w)/k) and across it
// (b = (-kz u + kx w)/k), the pressure only acts on a and v:
//   (lam - nu D^2) a + i k p = f_a   (Chebyshev rows 0..N-2)
//   (lam - nu D^2) v + D p   = f_v   (rows 0..N-2)
//   i k a + D v = 0                  (every coefficient 0..N)
//   a(+-1) = v(+-1) = 0
//   (lam - nu D^2) b = f_b (rows 0..N-2),  b(+-1) = 0
// with lam = 1/dt + nu k^2. Writing a = i a~ makes the coupled block real.
// Even and odd Chebyshev degrees decouple: v of parity P couples with a~ and
// p of parity 1-P. For each parity the real system is factored once and its
// inverse, restricted to the momentum right-hand sides and to the v unknowns,
// gives v; a follows from continuity, a = (i/k) D v. Eliminating a~ and p with
// continuity and the a~-momentum rows shows that f~_a only enters through the
// reduced right-hand side g = f_v - (1/k) D f~_a (rows of parity P, the sum over
// the a~-momentum rows m > n), so v = V_P g: only the f_v columns of the
// restricted inverse are stored (the matrix V_P, nv_P x rb_P), and the kernels
// form g with one O(N) suffix sum.
// b uses the restricted inverse H_Q of the Dirichlet Helmholtz tau problem.
// The mean mode (0,0) uses H_Q with k = 0 for u and w.
//
// Laminar advection in L (Sec. 3.6, the closing proposal): M u = y du/dx + v e_x
// adds i kx Y (Y: multiplication by y on Chebyshev coefficients) to every
// momentum row and v to the x-momentum rows. In the rotated components
//   (lam - nu D^2 + i kx Y) a~ - i (kx/k) v + k p = f~_a
//   (lam - nu D^2 + i kx Y) v + D p            = f_v
//   (lam - nu D^2 + i kx Y) b = f_b + (kz/k) v
// Y couples the two parities and makes the system complex, but the elimination
// above goes through unchanged (the new terms are operator terms, not
// right-hand sides): v = V' g with the same reduced right-hand side g, now one
// complex operator over both parities, and b = H' (f_b + (kz/k) v) with the
// complex Helmholtz operator H'. The mean mode keeps the real H_Q (kx = 0 and
// v = 0 there).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <thread>

#include "sp_internal.h"

namespace {

// exact-where-possible cos(pi * k / N) for integer k
double cospi_frac(long k, long N) {
  long m = k % (2 * N);
  if (m < 0) m += 2 * N;
  if (m == 0) return 1.0;
  if (m == N) return -1.0;
  if (2 * m == N || 2 * m == 3 * N) return 0.0;
  return std::cos(M_PI * (double)m / (double)N);
}

bool make_fft_plan(int n, FftPlan* p) {
  p->n = n;
  p->nst = 0;
  int m = n;
  while (m % 4 == 0) { p->radix[p->nst++] = 4; m /= 4; }
  while (m % 3 == 0) { p->radix[p->nst++] = 3; m /= 3; }
  while (m % 2 == 0) { p->radix[p->nst++] = 2; m /= 2; }
  return m == 1 && p->nst <= 12;
}

using cplx = std::complex<double>;

// LU with partial pivoting, in place, row-major n x n (S = double or complex).
// Returns false if singular.
template <typename S>
bool lu_factor(std::vector<S>& A, int n, std::vector<int>& piv) {
  piv.resize(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::abs(A[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double v = std::abs(A[(size_t)i * n + k]);
      if (v > best) { best = v; p = i; }
    }
    if (best == 0.0) return false;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
    S inv = S(1.0) / A[(size_t)k * n + k];
    for (int i = k + 1; i < n; ++i) {
      S l = A[(size_t)i * n + k] * inv;
      A[(size_t)i * n + k] = l;
      if (l != S(0.0))
        for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
    }
  }
  return true;
}

template <typename S>
void lu_solve(const std::vector<S>& LU, int n, const std::vector<int>& piv, S* b) {
  for (int k = 0; k < n; ++k) {
    int p = piv[k];
    if (p != k) std::swap(b[k], b[p]);
  }
  for (int i = 0; i < n; ++i) {
    S s = b[i];
    for (int j = 0; j < i; ++j) s -= LU[(size_t)i * n + j] * b[j];
    b[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    S s = b[i];
    for (int j = i + 1; j < n; ++j) s -= LU[(size_t)i * n + j] * b[j];
    b[i] = s / LU[(size_t)i * n + i];
  }
}

struct ChebOps {
  int N;
  std::vector<double> D, D2;  // (N+1)^2 row-major: (Du)_n = sum_m D[n][m] u_m
  std::vector<double> Y;      // multiplication by y: y T_0 = T_1, y T_m = (T_(m+1) + T_(m-1))/2
  explicit ChebOps(int N_) : N(N_) {
    int n1 = N + 1;
    Y.assign((size_t)n1 * n1, 0.0);
    Y[(size_t)1 * n1 + 0] = 1.0;
    for (int m = 1; m < n1; ++m) {
      Y[(size_t)(m - 1) * n1 + m] += 0.5;
      if (m + 1 < n1) Y[(size_t)(m + 1) * n1 + m] += 0.5;
    }
    D.assign((size_t)n1 * n1, 0.0);
    for (int n = 0; n < n1; ++n)
      for (int p = n + 1; p < n1; ++p)
        if ((p + n) & 1) D[(size_t)n * n1 + p] = 2.0 * p / (n == 0 ? 2.0 : 1.0);
    D2.assign((size_t)n1 * n1, 0.0);
    for (int i = 0; i < n1; ++i)
      for (int k = 0; k < n1; ++k) {
        double d = D[(size_t)i * n1 + k];
        if (d == 0.0) continue;
        for (int j = 0; j < n1; ++j) D2[(size_t)i * n1 + j] += d * D[(size_t)k * n1 + j];
      }
  }
};

// V_P: rows = v unknowns of parity P (increasing n), columns = f_v rows of
// parity P (n <= N-2): the restricted inverse applied to g (see above).
bool build_vop(const ChebOps& C, int P, double k, double lam, double nu, double* out) {
  const int N = C.N, n1 = N + 1;
  std::vector<int> vi, ai;
  for (int n = 0; n <= N; ++n) ((n % 2 == P) ? vi : ai).push_back(n);
  const int nv = (int)vi.size(), na = (int)ai.size();
  const int nt = nv + 2 * na;  // v, a~, p (p has the parity of a~)
  std::vector<int> iv(n1, -1), ia(n1, -1);
  for (int i = 0; i < nv; ++i) iv[vi[i]] = i;
  for (int i = 0; i < na; ++i) ia[ai[i]] = i;
  auto col_v = [&](int n) { return iv[n]; };
  auto col_a = [&](int n) { return nv + ia[n]; };
  auto col_p = [&](int n) { return nv + na + ia[n]; };
  std::vector<double> A((size_t)nt * nt, 0.0);
  std::vector<int> rhs_rows;  // row index of each RHS column, in V_P column order
  int r = 0;
  std::vector<int> vrows, arows;
  for (int n = 0; n <= N - 2; ++n) {
    if (n % 2 == P) {  // v-momentum
      for (int m : vi) A[(size_t)r * nt + col_v(m)] = (n == m ? lam : 0.0) - nu * C.D2[(size_t)n * n1 + m];
      for (int m : ai) A[(size_t)r * nt + col_p(m)] = C.D[(size_t)n * n1 + m];
      vrows.push_back(r++);
    }
  }
  for (int n = 0; n <= N - 2; ++n) {
    if (n % 2 != P) {  // a~-momentum: (lam - nu D^2) a~ + k p = f~_a
      for (int m : ai) A[(size_t)r * nt + col_a(m)] = (n == m ? lam : 0.0) - nu * C.D2[(size_t)n * n1 + m];
      A[(size_t)r * nt + col_p(n)] += k;
      arows.push_back(r++);
    }
  }
  for (int n = 0; n <= N; ++n) {
    if (n % 2 != P) {  // continuity: -k a~_n + (D v)_n = 0
      A[(size_t)r * nt + col_a(n)] = -k;
      for (int m : vi) A[(size_t)r * nt + col_v(m)] = C.D[(size_t)n * n1 + m];
      ++r;
    }
  }
  for (int m : vi) A[(size_t)r * nt + col_v(m)] = 1.0;  // v(+1) = 0 (= v(-1) up to sign)
  ++r;
  for (int m : ai) A[(size_t)r * nt + col_a(m)] = 1.0;  // a(+1) = 0
  ++r;
  if (r != nt) return false;
  std::vector<int> piv;
  if (!lu_factor(A, nt, piv)) return false;
  rhs_rows = vrows;  // the f_v rows only: f~_a enters through g
  const int ncol = (int)rhs_rows.size();
  std::vector<double> b(nt);
  for (int cidx = 0; cidx < ncol; ++cidx) {
    std::fill(b.begin(), b.end(), 0.0);
    b[rhs_rows[cidx]] = 1.0;
    lu_solve(A, nt, piv, b.data());
    for (int i = 0; i < nv; ++i) out[(size_t)cidx * nv + i] = b[i];  // column-major
  }
  return true;
}

// H_Q: rows = unknowns of parity Q, columns = momentum rows of parity Q (n <= N-2).
bool build_hop(const ChebOps& C, int Q, double lam, double nu, double* out) {
  const int N = C.N, n1 = N + 1;
  std::vector<int> bi;
  for (int n = Q; n <= N; n += 2) bi.push_back(n);
  const int nb = (int)bi.size();
  std::vector<double> A((size_t)nb * nb, 0.0);
  std::vector<int> rows;
  int r = 0;
  for (int n = Q; n <= N - 2; n += 2) {
    for (int i = 0; i < nb; ++i) {
      int m = bi[i];
      A[(size_t)r * nb + i] = (n == m ? lam : 0.0) - nu * C.D2[(size_t)n * n1 + m];
    }
    rows.push_back(r++);
  }
  for (int i = 0; i < nb; ++i) A[(size_t)r * nb + i] = 1.0;
  ++r;
  if (r != nb) return false;
  std::vector<int> piv;
  if (!lu_factor(A, nb, piv)) return false;
  const int ncol = (int)rows.size();
  std::vector<double> b(nb);
  for (int cidx = 0; cidx < ncol; ++cidx) {
    std::fill(b.begin(), b.end(), 0.0);
    b[rows[cidx]] = 1.0;
    lu_solve(A, nb, piv, b.data());
    for (int i = 0; i < nb; ++i) out[(size_t)cidx * nb + i] = b[i];  // column-major
  }
  return true;
}

// V': the v unknowns n = 0..N (rows) against the reduced right-hand side g in the
// parity order of the kernel (column j < N/2: row 2j; j >= N/2: row 2(j - N/2) + 1),
// complex, column-major, (re, im) pairs. Laminar advection in L (see the top).
bool build_vop_la(const ChebOps& C, double kx, double k, double lam, double nu, double* out) {
  const int N = C.N, n1 = N + 1, nt = 3 * n1;
  const cplx ikx(0.0, kx);
  auto col_v = [&](int n) { return n; };
  auto col_a = [&](int n) { return n1 + n; };
  auto col_p = [&](int n) { return 2 * n1 + n; };
  std::vector<cplx> A((size_t)nt * nt, cplx(0.0));
  std::vector<int> vrow(n1, -1);
  int r = 0;
  auto op = [&](int n, int m) {
    return cplx((n == m ? lam : 0.0) - nu * C.D2[(size_t)n * n1 + m]) + ikx * C.Y[(size_t)n * n1 + m];
  };
  for (int n = 0; n <= N - 2; ++n) {  // v-momentum
    for (int m = 0; m < n1; ++m) {
      A[(size_t)r * nt + col_v(m)] = op(n, m);
      A[(size_t)r * nt + col_p(m)] = C.D[(size_t)n * n1 + m];
    }
    vrow[n] = r++;
  }
  for (int n = 0; n <= N - 2; ++n) {  // a~-momentum
    for (int m = 0; m < n1; ++m) A[(size_t)r * nt + col_a(m)] = op(n, m);
    A[(size_t)r * nt + col_v(n)] += cplx(0.0, -kx / k);
    A[(size_t)r * nt + col_p(n)] += k;
    ++r;
  }
  for (int n = 0; n <= N; ++n) {  // continuity: -k a~_n + (D v)_n = 0
    A[(size_t)r * nt + col_a(n)] = -k;
    for (int m = 0; m < n1; ++m) A[(size_t)r * nt + col_v(m)] = C.D[(size_t)n * n1 + m];
    ++r;
  }
  for (int m = 0; m < n1; ++m) {  // v(+1) = v(-1) = a(+1) = a(-1) = 0
    const double sg = (m & 1) ? -1.0 : 1.0;
    A[(size_t)r * nt + col_v(m)] = 1.0;
    A[(size_t)(r + 1) * nt + col_v(m)] = sg;
    A[(size_t)(r + 2) * nt + col_a(m)] = 1.0;
    A[(size_t)(r + 3) * nt + col_a(m)] = sg;
  }
  r += 4;
  if (r != nt) return false;
  std::vector<int> piv;
  if (!lu_factor(A, nt, piv)) return false;
  const int cv = N / 2;
  std::vector<cplx> b(nt);
  for (int j = 0; j < N - 1; ++j) {
    const int n = j < cv ? 2 * j : 2 * (j - cv) + 1;
    std::fill(b.begin(), b.end(), cplx(0.0));
    b[vrow[n]] = 1.0;
    lu_solve(A, nt, piv, b.data());
    for (int i = 0; i < n1; ++i) {
      out[((size_t)j * n1 + i) * 2 + 0] = b[col_v(i)].real();
      out[((size_t)j * n1 + i) * 2 + 1] = b[col_v(i)].imag();
    }
  }
  return true;
}

// H': the Dirichlet problem (lam - nu D^2 + i kx Y) b = r on rows 0..N-2, b(+-1) = 0;
// rows = unknowns n = 0..N, columns = momentum rows 0..N-2, complex, column-major.
bool build_hop_la(const ChebOps& C, double kx, double lam, double nu, double* out) {
  const int N = C.N, n1 = N + 1;
  std::vector<cplx> A((size_t)n1 * n1, cplx(0.0));
  for (int n = 0; n <= N - 2; ++n)
    for (int m = 0; m < n1; ++m)
      A[(size_t)n * n1 + m] = cplx((n == m ? lam : 0.0) - nu * C.D2[(size_t)n * n1 + m], kx * C.Y[(size_t)n * n1 + m]);
  for (int m = 0; m < n1; ++m) {
    A[(size_t)(N - 1) * n1 + m] = 1.0;
    A[(size_t)N * n1 + m] = (m & 1) ? -1.0 : 1.0;
  }
  std::vector<int> piv;
  if (!lu_factor(A, n1, piv)) return false;
  std::vector<cplx> b(n1);
  for (int j = 0; j <= N - 2; ++j) {
    std::fill(b.begin(), b.end(), cplx(0.0));
    b[j] = 1.0;
    lu_solve(A, n1, piv, b.data());
    for (int i = 0; i < n1; ++i) {
      out[((size_t)j * n1 + i) * 2 + 0] = b[i].real();
      out[((size_t)j * n1 + i) * 2 + 1] = b[i].imag();
    }
  }
  return true;
}

// ------------------------------------------------------------ O(N) chains
// The same per-mode tau problems, solved in O(N) per right-hand side (the batched
// tangent's solve, solve_chain.cu). For a Dirichlet Helmholtz tau problem
//   (l' - n' D^2) x = f on rows n <= N-2 of parity Q,  sum over parity Q of x_n = bc,
// the identity between the Chebyshev coefficients of x and of x'' (for n >= 2)
//   x_n = c_{n-2} x''_{n-2} / (4n(n-1)) - x''_n / (2(n^2-1)) + x''_{n+2} / (4n(n+1)),
// with x''_k = (l' x_k - f_k) / n' on the tau rows and 0 above them, turns rows
// n = 2..N into a tridiagonal system in the coefficients of parity Q:
//   -l' c_{n-2} / (4n(n-1)) x_{n-2} + (n' + [n <= N-2] l' / (2(n^2-1))) x_n
//     - [n+2 <= N-2] l' / (4n(n+1)) x_{n+2}
//   = -c_{n-2} f_{n-2} / (4n(n-1)) + [n <= N-2] f_n / (2(n^2-1)) - [n+2 <= N-2] f_{n+2} / (4n(n+1)),
// an invertible recombination of the tau rows (so the solution is the tau
// solution), which together with the boundary row is solved by one elimination
// sweep from the top and one substitution sweep from the bottom. Per unknown
// i = 1..m (n = 2i + Q) the sweep is beta_i = r_i q_i - p_i beta_{i+1} with r_i the
// right-hand side of row n above, the boundary-row weights psi_i give
// x_0 = (bc - sum_i psi_i beta_i) g, and the substitution is x_i = alpha_i x_{i-1} + beta_i.
// The device record of unknown i holds (q w_0, q w_1, q w_2, p, psi, alpha), w_k the
// weights of f_{n-2}, f_n, f_{n+2} in r_i: the sweep then costs one product and three
// fused multiply-adds per real component.
// H uses (l', n') = (lam, nu); K uses (-k^2, -1), i.e. (D^2 - k^2) x = f.
//
// The coupled (v, a, p) problem of parity P is the fourth-order tau problem
//   (lam - nu D^2)(D^2 - k^2) v = -k^2 g + tau h   on rows n <= N-2 of parity P,
//   v(+-1) = Dv(+-1) = 0,
// where h_n = 1/c_n carries the one pressure coefficient (p_{N-1} or p_N) that no
// tau row fixes. With w = (D^2 - k^2) v it is two Helmholtz problems: w = w_A +
// sigma psi_w + tau w_h from H (w_A: right-hand side -k^2 g, bc 0; psi_w: bc 1;
// w_h: right-hand side h), then v = K(w) with v(+-1) = 0, and sigma, tau from the
// two conditions left: the top coefficient of w = (D^2 - k^2) v (w_top = -k^2 v_top,
// the tau problem for v leaves it free) and Dv(+-1) = 0 (sum n^2 v_n = 0). The
// record stores v_psi = K(psi_w), v_h = K(w_h) and the inverse of the 2 x 2
// influence matrix of these two conditions.
struct TriOp {
  std::vector<double> q, p, psi, alpha;  // index 1..m
  double g = 0.0;                        // 1 / sum_i gamma_i
};

// RHS weights of row n of the tridiagonal form (universal: depend on n and N only)
void chain_weights(int N, int n, double* w) {
  const double cm2 = (n - 2 == 0) ? 2.0 : 1.0;
  w[0] = -cm2 / (4.0 * n * (n - 1));
  w[1] = (n <= N - 2) ? 1.0 / (2.0 * ((double)n * n - 1.0)) : 0.0;
  w[2] = (n + 2 <= N - 2) ? -1.0 / (4.0 * n * (n + 1.0)) : 0.0;
}

TriOp tri_factor(int N, int Q, double lp, double np_) {
  const int m = (N - Q) / 2;  // unknowns i = 0..m
  TriOp t;
  t.q.assign(m + 2, 0.0);
  t.p.assign(m + 2, 0.0);
  t.psi.assign(m + 2, 0.0);
  t.alpha.assign(m + 2, 0.0);
  for (int i = m; i >= 1; --i) {
    const int n = 2 * i + Q;
    const double cm2 = (n - 2 == 0) ? 2.0 : 1.0;
    const double l = -lp * cm2 / (4.0 * n * (n - 1));
    const double d = np_ + ((n <= N - 2) ? lp / (2.0 * ((double)n * n - 1.0)) : 0.0);
    const double u = (n + 2 <= N - 2) ? -lp / (4.0 * n * (n + 1.0)) : 0.0;
    const double den = d + u * t.alpha[i + 1];
    t.alpha[i] = -l / den;
    t.q[i] = 1.0 / den;
    t.p[i] = u / den;
  }
  double gsum = 1.0, gam = 1.0;
  for (int i = 1; i <= m; ++i) {
    gam *= t.alpha[i];
    gsum += gam;
  }
  t.g = 1.0 / gsum;
  t.psi[m] = 1.0;
  for (int k = m - 1; k >= 1; --k) t.psi[k] = 1.0 + t.alpha[k + 1] * t.psi[k + 1];
  return t;
}

// x (parity Q, index i <-> n = 2i + Q) solving the Helmholtz tau problem with
// right-hand side f (full Chebyshev index, rows <= N-2 read) and boundary value bc
std::vector<double> tri_solve(int N, int Q, const TriOp& t, const std::vector<double>& f, double bc) {
  const int m = (N - Q) / 2;
  std::vector<double> beta(m + 2, 0.0), x(m + 1, 0.0);
  auto F = [&](int n) { return (n >= 0 && n <= N - 2) ? f[n] : 0.0; };
  double acc = 0.0;
  for (int i = m; i >= 1; --i) {
    const int n = 2 * i + Q;
    double w[3];
    chain_weights(N, n, w);
    const double r = w[0] * F(n - 2) + w[1] * F(n) + w[2] * F(n + 2);
    beta[i] = r * t.q[i] - t.p[i] * beta[i + 1];
    acc += t.psi[i] * beta[i];
  }
  x[0] = (bc - acc) * t.g;
  for (int i = 1; i <= m; ++i) x[i] = t.alpha[i] * x[i - 1] + beta[i];
  return x;
}

// the sweep record of one tridiagonal operator (6 doubles per unknown i = 1..m, see above)
void put_sweep_record(int N, int Q, const TriOp& t, double* r6) {
  const int m = (N - Q) / 2;
  for (int i = 1; i <= m; ++i) {
    double w[3];
    chain_weights(N, 2 * i + Q, w);
    r6[6 * i + 0] = t.q[i] * w[0];
    r6[6 * i + 1] = t.q[i] * w[1];
    r6[6 * i + 2] = t.q[i] * w[2];
    r6[6 * i + 3] = t.p[i];
    r6[6 * i + 4] = t.psi[i];
    r6[6 * i + 5] = t.alpha[i];
  }
}

// the record of one parity: [H x 6 NH][K x 6 NH][(v_psi, v_h) x NH][8 scalars]
void build_chain_parity(int N, int P, double k, double lam, double nu, bool mean, double* out) {
  const int NH = N / 2 + 1, m = (N - P) / 2;
  const TriOp H = tri_factor(N, P, lam, nu);
  double* v2 = out + 12 * NH;
  double* sc = out + 14 * NH;
  put_sweep_record(N, P, H, out);
  sc[0] = H.g;
  if (mean) return;
  const double k2 = k * k;
  const TriOp K = tri_factor(N, P, -k2, -1.0);
  put_sweep_record(N, P, K, out + 6 * NH);
  sc[1] = K.g;
  const int n1 = N + 1;
  std::vector<double> zero(n1, 0.0), h(n1, 0.0);
  for (int n = P; n <= N - 2; n += 2) h[n] = (n == 0) ? 0.5 : 1.0;
  const std::vector<double> wpsi = tri_solve(N, P, H, zero, 1.0);
  const std::vector<double> wh = tri_solve(N, P, H, h, 0.0);
  auto full = [&](const std::vector<double>& x) {
    std::vector<double> f(n1, 0.0);
    for (int i = 0; i <= m; ++i) f[2 * i + P] = x[i];
    return f;
  };
  const std::vector<double> vpsi = tri_solve(N, P, K, full(wpsi), 0.0);
  const std::vector<double> vh = tri_solve(N, P, K, full(wh), 0.0);
  double n2psi = 0.0, n2h = 0.0;
  for (int i = 0; i <= m; ++i) {
    const double n = 2.0 * i + P;
    n2psi += n * n * vpsi[i];
    n2h += n * n * vh[i];
    v2[2 * i + 0] = vpsi[i];
    v2[2 * i + 1] = vh[i];
  }
  const double e00 = wpsi[m] + k2 * vpsi[m], e01 = wh[m] + k2 * vh[m];
  const double e10 = n2psi, e11 = n2h;
  const double det = e00 * e11 - e01 * e10;
  sc[2] = e11 / det;
  sc[3] = -e01 / det;
  sc[4] = -e10 / det;
  sc[5] = e00 / det;
}

}  // namespace

// unique mode u -> (pos, iz): positions 0..Kx keep every iz, negative ix skip iz = 0
void sp_unique_mode(const sp_ctx* c, int u, int* pos, int* iz) {
  int first = (c->Kx + 1) * c->MZ;
  if (u < first) {
    *pos = u / c->MZ;
    *iz = u % c->MZ;
  } else {
    int v = u - first;
    *pos = c->Kx + 1 + v / (c->MZ - 1);
    *iz = 1 + v % (c->MZ - 1);
  }
}

sp_status sp_build_plan(sp_ctx* c) {
  const int N = c->N, n1 = N + 1, NH = c->NH;
  // Chebyshev tables on the half grid j = 0..N/2
  std::vector<double> Th((size_t)NH * n1), TDh((size_t)NH * n1), Cfh((size_t)n1 * NH);
  for (int j = 0; j < NH; ++j) {
    for (int n = 0; n < n1; ++n) {
      Th[(size_t)j * n1 + n] = cospi_frac((long)j * n, N);
      // T_n'(cos th) = n sin(n th) / sin(th); T_n'(1) = n^2
      double d;
      if (j == 0) d = (double)n * n;
      else d = n * cospi_frac((long)N - 2L * j * n, 2L * N) / cospi_frac((long)N - 2L * j, 2L * N);
      TDh[(size_t)j * n1 + n] = d;
    }
  }
  for (int n = 0; n < n1; ++n) {
    double cbn = (n == 0 || n == N) ? 2.0 : 1.0;
    for (int j = 0; j < NH; ++j) {
      double cbj = (j == 0) ? 2.0 : 1.0;  // j = N is not on the half grid
      Cfh[(size_t)n * NH + j] = 2.0 / (N * cbn) * cospi_frac((long)j * n, N) / cbj;
    }
  }
  // the second level of the even/odd split (N divisible by 4): at y_{N/2-jq}, odd degrees
  // n = 2m+1 give T_n = (-1)^m sin(pi jq n / N) and T_n' = (-1)^m n cos(pi jq n / N) / cos(pi jq / N)
  const int NQ = N / 4 + 1;
  const bool q2 = N % 4 == 0 && N >= 4;
  std::vector<double> Tp, TDp, tq, Cq;
  if (q2) {
    Cq.assign((size_t)n1 * NQ, 0.0);
    for (int n = 0; n < n1; n += 2) {
      const double cbn = (n == 0 || n == N) ? 2.0 : 1.0;
      for (int jq = 0; jq < NQ; ++jq) Cq[(size_t)n * NQ + jq] = 2.0 / (N * cbn) * cospi_frac((long)jq * n, N);
    }
    Tp.assign((size_t)NQ * n1, 0.0);
    TDp.assign((size_t)NQ * n1, 0.0);
    tq.assign(NQ, 0.0);
    for (int jq = 0; jq < NQ; ++jq) {
      const double cj = cospi_frac(jq, N), sj = cospi_frac((long)N - 2L * jq, 2L * N);
      tq[jq] = sj / cj;
      for (int n = 1; n < n1; n += 2) {
        const double sg = (((n - 1) / 2) & 1) ? -1.0 : 1.0;
        Tp[(size_t)jq * n1 + n] = sg * cospi_frac((long)N - 2L * jq * n, 2L * N);
        TDp[(size_t)jq * n1 + n] = sg * n * cospi_frac((long)jq * n, N) / cj;
      }
    }
  }
  // twiddles exp(-2 pi i k / n)
  std::vector<double> yv(n1), lam6((size_t)n1 * 6, 0.0);
  for (int j = 0; j < n1; ++j) {
    yv[j] = cospi_frac(j, N);
    lam6[(size_t)j * 6 + 0] = yv[j];   // U_lam = y e_x
    lam6[(size_t)j * 6 + 5] = -1.0;    // curl U_lam = -e_z
  }

  // per-mode operators
  c->nv0 = N / 2 + 1;
  c->nv1 = N / 2;
  c->rb0 = N / 2;      // momentum rows of parity 0 (n <= N-2): columns of V_0 and H_0
  c->rb1 = N / 2 - 1;  // parity 1: columns of V_1 and H_1
  c->cv = N / 2;       // stride of the per-parity right-hand sides in shared memory
  c->off_v0 = 0;
  c->off_v1 = c->off_v0 + c->nv0 * c->rb0;
  c->off_h0 = c->off_v1 + c->nv1 * c->rb1;
  c->off_h1 = c->off_h0 + c->nv0 * c->rb0;
  c->op_stride = c->off_h1 + c->nv1 * c->rb1;
  const bool la = c->cfg.lam_adv != 0;
  if (la) {
    // complex V' and H', (N - 1) columns of N + 1 rows each; the mean mode keeps H_Q
    c->off_vc = 0;
    c->off_hc = 2 * (N - 1) * n1;
    c->op_stride = std::max(c->op_stride, 4 * (N - 1) * n1);
    c->op_stride += c->op_stride & 1;  // 16-byte aligned complex columns
  }
  std::vector<double> ops((size_t)c->n_unique * c->op_stride, 0.0);
  ChebOps C(N);
  int nthreads = (int)std::thread::hardware_concurrency();
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 32) nthreads = 32;
  std::vector<int> bad(nthreads, 0);
  auto work = [&](int tid) {
    for (int u = tid; u < c->n_unique; u += nthreads) {
      int pos, iz;
      sp_unique_mode(c, u, &pos, &iz);
      int ix = pos <= c->Kx ? pos : pos - c->MX;
      double kx = c->alpha * ix, kz = c->beta * iz;
      double k2 = kx * kx + kz * kz, k = std::sqrt(k2);
      double lam = 1.0 / c->dt + c->nu * k2;
      double* o = ops.data() + (size_t)u * c->op_stride;
      bool ok = true;
      if (la && u != 0) {
        ok = ok && build_vop_la(C, kx, k, lam, c->nu, o + c->off_vc);
        ok = ok && build_hop_la(C, kx, lam, c->nu, o + c->off_hc);
      } else {
        if (u != 0) {
          ok = ok && build_vop(C, 0, k, lam, c->nu, o + c->off_v0);
          ok = ok && build_vop(C, 1, k, lam, c->nu, o + c->off_v1);
        }
        ok = ok && build_hop(C, 0, lam, c->nu, o + c->off_h0);
        ok = ok && build_hop(C, 1, lam, c->nu, o + c->off_h1);
      }
      if (!ok) bad[tid] = 1;
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t) th.emplace_back(work, t);
  for (auto& t : th) t.join();
  for (int b : bad)
    if (b) return sp_fail(c, SP_EINVAL, "singular per-mode Stokes system");

  // O(N) chain records and the universal row weights (the batched tangent's solve)
  c->use_chain =
      (c->cfg.max_batch >= kChainMinBatch && !la && N < kChainMaxRows) ? 1 : 0;
  std::vector<double> chain;
  if (c->use_chain) {
    c->chain_par = 14 * NH + 8;
    c->chain_stride = 2 * c->chain_par;
    chain.assign((size_t)c->n_unique * c->chain_stride, 0.0);
    for (int u = 0; u < c->n_unique; ++u) {
      int pos, iz;
      sp_unique_mode(c, u, &pos, &iz);
      const int ix = pos <= c->Kx ? pos : pos - c->MX;
      const double kx = c->alpha * ix, kz = c->beta * iz, k = std::sqrt(kx * kx + kz * kz);
      const double lam = 1.0 / c->dt + c->nu * k * k;
      for (int P = 0; P < 2; ++P)
        build_chain_parity(N, P, k, lam, c->nu, u == 0, chain.data() + (size_t)u * c->chain_stride + P * c->chain_par);
    }
  }

  // float copies
  std::vector<float> Thf(Th.begin(), Th.end()), TDhf(TDh.begin(), TDh.end()),
      Cfhf(Cfh.begin(), Cfh.end());

  auto up = [&](void** dst, const void* src, size_t bytes) -> bool {
    if (cudaMalloc(dst, bytes) != cudaSuccess) return false;
    return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  bool ok = up((void**)&c->Th, Th.data(), Th.size() * 8) && up((void**)&c->TDh, TDh.data(), TDh.size() * 8) &&
            up((void**)&c->Cfh, Cfh.data(), Cfh.size() * 8) && up((void**)&c->Th_f, Thf.data(), Thf.size() * 4) &&
            up((void**)&c->TDh_f, TDhf.data(), TDhf.size() * 4) && up((void**)&c->Cfh_f, Cfhf.data(), Cfhf.size() * 4) &&
            up((void**)&c->ops, ops.data(), ops.size() * 8) && up((void**)&c->yv, yv.data(), yv.size() * 8) &&
            up((void**)&c->lam6, lam6.data(), lam6.size() * 8) &&
            (!c->use_chain || up((void**)&c->chain, chain.data(), chain.size() * 8));
  if (!ok) return sp_fail(c, SP_ENOMEM, "device allocation of plan tables failed");
  // the tensor-core inverse transform's constant operands: the full T and T' (all NY points)
  if (c->geom == 0 && c->NY >= 41 && c->NY <= 72) {
    std::vector<double> th((size_t)n1 * n1), td((size_t)n1 * n1);
    for (int j = 0; j < n1; ++j)
      for (int n = 0; n < n1; ++n) {
        th[(size_t)j * n1 + n] = cospi_frac((long)j * n, N);
        double d;
        if (j == 0) d = (double)n * n;
        else if (j == N) d = ((n + 1) % 2 == 0 ? 1.0 : -1.0) * n * n;
        else d = n * cospi_frac((long)N - 2L * j * n, 2L * N) / cospi_frac((long)N - 2L * j, 2L * N);
        td[(size_t)j * n1 + n] = d;
      }
    const std::vector<float> img = yinv_tc_image(th.data(), td.data(), n1);
    if (!up((void**)&c->yinv_tc_mat, img.data(), img.size() * 4))
      return sp_fail(c, SP_ENOMEM, "device allocation of plan tables failed");
    // the forward transform's: C[n][j] = 2 T_n(y_j) / (N cbar_n cbar_j) on the tau rows n <= N - 2
    const int NR = N - 1;
    std::vector<double> cf((size_t)NR * n1);
    for (int n = 0; n < NR; ++n) {
      const double cbn = n == 0 ? 2.0 : 1.0;
      for (int j = 0; j < n1; ++j) {
        const double cbj = (j == 0 || j == N) ? 2.0 : 1.0;
        cf[(size_t)n * n1 + j] = 2.0 / (N * cbn) * cospi_frac((long)j * n, N) / cbj;
      }
    }
    const std::vector<float> imf = rhs_tc_image(cf.data(), n1, NR);
    if (!up((void**)&c->rhs_tc_mat, imf.data(), imf.size() * 4))
      return sp_fail(c, SP_ENOMEM, "device allocation of plan tables failed");
  }
  if (q2) {
    std::vector<float> Tpf(Tp.begin(), Tp.end()), TDpf(TDp.begin(), TDp.end()), tqf(tq.begin(), tq.end()),
        Cqf(Cq.begin(), Cq.end());
    ok = up((void**)&c->Cq, Cq.data(), Cq.size() * 8) && up((void**)&c->Cq_f, Cqf.data(), Cqf.size() * 4) &&
         up((void**)&c->Tp, Tp.data(), Tp.size() * 8) && up((void**)&c->TDp, TDp.data(), TDp.size() * 8) &&
         up((void**)&c->tq, tq.data(), tq.size() * 8) && up((void**)&c->Tp_f, Tpf.data(), Tpf.size() * 4) &&
         up((void**)&c->TDp_f, TDpf.data(), TDpf.size() * 4) && up((void**)&c->tq_f, tqf.data(), tqf.size() * 4);
    if (!ok) return sp_fail(c, SP_ENOMEM, "device allocation of plan tables failed");
  }
  return sp_build_fft_tables(c);
}

// FFT plans and twiddle tables exp(-2 pi i k / n) of the two periodic directions
sp_status sp_build_fft_tables(sp_ctx* c) {
  if (!make_fft_plan(c->nx, &c->px) || !make_fft_plan(c->nz, &c->pz))
    return sp_fail(c, SP_EINVAL, "the periodic grid sizes must be products of 2 and 3");
  // twiddles exp(-2 pi i k / n); sin(pi m / N) = cos(pi (N - 2m) / (2N))
  auto tw = [](int n) {
    std::vector<double2> t(n);
    for (int k = 0; k < n; ++k) {
      t[k].x = cospi_frac(2L * k, n);
      t[k].y = -cospi_frac((long)n - 4L * k, 2L * n);
    }
    return t;
  };
  std::vector<double2> twx = tw(c->nx), twz = tw(c->nz);
  std::vector<float2> twxf(c->nx), twzf(c->nz);
  for (int k = 0; k < c->nx; ++k) twxf[k] = make_float2((float)twx[k].x, (float)twx[k].y);
  for (int k = 0; k < c->nz; ++k) twzf[k] = make_float2((float)twz[k].x, (float)twz[k].y);
  auto up = [&](void** dst, const void* src, size_t bytes) -> bool {
    if (cudaMalloc(dst, bytes) != cudaSuccess) return false;
    return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  const bool ok = up((void**)&c->twx, twx.data(), twx.size() * 16) && up((void**)&c->twz, twz.data(), twz.size() * 16) &&
                  up((void**)&c->twx_f, twxf.data(), twxf.size() * 8) && up((void**)&c->twz_f, twzf.data(), twzf.size() * 8);
  if (!ok) return sp_fail(c, SP_ENOMEM, "device allocation of twiddle tables failed");
  return SP_OK;
}
