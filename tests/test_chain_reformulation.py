"""The O(N) per-mode Stokes solve of the batched tangent (Sec. 2, Eq. befe; Sec. 3.2: the exact
per-mode Chebyshev-tau inversion) restated in numpy, step for step as the chain kernel takes it, and
checked against the oracle's dense tau system of the same mode.

The reformulation: the Dirichlet Helmholtz tau problem (l' - n' D^2) x = f on the rows n <= N-2 of
one parity, with the identity between the Chebyshev coefficients of x and of x'', becomes a
tridiagonal system plus the boundary row, solved by one elimination sweep from the top and one
substitution from the bottom. The coupled (v, a, p) problem of parity P is the fourth-order problem
(lam - nu D^2)(D^2 - k^2) v = -k^2 g + tau h with v(+-1) = Dv(+-1) = 0: two Helmholtz solves (w_A,
then v_A) and a 2 x 2 influence correction (the top coefficient of w = (D^2 - k^2) v, and
sum n^2 v_n = 0). The rotated velocity b of parity 1 - P is one more Helmholtz solve. Each
(mode, parity) item writes G = u_new - u on its own rows; here every output row must be written
exactly once, and the mean mode solves two Dirichlet Helmholtz problems.

This is a restatement of the design, independent of the CUDA sources; the GPU tests compare the
kernel itself with the oracle."""
import math

import numpy as np
import pytest

from oracle.couette import Couette


def row_weights(N, n):
    """Weights of f_{n-2}, f_n, f_{n+2} in the right-hand side of tridiagonal row n."""
    cm2 = 2.0 if n - 2 == 0 else 1.0
    return (-cm2 / (4.0 * n * (n - 1)), 1.0 / (2.0 * (n * n - 1.0)) if n <= N - 2 else 0.0,
            -1.0 / (4.0 * n * (n + 1.0)) if n + 2 <= N - 2 else 0.0)


def tri_factor(N, Q, lp, np_):
    """Elimination coefficients of (lp - np_ D^2) x = f on the rows of parity Q."""
    m = (N - Q) // 2
    q, p, psi, al = (np.zeros(m + 2) for _ in range(4))
    for i in range(m, 0, -1):
        n = 2 * i + Q
        cm2 = 2.0 if n - 2 == 0 else 1.0
        lo = -lp * cm2 / (4.0 * n * (n - 1))
        d = np_ + (lp / (2.0 * (n * n - 1.0)) if n <= N - 2 else 0.0)
        up = -lp / (4.0 * n * (n + 1.0)) if n + 2 <= N - 2 else 0.0
        den = d + up * al[i + 1]
        al[i], q[i], p[i] = -lo / den, 1.0 / den, up / den
    gs, gam = 1.0, 1.0
    for i in range(1, m + 1):
        gam *= al[i]
        gs += gam
    psi[m] = 1.0
    for i in range(m - 1, 0, -1):
        psi[i] = 1.0 + al[i + 1] * psi[i + 1]
    return dict(q=q, p=p, psi=psi, al=al, g=1.0 / gs)


def sweep(N, Q, T, rhs, bc):
    """x_i (n = 2i + Q) of the Dirichlet problem; rhs(n) is called from the top row down."""
    m = (N - Q) // 2
    X = np.zeros(m + 1, complex)
    r_hi, r_mid, b_next, acc = 0.0, rhs(2 * m + Q), 0.0, 0.0
    for i in range(m, 0, -1):
        n = 2 * i + Q
        r_lo = rhs(n - 2)
        w = row_weights(N, n)
        b = (w[0] * r_lo + w[1] * r_mid + w[2] * r_hi) * T["q"][i] - T["p"][i] * b_next
        acc += T["psi"][i] * b
        X[i] = b
        b_next, r_hi, r_mid = b, r_mid, r_lo
    x = (bc - acc) * T["g"]
    X[0] = x
    for i in range(1, m + 1):
        x = X[i] + x * T["al"][i]
        X[i] = x
    return X, x


def records(N, P, k, lam, nu):
    """Per (mode, parity): the two operators, the influence solutions and the inverse 2 x 2 matrix."""
    H, K = tri_factor(N, P, lam, nu), tri_factor(N, P, -k * k, -1.0)
    m = (N - P) // 2
    h = np.zeros(N + 1)
    h[P:N - 1:2] = 1.0
    if P == 0:
        h[0] = 0.5
    w_psi, _ = sweep(N, P, H, lambda n: 0.0, 1.0)
    w_h, _ = sweep(N, P, H, lambda n: h[n] if n <= N - 2 else 0.0, 0.0)

    def on_rows(x):
        f = np.zeros(N + 1, complex)
        f[P::2][:m + 1] = x
        return f
    fp, fh = on_rows(w_psi), on_rows(w_h)
    v_psi, _ = sweep(N, P, K, lambda n: fp[n] if n <= N - 2 else 0.0, 0.0)
    v_h, _ = sweep(N, P, K, lambda n: fh[n] if n <= N - 2 else 0.0, 0.0)
    ns = np.arange(P, N + 1, 2, dtype=float)[:m + 1]
    E = np.array([[w_psi[m] + k * k * v_psi[m], w_h[m] + k * k * v_h[m]],
                  [np.sum(ns ** 2 * v_psi), np.sum(ns ** 2 * v_h)]]).real
    return dict(H=H, K=K, v_psi=v_psi.real, v_h=v_h.real, Ei=np.linalg.inv(E))


def item(N, P, kx, kz, rec, f, du):
    """Outputs {(component, row): G} of the item (mode, parity P)."""
    Q = 1 - P
    k2 = kx * kx + kz * kz
    ik = 1.0 / math.sqrt(k2)
    cx, cz = kx * ik, kz * ik
    rP, rQ, m = rec[P], rec[Q], (N - P) // 2

    def fval(c, n):
        return f[c][n] if 0 <= n <= N - 2 else 0.0
    # (1) w_A: right-hand side -k^2 g, g_n = f_v,n - (2 / (c_n k)) S_n, S_n the suffix sum over the
    # rows m' > n of parity Q of m' (-i f_a,m'), built while the sweep descends
    state = {"S": 0j, "next": 2 * m + P - 1}

    def gneg(n):
        if n > N - 2:
            return 0.0
        while state["next"] > n:
            na = state["next"]
            if na <= N - 2:
                fa = fval(0, na) * cx + fval(2, na) * cz
                state["S"] += na * (-1j * fa)
            state["next"] -= 2
        return -k2 * (fval(1, n) - (1.0 if n == 0 else 2.0) * ik * state["S"])
    S1, w_top = sweep(N, P, rP["H"], gneg, 0.0)
    # (2) v_A from w_A; (3) the influence correction
    S2, v_top = sweep(N, P, rP["K"], lambda n: S1[(n - P) // 2] if n <= N - 2 else 0.0, 0.0)
    e1 = w_top + k2 * v_top
    e2 = sum((2 * i + P) ** 2 * S2[i] for i in range(m + 1))
    Ei = rP["Ei"]
    sig, tau = -(Ei[0, 0] * e1 + Ei[0, 1] * e2), -(Ei[1, 0] * e1 + Ei[1, 1] * e2)
    # (4) v and G_v; a = (i/k) D v on the rows of parity Q by a suffix sum
    out, Sa, a = {}, 0j, {}
    for i in range(m, -1, -1):
        n = 2 * i + P
        v = S2[i] + sig * rP["v_psi"][i] + tau * rP["v_h"][i]
        out[(1, n)] = v - du[1][n]
        Sa += n * v
        if n >= 1:
            a[n - 1] = 1j * (1.0 if n - 1 == 0 else 2.0) * ik * Sa
    # (5) b of parity Q, then u = cx a - cz b, w = cz a + cx b
    B, _ = sweep(N, Q, rQ["H"], lambda n: -cz * fval(0, n) + cx * fval(2, n), 0.0)
    for i in range((N - Q) // 2 + 1):
        n = 2 * i + Q
        an = a.get(n, 0.0)
        out[(0, n)] = cx * an - cz * B[i] - du[0][n]
        out[(2, n)] = cz * an + cx * B[i] - du[2][n]
    return out


def mean_item(N, P, lam, nu, f, du):
    H = tri_factor(N, P, lam, nu)
    X0, _ = sweep(N, P, H, lambda n: f[0][n] if n <= N - 2 else 0.0, 0.0)
    X2, _ = sweep(N, P, H, lambda n: f[2][n] if n <= N - 2 else 0.0, 0.0)
    out = {}
    for i in range((N - P) // 2 + 1):
        n = 2 * i + P
        out[(0, n)], out[(1, n)], out[(2, n)] = X0[i] - du[0][n], -du[1][n], X2[i] - du[2][n]
    return out


def gather(N, items):
    got = np.full((3, N + 1), np.nan, complex)
    for outs in items:
        for (c, n), v in outs.items():
            assert np.isnan(got[c, n]), f"row {n} of component {c} written twice"
            got[c, n] = v
    assert not np.any(np.isnan(got)), "a row was not written"
    return got


CASES = [(16, 400.0, 100.0, 1.14, 2.5), (32, 400.0, 100.0, 5.7, 0.0), (64, 1000.0, 100.0, 0.57, 1.25),
         (64, 400.0, 1e-3, 0.0, 2.5), (96, 400.0, 100.0, 17.1, 37.5), (128, 1000.0, 1e12, 2.28, 5.0),
         (256, 400.0, 100.0, 1.14, 10.0)]


@pytest.mark.parametrize("N,re,dt,kx,kz", CASES)
def test_chain_solve_equals_dense_tau_solve(N, re, dt, kx, kz):
    rng = np.random.default_rng(N + int(kx * 100))
    g = Couette(8, N + 1, 8, re=re, dt=dt)
    nu, k = 1.0 / re, math.hypot(kx, kz)
    lam = 1.0 / dt + nu * k * k
    rec = [records(N, P, k, lam, nu) for P in (0, 1)]
    f = rng.standard_normal((3, N + 1)) + 1j * rng.standard_normal((3, N + 1))
    f[:, N - 1:] = 0.0
    du = rng.standard_normal((3, N + 1)) + 1j * rng.standard_normal((3, N + 1))
    n1 = N + 1
    rhs = np.zeros(4 * n1, complex)
    for c in range(3):
        rhs[c * (N - 1):(c + 1) * (N - 1)] = f[c, :N - 1]
    x = np.linalg.solve(g.assemble_mode(kx, kz, lam), rhs)
    ref = np.stack([x[:n1], x[n1:2 * n1], x[2 * n1:3 * n1]]) - du
    got = gather(N, [item(N, P, kx, kz, rec, f, du) for P in (0, 1)])
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("N,dt", [(16, 100.0), (64, 1e-3), (96, 1e12)])
def test_chain_mean_mode_equals_dense_dirichlet_solve(N, dt):
    rng = np.random.default_rng(7 + N)
    re = 400.0
    g = Couette(8, N + 1, 8, re=re, dt=dt)
    nu, lam = 1.0 / re, 1.0 / dt
    f = rng.standard_normal((3, N + 1)) + 1j * rng.standard_normal((3, N + 1))
    f[:, N - 1:] = 0.0
    du = rng.standard_normal((3, N + 1)) + 1j * rng.standard_normal((3, N + 1))
    n1 = N + 1
    A = np.zeros((n1, n1))
    A[:N - 1] = (lam * np.eye(n1) - nu * g.D2)[:N - 1]
    A[N - 1] = 1.0                                # u(+1) = 0
    A[N] = (-1.0) ** np.arange(n1)                # u(-1) = 0
    ref = np.zeros((3, n1), complex)
    for c in (0, 2):
        ref[c] = np.linalg.solve(A, np.concatenate([f[c, :N - 1], [0.0, 0.0]]))
    ref -= du
    got = gather(N, [mean_item(N, P, lam, nu, f, du) for P in (0, 1)])
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))
