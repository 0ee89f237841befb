"""Newton-GMRES with a hookstep trust region, written plainly (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2 (Eqs. linear, biglin): solve G_U du = G(U) and update U <- U - du.
The linear system is solved matrix-free by GMRES without restarts (Sec. 2,
Eq. Kspace; Sec. 3.2): the Krylov basis is orthonormalised by modified
Gram-Schmidt in the problem's own inner product, every basis vector is kept
(K(K-1)/2 inner products, Eq. CPU). Iterations stop when the least-squares
residual falls below eta*|G(U)| (the relaxed tolerance of Sec. 3.6) or at the
Krylov cap.

The step is constrained by a hookstep (Sec. 3.2): with the Arnoldi relation
G_U V_k = V_{k+1} H_k and du = V_k y, minimise |beta e1 - H_k y| subject to
|y| <= Delta, using the SVD H_k = P diag(s) Q^T: y = Q z with
z_i = s_i p_i / (s_i^2 + mu), p = P^T beta e1, and mu >= 0 chosen so |z| = Delta
when the plain least-squares step is longer than Delta. Delta follows the
usual ratio test between the actual and the predicted decrease of |G|^2
(the paper gives no constants; the ones below are this library's reading).
"""
from __future__ import annotations

import math

import numpy as np


def _hook(s, p, delta):
    """z minimising |p - diag(s) z| subject to |z| <= delta."""
    z = p / s
    if np.linalg.norm(z) <= delta:
        return z
    lo, hi = 0.0, float(np.max(s * np.abs(p)) / delta + np.max(s) ** 2)
    for _ in range(200):
        mu = 0.5 * (lo + hi)
        z = s * p / (s * s + mu)
        if np.linalg.norm(z) > delta:
            lo = mu
        else:
            hi = mu
    return s * p / (s * s + hi)


def gmres(apply_j, rhs, inner, max_k, eta):
    """Unrestarted GMRES (modified Gram-Schmidt). Returns (V, H, beta, residuals)."""
    beta = math.sqrt(inner(rhs, rhs))
    V = [rhs / beta]
    H = np.zeros((max_k + 1, max_k))
    res = [beta]
    k = 0
    for j in range(max_k):
        w = apply_j(V[j])
        for i in range(j + 1):
            h = inner(V[i], w)
            H[i, j] = h
            w = w - h * V[i]
        hn = math.sqrt(max(inner(w, w), 0.0))
        H[j + 1, j] = hn
        k = j + 1
        e1 = np.zeros(k + 1)
        e1[0] = beta
        y, *_ = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)
        r = float(np.linalg.norm(e1 - H[:k + 1, :k] @ y))
        res.append(r)
        if hn == 0.0:
            break
        V.append(w / hn)
        if r <= eta * beta:
            break
    return V, H[:k + 1, :k], beta, res


def newton_hookstep(G, make_jvp, inner, U0, tol=1e-10, max_newton=20, max_k=30,
                    eta=1e-3, delta0=None, max_hook=12, log=None):
    """Find a root of G from U0. ``make_jvp(U)`` returns du -> G_U du.

    Returns (U, history) where history is a list of dicts per Newton step.
    """
    U = U0
    F = G(U)
    nF = math.sqrt(inner(F, F))
    delta = delta0 if delta0 is not None else 0.1 * max(math.sqrt(inner(U, U)), 1.0)
    history = [{"newton": 0, "norm_F": nF, "krylov": 0, "delta": delta}]
    for it in range(1, max_newton + 1):
        if nF < tol:
            break
        jv = make_jvp(U)
        V, H, beta, res = gmres(jv, F, inner, max_k, eta)
        k = H.shape[1]
        P, s, Qt = np.linalg.svd(H, full_matrices=False)
        p = P.T @ np.concatenate([[beta], np.zeros(k)])
        accepted = False
        for _ in range(max_hook):
            z = _hook(s, p, delta)
            y = Qt.T @ z
            du = sum(y[i] * V[i] for i in range(k))
            U_try = U - du
            F_try = G(U_try)
            n_try = math.sqrt(inner(F_try, F_try))
            e1 = np.zeros(k + 1)
            e1[0] = beta
            pred = float(np.linalg.norm(e1 - H @ y))
            denom = nF * nF - pred * pred
            rho = (nF * nF - n_try * n_try) / denom if denom > 0 else -1.0
            ylen = float(np.linalg.norm(y))
            if rho < 0.01 or not np.isfinite(n_try):
                delta = 0.5 * ylen
                continue
            if rho > 0.75 and ylen >= 0.99 * delta:
                delta = 2.0 * delta
            elif rho < 0.25:
                delta = 0.5 * delta
            accepted = True
            break
        if not accepted:
            # take the shortest step tried: the trust region has collapsed
            history.append({"newton": it, "norm_F": nF, "krylov": k, "delta": delta,
                            "rejected": True, "gmres_res": res})
            break
        U, F, nF = U_try, F_try, n_try
        rec = {"newton": it, "norm_F": nF, "krylov": k, "delta": delta, "gmres_res": res}
        history.append(rec)
        if log is not None:
            log(rec)
    return U, history


# --------------------------------------------------------------------------
# Short-recurrence Krylov solvers (Sec. 3.6 names BiCGSTAB(l) and IDR as the
# remedy for GMRES's K^2 orthogonalisation cost). Both solve A x = b from
# x = 0 with the problem's inner product and stop when |r| <= eta |b| or after
# max_act actions of A. They return (x, hist, acts): hist lists |r| at the
# points the algorithms update r (BiCGSTAB(l): once per outer cycle, after the
# minimal-residual part; IDR(s): after every residual update), starting with
# |b|.

def bicgstab_ell(apply_a, b, inner, ell, max_act, eta, r_shadow=None):
    """BiCGSTAB(l) of Sleijpen and Fokkema (1993), in the paper's order:
    l BiCG steps extend the bases r_0..r_l and u_0..u_l, then a minimal-residual
    polynomial of degree l (modified Gram-Schmidt on r_1..r_l) updates x, r_0, u_0."""
    nb = math.sqrt(inner(b, b))
    x = np.zeros_like(b)
    r = [b.copy()] + [np.zeros_like(b) for _ in range(ell)]
    u = [np.zeros_like(b) for _ in range(ell + 1)]
    rt = b.copy() if r_shadow is None else r_shadow
    rho0, alpha, omega = 1.0, 0.0, 1.0
    hist, acts = [nb], 0
    rn = nb
    while acts < max_act and rn > eta * nb:
        rho0 = -omega * rho0
        # BiCG part
        for j in range(ell):
            rho1 = inner(r[j], rt)
            beta = alpha * rho1 / rho0
            rho0 = rho1
            for i in range(j + 1):
                u[i] = r[i] - beta * u[i]
            u[j + 1] = apply_a(u[j])
            gamma = inner(u[j + 1], rt)
            alpha = rho0 / gamma
            for i in range(j + 1):
                r[i] = r[i] - alpha * u[i + 1]
            r[j + 1] = apply_a(r[j])
            x = x + alpha * u[0]
            acts += 2
        # minimal-residual part
        tau = np.zeros((ell + 1, ell + 1))
        sigma = np.zeros(ell + 1)
        gp = np.zeros(ell + 1)
        for j in range(1, ell + 1):
            for i in range(1, j):
                tau[i, j] = inner(r[j], r[i]) / sigma[i]
                r[j] = r[j] - tau[i, j] * r[i]
            sigma[j] = inner(r[j], r[j])
            gp[j] = inner(r[0], r[j]) / sigma[j]
        g = np.zeros(ell + 1)
        g[ell] = gp[ell]
        omega = g[ell]
        for j in range(ell - 1, 0, -1):
            g[j] = gp[j] - sum(tau[j, i] * g[i] for i in range(j + 1, ell + 1))
        gpp = np.zeros(ell + 1)
        for j in range(1, ell):
            gpp[j] = g[j + 1] + sum(tau[j, i] * g[i + 1] for i in range(j + 1, ell))
        x = x + g[1] * r[0]
        r[0] = r[0] - gp[ell] * r[ell]
        u[0] = u[0] - g[ell] * u[ell]
        for j in range(1, ell):
            u[0] = u[0] - g[j] * u[j]
            x = x + gpp[j] * r[j]
            r[0] = r[0] - gp[j] * r[j]
        rn = math.sqrt(inner(r[0], r[0]))
        hist.append(rn)
        if not np.isfinite(rn):
            break
    return x, hist, acts


def idr_s(apply_a, b, inner, P, max_act, eta, kappa=0.7):
    """IDR(s) with biorthogonalised bases (van Gijzen and Sonneveld, 2011), in their
    order: per cycle s directions u_k (g_k = A u_k) made biorthogonal to the shadow
    vectors P, each followed by a residual update; then the dimension-reduction
    step with the minimal-residual omega, raised to kappa |r|/|t| relative size when
    the angle between t = A r and r is small ("maintaining the convergence";
    kappa = 0 turns that off)."""
    s = len(P)
    nb = math.sqrt(inner(b, b))
    x = np.zeros_like(b)
    r = b.copy()
    g = [np.zeros_like(b) for _ in range(s)]
    u = [np.zeros_like(b) for _ in range(s)]
    M = np.eye(s)
    omega = 1.0
    hist, acts = [nb], 0
    rn = nb
    while acts < max_act and rn > eta * nb:
        f = np.array([inner(P[i], r) for i in range(s)])
        for k in range(s):
            c = np.zeros(s)
            for i in range(k, s):  # M[k:, k:] c = f[k:], lower triangular
                c[i] = (f[i] - sum(M[i, j] * c[j] for j in range(k, i))) / M[i, i]
            v = r - sum(c[i] * g[i] for i in range(k, s))
            u[k] = omega * v + sum(c[i] * u[i] for i in range(k, s))
            g[k] = apply_a(u[k])
            acts += 1
            for i in range(k):
                a = inner(P[i], g[k]) / M[i, i]
                g[k] = g[k] - a * g[i]
                u[k] = u[k] - a * u[i]
            for i in range(k, s):
                M[i, k] = inner(P[i], g[k])
            beta = f[k] / M[k, k]
            r = r - beta * g[k]
            x = x + beta * u[k]
            rn = math.sqrt(inner(r, r))
            hist.append(rn)
            if rn <= eta * nb or acts >= max_act:
                break
            for i in range(k + 1, s):
                f[i] = f[i] - beta * M[i, k]
        if rn <= eta * nb or acts >= max_act:
            break
        t = apply_a(r)
        acts += 1
        tt, tr = inner(t, t), inner(t, r)
        omega = tr / tt
        rho = abs(tr) / (math.sqrt(tt) * rn)
        if rho < kappa:
            omega = omega * kappa / rho
        x = x + omega * r
        r = r - omega * t
        rn = math.sqrt(inner(r, r))
        hist.append(rn)
    return x, hist, acts
