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
