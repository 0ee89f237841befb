"""Pins of the oracle's Newton-GMRES-hookstep (Sec. 2, Eqs. linear, biglin, Kspace).

The root it must find is known in closed form: laminar Couette flow, u = 0,
is a fixed point of the BEFE step for every dt (Eq. mycalc), and near a small
perturbed-laminar guess it is the only root.
"""
import numpy as np

import seeded_inputs as si
from oracle.couette import Couette
from oracle.newton import gmres, newton_hookstep


def test_gmres_arnoldi_orthonormal_and_monotone():
    g = Couette(8, 17, 8, re=100.0)
    a, b, c = si.couette_random_coeffs(1000, 8, 17, 8)
    u = g.seed_state(a, b, c, 0.05)
    F = g.step(u)
    base = g.base(u)
    V, H, beta, res = gmres(lambda d: g.jvp(base, d), F, g.inner, 25, 0.0)
    k = H.shape[1]
    gram = np.array([[g.inner(V[i], V[j]) for j in range(k)] for i in range(k)])
    assert np.max(np.abs(gram - np.eye(k))) < 1e-12
    assert all(res[i + 1] <= res[i] * (1 + 1e-12) for i in range(len(res) - 1))
    # the Arnoldi relation J V_k = V_{k+1} H_k
    for j in range(k):
        lhs = g.jvp(base, V[j])
        rhs = sum(H[i, j] * V[i] for i in range(min(k + 1, len(V))))
        assert np.max(np.abs(lhs - rhs)) < 1e-11 * max(1.0, np.max(np.abs(lhs)))


def test_newton_converges_to_laminar():
    g = Couette(8, 17, 8, re=100.0)
    a, b, c = si.couette_random_coeffs(1000, 8, 17, 8)
    u = g.seed_state(a, b, c, 0.05)
    U, hist = newton_hookstep(g.step, lambda U: (lambda d, B=g.base(U): g.jvp(B, d)),
                              g.inner, u, tol=1e-10, max_newton=12, max_k=60)
    assert hist[-1]["norm_F"] < 1e-10
    assert g.norm(U) < 1e-9
    # quadratic convergence at the end
    nf = [h["norm_F"] for h in hist]
    assert nf[-1] < 1e-2 * nf[-2]
