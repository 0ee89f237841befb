"""Writes eq_12x25x12_re500.npz: a nontrivial plane Couette equilibrium, computed by the
FP64 oracle alone (this script imports nothing but oracle/ and seeded_inputs).

Recipe: box 2pi/1.14 x 2 x 2pi/2.5 (Sec. 3.3), grid 12 x 25 x 12. Newton-GMRES-hookstep
(oracle/newton.py) on the step with laminar advection folded into L (Sec. 3.6; same fixed
points as the Stokes step) from the seeded perturbed-laminar guess seed 7113, modes
|ix|, |iz| <= 1, amplitude 0.3, at Re 400; then continued to Re 450 and Re 500. The file
also holds the leading eigenvalues of L + N_U at Re 500, from the oracle's dense Jacobian
of G^Stokes_T with T = 1e-4 rescaled by (1 + T)/T (Eq. beaumescale), restricted to the
physical subspace.

Run from the repository root:  python tests/golden/make_equilibrium.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import seeded_inputs as si  # noqa: E402
from oracle.couette import Couette  # noqa: E402
from oracle.newton import newton_hookstep  # noqa: E402

GRID = (12, 25, 12)
SEED, AMP, MMAX = 7113, 0.3, 1
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "eq_12x25x12_re500.npz")


def newton(re, U):
    o = Couette(*GRID, re=re, lam_adv=True)
    jv = lambda V: (lambda d, b=o.base(V): o.jvp(b, d))
    U, hist = newton_hookstep(o.step, jv, o.inner, U, tol=1e-12, max_newton=60, max_k=150)
    return U, hist[-1]["norm_F"]


def real_matrix(o, fn):
    shape = o.zeros().shape
    n = int(np.prod(shape))
    cols = []
    for k in range(2 * n):
        e = np.zeros(2 * n)
        e[k] = 1.0
        j = fn((e[:n] + 1j * e[n:]).reshape(shape)).reshape(-1)
        cols.append(np.concatenate([j.real, j.imag]))
    return np.array(cols).T


def main():
    o = Couette(*GRID, re=400.0)
    a, b, c = si.couette_random_coeffs(SEED, *GRID, mmax=MMAX)
    U = o.seed_state(a, b, c, AMP)
    for re in (400.0, 450.0, 500.0):
        U, nF = newton(re, U)
        print(f"Re {re:g}: |G| = {nF:.2e}, |U| = {o.norm(U):.6f}")
    T = 1e-4
    g = Couette(*GRID, re=500.0, dt=T)
    base = g.base(U)
    J = real_matrix(g, lambda d: g.jvp(base, d))
    P = real_matrix(g, g.sym)
    ev = np.linalg.eigvals(J + P)
    ev = ev[np.abs(ev) > 1e-9] - 1.0  # the complement of the physical subspace has eigenvalue -1 + 1 = 0
    ev = ev * (1 + T) / T
    lead = ev[np.argsort(-ev.real)[:6]]
    print("leading eigenvalues of L + N_U:", lead)
    np.savez(OUT, U=U, re=500.0, grid=np.array(GRID), seed=SEED, amp=AMP, mmax=MMAX, leading=lead)


if __name__ == "__main__":
    main()
