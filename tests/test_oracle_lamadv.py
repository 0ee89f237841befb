"""Pins of the oracle's laminar-advection variant (Sec. 3.6, closing proposal).

With laminar advection in L the step solves
    (1/dt - nu lap + M) u_new + grad p = u/dt + N(u) + M u,  M u = y du/dx + v e_x.
The pins below check it against things the oracle does not compute itself:
  * numpy's Chebyshev multiplication by x (the matrix Y);
  * a manufactured polynomial solution, built with numpy.polynomial, which the
    per-mode tau system must reproduce exactly (so every term of the modified
    momentum rows, their signs and the v coupling are fixed);
  * consistency: the two splittings approximate the same ODE, so the steps
    differ by O(dt^2) as dt -> 0 (a wrong M on either side leaves O(dt));
  * at laminar flow the linearised nonlinear part of N + M is a gradient, so
    G'_U -> -I as dt -> infinity, unlike the Stokes step's G_U;
  * plane Couette flow is linearly stable (Romanov 1973): at laminar flow every
    eigenvalue of G'_U + I lies inside the unit disc.
"""
import math

import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest

import seeded_inputs as si
from oracle.couette import Couette


def test_y_matrix_against_numpy():
    g = Couette(4, 17, 4, lam_adv=True)
    rng = np.random.default_rng(1)
    for _ in range(5):
        a = rng.standard_normal(g.NY)
        ref = npc.chebmulx(a)[:g.NY]
        assert np.max(np.abs(g.Y @ a - ref)) < 1e-14


def _pad(c, n):
    out = np.zeros(n, complex)
    m = min(n, len(c))
    out[:m] = c[:m]
    return out


def manufactured(g, seed):
    """Divergence-free, no-slip polynomial velocity and a pressure per mode, and the
    right-hand side f that the modified Stokes rows give for them (numpy.polynomial)."""
    rng = np.random.default_rng(seed)
    N, n1 = g.N, g.NY
    bump = np.array([0.5, 0.0, -0.5])            # 1 - y^2 in Chebyshev coefficients
    bump2 = npc.chebmul(bump, bump)
    dt, nu = g.dt, g.nu
    c = g.zeros()
    f = g.zeros()
    cplx = lambda n: rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for p in range(g.MX):
        for iz in range(g.MZ):
            kx, kz = g.kx[p], g.kz[iz]
            k2 = kx * kx + kz * kz
            lam = 1.0 / dt + nu * k2
            if p == 0 and iz == 0:
                u = _pad(npc.chebmul(bump, rng.standard_normal(N - 1)), n1)
                w = _pad(npc.chebmul(bump, rng.standard_normal(N - 1)), n1)
                v = np.zeros(n1, complex)
                pr = np.zeros(n1, complex)
            else:
                v = _pad(npc.chebmul(bump2, cplx(N - 3)), n1)
                eta = _pad(npc.chebmul(bump, cplx(N - 1)), n1)
                dv = _pad(npc.chebder(v), n1)
                u = 1j * (kx * dv - kz * eta) / k2
                w = 1j * (kz * dv + kx * eta) / k2
                pr = cplx(n1)
            vel = [u, v, w]
            grad = [1j * kx * pr, _pad(npc.chebder(pr), n1), 1j * kz * pr]
            for comp in range(3):
                q = vel[comp]
                rhs = lam * q - nu * _pad(npc.chebder(q, 2), n1) + grad[comp]
                if g.lam_adv:
                    rhs = rhs + 1j * kx * _pad(npc.chebmulx(q), n1)
                    if comp == 0:
                        rhs = rhs + v
                c[comp, p, iz] = q
                f[comp, p, iz] = rhs
    return c, f


@pytest.mark.parametrize("lam_adv", [False, True])
@pytest.mark.parametrize("dt", [100.0, 0.5])
def test_manufactured_solution_is_reproduced(lam_adv, dt):
    g = Couette(12, 17, 12, re=400.0, dt=dt, lam_adv=lam_adv)
    c, f = manufactured(g, 7)
    got = g.solve(f)
    assert np.max(np.abs(got - c)) < 1e-10 * np.max(np.abs(c))
    if lam_adv:
        # the same right-hand side through the Stokes rows does not give c back
        plain = Couette(12, 17, 12, re=400.0, dt=dt)
        assert np.max(np.abs(plain.solve(f) - c)) > 1e-3 * np.max(np.abs(c))


def seeded(g, seed, amp, mmax=2):
    a, b, cm = si.couette_random_coeffs(seed, g.nx, g.ny, g.nz, mmax=mmax)
    return g.seed_state(a, b, cm, amp)


def test_laminar_is_a_fixed_point():
    g = Couette(12, 17, 12, lam_adv=True)
    # N(0) = y e_y is a gradient: the pressure takes it up to rounding
    assert np.max(np.abs(g.step(g.zeros()))) < 1e-13


def test_same_ode_as_dt_vanishes():
    """B'_dt(u) - B_dt(u) = O(dt^2): both are first-order steps of du/dt = Lu + N(u)."""
    diffs = []
    for dt in (1e-3, 1e-4):
        a = Couette(8, 17, 8, re=400.0, dt=dt, lam_adv=True)
        b = Couette(8, 17, 8, re=400.0, dt=dt)
        u = seeded(a, 11, 0.3)
        diffs.append(a.norm(a.befe(u) - b.befe(u)))
    ratio = diffs[0] / diffs[1]
    assert 70.0 < ratio < 130.0, ratio


def test_jvp_matches_finite_differences():
    g = Couette(8, 17, 8, re=400.0, dt=100.0, lam_adv=True)
    u = seeded(g, 21, 0.2)
    d = seeded(g, 22, 1.0)
    j = g.jvp(g.base(u), d)
    # G is quadratic in u, so central differences are exact up to rounding
    h = 1e-3
    jc = (g.step(u + h * d) - g.step(u - h * d)) / (2 * h)
    assert g.norm(j - jc) < 1e-9 * g.norm(j)


def _low_degree(g, seed, deg):
    """A seeded direction whose Chebyshev degrees stay below N - 1 after y * u."""
    a, b, cm = si.couette_random_coeffs(seed, g.nx, g.ny, g.nz)
    for arr in (a, b, cm):
        arr[..., deg:] = 0.0
    return g.seed_state(a, b, cm, 1.0)


def test_jacobian_at_laminar_tends_to_minus_identity():
    res = {}
    for lam_adv in (False, True):
        r = []
        for dt in (1e4, 1e5):
            g = Couette(8, 17, 8, re=400.0, dt=dt, lam_adv=lam_adv)
            d = _low_degree(g, 31, 6)
            j = g.jvp(g.base(g.zeros()), d)
            r.append(g.norm(j + d))
        res[lam_adv] = r
    # laminar advection in L: G'_U + I = (I - dt L')^-1 = O(1/dt)
    assert 9.5 < res[True][0] / res[True][1] < 10.5
    assert res[True][0] < 0.05
    # Stokes step: G_U + I -> -L^-1 N_U, of order one
    assert 0.9 < res[False][0] / res[False][1] < 1.1
    assert res[False][1] > 0.1


def dense_matrix(g, fn):
    """Real matrix of a real-linear map of states on the stored real coordinates."""
    shape = g.zeros().shape
    n = int(np.prod(shape))
    cols = []
    for k in range(2 * n):
        e = np.zeros(2 * n)
        e[k] = 1.0
        d = (e[:n] + 1j * e[n:]).reshape(shape)
        j = fn(d).reshape(-1)
        cols.append(np.concatenate([j.real, j.imag]))
    return np.array(cols).T


def test_laminar_spectrum_inside_unit_disc():
    g = Couette(6, 13, 6, re=1000.0, dt=10.0, lam_adv=True)
    base = g.base(g.zeros())
    J = dense_matrix(g, lambda d: g.jvp(base, d))
    P = dense_matrix(g, g.sym)
    # J + P maps every state into the physical (divergence-free, no-slip, Hermitian)
    # subspace and acts there as (I - dt L')^-1: zero eigenvalues off it
    ev = np.linalg.eigvals(J + P)
    assert np.max(np.abs(ev)) < 1.0
    # the i kx y term makes the spectrum complex for kx != 0
    assert np.max(np.abs(ev.imag)) > 1e-3
