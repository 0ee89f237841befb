"""Pins of the multi-step operator G^int = (B_dt)^n - I (Eq. Gint) in the oracle.

Each pin comes from outside the composition itself: a closed form of the
discrete dynamics, the first-order convergence of n BEFE steps to the flow map
at fixed T = n dt, and central differences of G^int for its tangent.
"""
import math

import numpy as np
import numpy.polynomial.chebyshev as C

import seeded_inputs as si
from oracle.couette import Couette
from oracle.gint import jvp_n, step_n


def mean_flow_mode(orc, eps):
    """eps cos(pi y / 2) e_x in the (0, 0) mode: a streamwise mean-flow perturbation."""
    u = orc.zeros()
    coef = C.chebinterpolate(lambda y: np.cos(np.pi * y / 2), orc.ny - 1)
    u[0, 0, 0, :] = eps * coef
    return u


def test_mean_flow_decays_in_closed_form():
    # For u = (u00(y), 0, 0) the product U_tot x Omega_tot = (0, (y + u00)(1 + u00'), 0) is the
    # gradient of (y + u00)^2 / 2: the pressure absorbs it, so each BEFE step only diffuses,
    # (1 - dt nu D^2) u_new = u, and cos(pi y / 2) decays by 1 / (1 + dt nu pi^2 / 4) per step.
    orc = Couette(8, 33, 8, re=400.0, dt=0.05)
    u = mean_flow_mode(orc, 0.3)
    for n in (1, 4, 13):
        g = step_n(orc, u, n)
        fac = (1.0 + orc.dt * orc.nu * math.pi ** 2 / 4) ** (-n) - 1.0
        assert np.max(np.abs(g - fac * u)) < 1e-12 * np.max(np.abs(u))


def test_first_order_in_dt_at_fixed_T():
    # B^(T/dt) approximates the flow map with error O(dt): halving dt halves the error,
    # so successive differences shrink by a factor close to 2 (Richardson)
    T = 0.4
    gs = []
    for dt in (0.1, 0.05, 0.025):
        orc = Couette(8, 17, 8, re=300.0, dt=dt)
        u = orc.seed_state(*si.couette_random_coeffs(11, 8, 17, 8), 0.2)
        gs.append(step_n(orc, u, int(round(T / dt))))
    d1 = np.max(np.abs(gs[0] - gs[1]))
    d2 = np.max(np.abs(gs[1] - gs[2]))
    assert 1.7 < d1 / d2 < 2.3


def test_tangent_matches_central_differences():
    orc = Couette(8, 17, 8, re=400.0, dt=0.05)
    u = orc.seed_state(*si.couette_random_coeffs(12, 8, 17, 8), 0.2)
    du = orc.seed_state(*si.couette_random_coeffs(13, 8, 17, 8), 1.0)
    n = 6
    J = jvp_n(orc, u, n, du)
    h = 1e-4
    fd = (step_n(orc, u + h * du, n) - step_n(orc, u - h * du, n)) / (2 * h)
    # G^int is a polynomial of high degree in u: the central difference is exact to O(h^2)
    assert np.max(np.abs(J - fd)) < 1e-7 * np.max(np.abs(J))


def test_single_step_and_laminar():
    orc = Couette(8, 17, 8, re=400.0, dt=0.05)
    u = orc.seed_state(*si.couette_random_coeffs(14, 8, 17, 8), 0.1)
    assert np.max(np.abs(step_n(orc, u, 1) - orc.step(u))) == 0.0
    assert np.max(np.abs(step_n(orc, orc.zeros(), 7))) < 1e-14


def test_befe_loop_unstable_at_large_kx():
    """One BEFE step treats the advection explicitly (forward Euler), so at laminar flow a mode
    with streamwise wavenumber kx near walls moving at |U| = 1 is amplified by up to
    sqrt(1 + (dt kx)^2) / (1 + dt nu k^2) per step. At dt = 1/32 and kx = 15 x 1.14 that
    exceeds one: B_dt^n grows with n and G^int_T = B^n - I becomes ill conditioned for
    T >= 1. At dt = 1/256 the same mode decays. (Power iteration on B_U = G_U + I restricted
    to the ix = Kx modes, which B_U leaves invariant at laminar flow.)"""
    rad = {}
    for dt in (1 / 32, 1 / 256):
        o = Couette(48, 17, 4, re=380.0, dt=dt)
        base = o.base(o.zeros())
        rng = np.random.default_rng(0)
        d = o.zeros()
        d[:, o.Kx, 0, :] = rng.standard_normal((3, o.NY)) + 1j * rng.standard_normal((3, o.NY))
        d = o.befe(o.sym(d)) - o.befe(o.zeros())
        lam = 0.0
        for _ in range(80):
            d = d / o.norm(d)
            e = o.jvp(base, d) + d
            lam = o.norm(e)
            d = e
        rad[dt] = lam
        kx = o.kx[o.Kx]
        bound = math.sqrt(1 + (dt * kx) ** 2)
        assert lam < bound
    assert rad[1 / 32] > 1.02
    assert rad[1 / 256] < 1.0
