"""Pins of the pipe oracle (oracle/pipe.py) against closed forms and exact identities.

Finite differences on the clustered radial grid are exact for polynomials of degree
<= 8 (9-point stencils) with the right parity; Bessel zeros give the Helmholtz
eigenvalues; Hagen-Poiseuille flow is a fixed point for every dt and speed c; the
step is bilinear in (u, c) plus quadratic in u, so central differences are exact.
"""
import math

import numpy as np
import pytest
from scipy.special import jn_zeros

import seeded_inputs as si
from oracle.newton import newton_hookstep
from oracle.pipe import Pipe, fd_weights, poloidal_fields, seed_state


def small():
    return Pipe(nr=32, mt=4, kz=4, nt=15, nz=16, re=2500.0, dt=50.0)


def test_fd_weights_exact_on_polynomials():
    x = np.array([0.0, 0.1, 0.25, 0.3, 0.5, 0.55, 0.7, 0.9, 1.0])
    for order in (1, 2):
        w = fd_weights(0.33, x, order)
        for deg in range(9):
            exact = math.factorial(deg) / math.factorial(deg - order) * 0.33 ** (deg - order) if deg >= order else 0.0
            assert abs(np.dot(w, x ** deg) - exact) < 1e-9 * max(1.0, abs(exact))


@pytest.mark.parametrize("par", [0, 1])
def test_radial_derivatives_with_parity(par):
    P = small()
    r = P.r
    a = 2 + par  # r^a (1 - r^2): parity (-1)^a, degree a + 2 <= 8
    f = r ** a * (1 - r ** 2)
    d1 = a * r ** (a - 1) - (a + 2) * r ** (a + 1)
    d2 = a * (a - 1) * r ** (a - 2) - (a + 2) * (a + 1) * r ** a
    D1, D2 = P.D[par]
    assert np.max(np.abs(D1 @ f - d1)) < 1e-9
    assert np.max(np.abs(D2 @ f - d2)) < 1e-7


@pytest.mark.parametrize("c", [0.0, 0.7])
def test_hagen_poiseuille_is_fixed_point(c):
    P = small()
    u, _ = P.zeros()
    G, gc = P.step((u, c))
    assert np.max(np.abs(G)) < 1e-13 and gc == 0.0


@pytest.mark.parametrize("q,par", [(0, 0), (1, 1), (2, 0)])
def test_helmholtz_eigenvalues_bessel(q, par):
    """Eigenvalues of D2 + D1/r - q^2/r^2 with u(1) = 0 tend to -j_{q,n}^2."""
    P = Pipe(nr=64, mt=2, kz=2, nt=9, nz=8)
    L = P.lap(q, par, 0.0)
    ev = np.sort(np.linalg.eigvals(L[1:, 1:]).real)[::-1]
    ref = jn_zeros(q, 4) ** 2
    got = -ev[:4]
    assert np.max(np.abs(got - ref) / ref) < 1e-6, (got, ref)


def test_curl_of_polynomial_field_exact():
    """omega from the oracle's curl against the analytic curl (exact: degree <= 8)."""
    P = small()
    r = P.r
    p, q = 1, 1  # kz = 1, m' = 1
    m, k = P.m[q], P.k[p]
    u = np.zeros((3, P.MK, P.MT, P.nr), complex)
    ur = (1 - r ** 2) * r ** (m - 1)
    ut = 0.3j * (1 - r ** 2) * r ** (m + 1)
    uz = r ** m * (1 - r ** 2) ** 2
    u[0, p, q], u[1, p, q], u[2, p, q] = ur, ut, uz
    f = P.fields(u)
    # analytic omega of the single mode (m, k)
    dz = m * r ** (m - 1) * (1 - r ** 2) ** 2 - 4 * r ** (m + 1) * (1 - r ** 2)
    dt = 0.3j * ((m + 1) * r ** m - (m + 3) * r ** (m + 2))
    om = np.zeros((6, P.MK, P.MT, P.nr), complex)
    om[0, p, q], om[1, p, q], om[2, p, q] = ur, ut, uz
    om[3, p, q] = 1j * m / r * uz - 1j * k * ut
    om[4, p, q] = 1j * k * ur - dz
    om[5, p, q] = dt + ut / r - 1j * m / r * ur
    ref = P.to_physical(om)
    assert np.max(np.abs(f - ref)) < 1e-9 * np.max(np.abs(ref))


def test_solve_divergence_smooth_and_wall_exact():
    P = Pipe(nr=64, mt=3, kz=3, nt=12, nz=12)
    r = P.r
    f = np.zeros((3, P.MK, P.MT, P.nr), complex)
    for (p, q) in [(1, 1), (2, 0), (0, 2)]:
        ur, ut, uz = poloidal_fields(r, int(P.m[q]), P.k[p], np.array([1.0, 0.5]))
        f[0, p, q], f[1, p, q], f[2, p, q] = ur + 0.3 * r ** (P.m[q] + 1), ut, uz
    f = P.sym(f)
    u = P.solve(f)
    div = P.divergence(u)
    scale = np.max(np.abs(u))
    assert np.max(np.abs(div[:, :, 0])) < 1e-11 * scale * P.nr ** 2  # continuity row at the wall
    assert np.max(np.abs(div)) < 1e-5 * scale * P.nr ** 2             # FD consistency inside
    assert np.max(np.abs(u[:, :, :, 0])) < 1e-14 * scale              # no-slip


def test_jvp_central_difference_exact_and_phase():
    P = small()
    st, pol = si.pipe_random_coeffs(4000, P.kzmax, P.mt)
    u, c = seed_state(P, st, pol)
    base = P.base((u, c))
    rng = np.random.default_rng(3)
    du = P.sym(rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape))
    dc = 0.37
    J, ph = P.jvp(base, (du, dc))
    h = 0.5
    Gp, _ = P.step((u + h * du, c + h * dc))
    Gm, _ = P.step((u - h * du, c - h * dc))
    assert np.max(np.abs(J - (Gp - Gm) / (2 * h))) < 1e-11 * np.max(np.abs(J))
    dzu = 1j * P.k[None, :, None, None] * u
    assert abs(ph - P.inner((dzu, 0.0), (P.sym(du), 0.0))) < 1e-12 * max(1.0, abs(ph))


def test_translation_equivariance():
    P = small()
    st, pol = si.pipe_random_coeffs(4001, P.kzmax, P.mt)
    u, c = seed_state(P, st, pol)
    sz, st_ = 3 * (2 * np.pi / P.alpha) / P.nz, 2 * (2 * np.pi / P.ms) / P.nt
    ph = np.exp(1j * (P.k[:, None, None] * sz + P.m[None, :, None] * st_))
    G1, _ = P.step((u * ph, c))
    G0, _ = P.step((u, c))
    assert np.max(np.abs(G1 - G0 * ph)) < 1e-12


def test_newton_reaches_a_root():
    """Traveling-wave Newton (speed as unknown, phase condition) from the seeded guess."""
    # Re = 100: GMRES converges in ~50 actions here (the count grows with Re, Sec. 3.3)
    P = Pipe(nr=16, mt=2, kz=2, nt=9, nz=8, re=100.0, dt=50.0)
    st, pol = si.pipe_random_coeffs(4000, P.kzmax, P.mt)
    state = seed_state(P, st, pol, amp_streak=0.01)

    def G(s):
        return P.step(s)

    def make_jvp(s):
        b = P.base(s)
        return lambda d: P.jvp(b, d)

    U, hist = newton_hookstep_tuple(G, make_jvp, P.inner, state)
    assert hist[-1] < 1e-10


def newton_hookstep_tuple(G, make_jvp, inner, U0):
    """Plain Newton-GMRES (no trust region) on (field, speed) tuples; returns |G| history."""
    from oracle.newton import gmres
    U = U0
    hist = []

    class T(tuple):
        def __add__(self, o):
            return T((self[0] + o[0], self[1] + o[1]))

        def __sub__(self, o):
            return T((self[0] - o[0], self[1] - o[1]))

        def __mul__(self, s):
            return T((self[0] * s, self[1] * s))

        __rmul__ = __mul__

        def __truediv__(self, s):
            return T((self[0] / s, self[1] / s))

    U = T(U)
    for _ in range(12):
        F = T(G(U))
        nF = math.sqrt(inner(F, F))
        hist.append(nF)
        if nF < 1e-10:
            break
        jv = make_jvp(U)
        V, H, beta, res = gmres(lambda d: T(jv(d)), F, inner, 80, 1e-10)
        k = H.shape[1]
        e1 = np.zeros(k + 1)
        e1[0] = beta
        y, *_ = np.linalg.lstsq(H, e1, rcond=None)
        du = sum((V[i] * float(y[i]) for i in range(k)), T((0 * U[0], 0.0)))
        U = U - du
    return U, hist


def test_laminar_total_fields_closed_form():
    """U_tot = (1 - r^2) e_z and Omega_tot = curl U_tot = 2 r e_theta for u = 0."""
    P = small()
    u, _ = P.zeros()
    f = P.total_fields(u)
    r = P.r[:, None, None]
    assert np.max(np.abs(f[2] - (1 - r ** 2))) < 1e-15
    assert np.max(np.abs(f[4] - 2 * r)) < 1e-15
    for i in (0, 1, 3, 5):
        assert np.max(np.abs(f[i])) == 0.0


def test_nonlinear_term_of_streak_brute_force():
    """N(u) for an axial streak u_z = a(r) cos(m theta) against U_tot x Omega_tot on the grid."""
    P = small()
    r = P.r
    q = 1
    m = P.m[q]
    a = 0.2 * (1 - r ** 2) * r ** m
    u = np.zeros((3, P.MK, P.MT, P.nr), complex)
    u[2, 0, q] = a
    th = np.arange(P.nt) * (2 * np.pi / P.ms) / P.nt
    da = 0.2 * (m * r ** (m - 1) - (m + 2) * r ** (m + 1))
    # physical fields: u_z = 2 a cos(m th); omega_r = (1/r) d_th u_z; omega_theta = -d_r u_z
    uz = 2 * a[:, None] * np.cos(m * th)[None, :]
    om_r = -2 * m * a[:, None] / r[:, None] * np.sin(m * th)[None, :]
    om_t = -2 * da[:, None] * np.cos(m * th)[None, :]
    Uz = uz + (1 - r ** 2)[:, None]
    Ot = om_t + 2 * r[:, None]
    # U_tot = (0, 0, Uz), Omega_tot = (om_r, Ot, 0): U x Omega = (-Uz Ot, Uz om_r, 0)
    ref = np.zeros((3, P.nr, P.nz, P.nt))
    ref[0] = (-Uz * Ot)[:, None, :]
    ref[1] = (Uz * om_r)[:, None, :]
    n = P.nonlinear(u)
    expect = P.to_spectral(ref)
    assert np.max(np.abs(n - expect)) < 1e-10 * np.max(np.abs(expect))


@pytest.mark.parametrize("q,p", [(1, 0), (0, 1), (1, 3), (6, 10), (12, 24)])
def test_continuity_at_every_point_reading_is_numerically_singular(q, p):
    """The per-mode system's reading (Sec. 3.2, 3.4): the pressure Poisson equation at the interior
    points plus continuity at the wall. The other natural reading, continuity at every radial
    point, leaves a system whose smallest singular value is 1e-13 to 4e-12 of the largest at
    Nr = 64, against 6e-10 to 2e-8 for the Poisson reading: the first is not usable."""
    P = Pipe(nr=64)
    m, k = P.m[q], P.k[p]
    A = P.assemble_mode(m, k, 1.0 / P.dt)
    B = A.copy()
    B[3 * P.nr:, :] = 0.0
    B[3 * P.nr:, :3 * P.nr] = P.div_rows(m, k)
    sa = np.linalg.svd(A, compute_uv=False)
    sb = np.linalg.svd(B, compute_uv=False)
    assert sb[-1] / sb[0] < 1e-11
    assert sa[-1] / sa[0] > 1e-10
