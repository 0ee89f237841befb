"""Pins of the Couette oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
library routines (numpy.polynomial.chebyshev, numpy.fft), analytic Stokes
eigenvalues, brute-force pointwise evaluation on tiny grids, exact algebraic
identities of the BEFE step (Eq. mycalc) and of a quadratic map.
"""
import math

import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest
from scipy.linalg import eig
from scipy.optimize import brentq

import seeded_inputs as si
from oracle.couette import Couette


def rand_state(g, seed):
    return g.sym(si.couette_random_full(seed, g.nx, g.ny, g.nz))


# ------------------------------------------------------------------ transforms
def test_chebyshev_values_closed_form():
    g = Couette(4, 17, 4)
    N = g.N
    for n in range(N + 1):
        e = np.zeros(N + 1)
        e[n] = 1.0
        vals = g.cheb_values(e)
        ref = np.array([math.cos(n * math.pi * j / N) for j in range(N + 1)])
        assert np.max(np.abs(vals - ref)) < 1e-14


def test_chebyshev_against_numpy():
    g = Couette(4, 17, 4)
    rng = np.random.default_rng(0)
    a = rng.standard_normal(g.NY)
    assert np.allclose(g.cheb_values(a), npc.chebval(g.y, a), atol=1e-13, rtol=0)
    assert np.allclose(g.cheb_coeffs(g.cheb_values(a)), a, atol=1e-13, rtol=0)
    # interpolation through the Gauss-Lobatto points is the forward transform
    f = np.exp(g.y) * np.sin(3 * g.y)
    assert np.allclose(g.cheb_coeffs(f), npc.chebfit(g.y, f, g.N), atol=1e-12, rtol=0)
    # coefficient-space derivative
    d = np.zeros(g.NY)
    d[:g.N] = npc.chebder(a)
    assert np.allclose(g.D @ a, d, atol=1e-11, rtol=0)


def test_fourier_single_mode_and_numpy():
    g = Couette(12, 9, 12)
    c = np.zeros((g.MX, g.MZ, g.NY), complex)
    p = 2  # ix = 2
    c[p, 1, 3] = 0.3 - 0.7j
    phys = g.to_physical(c)
    x = np.arange(g.nx) * g.lx / g.nx
    z = np.arange(g.nz) * g.lz / g.nz
    th = g.kx[p] * x[:, None] + g.kz[1] * z[None, :]
    ref = 2 * ((0.3 - 0.7j) * np.exp(1j * th)).real
    assert np.max(np.abs(phys[3] - ref)) < 1e-14
    assert np.max(np.abs(np.delete(phys, 3, axis=0))) == 0.0
    # forward transform matches numpy's FFT on retained modes
    rng = np.random.default_rng(1)
    f = rng.standard_normal((g.NY, g.nx, g.nz))
    ff = np.fft.fft2(f, axes=(1, 2)) / (g.nx * g.nz)
    spec = g.to_spectral(f)
    for pos in range(g.MX):
        for iz in range(g.MZ):
            assert abs(spec[pos, iz, 0] - ff[0, g.ixs[pos] % g.nx, iz]) < 1e-14
    # round trip on a Hermitian state of retained modes
    s = g.sym(si.couette_random_full(2, g.nx, g.ny, g.nz))[0]
    assert np.max(np.abs(g.to_spectral(g.to_physical(s)) - s)) < 1e-13


# -------------------------------------------------------- Stokes eigenvalues
def _analytic_q(k, qmax):
    """Wall-normal wavenumbers q of Stokes modes: mu = -nu (k^2 + q^2)."""
    qs = []
    n = 1
    while n * math.pi / 2 < qmax:
        qs.append(n * math.pi / 2)  # modes of the wall-parallel vorticity
        n += 1
    fe = lambda q: q * math.tan(q) + k * math.tanh(k)        # even v-modes
    fo = lambda q: q / math.tan(q) - k / math.tanh(k)        # odd v-modes
    for m in range(0, int(qmax / math.pi) + 2):
        lo, hi = m * math.pi + 1e-9, (m + 1) * math.pi - 1e-9
        for f, brk in ((fe, m * math.pi + math.pi / 2), (fo, m * math.pi)):
            # scan the branch between poles for sign changes
            grid = np.linspace(lo, hi, 2001)
            vals = [f(q) for q in grid]
            for i in range(len(grid) - 1):
                if np.isfinite(vals[i]) and np.isfinite(vals[i + 1]) and vals[i] * vals[i + 1] < 0 \
                        and abs(vals[i]) < 1e3 and abs(vals[i + 1]) < 1e3:
                    r = brentq(f, grid[i], grid[i + 1], xtol=1e-15)
                    if r < qmax:
                        qs.append(r)
    return np.sort(np.array(qs))


@pytest.mark.parametrize("kx,kz", [(1.14, 2.5), (0.0, 2.5), (2.28, 0.0)])
def test_stokes_eigenvalues_analytic(kx, kz):
    """Generalised eigenvalues of the tau pencil = analytic Stokes eigenvalues."""
    g = Couette(4, 33, 4, re=400.0)
    A0 = g.assemble_mode(kx, kz, 0.0)
    B = g.assemble_mode(kx, kz, 1.0) - A0
    s = eig(A0, B, right=False)
    s = s[np.isfinite(s)]
    # A(lam) = A0 + lam B is singular at lam* = -s and lam* = -nu q^2
    q2 = np.sort((s / g.nu).real)
    assert np.max(np.abs((s / g.nu).imag)) < 1e-6 * np.max(np.abs(q2))
    k = math.hypot(kx, kz)
    qa = _analytic_q(k, 12.0)
    got = np.sqrt(q2[:len(qa)])
    assert np.max(np.abs(got - qa) / qa) < 1e-10, (got, qa)


def test_solve_on_stokes_eigenmode():
    """S(u/dt) = u/(1 - dt mu) on an eigenmode: G = dt mu/(1 - dt mu) u (N = 0)."""
    g = Couette(4, 33, 4, re=400.0, dt=100.0)
    p, iz = 1, 1
    kx, kz = g.kx[p], g.kz[iz]
    A0 = g.assemble_mode(kx, kz, 0.0)
    B = g.assemble_mode(kx, kz, 1.0) - A0
    s, vecs = eig(A0, B)
    ok = np.isfinite(s)
    s, vecs = s[ok], vecs[:, ok]
    i = np.argmin(s.real)
    n1 = g.NY
    mode = vecs[:, i]
    mu = -s[i].real - g.nu * (kx * kx + kz * kz)
    f = g.zeros()
    for comp in range(3):
        f[comp, p, iz] = mode[comp * n1:(comp + 1) * n1] / g.dt
    out = g.solve(f)
    expect = f * g.dt / (1.0 - g.dt * mu)
    assert np.max(np.abs(out - expect)) < 1e-10 * np.max(np.abs(expect))


# ---------------------------------------------------------- step properties
@pytest.mark.parametrize("dt", [1e-4, 1.0, 100.0, 1e12])
def test_laminar_is_fixed_point(dt):
    g = Couette(8, 17, 8, dt=dt)
    assert np.max(np.abs(g.step(g.zeros()))) < 1e-13


def test_step_divergence_free_and_no_slip():
    g = Couette(8, 17, 8)
    u = rand_state(g, 3)
    un = g.befe(u)
    scale = np.max(np.abs(un))
    assert np.max(np.abs(g.divergence(un))) < 1e-13 * scale * 40
    for wv in g.wall_values(un):
        assert np.max(np.abs(wv)) < 1e-13 * scale * 10


def test_nonlinear_term_brute_force():
    """N(u) against pointwise series evaluation on a tiny grid (library routines)."""
    g = Couette(8, 9, 8)
    c = rand_state(g, 4)
    N = g.N
    xs = np.arange(g.nx) * g.lx / g.nx
    zs = np.arange(g.nz) * g.lz / g.nz
    nl = np.zeros((3, g.NY, g.nx, g.nz))
    for j, yv in enumerate(g.y):
        for i, xv in enumerate(xs):
            for k, zv in enumerate(zs):
                vel = np.zeros(3, complex)
                grad = np.zeros((3, 3), complex)  # grad[comp, direction]
                for pos in range(g.MX):
                    for iz in range(g.MZ):
                        wgt = 1.0 if iz == 0 else 2.0
                        e = wgt * np.exp(1j * (g.kx[pos] * xv + g.kz[iz] * zv))
                        for comp in range(3):
                            a = c[comp, pos, iz]
                            val = npc.chebval(yv, a)
                            dy = npc.chebval(yv, npc.chebder(a))
                            vel[comp] += e * val
                            grad[comp, 0] += e * 1j * g.kx[pos] * val
                            grad[comp, 1] += e * dy
                            grad[comp, 2] += e * 1j * g.kz[iz] * val
                vel, grad = vel.real, grad.real
                om = np.array([grad[2, 1] - grad[1, 2], grad[0, 2] - grad[2, 0],
                               grad[1, 0] - grad[0, 1]])
                U = vel + np.array([yv, 0.0, 0.0])
                O = om + np.array([0.0, 0.0, -1.0])
                nl[:, j, i, k] = np.cross(U, O)
    ff = np.fft.fft2(nl, axes=(2, 3)) / (g.nx * g.nz)
    ref = np.zeros_like(c)
    for comp in range(3):
        for pos in range(g.MX):
            for iz in range(g.MZ):
                col = ff[comp, :, g.ixs[pos] % g.nx, iz]
                ref[comp, pos, iz] = npc.chebfit(g.y, col.real, N) + 1j * npc.chebfit(g.y, col.imag, N)
    got = g.nonlinear(c)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_befe_identity_mycalc():
    """B - I = (I - dt L)^-1 dt (L + N) for an admissible state (Eq. mycalc)."""
    for dt in (1e-4, 1.0, 100.0, 1e12):
        g = Couette(8, 17, 8, dt=dt)
        a, b, cm = si.couette_random_coeffs(10, 8, 17, 8)
        u = g.seed_state(a, b, cm, 0.1)
        lhs = g.step(u)
        # S = dt (I - dt L)^-1 solves (1/dt - nu lap) x + grad p = f
        rhs = g.sym(g.solve(g.laplacian_part(u) + g.nonlinear(u)))
        assert np.max(np.abs(lhs - rhs)) < 1e-11 * max(1.0, np.max(np.abs(lhs)))


def test_small_and_large_dt_limits():
    """G ~ dt (L+N) for small dt; G -> -L^-1 (L+N) for large dt (Eqs. smalldt, largedt)."""
    a, b, cm = si.couette_random_coeffs(11, 8, 17, 8)
    g1 = Couette(8, 17, 8, dt=1e-7)
    u = g1.seed_state(a, b, cm, 0.1)
    G1 = g1.step(u)
    g2 = Couette(8, 17, 8, dt=2e-7)
    G2 = g2.step(u)
    assert np.max(np.abs(G2 - 2 * G1)) < 1e-5 * np.max(np.abs(G2))
    gl = Couette(8, 17, 8, dt=1e8)
    gh = Couette(8, 17, 8, dt=1e12)
    Gl, Gh = gl.step(u), gh.step(u)
    assert np.max(np.abs(Gl - Gh)) < 1e-6 * np.max(np.abs(Gh))


def test_translation_equivariance():
    """Shifting the flow in x and z commutes with the step."""
    g = Couette(8, 17, 8)
    a, b, cm = si.couette_random_coeffs(12, 8, 17, 8)
    u = g.seed_state(a, b, cm, 0.1)
    sx, sz = 3 * g.lx / g.nx, 5 * g.lz / g.nz
    ph = np.exp(1j * (g.kx[:, None, None] * sx + g.kz[None, :, None] * sz))
    assert np.max(np.abs(g.step(u * ph) - g.step(u) * ph)) < 1e-12


def test_seed_state_admissible():
    g = Couette(16, 33, 16)
    a, b, cm = si.couette_random_coeffs(1000, 16, 33, 16)
    u = g.seed_state(a, b, cm, 0.1)
    assert abs(g.norm(u) - 0.1) < 1e-15
    scale = np.max(np.sum(np.abs(u), axis=-1))  # l1 norm of a Chebyshev series
    assert np.max(np.abs(g.divergence(u))) < 1e-13 * scale * g.N
    for wv in g.wall_values(u):
        assert np.max(np.abs(wv)) < 1e-12 * scale  # Dv amplifies rounding by ~N^2
    assert np.max(np.abs(g.sym(u) - u)) == 0.0


# ------------------------------------------------------- tangent and adjoint
def dense_jacobian_fd(g, u, h=0.5):
    """Columns of G_U from central differences of G; exact since G is quadratic."""
    shape = u.shape
    n = u.size
    cols = []
    for comp in (1.0, 1j):
        for i in range(n):
            e = np.zeros(n, complex)
            e[i] = comp
            e = e.reshape(shape)
            cols.append((g.step(u + h * e) - g.step(u - h * e)) / (2 * h))
    return cols


def to_real(a):
    return np.concatenate([a.real.ravel(), a.imag.ravel()])


def test_dense_jacobian_4x9x4():
    """sp_jvp's oracle against the brute-force dense Jacobian (n_real = 324)."""
    g = Couette(4, 9, 4)
    a, b, cm = si.couette_random_coeffs(20, 4, 9, 4, mmax=1)
    u = g.seed_state(a, b, cm, 0.3)
    cols = dense_jacobian_fd(g, u)
    J = np.stack([to_real(cc) for cc in cols], axis=1)
    assert J.shape == (324, 324)
    base = g.base(u)
    rng = np.random.default_rng(5)
    for _ in range(4):
        d = rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape)
        got = to_real(g.jvp(base, d))
        ref = J @ to_real(d)
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    # adjoint in the weighted inner product: J^* = W^-1 J^T W
    w = np.broadcast_to(g.wz[None, None, :, None], u.shape).astype(float)
    wr = np.concatenate([w.ravel(), w.ravel()])
    Jstar = (J.T * wr[None, :]) / wr[:, None]
    for _ in range(4):
        r = rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape)
        got = to_real(g.vjp(base, r))
        ref = Jstar @ to_real(r)
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_jvp_central_difference_exact():
    """G is quadratic, so a central difference is exact for any step h."""
    g = Couette(8, 17, 8)
    u = rand_state(g, 30) * 0.2
    d = rand_state(g, 31)
    base = g.base(u)
    j = g.jvp(base, d)
    for h in (1e-2, 1.0):
        fd = (g.step(u + h * d) - g.step(u - h * d)) / (2 * h)
        assert np.max(np.abs(fd - j)) < 1e-11 * np.max(np.abs(j))


def test_vjp_dot_product():
    g = Couette(8, 17, 8)
    u = rand_state(g, 40) * 0.2
    base = g.base(u)
    for s in range(3):
        d = si.couette_random_full(41 + s, 8, 17, 8)
        r = si.couette_random_full(51 + s, 8, 17, 8)
        lhs = g.inner(g.jvp(base, d), r)
        rhs = g.inner(d, g.vjp(base, r))
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_fd_jvp_matches_tangent():
    g = Couette(8, 17, 8)
    a, b, cm = si.couette_random_coeffs(60, 8, 17, 8)
    u = g.seed_state(a, b, cm, 0.1)
    d = g.seed_state(*si.couette_random_coeffs(61, 8, 17, 8), 1.0)
    j = g.jvp(g.base(u), d)
    fd = g.jvp_fd(u, d)
    assert np.max(np.abs(fd - j)) < 1e-5 * np.max(np.abs(j))
