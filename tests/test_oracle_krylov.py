"""Pins of the oracle's short-recurrence Krylov solvers (Sec. 3.6: BiCGSTAB(l), IDR(s)).

Each solver is checked against something other than itself:
  * numpy.linalg.solve on dense nonsymmetric systems, and on the dense Jacobian
    of the oracle's tangent step restricted to the Hermitian (physical) subspace;
  * BiCGSTAB(1) against van der Vorst's classical BiCGSTAB (a different
    recurrence with the same iterates in exact arithmetic);
  * IDR(1) without the angle safeguard against the same BiCGSTAB: with the
    shadow vector as P, its residuals after every dimension-reduction step are
    BiCGSTAB's (Sonneveld and van Gijzen's equivalence);
  * IDR(s)'s finite termination: at most N + N/s actions on an N x N system.
A dropped term, a wrong sign or a transposed coefficient in either recurrence
breaks one of these.
"""
import math

import numpy as np
import pytest

import seeded_inputs as si
from oracle.couette import Couette
from oracle.newton import bicgstab_ell, idr_s


def euclid(a, b):
    return float(np.dot(a, b))


def dense_system(n, seed, shift=3.0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) / math.sqrt(n) + shift * np.eye(n)
    b = rng.standard_normal(n)
    return A, b


def shadow_space(n, s, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, s)))
    return [Q[:, i].copy() for i in range(s)]


def classical_bicgstab(A, b, r_shadow, cycles):
    """van der Vorst (1992), written independently: residual norm after every cycle."""
    x = np.zeros_like(b)
    r = b.copy()
    p = np.zeros_like(b)
    v = np.zeros_like(b)
    rho, alpha, omega = 1.0, 1.0, 1.0
    hist = [np.linalg.norm(r)]
    for _ in range(cycles):
        rho_new = r_shadow @ r
        beta = (rho_new / rho) * (alpha / omega)
        rho = rho_new
        p = r + beta * (p - omega * v)
        v = A @ p
        alpha = rho / (r_shadow @ v)
        s = r - alpha * v
        t = A @ s
        omega = (t @ s) / (t @ t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        hist.append(np.linalg.norm(r))
    return x, hist


@pytest.mark.parametrize("ell", [1, 2, 4])
def test_bicgstab_ell_solves_dense_system(ell):
    A, b = dense_system(40, 11)
    x, hist, acts = bicgstab_ell(lambda v: A @ v, b, euclid, ell, 400, 1e-12)
    ref = np.linalg.solve(A, b)
    assert np.max(np.abs(x - ref)) < 1e-9 * np.max(np.abs(ref))
    # the recursively updated residual is the true one (no term dropped from x)
    assert abs(np.linalg.norm(b - A @ x) - hist[-1]) < 1e-9 * np.linalg.norm(b)
    assert hist[-1] <= 1e-12 * hist[0]


@pytest.mark.parametrize("s", [1, 2, 4, 8])
def test_idr_solves_dense_system(s):
    A, b = dense_system(40, 12)
    P = shadow_space(40, s, 13)
    x, hist, acts = idr_s(lambda v: A @ v, b, euclid, P, 400, 1e-12)
    ref = np.linalg.solve(A, b)
    assert np.max(np.abs(x - ref)) < 1e-9 * np.max(np.abs(ref))
    assert abs(np.linalg.norm(b - A @ x) - hist[-1]) < 1e-9 * np.linalg.norm(b)


def test_bicgstab_one_is_classical_bicgstab():
    A, b = dense_system(30, 21, shift=1.5)
    rt = np.random.default_rng(22).standard_normal(30)
    _, hist, _ = bicgstab_ell(lambda v: A @ v, b, euclid, 1, 24, 0.0, r_shadow=rt)
    _, ref = classical_bicgstab(A, b, rt, 12)
    h = np.array(hist[:13])
    assert np.max(np.abs(h - np.array(ref)) / np.array(ref)) < 1e-8


def test_idr_one_is_bicgstab_at_cycle_ends():
    A, b = dense_system(30, 31, shift=1.5)
    rt = np.random.default_rng(32).standard_normal(30)
    _, hist, _ = idr_s(lambda v: A @ v, b, euclid, [rt], 40, 0.0, kappa=0.0)
    _, ref = classical_bicgstab(A, b, rt, 12)
    # IDR(1) updates r twice per cycle (the direction step, the reduction step):
    # entries 0, 2, 4, ... are BiCGSTAB's residuals
    ends = np.array(hist[0:25:2])
    assert np.max(np.abs(ends - np.array(ref)) / np.array(ref)) < 1e-7


@pytest.mark.parametrize("s", [2, 4, 8])
def test_idr_finite_termination(s):
    """A spread spectrum (eigenvalues 1..100) keeps the residual large until the
    theoretical bound of n + n/s actions, where it collapses."""
    n = 24
    rng = np.random.default_rng(40)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.linspace(1.0, 100.0, n)) @ Q.T + 0.5 * rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    P = shadow_space(n, s, 42)
    _, hist, acts = idr_s(lambda v: A @ v, b, euclid, P, 10 * n, 1e-10)
    assert hist[-1] <= 1e-10 * hist[0]
    assert acts <= n + n // s
    assert hist[len(hist) // 2] > 1e-6 * hist[0]  # not a trivially easy system


def physical_basis(g):
    """Orthonormal basis of the Hermitian subspace of stored states (the range of sym)."""
    shape = g.zeros().shape
    n = 2 * int(np.prod(shape))
    cols = []
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        cols.append(g.sym(e.view(np.complex128).reshape(shape)).view(np.float64).ravel())
    S = np.array(cols).T
    U, sv, _ = np.linalg.svd(S, full_matrices=False)
    return U[:, sv > 1e-8 * sv[0]]


@pytest.fixture(scope="module")
def jacobian_problem():
    g = Couette(8, 9, 8, re=100.0)
    a, b, c = si.couette_random_coeffs(1000, 8, 9, 8)
    u = g.seed_state(a, b, c, 0.1)
    F = g.step(u)
    base = g.base(u)
    shape = F.shape
    Q = physical_basis(g)
    J = lambda v: g.jvp(base, v)
    JQ = np.array([J(Q[:, i].view(np.complex128).reshape(shape)).view(np.float64).ravel()
                   for i in range(Q.shape[1])]).T
    y = np.linalg.solve(Q.T @ JQ, Q.T @ F.view(np.float64).ravel())
    return g, base, F, (Q @ y).view(np.complex128).reshape(shape)


@pytest.mark.parametrize("solver,par", [("bicgstab", 2), ("bicgstab", 4), ("idr", 4), ("idr", 8)])
def test_krylov_on_the_tangent_against_dense_solve(jacobian_problem, solver, par):
    g, base, F, ref = jacobian_problem
    J = lambda v: g.jvp(base, v)
    if solver == "bicgstab":
        x, hist, acts = bicgstab_ell(J, F, g.inner, par, 4000, 1e-11)
    else:
        P = [g.sym(p) for p in si.idr_shadow(par, 8, 9, 8, seed=77)]
        x, hist, acts = idr_s(J, F, g.inner, P, 4000, 1e-11)
    assert hist[-1] <= 1e-11 * hist[0]
    assert g.norm(x - ref) < 1e-8 * g.norm(ref)
