"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP64 mode rel. 1e-12 (max abs difference over max abs value);
mixed mode 1e-5 for the tangent (float transforms and products, double solve).
"""
import numpy as np
import pytest
import torch

import seeded_inputs as si
from gpu_util import dev, host, make, rel, seeded

pytestmark = pytest.mark.gpu

# (96, 33, 96) keeps its FP64 plane buffers in global memory (too large for shared memory)
GRIDS = [(4, 9, 4), (8, 17, 8), (16, 33, 16), (18, 17, 24), (24, 33, 12), (48, 65, 48), (96, 33, 96)]


@pytest.mark.parametrize("grid", [(8, 17, 8), (16, 33, 16)])
def test_seed_state_matches_oracle(grid):
    ctx, orc = make(*grid)
    a, b, c = si.couette_random_coeffs(1000, *grid)
    ref = orc.seed_state(a, b, c, 0.1)
    U = ctx.zeros()
    ctx.sp_seed_state(dev(a), dev(b), dev(c), 0.1, U)
    assert rel(host(U), ref) < 1e-13


@pytest.mark.parametrize("grid", GRIDS)
def test_step_parity(grid):
    ctx, orc = make(*grid)
    u = seeded(orc, 1000, 0.1)
    G = ctx.zeros()
    ctx.sp_step(dev(u), G)
    ref = orc.step(u)
    assert rel(host(G), ref) < 1e-12


@pytest.mark.parametrize("dt", [1e-3, 1.0, 10.0, 1e6])
def test_step_parity_dt(dt):
    # G = u_new - u cancels to O(dt |u|) for small dt: the rounding of the two
    # O(|u|) terms sets the floor, so the scale is max(|G|, |u|)
    ctx, orc = make(16, 33, 16, dt=dt)
    u = seeded(orc, 1001, 0.1)
    G = ctx.zeros()
    ctx.sp_step(dev(u), G)
    ref = orc.step(u)
    scale = max(np.max(np.abs(ref)), np.max(np.abs(u)))
    assert np.max(np.abs(host(G) - ref)) < 1e-12 * scale


def test_step_non_hermitian_input_projected():
    ctx, orc = make(8, 17, 8)
    u = si.couette_random_full(7, 8, 17, 8) * 0.05   # not Hermitian, not divergence-free
    G = ctx.zeros()
    ctx.sp_step(dev(u), G)
    assert rel(host(G), orc.step(u)) < 1e-12


def test_laminar_fixed_point():
    ctx, orc = make(16, 33, 16)
    U = ctx.zeros()
    G = ctx.zeros()
    ctx.sp_step(U, G)
    assert float(host(G).__abs__().max()) < 1e-13


@pytest.mark.parametrize("grid", GRIDS)
def test_jvp_parity_fp64(grid):
    ctx, orc = make(*grid, max_batch=3)
    u = seeded(orc, 1000, 0.1)
    ctx.sp_set_base(dev(u))
    base = orc.base(u)
    ds = np.stack([si.couette_random_full(20 + i, *grid) for i in range(3)])
    out = ctx.zeros(3)
    ctx.sp_jvp(dev(ds), out)
    got = host(out)
    for i in range(3):
        assert rel(got[i], orc.jvp(base, ds[i])) < 1e-12


# square grids up to 64 take the register-FFT plane kernel, others the Stockham one
@pytest.mark.parametrize("grid", [(16, 33, 16), (24, 33, 24), (32, 33, 32), (48, 65, 48), (64, 65, 64),
                                  (18, 17, 24), (96, 33, 96)])
def test_jvp_parity_mixed(grid):
    ctx, orc = make(*grid, prec=1, max_batch=2)
    u = seeded(orc, 1000, 0.1)
    ctx.sp_set_base(dev(u))
    base = orc.base(u)
    ds = np.stack([orc.seed_state(*si.couette_random_coeffs(30 + i, *grid), 1.0) for i in range(2)])
    out = ctx.zeros(2)
    ctx.sp_jvp(dev(ds), out)
    got = host(out)
    for i in range(2):
        ref = orc.jvp(base, ds[i])
        for c in range(3):  # per velocity component
            assert rel(got[i, c], ref[c]) < 1e-5


def test_jvp_batch_larger_than_pass():
    ctx, orc = make(8, 17, 8, max_batch=2)
    u = seeded(orc, 5, 0.1)
    ctx.sp_set_base(dev(u))
    base = orc.base(u)
    ds = np.stack([si.couette_random_full(40 + i, 8, 17, 8) for i in range(5)])
    out = ctx.zeros(5)
    ctx.sp_jvp(dev(ds), out)
    got = host(out)
    for i in range(5):
        assert rel(got[i], orc.jvp(base, ds[i])) < 1e-12


def test_dense_jacobian_4x9x4():
    """sp_jvp on every basis vector against the oracle's brute-force dense Jacobian."""
    from test_oracle_couette import dense_jacobian_fd, to_real
    ctx, orc = make(4, 9, 4, max_batch=64)
    a, b, c = si.couette_random_coeffs(20, 4, 9, 4, mmax=1)
    u = orc.seed_state(a, b, c, 0.3)
    cols = dense_jacobian_fd(orc, u)
    J = np.stack([to_real(cc) for cc in cols], axis=1)
    n = u.size
    basis = np.zeros((2 * n,) + u.shape, complex)
    for i in range(n):
        basis[i].flat[i] = 1.0
        basis[n + i].flat[i] = 1j
    ctx.sp_set_base(dev(u))
    out = ctx.zeros(2 * n)
    ctx.sp_jvp(dev(basis), out)
    got = host(out)
    Jg = np.stack([to_real(got[i]) for i in range(2 * n)], axis=1)
    assert np.max(np.abs(Jg - J)) < 1e-12 * np.max(np.abs(J))


def test_jvp_fd_matches_oracle():
    ctx, orc = make(16, 33, 16)
    u = seeded(orc, 1000, 0.1)
    d = orc.seed_state(*si.couette_random_coeffs(50, 16, 33, 16), 1.0)
    ctx.sp_set_base(dev(u))
    out = ctx.zeros()
    ctx.sp_jvp_fd(dev(d), out)
    ref = orc.jvp(orc.base(u), d)
    assert rel(host(out), ref) < 1e-6


def test_inner_product():
    ctx, orc = make(8, 17, 8)
    a = si.couette_random_full(1, 8, 17, 8)
    b = si.couette_random_full(2, 8, 17, 8)
    got = ctx.sp_inner(dev(a), dev(b))[0]
    assert abs(got - orc.inner(a, b)) < 1e-12 * abs(orc.inner(a, b))


def test_newton_converges_to_laminar():
    ctx, orc = make(8, 17, 8, re=100.0)
    u = seeded(orc, 1000, 0.05)
    U = dev(u)
    rep = ctx.sp_newton_gmres(U, max_newton=12, max_krylov=60, tol=1e-10)
    assert rep["converged"], rep
    assert rep["norm_F"] < 1e-10
    assert float(np.sqrt(orc.inner(host(U), host(U)))) < 1e-9


def test_newton_with_gradient_direction_converges():
    """Hookstep over the Krylov space augmented with J^* F (the dogleg direction)."""
    ctx, orc = make(8, 17, 8, re=100.0)
    u = seeded(orc, 1000, 0.05)
    U = dev(u)
    rep = ctx.sp_newton_gmres(U, max_newton=12, max_krylov=60, tol=1e-10, use_gradient=True)
    assert rep["converged"], rep
    assert float(np.sqrt(orc.inner(host(U), host(U)))) < 1e-9


def test_newton_mixed_precision_reaches_fp64_tolerance():
    """Inexact (float-transform) tangents inside GMRES, FP64 residual: |G| < 1e-10."""
    ctx, orc = make(16, 33, 16, prec=1)
    u = seeded(orc, 1000, 0.1)
    U = dev(u)
    rep = ctx.sp_newton_gmres(U, max_newton=20, max_krylov=300, tol=1e-10)
    assert rep["converged"], rep
    G = orc.step(host(U))
    assert np.sqrt(orc.inner(G, G)) < 1e-10
