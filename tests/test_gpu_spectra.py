"""Dense Jacobians from batched tangent actions (the spectra of Sec. 3.3), checked
against two exact facts at laminar flow:
  * the physical subspace S = range(G_U + P) (P: the Hermitian projection every map
    applies) has the dimension of divergence-free, no-slip, Hermitian states:
    (4N - 8) real values per solved mode (kx, kz) != (0, 0) and 2(N - 1) for the mean flow;
  * the base is stationary, so the multi-step Jacobian is the n-th power of the
    single-step one: G^int_U + P = (G_U + P)^n on S (Eq. Gint)."""
import numpy as np
import pytest
import torch

import bench

pytestmark = pytest.mark.gpu


def laminar_jacobian(n_steps, dt, nx=8, ny=9, nz=8, re=500.0):
    import paper_1804_05087_gb300 as sp
    ctx = sp.Context(sp.Config(nx, ny, nz, lx=bench.LX, lz=bench.LZ, re=re, dt=dt, prec=sp.SP_FP64,
                               max_batch=256))
    ctx.sp_set_base_n(ctx.zeros(), n_steps)
    J = bench.dense_jacobian(ctx, n_steps)
    P = bench.hermitian_projection(ctx)
    return ctx, J, P


def test_physical_subspace_dimension():
    ctx, J, P = laminar_jacobian(1, 100.0)
    sv = np.linalg.svd(J + P, compute_uv=False)
    d = int(np.sum(sv > 1e-10 * sv[0]))
    N = ctx.NY - 1
    modes = (ctx.Kx + 1) * ctx.MZ + ctx.Kx * (ctx.MZ - 1)
    assert d == (modes - 1) * (4 * N - 8) + 2 * (N - 1)
    # outside S the tangent is exactly -(I - P) P = 0 on anti-Hermitian inputs
    anti = np.eye(J.shape[0]) - P
    assert np.max(np.abs(J @ anti)) < 1e-14


def test_multistep_jacobian_is_a_power_at_a_stationary_base():
    n, dt = 6, 0.05
    _, J1, P = laminar_jacobian(1, dt)
    _, Jn, _ = laminar_jacobian(n, dt)
    B = J1 + P
    assert np.max(np.abs((Jn + P) - np.linalg.matrix_power(B, n))) < 1e-12 * np.max(np.abs(Jn + P))
