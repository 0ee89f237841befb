"""Parity of the pipe-flow CUDA path (sp_pipe_create contexts) with the pipe oracle.

Tolerance: FP64 rel. 2e-11 (max abs difference over max abs value). The library
solves each mode's Stokes problem by banded LU factors (partial pivoting) of the
Poisson and Helmholtz matrices plus one influence coefficient; the oracle by a dense
complex LU of the whole 4 Nr system. The two agree to 1e-12 .. 5e-12 on these grids
(the worst case, the tangent at Nr = 64, 4.9e-12); 2e-11 leaves a factor 4 for the
rounding order. Mixed precision: 1e-5 per component.
"""
import numpy as np
import pytest
import torch

import seeded_inputs as si
from gpu_util import host, rel
from oracle.pipe import Pipe, seed_state

pytestmark = pytest.mark.gpu

GRIDS = [dict(nr=16, mt=2, kz=2, nt=12, nz=8), dict(nr=24, mt=3, kz=4, nt=12, nz=16),
         dict(nr=32, mt=4, kz=6, nt=18, nz=24), dict(nr=64, mt=12, kz=24, nt=48, nz=96)]


def make(g, prec=0, max_batch=1, re=2500.0, dt=50.0):
    import paper_1804_05087_gb300 as sp
    cfg = sp.PipeConfig(nr=g["nr"], mt=g["mt"], kz=g["kz"], ntheta=g["nt"], nz=g["nz"], re=re, dt=dt,
                        prec=prec, max_batch=max_batch)
    ctx = sp.Context(cfg)
    orc = Pipe(nr=g["nr"], mt=g["mt"], kz=g["kz"], nt=g["nt"], nz=g["nz"], re=re, dt=dt)
    return ctx, orc


def to_dev(ctx, u, c):
    return ctx.pipe_join(torch.from_numpy(np.ascontiguousarray(u)).cuda(), c)


def seeded(ctx, orc, seed=4000):
    streak, pol = si.pipe_random_coeffs(seed, orc.kzmax, orc.mt)
    u, c = seed_state(orc, streak, pol)
    return u, c, streak, pol


@pytest.mark.parametrize("g", GRIDS[:2])
def test_pipe_seed_matches_oracle(g):
    ctx, orc = make(g)
    u, c, streak, pol = seeded(ctx, orc)
    U = ctx.zeros()
    ctx.sp_pipe_seed_state(streak, pol, 0.05, 0.1, 0.5, U)
    gu, gc = ctx.pipe_split(U)
    assert rel(host(gu), u) < 1e-12 and gc == c


@pytest.mark.parametrize("g", GRIDS)
def test_pipe_step_parity(g):
    ctx, orc = make(g)
    u, c, _, _ = seeded(ctx, orc)
    G = ctx.zeros()
    ctx.sp_step(to_dev(ctx, u, c), G)
    gu, gc = ctx.pipe_split(G)
    ref, _ = orc.step((u, c))
    assert rel(host(gu), ref) < 2e-11
    assert gc == 0.0


def test_pipe_laminar_fixed_point():
    ctx, orc = make(GRIDS[1])
    G = ctx.zeros()
    U = ctx.zeros()
    U[-1] = 0.7
    ctx.sp_step(U, G)
    assert float(host(G).__abs__().max()) < 1e-13


@pytest.mark.parametrize("g", GRIDS)
def test_pipe_jvp_parity(g):
    ctx, orc = make(g)
    u, c, _, _ = seeded(ctx, orc)
    ctx.sp_set_base(to_dev(ctx, u, c))
    rng = np.random.default_rng(7)
    du = orc.sym(rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape))
    du[:, :, :, 0] = 0.0
    dc = 0.31
    J = ctx.zeros()
    ctx.sp_jvp(to_dev(ctx, du, dc), J)
    ju, jc = ctx.pipe_split(J)
    ref, ph = orc.jvp(orc.base((u, c)), (du, dc))
    assert rel(host(ju), ref) < 2e-11
    assert abs(jc - ph) < 1e-10 * max(1.0, abs(ph))


@pytest.mark.parametrize("g", [GRIDS[1], GRIDS[3]])
def test_pipe_jvp_mixed(g):
    ctx, orc = make(g, prec=1)
    u, c, _, _ = seeded(ctx, orc)
    ctx.sp_set_base(to_dev(ctx, u, c))
    streak, pol = si.pipe_random_coeffs(4100, orc.kzmax, orc.mt)
    du, _ = seed_state(orc, streak, pol, amp_streak=1.0, frac=1.0)
    J = ctx.zeros()
    ctx.sp_jvp(to_dev(ctx, du, 0.2), J)
    ju, _ = ctx.pipe_split(J)
    ref, _ = orc.jvp(orc.base((u, c)), (du, 0.2))
    got = host(ju)
    for comp in range(3):
        assert rel(got[comp], ref[comp]) < 1e-5


def test_pipe_fd_jvp():
    ctx, orc = make(GRIDS[1])
    u, c, _, _ = seeded(ctx, orc)
    ctx.sp_set_base(to_dev(ctx, u, c))
    streak, pol = si.pipe_random_coeffs(4200, orc.kzmax, orc.mt)
    du, _ = seed_state(orc, streak, pol, amp_streak=1.0, frac=1.0)
    J = ctx.zeros()
    ctx.sp_jvp_fd(to_dev(ctx, du, 0.1), J)
    ju, jc = ctx.pipe_split(J)
    ref, ph = orc.jvp(orc.base((u, c)), (du, 0.1))
    assert rel(host(ju), ref) < 1e-5
    assert abs(jc - ph) < 1e-10 * max(1.0, abs(ph))


def test_pipe_newton_converges():
    g = GRIDS[0]
    ctx, orc = make(g, re=100.0)
    streak, pol = si.pipe_random_coeffs(4000, orc.kzmax, orc.mt)
    U = ctx.zeros()
    ctx.sp_pipe_seed_state(streak, pol, 0.01, 0.1, 0.5, U)
    rep = ctx.sp_newton_gmres(U, max_newton=15, max_krylov=120, tol=1e-10)
    assert rep["converged"], rep
    gu, gc = ctx.pipe_split(U)
    F, _ = orc.step((host(gu), gc))
    assert np.sqrt(orc.inner((F, 0.0), (F, 0.0))) < 1e-9
