"""The multi-step operator G^int = (B_dt)^n - I (Eq. Gint) on the GPU against the
oracle's composition of single steps (FP64 rel. 1e-12; mixed tangent 1e-5)."""
import math

import numpy as np
import pytest
import torch

import seeded_inputs as si
from gpu_util import dev, host, make, rel, seeded
from oracle.gint import jvp_n, step_n
from test_oracle_gint import mean_flow_mode

pytestmark = pytest.mark.gpu


def close(got, ref, x, tol):
    """G = B^n(x) - x cancels to O(n dt |x|) for small dt: the rounding of the O(|x|) terms
    sets the floor, so the scale is max(|G|, |x|) (as for a single step with small dt)."""
    scale = max(np.max(np.abs(ref)), np.max(np.abs(x)))
    return np.max(np.abs(got - ref)) < tol * scale


def test_step_n_parity():
    ctx, orc = make(16, 33, 16, dt=0.05)
    u = seeded(orc, 1000, 0.1)
    G = ctx.zeros()
    ctx.sp_step_n(dev(u), G, 7)
    assert close(host(G), step_n(orc, u, 7), u, 1e-12)


def test_step_n_mean_flow_closed_form():
    ctx, orc = make(8, 33, 8, dt=0.05)
    u = mean_flow_mode(orc, 0.3)
    G = ctx.zeros()
    ctx.sp_step_n(dev(u), G, 13)
    fac = (1.0 + orc.dt * orc.nu * math.pi ** 2 / 4) ** (-13) - 1.0
    assert np.max(np.abs(host(G) - fac * u)) < 1e-12 * np.max(np.abs(u))


@pytest.mark.parametrize("prec", [0, 1])
def test_jvp_n_parity(prec):
    ctx, orc = make(16, 33, 16, prec=prec, max_batch=2, dt=0.05)
    u = seeded(orc, 1001, 0.1)
    ds = np.stack([seeded(orc, 2000 + i, 1.0) for i in range(3)])
    ctx.sp_set_base_n(dev(u), 5)
    J = ctx.zeros(3)
    ctx.sp_jvp_n(dev(ds), J)   # 3 directions in passes of max_batch = 2
    got = host(J)
    tol = 1e-12 if prec == 0 else 1e-5
    for k in range(3):
        assert close(got[k], jvp_n(orc, u, 5, ds[k]), ds[k], tol)


def test_jvp_fd_follows_the_trajectory():
    ctx, orc = make(16, 33, 16, dt=0.05)
    u = seeded(orc, 1002, 0.1)
    d = seeded(orc, 2100, 1.0)
    ctx.sp_set_base_n(dev(u), 4)
    out = ctx.zeros()
    ctx.sp_jvp_fd(dev(d), out)
    assert close(host(out), jvp_n(orc, u, 4, d), d, 1e-5)
    # back to the single step
    ctx.sp_set_base(dev(u))
    ctx.sp_jvp_n(dev(d), out)
    assert close(host(out), orc.jvp(orc.base(u), d), d, 1e-12)


def test_newton_on_gint_converges():
    ctx, orc = make(16, 33, 16, prec=1, dt=0.05)
    U = dev(seeded(orc, 1003, 0.05))
    rep = ctx.sp_newton_gmres(U, max_newton=20, max_krylov=100, tol=1e-10, int_steps=20)
    assert rep["converged"], rep
    assert float(torch.linalg.vector_norm(U)) < 1e-8
    # each residual and each accepted trial costs 20 steps
    assert rep["total_steps"] % 20 == 0
