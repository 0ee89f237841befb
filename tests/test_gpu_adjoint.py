"""The hand-written adjoint step (sp_vjp, sp_vjp_euclid, StokesStep.backward).

Checks: the dot-product identity <J d, r> = <d, J* r> in the weighted inner
product, parity with the oracle's adjoint (FP64 rel. 1e-12, mixed 1e-5 per
component), the brute-force dense transpose on 4x9x4, and torch.autograd.
"""
import numpy as np
import pytest
import torch

import seeded_inputs as si
from gpu_util import dev, host, make, rel, seeded

pytestmark = pytest.mark.gpu


def weights(orc):
    return np.broadcast_to(orc.wz[None, None, :, None], (3, orc.MX, orc.MZ, orc.NY))


@pytest.mark.parametrize("grid", [(8, 17, 8), (16, 33, 16), (18, 17, 24), (48, 65, 48)])
def test_vjp_parity_and_dot_product(grid):
    ctx, orc = make(*grid, max_batch=2)
    u = seeded(orc, 1000, 0.1)
    ctx.sp_set_base(dev(u))
    base = orc.base(u)
    rs = np.stack([si.couette_random_full(60 + i, *grid) for i in range(2)])
    out = ctx.zeros(2)
    ctx.sp_vjp(dev(rs), out)
    got = host(out)
    for i in range(2):
        assert rel(got[i], orc.vjp(base, rs[i])) < 1e-12
    d = si.couette_random_full(70, *grid)
    jd = ctx.zeros()
    ctx.sp_jvp(dev(d), jd)
    lhs = orc.inner(host(jd), rs[0])
    rhs = orc.inner(d, got[0])
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0)


def test_vjp_dense_transpose_4x9x4():
    from test_oracle_couette import dense_jacobian_fd, to_real
    ctx, orc = make(4, 9, 4, max_batch=64)
    a, b, c = si.couette_random_coeffs(20, 4, 9, 4, mmax=1)
    u = orc.seed_state(a, b, c, 0.3)
    J = np.stack([to_real(cc) for cc in dense_jacobian_fd(orc, u)], axis=1)
    w = weights(orc).astype(float)
    wr = np.concatenate([w.ravel(), w.ravel()])
    Jstar = (J.T * wr[None, :]) / wr[:, None]
    n = u.size
    basis = np.zeros((2 * n,) + u.shape, complex)
    for i in range(n):
        basis[i].flat[i] = 1.0
        basis[n + i].flat[i] = 1j
    ctx.sp_set_base(dev(u))
    out = ctx.zeros(2 * n)
    ctx.sp_vjp(dev(basis), out)
    got = host(out)
    Jg = np.stack([to_real(got[i]) for i in range(2 * n)], axis=1)
    assert np.max(np.abs(Jg - Jstar)) < 1e-12 * np.max(np.abs(Jstar))


@pytest.mark.parametrize("grid", [(16, 33, 16), (48, 65, 48), (64, 65, 64), (18, 17, 24)])
def test_vjp_mixed(grid):
    ctx, orc = make(*grid, prec=1)
    u = seeded(orc, 1000, 0.1)
    ctx.sp_set_base(dev(u))
    r = orc.seed_state(*si.couette_random_coeffs(80, *grid), 1.0)
    out = ctx.zeros()
    ctx.sp_vjp(dev(r), out)
    ref = orc.vjp(orc.base(u), r)
    got = host(out)
    for c in range(3):
        assert rel(got[c], ref[c]) < 1e-5


def test_vjp_euclid_is_plain_transpose():
    ctx, orc = make(16, 33, 16)
    u = seeded(orc, 1000, 0.1)
    ctx.sp_set_base(dev(u))
    g = si.couette_random_full(90, 16, 33, 16)
    out = ctx.zeros()
    ctx.sp_vjp_euclid(dev(g), out)
    w = weights(orc)
    ref = w * orc.vjp(orc.base(u), g / w)
    assert rel(host(out), ref) < 1e-12


def test_autograd_function():
    import paper_1804_05087_gb300 as sp
    ctx, orc = make(16, 33, 16)
    u = seeded(orc, 1000, 0.1)
    R = si.couette_random_full(91, 16, 33, 16)
    U = dev(u).requires_grad_(True)
    G = sp.StokesStep.apply(U, ctx)
    assert rel(host(G.detach()), orc.step(u)) < 1e-12
    loss = (G.conj() * dev(R)).real.sum()
    loss.backward()
    # d loss = sum Re(conj(R) dG) = <R, J dU>_euclid  =>  grad = J^T R (Euclidean)
    w = weights(orc)
    ref = w * orc.vjp(orc.base(u), R / w)
    assert rel(host(U.grad), ref) < 1e-12
    # forward mode: the tangent step
    import torch.autograd.forward_ad as fwAD
    d = si.couette_random_full(92, 16, 33, 16)
    with fwAD.dual_level():
        Ud = fwAD.make_dual(dev(u), dev(d))
        Gd = sp.StokesStep.apply(Ud, ctx)
        tangent = fwAD.unpack_dual(Gd).tangent
    assert rel(host(tangent), orc.jvp(orc.base(u), d)) < 1e-12


def test_gradient_of_half_residual_squared_matches_central_fd():
    """J^T F = grad (1/2)|F|^2 (the hookstep/dogleg direction): central FD, h = 1e-7."""
    ctx, orc = make(16, 33, 16)
    u = seeded(orc, 1000, 0.1)
    U = dev(u)
    F = ctx.zeros()
    ctx.sp_step(U, F)
    ctx.sp_set_base(U)
    g = ctx.zeros()
    ctx.sp_vjp(F, g)
    gh = host(g)
    for s in range(4):
        d = orc.seed_state(*si.couette_random_coeffs(5000 + s, 16, 33, 16), 1.0)
        h = 1e-7
        Fp, Fm = ctx.zeros(), ctx.zeros()
        ctx.sp_step(dev(u + h * d), Fp)
        ctx.sp_step(dev(u - h * d), Fm)
        fp, fm = host(Fp), host(Fm)
        fd = (0.5 * orc.inner(fp, fp) - 0.5 * orc.inner(fm, fm)) / (2 * h)
        an = orc.inner(gh, d)
        assert abs(fd - an) < 1e-6 * max(abs(an), 1e-3)
