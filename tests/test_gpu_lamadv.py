"""Laminar advection folded into L (Sec. 3.6, the closing proposal): the CUDA path
against the FP64 oracle's variant of the step.

Tolerances as for the Stokes step: FP64 rel. 1e-12, mixed tangent 1e-5 per
velocity component. The tile shapes of the per-mode solve compute the same
arithmetic per mode, so they agree bit for bit.
"""
import numpy as np
import pytest

import seeded_inputs as si
from gpu_util import dev, host, make, rel, seeded

pytestmark = pytest.mark.gpu

# register-FFT and Stockham plane kernels, ragged boxes, a mode count that leaves a
# partial tile (18 x 17 x 24: 5 x 8 retained modes), and the full 48 x 65 x 48 grid
GRIDS = [(8, 17, 8), (16, 33, 16), (18, 17, 24), (24, 33, 12), (48, 65, 48)]


def la(*grid, **kw):
    return make(*grid, lam_adv=1, **kw)


@pytest.mark.parametrize("grid", GRIDS)
def test_step_parity(grid):
    ctx, orc = la(*grid)
    u = seeded(orc, 1100, 0.1)
    G = ctx.zeros()
    ctx.sp_step(dev(u), G)
    assert rel(host(G), orc.step(u)) < 1e-12


@pytest.mark.parametrize("dt", [1e-3, 1.0, 1e6])
def test_step_parity_dt(dt):
    ctx, orc = la(16, 33, 16, dt=dt)
    u = seeded(orc, 1101, 0.1)
    G = ctx.zeros()
    ctx.sp_step(dev(u), G)
    ref = orc.step(u)
    scale = max(np.max(np.abs(ref)), np.max(np.abs(u)))
    assert np.max(np.abs(host(G) - ref)) < 1e-12 * scale


def test_step_other_box_and_re():
    ctx, orc = la(18, 17, 24, lx=4.0, lz=2.0, re=1000.0)
    u = seeded(orc, 1102, 0.2)
    G = ctx.zeros()
    ctx.sp_step(dev(u), G)
    assert rel(host(G), orc.step(u)) < 1e-12


def test_non_hermitian_input_projected():
    ctx, orc = la(8, 17, 8)
    u = si.couette_random_full(9, 8, 17, 8) * 0.05   # not Hermitian, not divergence-free
    G = ctx.zeros()
    ctx.sp_step(dev(u), G)
    assert rel(host(G), orc.step(u)) < 1e-12


def test_laminar_fixed_point():
    ctx, orc = la(16, 33, 16)
    U = ctx.zeros()
    G = ctx.zeros()
    ctx.sp_step(U, G)
    assert float(np.abs(host(G)).max()) < 1e-13


@pytest.mark.parametrize("grid", [(8, 17, 8), (18, 17, 24), (24, 33, 12)])
def test_jvp_parity_fp64(grid):
    ctx, orc = la(*grid, max_batch=3)
    u = seeded(orc, 1103, 0.1)
    ctx.sp_set_base(dev(u))
    base = orc.base(u)
    ds = np.stack([si.couette_random_full(60 + i, *grid) for i in range(3)])
    out = ctx.zeros(3)
    ctx.sp_jvp(dev(ds), out)
    got = host(out)
    for i in range(3):
        assert rel(got[i], orc.jvp(base, ds[i])) < 1e-12


@pytest.mark.parametrize("grid", [(16, 33, 16), (18, 17, 24), (48, 65, 48)])
def test_jvp_parity_mixed(grid):
    ctx, orc = la(*grid, prec=1, max_batch=2)
    u = seeded(orc, 1104, 0.1)
    ctx.sp_set_base(dev(u))
    base = orc.base(u)
    ds = np.stack([orc.seed_state(*si.couette_random_coeffs(70 + i, *grid), 1.0) for i in range(2)])
    out = ctx.zeros(2)
    ctx.sp_jvp(dev(ds), out)
    got = host(out)
    for i in range(2):
        ref = orc.jvp(base, ds[i])
        for c in range(3):
            assert rel(got[i, c], ref[c]) < 1e-5


def test_full_size_batch_sampled():
    """48 x 65 x 48, 256 directions in one mixed-precision pass (the throughput
    workload with laminar advection in L): sampled directions against the oracle."""
    grid = (48, 65, 48)
    ctx, orc = la(*grid, prec=1, max_batch=256)
    ctx.sp_autotune(256)
    u = seeded(orc, 1105, 0.1)
    ctx.sp_set_base(dev(u))
    base = orc.base(u)
    D = ctx.zeros(256)
    ds = {}
    for i in (0, 101, 255):
        ds[i] = orc.seed_state(*si.couette_random_coeffs(80 + i, *grid), 1.0)
        D[i].copy_(dev(ds[i]))
    out = ctx.zeros(256)
    ctx.sp_jvp(D, out)
    got = host(out)
    for i, d in ds.items():
        ref = orc.jvp(base, d)
        for c in range(3):
            assert rel(got[i, c], ref[c]) < 1e-5
    # zero directions give zero
    assert np.max(np.abs(got[1])) == 0.0


def test_jvp_fd_matches_oracle():
    ctx, orc = la(16, 33, 16)
    u = seeded(orc, 1106, 0.1)
    d = orc.seed_state(*si.couette_random_coeffs(90, 16, 33, 16), 1.0)
    ctx.sp_set_base(dev(u))
    out = ctx.zeros()
    ctx.sp_jvp_fd(dev(d), out)
    assert rel(host(out), orc.jvp(orc.base(u), d)) < 1e-6


@pytest.mark.parametrize("prec", [0, 1])
def test_every_shape_bit_identical(prec):
    grid = (24, 49, 24)
    ctx, orc = la(*grid, prec=prec, max_batch=3)
    u = seeded(orc, 1107, 0.1)
    ds = np.stack([seeded(orc, 2100 + i, 1.0) for i in range(3)])
    U, D = dev(u), dev(ds)
    rep = ctx.sp_autotune(3)
    ref_J = ref_G = None
    for i in range(len(rep["shapes"])):
        if rep["ms_tangent"][i] < 0 or rep["ms_step"][i] < 0:
            continue
        ctx.sp_set_solve_shape(i, i)
        G = ctx.zeros()
        ctx.sp_step(U, G)
        ctx.sp_set_base(U)
        J = ctx.zeros(3)
        ctx.sp_jvp(D, J)
        if ref_J is None:
            ref_J, ref_G = host(J), host(G)
            assert rel(ref_G, orc.step(u)) < 1e-12
        else:
            assert np.array_equal(host(J), ref_J)
            assert np.array_equal(host(G), ref_G)


def test_static_entry_point():
    ctx, orc = la(8, 17, 8)
    u = seeded(orc, 1108, 0.1)
    d = seeded(orc, 1109, 1.0)
    ctx.sp_set_base(dev(u))
    a, b = ctx.zeros(), ctx.zeros()
    ctx.sp_jvp(dev(d), a)
    ctx.sp_jvp_static(dev(d), b)
    assert np.array_equal(host(a), host(b))


def test_adjoint_and_mixed_groups_rejected():
    import paper_1804_05087_gb300 as sp
    ctx, orc = la(8, 17, 8)
    ctx.sp_set_base(ctx.zeros())
    with pytest.raises(sp.SpError):
        ctx.sp_vjp(ctx.zeros(), ctx.zeros())
    with pytest.raises(sp.SpError):
        ctx.sp_newton_gmres(ctx.zeros(), use_gradient=True)
    with pytest.raises(sp.SpError):
        sp.Group([sp.Config(8, 17, 8, lam_adv=1), sp.Config(8, 17, 8, lam_adv=0)])


def test_newton_converges_with_fewer_actions():
    """Newton-GMRES with laminar advection in L reaches the same root (laminar flow
    from a perturbed-laminar guess) with fewer Jacobian actions than the Stokes step."""
    reps = {}
    for lam_adv in (0, 1):
        ctx, orc = make(16, 33, 16, prec=1, lam_adv=lam_adv)
        U = dev(seeded(orc, 1110, 0.1))
        rep = ctx.sp_newton_gmres(U, max_newton=20, max_krylov=300, tol=1e-10)
        assert rep["converged"], rep
        assert float(np.sqrt(orc.inner(host(U), host(U)))) < 1e-8
        G = orc.step(host(U))
        assert np.sqrt(orc.inner(G, G)) < 1e-10
        reps[lam_adv] = rep
    assert reps[1]["total_jvps"] < reps[0]["total_jvps"], reps
