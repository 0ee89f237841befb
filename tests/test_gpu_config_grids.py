"""Oracle parity on the workloads' own grids (Sec. 3.3 workloads, Sec. 2 step and tangent).

* 96x97x96, doubled box (4 pi/1.14 x 2 x 4 pi/2.5), Re 1000: the Newton-hookstep
  workload with the adjoint (step, tangent, adjoint; FP64 and mixed).
* 32x49x32, Re 700: a member grid of the batched continuation (64 instances).
* 48x65x48 with a linearisation point that populates every retained mode, so the
  high-wavenumber parts of the base fields enter the plane stage.

Tolerances as elsewhere: FP64 rel. 1e-12 (max abs difference over max abs value);
mixed 1e-5 per velocity component (float transforms and products, FP64 solve) for
inputs with the spectral decay of the workloads' states. Inputs with O(1) random
coefficients at every Chebyshev degree and Fourier mode are far less well conditioned:
measured with the oracle, one rounding of the solve's right-hand side at the size of its
largest entry moves the result by 8e-14 (48x65x48), 1e-13 (32x49x32) and 4e-13
(96x97x96) per component, against 2e-15 to 7e-15 for the seeded inputs; the plane
stage rounds tens of times, and a float rounding is 5.4e8 times an FP64 one. So for
these inputs: FP64 1e-11, mixed 1e-4 (N <= 64) and 1e-3 (N = 96) per component.
"""
import math

import numpy as np
import pytest

import seeded_inputs as si
from gpu_util import dev, host, make, rel

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

CASES = {
    "96x97x96": dict(grid=(96, 97, 96), lx=4 * math.pi / 1.14, lz=4 * math.pi / 2.5, re=1000.0, seed=5000),
    "32x49x32": dict(grid=(32, 49, 32), lx=2 * math.pi / 1.14, lz=2 * math.pi / 2.5, re=700.0, seed=3001),
}


def full_mixed_tol(ctx):
    return 1e-4 if ctx.NY <= 65 else 1e-3


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    p = CASES[request.param]
    grid = p["grid"]
    kw = dict(lx=p["lx"], lz=p["lz"], re=p["re"], dt=100.0)
    ctx64, orc = make(*grid, prec=0, max_batch=2, **kw)
    ctx32, _ = make(*grid, prec=1, max_batch=2, **kw)
    u = orc.seed_state(*si.couette_random_coeffs(p["seed"], *grid), 0.1)
    base = orc.base(u)
    ds = np.stack([si.couette_random_full(p["seed"] + 1, *grid),
                   orc.seed_state(*si.couette_random_coeffs(p["seed"] + 2, *grid), 1.0)])
    ref = {"step": orc.step(u),
           "jvp": [orc.jvp(base, d) for d in ds],
           "vjp": [orc.vjp(base, d) for d in ds]}
    return ctx64, ctx32, u, ds, ref


def test_step_fp64(case):
    ctx64, _, u, _, ref = case
    G = ctx64.zeros()
    ctx64.sp_step(dev(u), G)
    assert rel(host(G), ref["step"]) < 1e-12


def test_jvp_fp64_and_mixed(case):
    ctx64, ctx32, u, ds, ref = case
    for ctx, prec in ((ctx64, 0), (ctx32, 1)):
        ctx.sp_set_base(dev(u))
        out = ctx.zeros(2)
        ctx.sp_jvp(dev(ds), out)
        got = host(out)
        for i in range(2):
            if prec == 0:
                assert rel(got[i], ref["jvp"][i]) < 1e-12
            else:
                tol = full_mixed_tol(ctx) if i == 0 else 1e-5  # ds[0]: full-spectrum direction
                for c in range(3):
                    assert rel(got[i, c], ref["jvp"][i][c]) < tol


def test_vjp_fp64_and_mixed(case):
    ctx64, ctx32, u, ds, ref = case
    for ctx, prec in ((ctx64, 0), (ctx32, 1)):
        ctx.sp_set_base(dev(u))
        out = ctx.zeros(2)
        ctx.sp_vjp(dev(ds), out)
        got = host(out)
        for i in range(2):
            if prec == 0:
                assert rel(got[i], ref["vjp"][i]) < 1e-12
            else:
                tol = full_mixed_tol(ctx) if i == 0 else 1e-5
                for c in range(3):
                    assert rel(got[i, c], ref["vjp"][i][c]) < tol


@pytest.mark.parametrize("prec", [0, 1])
def test_full_spectrum_base_48x65x48(prec):
    """Linearisation point with every retained mode populated (random, not a flow state:
    the tangent is defined for any point), and the physical state B(u) of one step."""
    grid = (48, 65, 48)
    ctx, orc = make(*grid, prec=prec, max_batch=2)
    u0 = orc.seed_state(*si.couette_random_coeffs(1001, *grid), 0.1)
    full = si.couette_random_full(1002, *grid)
    bases = [0.1 * full / orc.norm(full), u0 + orc.step(u0)]
    ds = np.stack([si.couette_random_full(1003, *grid), orc.seed_state(*si.couette_random_coeffs(2000, *grid), 1.0)])
    for k, ub in enumerate(bases):
        ctx.sp_set_base(dev(ub))
        b = orc.base(ub)
        out = ctx.zeros(2)
        ctx.sp_jvp(dev(ds), out)
        got = host(out)
        for i in range(2):
            ref = orc.jvp(b, ds[i])
            full = k == 0 or i == 0  # a full-spectrum base or direction
            if prec == 0:
                assert rel(got[i], ref) < (1e-11 if full else 1e-12)
            else:
                tol = full_mixed_tol(ctx) if full else 1e-5
                for c in range(3):
                    assert rel(got[i, c], ref[c]) < tol
