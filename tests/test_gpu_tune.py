"""Tile autotuner of the per-mode solve: every tile shape computes the same
arithmetic per mode, so the tangent and the step are bit-identical whatever
shape runs; sp_autotune only picks the fastest."""
import numpy as np
import pytest
import torch

import seeded_inputs as si
from gpu_util import dev, host, make, rel, seeded

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("grid", [(16, 33, 16), (24, 49, 24)])
def test_every_shape_bit_identical(prec, grid):
    ctx, orc = make(*grid, prec=prec, max_batch=3)
    u = seeded(orc, 1000, 0.1)
    ds = np.stack([seeded(orc, 2000 + i, 1.0) for i in range(3)])
    U, D = dev(u), dev(ds)
    ref_J, ref_G = None, None
    rep = ctx.sp_autotune(3)
    n = len(rep["shapes"])
    assert n >= 2
    for i in range(n):
        fits = rep["ms_tangent"][i] >= 0 and rep["ms_step"][i] >= 0
        if not fits:
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
            base = orc.base(u)
            tol = 1e-12 if prec == 0 else 1e-5
            for k in range(3):
                assert rel(ref_J[k], orc.jvp(base, ds[k])) < tol
        else:
            assert np.array_equal(host(J), ref_J)
            assert np.array_equal(host(G), ref_G)


def test_autotune_report_and_choice():
    ctx, orc = make(48, 65, 48, prec=1, max_batch=8)
    rep = ctx.sp_autotune(8)
    assert rep["tangent"] in rep["shapes"] and rep["step"] in rep["shapes"]
    i = rep["shapes"].index(rep["tangent"])
    ok = [t for t in rep["ms_tangent"] if t >= 0]
    assert rep["ms_tangent"][i] == min(ok)
    with pytest.raises(Exception):
        ctx.sp_set_solve_shape(99, -1)
