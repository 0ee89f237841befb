"""The mixed tangent with its inverse Chebyshev transform on the tensor cores, against the oracle.

Grids with 41 <= Ny <= 72 take the tcgen05 transform (TF32 with hi/lo operand splits, FP32
accumulation; rows a2 and a1 of the step, Sec. 3.2). The mixed tangent must stay within the
per-component tolerance of the mixed path, 1e-5 for seeded directions (1e-4 for a full-spectrum
random one, see tests/test_gpu_config_grids.py). The grids cover every K the kernel supports (48, 56,
64, 72) and mode counts that leave a ragged last tile of 16 modes.
"""
import numpy as np
import pytest

import seeded_inputs as si
from gpu_util import dev, host, make, rel, seeded

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("grid", [(16, 41, 16), (18, 49, 24), (24, 57, 24), (48, 65, 48), (16, 71, 16)])
def test_tensor_core_transform_tangent(grid):
    ctx, orc = make(*grid, prec=1, max_batch=3)
    u = seeded(orc, 1000, 0.1)
    ctx.sp_set_base(dev(u))
    base = orc.base(u)
    ds = np.stack([seeded(orc, 80, 1.0), seeded(orc, 81, 1.0), si.couette_random_full(82, *grid)])
    out = ctx.zeros(3)
    ctx.sp_jvp(dev(ds), out)
    got = host(out)
    assert np.all(np.isfinite(got))
    for i in range(3):
        ref = orc.jvp(base, ds[i])
        tol = 1e-4 if i == 2 else 1e-5
        for c in range(3):
            assert rel(got[i, c], ref[c]) < tol


@pytest.mark.parametrize("grid", [(16, 41, 16), (18, 49, 24), (16, 71, 16)])
@pytest.mark.parametrize("n_dir", [3, 20])
def test_tensor_core_forward_transform_chains(grid, n_dir):
    """Contexts with max_batch >= 32 solve the batched tangent by the O(N) chains, whose right-hand
    sides (forward transform of the plane-stage output plus u/dt, row a6) come from the tcgen05
    kernel as well; 20 directions write them directions fastest, 3 directions modes fastest."""
    ctx, orc = make(*grid, prec=1, max_batch=32)
    ctx.sp_set_tensor_cores(inverse=True, forward=True)
    u = seeded(orc, 1001, 0.1)
    ctx.sp_set_base(dev(u))
    base = orc.base(u)
    ds = np.stack([seeded(orc, 90 + i, 1.0) for i in range(n_dir - 1)] + [si.couette_random_full(89, *grid)])
    out = ctx.zeros(n_dir)
    ctx.sp_jvp(dev(ds), out)
    got = host(out)
    assert np.all(np.isfinite(got))
    for i in (0, n_dir // 2, n_dir - 1):
        ref = orc.jvp(base, ds[i])
        tol = 1e-4 if i == n_dir - 1 else 1e-5
        for c in range(3):
            assert rel(got[i, c], ref[c]) < tol


def test_tensor_core_forms_agree_with_cuda_core_kernels():
    """The same batched mixed tangent with every tensor-core form off and on: agreement to float
    accuracy (each is checked against the oracle above)."""
    grid = (18, 49, 24)
    ctx, orc = make(*grid, prec=1, max_batch=32)
    u = seeded(orc, 1002, 0.1)
    ctx.sp_set_base(dev(u))
    ds = np.stack([seeded(orc, 120 + i, 1.0) for i in range(20)])
    outs = []
    for inv, fwd in ((False, False), (True, True)):
        ctx.sp_set_tensor_cores(inverse=inv, forward=fwd)
        out = ctx.zeros(20)
        ctx.sp_jvp(dev(ds), out)
        outs.append(host(out))
    for i in range(20):
        for c in range(3):
            assert rel(outs[1][i, c], outs[0][i, c]) < 1e-5
