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
