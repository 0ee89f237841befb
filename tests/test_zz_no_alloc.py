"""sp_jvp_static, the tangent step that allocates nothing, against sp_jvp.

Collected last on purpose (file name), so that a run stopping at the first
failure has run every other test before it. It must pass both alone in a
fresh process and after the other tests: the static scratch array keeps the
contents of earlier calls, and the results must not depend on them.
"""
import numpy as np
import pytest

import seeded_inputs as si
from gpu_util import dev, host, make, rel, seeded

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("grid,prec,tol", [((16, 33, 16), 0, 1e-12), ((48, 65, 48), 0, 1e-12),
                                           ((48, 65, 48), 1, 1e-12)])
def test_static_scratch_matches_sp_jvp_twice(grid, prec, tol):
    ctx, orc = make(*grid, prec=prec)
    u = seeded(orc, 1000, 0.1)
    ctx.sp_set_base(dev(u))
    for call in range(2):  # two calls in a row, different directions
        d = dev(si.couette_random_full(900 + call, *grid))
        ref = ctx.zeros()
        ctx.sp_jvp(d, ref)
        out = ctx.zeros()
        ctx.sp_jvp_static(d, out)
        assert rel(host(out), host(ref)) < tol


def test_static_scratch_rejects_grids_beyond_its_size():
    import paper_1804_05087_gb300 as sp
    ctx, orc = make(64, 97, 64)  # 9 * 97 * 43 * 22 complex doubles > 8 MiB
    u = np.zeros(ctx.shape, complex)
    ctx.sp_set_base(dev(u))
    d = ctx.zeros()
    out = ctx.zeros()
    with pytest.raises(sp.SpError) as e:
        ctx.sp_jvp_static(d, out)
    assert e.value.status == 1
