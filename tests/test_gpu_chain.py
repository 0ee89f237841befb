"""The batched tangent's O(N) per-mode solve (contexts with max_batch >= 32) against the oracle.

The oracle solves every per-mode Chebyshev-tau system by dense LU (Sec. 2, Eq. befe;
Sec. 3.2); the library solves the same systems by tridiagonal sweeps and a 2 x 2
influence correction. Tolerances: FP64 rel. 1e-12, mixed 1e-5 per velocity component.
Calls of 3 directions put lanes over modes, calls of 16 or more over directions: the
arithmetic per (mode, direction) is the same, so the results are identical bit for bit.
"""
import numpy as np
import pytest
import torch

import seeded_inputs as si
from gpu_util import dev, host, make, rel, seeded

pytestmark = pytest.mark.gpu

GRIDS = [(8, 17, 8), (16, 33, 16), (24, 49, 24), (18, 17, 24), (48, 65, 48), (32, 97, 32)]


@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("n_dir", [3, 20])
def test_chain_tangent_fp64(grid, n_dir):
    ctx, orc = make(*grid, max_batch=32)
    u = seeded(orc, 1000, 0.1)
    ctx.sp_set_base(dev(u))
    base = orc.base(u)
    ds = np.stack([si.couette_random_full(50 + i, *grid) if i % 2 == 0 else seeded(orc, 60 + i, 1.0)
                   for i in range(n_dir)])
    out = ctx.zeros(n_dir)
    ctx.sp_jvp(dev(ds), out)
    got = host(out)
    for i in (0, 1, n_dir - 1):
        assert rel(got[i], orc.jvp(base, ds[i])) < 1e-12


@pytest.mark.parametrize("grid", [(16, 33, 16), (48, 65, 48)])
def test_chain_tangent_mixed(grid):
    ctx, orc = make(*grid, prec=1, max_batch=32)
    u = seeded(orc, 1000, 0.1)
    ctx.sp_set_base(dev(u))
    base = orc.base(u)
    ds = np.stack([seeded(orc, 70 + i, 1.0) for i in range(17)])
    out = ctx.zeros(17)
    ctx.sp_jvp(dev(ds), out)
    got = host(out)
    for i in (0, 16):
        ref = orc.jvp(base, ds[i])
        for c in range(3):
            assert rel(got[i, c], ref[c]) < 1e-5


@pytest.mark.parametrize("prec", [0, 1])
def test_chain_lane_mappings_bit_identical(prec):
    ctx, orc = make(24, 33, 24, prec=prec, max_batch=48)
    u = seeded(orc, 7, 0.1)
    ctx.sp_set_base(dev(u))
    D = dev(np.stack([seeded(orc, 100 + i, 1.0) for i in range(40)]))
    big = ctx.zeros(40)
    ctx.sp_jvp(D, big)
    small = ctx.zeros(3)
    ctx.sp_jvp(D[:3].contiguous(), small)
    one = ctx.zeros()
    ctx.sp_jvp(D[39].contiguous(), one)
    assert torch.equal(small, big[:3])
    assert torch.equal(one, big[39])


@pytest.mark.parametrize("dt", [1e-3, 1.0, 1e6])
def test_chain_tangent_dt(dt):
    # J du = B_dt' du - du cancels to O(dt |du|) for small dt: scale by max(|J du|, |du|)
    ctx, orc = make(16, 33, 16, max_batch=32, dt=dt)
    u = seeded(orc, 1001, 0.1)
    ctx.sp_set_base(dev(u))
    d = si.couette_random_full(9, 16, 33, 16)
    out = ctx.zeros()
    ctx.sp_jvp(dev(d), out)
    ref = orc.jvp(orc.base(u), d)
    scale = max(np.max(np.abs(ref)), np.max(np.abs(d)))
    assert np.max(np.abs(host(out) - ref)) < 1e-12 * scale


def test_chain_host_tangent_equals_device_tangent():
    ctx, orc = make(16, 33, 16, prec=1, max_batch=32)
    u = seeded(orc, 1000, 0.1)
    ds = np.stack([seeded(orc, 2000 + i, 1.0) for i in range(37)])  # chunks of 32, ragged last
    ctx.sp_set_base(dev(u))
    ref = ctx.zeros(37)
    ctx.sp_jvp(dev(ds), ref)
    hd = torch.from_numpy(ds).contiguous().pin_memory()
    ho = torch.zeros_like(hd).pin_memory()
    ctx.sp_jvp_host(hd, ho)
    torch.cuda.synchronize()
    got = ho.numpy()
    r = host(ref)
    # the chunks of 32 put lanes over directions like the whole batch; the ragged last
    # chunk of 5 puts them over modes: same arithmetic either way
    assert np.array_equal(got, r)
