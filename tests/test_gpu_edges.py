"""Edge cases of the C ABI on the GPU: empty batches, argument checks, the largest and
smallest grids the library accepts, and degenerate parameters.

Empty batches (n_dir = 0) are calls with valid pointers that must do nothing and
succeed; invalid arguments return SP_EINVAL without touching the outputs.
"""
import ctypes

import numpy as np
import pytest
import torch

from gpu_util import dev, host, make, rel, seeded

pytestmark = pytest.mark.gpu

SP_OK, SP_EINVAL = 0, 1


def lib():
    import paper_1804_05087_gb300 as sp
    return sp._lib


def ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_empty_batches_do_nothing():
    ctx, orc = make(8, 17, 8, max_batch=2)
    U = dev(seeded(orc, 1, 0.1))
    ctx.sp_set_base(U)
    d = ctx.zeros(2)
    out = torch.full_like(d, 7.0 + 3.0j)
    L = lib()
    for fn in (L.sp_jvp, L.sp_jvp_fd, L.sp_vjp, L.sp_vjp_euclid, L.sp_jvp_n):
        assert fn(ctx._h, ptr(d), ptr(out), 0, None) == SP_OK
    hd = d.cpu().pin_memory()
    ho = out.cpu().pin_memory()
    assert L.sp_jvp_host(ctx._h, ptr(hd), ptr(ho), 0, 0, None) == SP_OK
    torch.cuda.synchronize()
    assert torch.all(out == 7.0 + 3.0j)
    assert torch.all(ho == 7.0 + 3.0j)


def test_bad_arguments_rejected():
    ctx, orc = make(8, 17, 8)
    L = lib()
    U = ctx.zeros()
    G = ctx.zeros()
    # a tangent before any linearisation point
    assert L.sp_jvp(ctx._h, ptr(U), ptr(G), 1, None) == SP_EINVAL
    assert L.sp_vjp(ctx._h, ptr(U), ptr(G), 1, None) == SP_EINVAL
    # aliasing and null pointers, negative counts
    assert L.sp_step(ctx._h, ptr(U), ptr(U), None) == SP_EINVAL
    assert L.sp_step(ctx._h, None, ptr(G), None) == SP_EINVAL
    ctx.sp_set_base(U)
    assert L.sp_jvp(ctx._h, ptr(U), ptr(G), -1, None) == SP_EINVAL
    assert L.sp_jvp(ctx._h, ptr(U), ptr(U), 1, None) == SP_EINVAL
    assert L.sp_step_n(ctx._h, ptr(U), ptr(G), 0, None) == SP_EINVAL
    assert L.sp_set_solve_shape(ctx._h, 99, -1) == SP_EINVAL


def test_largest_chebyshev_degree():
    """ny = 257 is the largest accepted size (N = 256); 259 is rejected."""
    import paper_1804_05087_gb300 as sp
    ctx, orc = make(4, 257, 4)
    u = seeded(orc, 2, 0.1)
    G = ctx.zeros()
    ctx.sp_step(dev(u), G)
    # the per-mode tau systems are ill conditioned at N = 256 (Chebyshev D^2 grows like N^4):
    # two exact inverses agree to about 1e-9 relative there
    assert rel(host(G), orc.step(u)) < 1e-9
    with pytest.raises(sp.SpError):
        sp.Context(sp.Config(4, 259, 4))


def test_smallest_grid():
    """nx = nz = 4, ny = 5: one retained Fourier mode in each direction, N = 4."""
    ctx, orc = make(4, 5, 4, max_batch=2)
    u = seeded(orc, 3, 0.1)
    G = ctx.zeros()
    ctx.sp_step(dev(u), G)
    assert rel(host(G), orc.step(u)) < 1e-12
    ctx.sp_set_base(dev(u))
    d = np.stack([seeded(orc, 4 + i, 1.0) for i in range(2)])
    out = ctx.zeros(2)
    ctx.sp_jvp(dev(d), out)
    for i in range(2):
        assert rel(host(out)[i], orc.jvp(orc.base(u), d[i])) < 1e-12


@pytest.mark.parametrize("re", [1.0, 1e5])
def test_extreme_reynolds_numbers(re):
    ctx, orc = make(16, 33, 16, re=re)
    u = seeded(orc, 5, 0.1)
    G = ctx.zeros()
    ctx.sp_step(dev(u), G)
    ref = orc.step(u)
    scale = max(np.max(np.abs(ref)), np.max(np.abs(u)))
    assert np.max(np.abs(host(G) - ref)) < 1e-11 * scale


def test_large_batch_in_passes_matches_single_calls():
    """A batch of 7 directions in passes of 3 (a ragged last pass) equals seven single calls."""
    ctx, orc = make(12, 17, 12, max_batch=3, prec=1)
    u = seeded(orc, 6, 0.1)
    ctx.sp_set_base(dev(u))
    d = torch.stack([dev(seeded(orc, 10 + i, 1.0)) for i in range(7)])
    out = ctx.zeros(7)
    ctx.sp_jvp(d, out)
    for i in range(7):
        one = ctx.zeros()
        ctx.sp_jvp(d[i].contiguous(), one)
        assert torch.equal(one, out[i])
