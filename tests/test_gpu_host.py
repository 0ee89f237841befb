"""sp_jvp_host: the tangent of directions held in host memory, chunked so that the
copies of neighbouring chunks overlap the computation. Each direction's arithmetic is
that of sp_jvp, so the results are identical bit for bit."""
import numpy as np
import pytest
import torch

from gpu_util import dev, host, make, seeded

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("chunk", [0, 3, 7])
def test_host_tangent_equals_device_tangent(pinned, chunk):
    ctx, orc = make(16, 33, 16, prec=1, max_batch=4)
    u = seeded(orc, 1000, 0.1)
    ds = np.stack([seeded(orc, 2000 + i, 1.0) for i in range(7)])  # 7: ragged last chunk
    ctx.sp_set_base(dev(u))
    ref = ctx.zeros(7)
    ctx.sp_jvp(dev(ds), ref)
    hd = torch.from_numpy(ds).contiguous()
    ho = torch.zeros_like(hd)
    if pinned:
        hd, ho = hd.pin_memory(), ho.pin_memory()
    ctx.sp_jvp_host(hd, ho, chunk=chunk)
    torch.cuda.synchronize()
    assert np.array_equal(ho.numpy(), host(ref))


def test_host_tangent_pipe():
    import paper_1804_05087_gb300 as sp
    import seeded_inputs as si
    ctx = sp.Context(sp.PipeConfig(nr=16, mt=2, kz=2, ntheta=12, nz=8, prec=0, max_batch=2))
    st, pol = si.pipe_random_coeffs(4000, 2, 2)
    U = ctx.zeros()
    ctx.sp_pipe_seed_state(st, pol, 0.05, 0.1, 0.5, U)
    D = ctx.zeros(5)
    for i in range(5):
        st, pol = si.pipe_random_coeffs(4100 + i, 2, 2)
        ctx.sp_pipe_seed_state(st, pol, 1.0, 1.0, 0.1, D[i])
    ctx.sp_set_base(U)
    ref = ctx.zeros(5)
    ctx.sp_jvp(D, ref)
    ho = torch.zeros(D.shape, dtype=torch.complex128).pin_memory()
    ctx.sp_jvp_host(D.cpu().pin_memory(), ho)
    torch.cuda.synchronize()
    assert np.array_equal(ho.numpy(), ref.cpu().numpy())
