"""Helpers shared by the GPU tests: move oracle states to the library and back."""
import numpy as np
import torch

import seeded_inputs as si
from oracle.couette import Couette


def make(nx, ny, nz, prec=0, max_batch=1, **kw):
    import paper_1804_05087_gb300 as sp
    cfg = sp.Config(nx, ny, nz, prec=prec, max_batch=max_batch, **kw)
    ctx = sp.Context(cfg)
    orc = Couette(nx, ny, nz, lx=cfg.lx, lz=cfg.lz, re=cfg.re, dt=cfg.dt, lam_adv=bool(cfg.lam_adv))
    return ctx, orc


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def seeded(orc, seed, amp):
    a, b, c = si.couette_random_coeffs(seed, orc.nx, orc.ny, orc.nz)
    return orc.seed_state(a, b, c, amp)
