"""Newton-GMRES with the Arnoldi steps captured as CUDA graphs runs the same launches
as without: identical iterates and reports."""
import pytest
import torch

from gpu_util import dev, make, seeded

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("use_gradient,grid,re,kmax", [(False, (16, 33, 16), 400.0, 300),
                                                       (True, (8, 17, 8), 100.0, 60)])
def test_graph_replay_identical(use_gradient, grid, re, kmax):
    ctx, orc = make(*grid, prec=1, re=re)
    U1 = dev(seeded(orc, 1000, 0.05))
    U2 = U1.clone()
    r1 = ctx.sp_newton_gmres(U1, max_newton=20, max_krylov=kmax, tol=1e-10, use_graphs=True,
                             use_gradient=use_gradient)
    r2 = ctx.sp_newton_gmres(U2, max_newton=20, max_krylov=kmax, tol=1e-10, use_graphs=False,
                             use_gradient=use_gradient)
    assert r1["converged"] and r2["converged"], (r1, r2)
    assert torch.equal(U1, U2)
    for k in ("newton_iters", "total_jvps", "total_steps", "spec_jvps"):
        assert r1[k] == r2[k]
    # column j + 1 runs while the host tests column j: at most one discarded action per GMRES solve
    assert 0 <= r1["spec_jvps"] <= r1["newton_iters"] + 1


def test_graphs_survive_a_larger_basis():
    ctx, orc = make(8, 17, 8, prec=0)
    U = dev(seeded(orc, 1001, 0.05))
    r = ctx.sp_newton_gmres(U.clone(), max_newton=3, max_krylov=20, tol=1e-10)
    r = ctx.sp_newton_gmres(U.clone(), max_newton=3, max_krylov=60, tol=1e-10)   # reallocates: graphs dropped
    r = ctx.sp_newton_gmres(U.clone(), max_newton=3, max_krylov=40, tol=1e-10)   # smaller K reuses them
    assert r["newton_iters"] >= 1
