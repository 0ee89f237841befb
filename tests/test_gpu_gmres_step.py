"""One Newton-GMRES step on the GPU against the oracle's GMRES on the same linear system
(rows a9 and a10; Sec. 2, Eq. linear: G_U X = G(U), then U <- U - X). With eta = 0 both run
exactly K Arnoldi columns, so the Krylov space, the least-squares solution in it and the update
are the same up to rounding, although the GPU orthogonalises by classical Gram-Schmidt with a
selective second pass and the oracle by modified Gram-Schmidt. The trust radius is set far
above the step (delta0), and at amplitude 0.01 the step is accepted at once (the ratio of
actual to predicted decrease is 0.99 in the oracle). 8x17x8 takes the small-state column
(orth.cu), 32x65x32 (90,090 reals per state) the large-state one."""
import math

import numpy as np
import pytest

from gpu_util import dev, host, make, seeded
from oracle.newton import gmres

pytestmark = pytest.mark.gpu


def oracle_step(orc, u, K):
    F = orc.step(u)
    B = orc.base(u)
    V, H, beta, res = gmres(lambda d: orc.jvp(B, d), F, orc.inner, K, 0.0)
    assert H.shape[1] == K  # no breakdown
    e1 = np.zeros(K + 1)
    e1[0] = beta
    y = np.linalg.lstsq(H, e1, rcond=None)[0]
    X = sum(y[i] * V[i] for i in range(K))
    return u - X, X, res[-1] / beta


@pytest.mark.parametrize("grid,K,graphs", [((8, 17, 8), 24, False), ((8, 17, 8), 24, True),
                                           pytest.param((32, 65, 32), 16, False, marks=pytest.mark.slow)])
def test_one_newton_step_matches_oracle_gmres(grid, K, graphs):
    ctx, orc = make(*grid)
    u = seeded(orc, 1000, 0.01)
    U = dev(u)
    rep = ctx.sp_newton_gmres(U, max_newton=1, max_krylov=K, tol=0.0, eta=0.0, delta0=1e6, use_graphs=graphs)
    assert rep["newton_iters"] == 1 and rep["hook_trials"] == 1, rep
    assert rep["total_jvps"] == K and rep["spec_jvps"] == 0, rep
    u_new, X, lin_rel = oracle_step(orc, u, K)
    got = host(U)
    assert np.max(np.abs(got - u_new)) <= 1e-8 * np.max(np.abs(X))
    assert abs(rep["lin_rel"] - lin_rel) <= 1e-8 * lin_rel
    Fn = orc.step(u_new)
    assert abs(rep["norm_F"] - math.sqrt(orc.inner(Fn, Fn))) <= 1e-8 * rep["norm_F"]
