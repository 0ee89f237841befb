"""GPU BiCGSTAB(l) and IDR(s) against the oracle's (Sec. 3.6).

One Newton linear system G_U X = G(U) at a seeded state (8x9x8, Re 100, FP64
tangent): the library's solve (sp_krylov_solve) must follow the oracle's
residual history, |r| at every update, and reach the dense solution on the
physical subspace. Both sides take the same shadow vectors.
"""
import numpy as np
import pytest

import seeded_inputs as si
from gpu_util import dev, host, make
from test_oracle_krylov import jacobian_problem  # noqa: F401  (the dense reference, a fixture)

from oracle.newton import bicgstab_ell, idr_s

pytestmark = pytest.mark.gpu


def orthonormal(g, vs):
    """Modified Gram-Schmidt in the problem's inner product (the shadow space)."""
    out = []
    for v in vs:
        w = g.sym(v)
        for q in out:
            w = w - g.inner(q, w) * q
        out.append(w / g.norm(w))
    return out


@pytest.mark.parametrize("solver,par", [("bicgstab", 2), ("bicgstab", 4), ("idr", 4), ("idr", 8)])
def test_krylov_history_matches_oracle(jacobian_problem, solver, par):  # noqa: F811
    g, base, F, ref = jacobian_problem
    ctx, _ = make(8, 9, 8, re=100.0)
    a, b, c = si.couette_random_coeffs(1000, 8, 9, 8)
    U = g.seed_state(a, b, c, 0.1)
    ctx.sp_set_base(dev(U))
    if solver == "bicgstab":
        shadow = g.sym(si.idr_shadow(1, 8, 9, 8, seed=78)[0])
        xo, ho, ao = bicgstab_ell(lambda v: g.jvp(base, v), F, g.inner, par, 4000, 1e-11, r_shadow=shadow)
        sh = dev(shadow)
    else:
        P = orthonormal(g, si.idr_shadow(par, 8, 9, 8, seed=77))
        xo, ho, ao = idr_s(lambda v: g.jvp(base, v), F, g.inner, P, 4000, 1e-11)
        sh = dev(np.stack(P))
    X = ctx.zeros()
    hg, ag = ctx.sp_krylov_solve(dev(F), X, krylov=solver, param=par, max_act=4000, eta=1e-11, shadow=sh)
    x = host(X)
    ho, hg = np.array(ho), np.array(hg)
    # Rounding differences grow geometrically along these recurrences (by about 300 per
    # BiCGSTAB(4) cycle here), while a wrong coefficient shows at once: the first
    # updates agree to round-off, and agreement to 1e-6 lasts several updates.
    n = min(len(ho), len(hg))
    d = np.abs(hg[:n] - ho[:n]) / ho[:n]
    early = 2 if solver == "bicgstab" else par
    assert np.max(d[:early + 1]) < 1e-12
    first_bad = int(np.argmax(d > 1e-6)) if np.any(d > 1e-6) else n
    assert first_bad >= (4 if solver == "bicgstab" else 2 * par)
    assert hg[-1] <= 1e-11 * hg[0]
    assert abs(ag - ao) <= max(8, 0.2 * ao)
    assert g.norm(x - ref) < 1e-8 * g.norm(ref)
    assert g.norm(x - xo) < 1e-8 * g.norm(ref)


def test_krylov_solve_arguments():
    import paper_1804_05087_gb300 as sp
    ctx, g = make(8, 9, 8, re=100.0)
    F = ctx.zeros()
    X = ctx.zeros()
    with pytest.raises(sp.SpError):  # no linearisation point yet
        ctx.sp_krylov_solve(F, X)
    ctx.sp_set_base(ctx.zeros())
    with pytest.raises(sp.SpError):
        ctx.sp_krylov_solve(F, X, param=9)
    with pytest.raises(sp.SpError):
        ctx.sp_krylov_solve(F, F)
