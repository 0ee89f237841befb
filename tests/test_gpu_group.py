"""Groups of independent problems (sp_group_*): one launch per stage over all members.

A group changes no arithmetic, so each member's step and tangent are compared
with the FP64 oracle (rel. 1e-12, FP64 mode) and with the member's own context
(bit-identical: the grouped launch runs the same stage code on the same data).
"""
import numpy as np
import pytest
import torch

import seeded_inputs as si
from gpu_util import dev, host, rel
from oracle.couette import Couette

pytestmark = pytest.mark.gpu

# uneven members: several grids (register-FFT sizes and others), Re, boxes and dt
MEMBERS = [dict(nx=16, ny=33, nz=16, re=300.0), dict(nx=24, ny=33, nz=24, re=700.0),
           dict(nx=8, ny=17, nz=8, re=250.0, dt=10.0), dict(nx=32, ny=49, nz=32, re=1000.0),
           dict(nx=18, ny=17, nz=24, re=400.0, lx=4.0, lz=2.0), dict(nx=24, ny=33, nz=24, re=450.0)]


def make_group(prec, members=MEMBERS, lam_adv=0):
    import paper_1804_05087_gb300 as sp
    cfgs = [sp.Config(prec=prec, lam_adv=lam_adv, **m) for m in members]
    g = sp.Group(cfgs)
    orcs = [Couette(c.nx, c.ny, c.nz, lx=c.lx, lz=c.lz, re=c.re, dt=c.dt, lam_adv=bool(lam_adv)) for c in cfgs]
    return g, orcs


def seed_group(g, orcs, seed0, amp):
    """Group vector with member i seeded from seed0 + i by the oracle."""
    U = g.zeros()
    states = []
    for i, orc in enumerate(orcs):
        a, b, c = si.couette_random_coeffs(seed0 + i, orc.nx, orc.ny, orc.nz)
        u = orc.seed_state(a, b, c, amp)
        g.member_view(U, i).copy_(dev(u))
        states.append(u)
    return U, states


def test_group_layout():
    g, orcs = make_group(0)
    assert g.n == len(MEMBERS)
    for i, m in enumerate(g.members):
        assert g.offsets[i] % 32 == 0
        if i + 1 < g.n:
            assert g.offsets[i] + m.state_len <= g.offsets[i + 1]
    assert g.offsets[-1] + g.members[-1].state_len <= g.state_len


@pytest.mark.parametrize("lam_adv", [0, 1])
def test_group_step_matches_oracle_and_members(lam_adv):
    g, orcs = make_group(0, lam_adv=lam_adv)
    U, states = seed_group(g, orcs, 3000, 0.1)
    G = g.zeros()
    g.sp_group_step(U, G)
    for i, (m, orc) in enumerate(zip(g.members, orcs)):
        got = host(g.member_view(G, i))
        assert rel(got, orc.step(states[i])) < 1e-12
        own = m.zeros()
        m.sp_step(g.member_view(U, i).contiguous(), own)
        assert np.array_equal(got, host(own))


@pytest.mark.parametrize("lam_adv", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_group_jvp(prec, lam_adv):
    g, orcs = make_group(prec, lam_adv=lam_adv)
    U, states = seed_group(g, orcs, 3100, 0.1)
    D, dirs = seed_group(g, orcs, 3200, 1.0)
    g.sp_group_set_base(U)
    J = g.zeros()
    g.sp_group_jvp(D, J)
    for i, (m, orc) in enumerate(zip(g.members, orcs)):
        got = host(g.member_view(J, i))
        ref = orc.jvp(orc.base(states[i]), dirs[i])
        assert rel(got, ref) < (1e-12 if prec == 0 else 1e-5)
        own = m.zeros()
        m.sp_set_base(g.member_view(U, i).contiguous())
        m.sp_jvp(g.member_view(D, i).contiguous(), own)
        assert np.array_equal(got, host(own))


def test_group_inner_and_member_fd():
    g, orcs = make_group(0)
    U, states = seed_group(g, orcs, 3300, 0.1)
    D, dirs = seed_group(g, orcs, 3400, 1.0)
    ip = g.sp_group_inner(U, D)
    for i, orc in enumerate(orcs):
        assert abs(ip[i] - orc.inner(states[i], dirs[i])) < 1e-12 * max(1.0, abs(ip[i]))
    # the group's base also serves each member's finite-difference action
    g.sp_group_set_base(U)
    m = g.members[1]
    out = m.zeros()
    m.sp_jvp_fd(g.member_view(D, 1).contiguous(), out)
    assert rel(host(out), orcs[1].jvp(orcs[1].base(states[1]), dirs[1])) < 1e-5


# Newton from perturbed laminar flow: at Re = 1000 the Stokes-preconditioned Jacobian
# needs far more Krylov vectors, so the convergence tests keep Re <= 700
NEWTON_MEMBERS = MEMBERS[:3] + [dict(nx=32, ny=33, nz=32, re=500.0)]


@pytest.mark.parametrize("use_graphs", [False, True])
def test_group_newton_converges(use_graphs):
    g, orcs = make_group(1, NEWTON_MEMBERS)
    U, _ = seed_group(g, orcs, 3500, 0.02)
    ok, reps = g.sp_group_newton_gmres(U, max_newton=30, max_krylov=300, tol=1e-10, use_graphs=use_graphs)
    assert ok, reps
    for i, r in enumerate(reps):
        assert r["norm_F"] < 1e-10
        # perturbed-laminar guesses converge to laminar flow (zero deviation)
        assert float(torch.linalg.vector_norm(g.member_view(U, i))) < 1e-8


def test_group_newton_matches_single_contexts():
    members = MEMBERS[:3]
    g, orcs = make_group(1, members)
    U, states = seed_group(g, orcs, 3600, 0.02)
    U0 = U.clone()
    ok, reps = g.sp_group_newton_gmres(U, max_newton=20, max_krylov=200, tol=1e-10, use_graphs=True)
    assert ok
    U2 = U0.clone()
    ok2, reps2 = g.sp_group_newton_gmres(U2, max_newton=20, max_krylov=200, tol=1e-10, use_graphs=False)
    assert ok2
    # graph replay runs the same launches: identical iterates
    assert torch.equal(U, U2)
    for i, m in enumerate(g.members):
        u = g.member_view(U0, i).clone()
        rep = m.sp_newton_gmres(u, max_newton=20, max_krylov=200, tol=1e-10)
        assert rep["converged"]
        assert rep["newton_iters"] == reps[i]["newton_iters"]
        # the group's weighted dot products sum over other partial blocks than the single
        # context's: a GMRES stopping test may flip by one action at the threshold
        assert abs(rep["total_jvps"] - reps[i]["total_jvps"]) <= rep["newton_iters"]


def test_group_newton_laminar_advection_in_L():
    """Lock-step Newton with laminar advection in L (Sec. 3.6): every member converges, in
    fewer Jacobian actions than the same group with the Stokes step. The two steps have the
    same fixed points, so every root is checked with the oracle's Stokes step; from these
    guesses the 24 x 33 x 24, Re 700 member reaches a nontrivial equilibrium."""
    actions = {}
    for lam_adv in (0, 1):
        g, orcs = make_group(1, NEWTON_MEMBERS, lam_adv=lam_adv)
        U, _ = seed_group(g, orcs, 3500, 0.02)
        ok, reps = g.sp_group_newton_gmres(U, max_newton=30, max_krylov=300, tol=1e-10, use_graphs=True)
        assert ok, (lam_adv, [(r["newton_iters"], r["total_jvps"], r["norm_F"]) for r in reps])
        for i, (r, m) in enumerate(zip(reps, NEWTON_MEMBERS)):
            assert r["norm_F"] < 1e-10
            u = host(g.member_view(U, i))
            stokes = Couette(m["nx"], m["ny"], m["nz"], re=m["re"], dt=m.get("dt", 100.0))
            G = stokes.step(u)
            assert stokes.norm(G) < 1e-9 * max(1.0, stokes.norm(u))
        actions[lam_adv] = sum(r["total_jvps"] for r in reps)
    assert actions[1] < actions[0], actions
