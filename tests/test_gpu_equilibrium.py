"""The CUDA path at a nontrivial equilibrium (tests/golden/eq_12x25x12_re500.npz, written by
the oracle alone) and the paper's printed spectra of EQ1 at Re 500 (Sec. 3.5,
tests/golden/paper_eq1_spectra.txt).

Parity: step and tangent at the equilibrium against the oracle (FP64 1e-12, mixed 1e-5 per
component). Exact facts: the step vanishes there, and the x/z derivatives of the state are
null vectors of the tangent. Spectra: dense Jacobians from batched tangent actions, with the
leading eigenvalue of L + N_U against the oracle's stored value and the G^Stokes_0.1 and
G^int_10 spectra against the paper's numbers.
"""
import numpy as np
import pytest
import torch

import bench
from gpu_util import dev, host, make, rel
from test_oracle_equilibrium import load_eq, paper_values

pytestmark = pytest.mark.gpu


def eq_context(prec=0, lam_adv=0, dt=100.0, max_batch=1):
    U, re, grid, lead = load_eq()
    ctx, orc = make(*grid, prec=prec, re=re, dt=dt, lam_adv=lam_adv, max_batch=max_batch)
    return ctx, orc, U, lead


@pytest.mark.parametrize("lam_adv", [0, 1])
def test_step_vanishes_at_the_equilibrium(lam_adv):
    ctx, orc, U, _ = eq_context(lam_adv=lam_adv)
    G = ctx.zeros()
    ctx.sp_step(dev(U), G)
    g = host(G)
    assert np.max(np.abs(g - orc.step(U))) < 1e-12 * np.max(np.abs(U))
    assert orc.norm(g) < 1e-11


@pytest.mark.parametrize("lam_adv", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_tangent_parity_at_the_equilibrium(prec, lam_adv):
    import seeded_inputs as si
    ctx, orc, U, _ = eq_context(prec=prec, lam_adv=lam_adv, max_batch=2)
    ctx.sp_set_base(dev(U))
    base = orc.base(U)
    ds = np.stack([orc.seed_state(*si.couette_random_coeffs(400 + i, orc.nx, orc.ny, orc.nz), 1.0)
                   for i in range(2)])
    out = ctx.zeros(2)
    ctx.sp_jvp(dev(ds), out)
    got = host(out)
    for i in range(2):
        ref = orc.jvp(base, ds[i])
        if prec == 0:
            assert rel(got[i], ref) < 1e-12
        else:
            for c in range(3):
                assert rel(got[i, c], ref[c]) < 1e-5


def test_translation_modes_are_null_vectors():
    ctx, orc, U, _ = eq_context(max_batch=2)
    ctx.sp_set_base(dev(U))
    ikx = 1j * orc.kx[None, :, None, None]
    ikz = 1j * orc.kz[None, None, :, None]
    d = np.stack([ikx * U, ikz * U])
    out = ctx.zeros(2)
    ctx.sp_jvp(dev(d), out)
    got = host(out)
    for i in range(2):
        assert orc.norm(got[i]) < 1e-9 * orc.norm(d[i])


def test_newton_returns_to_the_equilibrium():
    """From a 1 % perturbation, Newton with laminar advection in L (mixed tangent) returns to
    the equilibrium (or a translated copy of it)."""
    import seeded_inputs as si
    ctx, orc, U, _ = eq_context(prec=1, lam_adv=1)
    d = orc.seed_state(*si.couette_random_coeffs(77, orc.nx, orc.ny, orc.nz), 0.01)
    X = dev(U + d)
    rep = ctx.sp_newton_gmres(X, max_newton=30, max_krylov=300, tol=1e-11)
    assert rep["converged"], rep
    # the nearest equilibrium may be a shifted copy: compare shift-invariant quantities
    x = host(X)
    assert abs(orc.norm(x) - orc.norm(U)) < 1e-8
    assert orc.norm(orc.step(x)) < 1e-10


def spectrum(T, n_steps, dt):
    """Eigenvalues of the G Jacobian at the equilibrium on the physical subspace (the
    complement, where G_U + P vanishes, removed)."""
    U, re, grid, _ = load_eq()
    ctx, orc = make(*grid, prec=0, re=re, dt=dt, max_batch=256)
    ctx.sp_set_base_n(dev(U), n_steps)
    J = bench.dense_jacobian(ctx, n_steps)
    P = bench.hermitian_projection(ctx)
    ev = np.linalg.eigvals(J + P)
    return ev[np.abs(ev) > 1e-9] - 1.0


def test_leading_eigenvalue_matches_the_oracle():
    _, _, _, lead = load_eq()
    T = 1e-4
    ev = spectrum(T, 1, T) * (1 + T) / T       # Eq. beaumescale
    top = np.sort(ev.real)[::-1]
    assert abs(top[0] - lead.real.max()) < 1e-6 * abs(lead.real.max())
    assert abs(top[1]) < 1e-6 and abs(top[2]) < 1e-6     # the two translation modes


def test_stokes_0p1_spectrum_against_the_paper():
    p = paper_values()
    T = 0.1
    ev = spectrum(T, 1, T) * (1 + T) / T
    lo = ev.real.min()
    # dominant eigenvalues with real parts near -10, inside a hull reaching -11 (Sec. 3.5)
    assert p["stokes0.1_hull_real_re500"] - 1.0 < lo < p["stokes0.1_dominant_real_re500"] + 1.0


def test_gint10_outlier_against_the_paper():
    p = paper_values()
    dt = 1.0 / 256            # a stable BEFE step (at dt = 1/32 the explicit advection grows)
    ev = spectrum(10.0, int(round(10.0 / dt)), dt)
    out = ev.real.max()
    assert abs(out - p["gint10_outlier_re500"]) < 0.1 * p["gint10_outlier_re500"]
    # the rest of the G^int_10 spectrum clusters at -1
    rest = np.sort(np.abs(ev + 1.0))
    assert rest[int(0.9 * len(rest))] < 0.2
