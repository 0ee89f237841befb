"""The host trust-region solver of Newton-GMRES-hookstep (hookstep.h; Sec. 3.2: the hookstep
minimises |g - R y| over the Krylov space subject to |y| <= delta) against a plain restatement:
y(mu) = (R^T R + mu I)^-1 R^T g with mu >= 0 the root of |y(mu)| = delta, from numpy's
symmetric eigendecomposition and a bracketing root finder; inside the radius, y = R^-1 g."""
import os
import shutil
import subprocess

import numpy as np
import pytest
from scipy.optimize import brentq

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1804_05087_gb300", "csrc")


@pytest.fixture(scope="module")
def solver(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("hook") / "hookstep_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "host", "hookstep_check.cpp"),
                    "-o", exe], check=True, capture_output=True)
    return exe


def run(exe, R, g, deltas):
    k = R.shape[0]
    parts = [f"{k} {len(deltas)}"]
    parts += [repr(float(R[i, j])) for j in range(k) for i in range(j + 1)]
    parts += [repr(float(x)) for x in g]
    parts += [repr(float(d)) for d in deltas]
    out = subprocess.run([exe], input=" ".join(parts), capture_output=True, text=True, check=True).stdout.split()
    vals = np.array([float(x) for x in out])
    res = []
    for t in range(len(deltas)):
        blk = vals[t * (k + 2):(t + 1) * (k + 2)]
        res.append((blk[0], blk[1], blk[2:]))
    return res


def reference(R, g, delta):
    k = R.shape[0]
    gk = g[:k]
    y0 = np.linalg.solve(R, gk)
    if np.linalg.norm(y0) <= delta:
        y = y0
    else:
        lam, Q = np.linalg.eigh(R.T @ R)
        c = Q.T @ (R.T @ gk)
        f = lambda mu: np.linalg.norm(c / (lam + mu)) - delta
        hi = np.linalg.norm(c) / delta
        mu = brentq(f, 0.0, hi, xtol=1e-300, rtol=1e-15, maxiter=500)
        y = Q @ (c / (lam + mu))
    pred = np.sqrt(np.linalg.norm(gk - R @ y) ** 2 + g[k] ** 2)
    return y, pred


def rotated_hessenberg(k, seed, span):
    """An upper triangle like the Givens-rotated Hessenberg matrix of GMRES (positive diagonal):
    the R factor of U diag(sigma) V^T with random orthogonal U, V and singular values sigma
    from 1 down to 10^-span, so that its condition number is 10^span."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.normal(size=(k, k)))
    V, _ = np.linalg.qr(rng.normal(size=(k, k)))
    sigma = 10.0 ** (-span * np.arange(k) / max(k - 1, 1))
    R = np.linalg.qr((U * sigma) @ V.T)[1]
    R = np.sign(np.diag(R))[:, None] * R
    return R, rng.uniform(-1, 1, k + 1)


@pytest.mark.parametrize("k,seed,span", [(1, 0, 0.0), (2, 1, 0.5), (3, 2, 1.0), (8, 3, 1.0), (40, 4, 0.0),
                                         (40, 5, 3.0), (120, 6, 2.0), (300, 7, 2.0)])
def test_trust_region_solution(solver, k, seed, span):
    R, g = rotated_hessenberg(k, seed, span)
    n0 = np.linalg.norm(np.linalg.solve(R, g[:k]))
    deltas = [1e-3 * n0, 0.1 * n0, 0.7 * n0, 2.0 * n0]
    for (ylen, pred, y), d in zip(run(solver, R, g, deltas), deltas):
        yr, pr = reference(R, g, d)
        assert np.max(np.abs(y - yr)) <= 1e-9 * np.max(np.abs(yr))
        assert abs(ylen - np.linalg.norm(yr)) <= 1e-9 * np.linalg.norm(yr)
        assert abs(pred - pr) <= 1e-9 * max(pr, 1e-300)
        if d < n0:
            assert abs(ylen - d) <= 1e-9 * d  # on the trust-region boundary
