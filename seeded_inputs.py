"""Seeded random inputs shared by the oracle and the CUDA path.

This module draws random numbers and lays them out; it holds none of the
method's arithmetic (no Chebyshev or Fourier operator, no solve, no product).
Both sides turn these arrays into a flow state with their own code:
the oracle in ``oracle/couette.py`` (``seed_state``), the library in its
``sp_seed_state`` kernel.

Recipe (perturbed laminar plane Couette state, Sec. 3.3 workloads):
  * perturbation only in the Fourier modes |ix| <= mmax, |iz| <= mmax;
  * for each such mode two random Chebyshev series, ``a`` (wall-normal
    velocity shape) and ``b`` (wall-normal vorticity shape), with complex
    standard-normal coefficients damped by 10**(-n/8);
  * the kz = 0 plane is Hermitian-consistent: entry (-ix, 0) is the complex
    conjugate of entry (ix, 0), and the (0, 0) entries are real;
  * ``a`` only fills degrees n <= N-4 and ``b`` degrees n <= N-2, so that
    multiplying by (1-y^2)^2 and (1-y^2) keeps the state inside P_N;
  * for the mean mode (0, 0) ``b`` holds the streamwise and ``c`` the spanwise
    mean-flow shape (real), ``a`` is zero there.

Arrays use the spectral layout of the library: modes [ix][iz] with ix in FFT
order (0..Kx, -Kx..-1) and iz in 0..Kz, Chebyshev degree n fastest.
"""
from __future__ import annotations

import numpy as np


def couette_dims(nx: int, ny: int, nz: int):
    """Retained Fourier ranges under the 2/3 rule: (Kx, Kz, MX, MZ, NY)."""
    kx = (nx - 1) // 3
    kz = (nz - 1) // 3
    return kx, kz, 2 * kx + 1, kz + 1, ny


def ix_of(pos: int, kx: int) -> int:
    """Signed x-wavenumber index of storage position ``pos`` (FFT order)."""
    return pos if pos <= kx else pos - (2 * kx + 1)


def pos_of(ix: int, kx: int) -> int:
    """Storage position of the signed x-wavenumber index ``ix``."""
    return ix if ix >= 0 else ix + 2 * kx + 1


def couette_random_coeffs(seed: int, nx: int, ny: int, nz: int, mmax: int = 2):
    """Random coefficient arrays (a, b, c), each complex128 [MX][MZ][NY].

    ``a`` and ``b`` carry the shapes of the wall-normal velocity and vorticity
    of every perturbed mode, ``c`` only the spanwise mean flow in mode (0, 0).
    Generator: numpy PCG64 ``default_rng(seed)``, drawn in a fixed order.
    """
    kx, kz, mx, mz, nyy = couette_dims(nx, ny, nz)
    n_deg = ny - 1
    rng = np.random.default_rng(seed)
    decay = 10.0 ** (-np.arange(nyy) / 8.0)
    a = np.zeros((mx, mz, nyy), np.complex128)
    b = np.zeros((mx, mz, nyy), np.complex128)
    c = np.zeros((mx, mz, nyy), np.complex128)
    lim_a = n_deg - 4 + 1  # degrees 0..N-4
    lim_b = n_deg - 2 + 1  # degrees 0..N-2
    mxx = min(mmax, kx)
    mzz = min(mmax, kz)
    for iz in range(0, mzz + 1):
        for ix in range(-mxx, mxx + 1):
            if iz == 0 and ix < 0:
                continue  # filled by Hermitian symmetry below
            p = pos_of(ix, kx)
            ra = rng.standard_normal((2, nyy))
            rb = rng.standard_normal((2, nyy))
            if iz == 0 and ix == 0:
                b[p, 0, :lim_b] = ra[0, :lim_b] * decay[:lim_b]
                c[p, 0, :lim_b] = rb[0, :lim_b] * decay[:lim_b]
                continue
            a[p, iz, :lim_a] = (ra[0, :lim_a] + 1j * ra[1, :lim_a]) * decay[:lim_a]
            b[p, iz, :lim_b] = (rb[0, :lim_b] + 1j * rb[1, :lim_b]) * decay[:lim_b]
            if iz == 0:
                q = pos_of(-ix, kx)
                a[q, 0] = np.conj(a[p, 0])
                b[q, 0] = np.conj(b[p, 0])
    return a, b, c


def random_directions(seed0: int, count: int, nx: int, ny: int, nz: int, mmax: int = 2):
    """``count`` coefficient triples for tangent directions, seeds seed0..seed0+count-1."""
    return [couette_random_coeffs(seed0 + i, nx, ny, nz, mmax) for i in range(count)]


def couette_random_full(seed: int, nx: int, ny: int, nz: int):
    """Dense random state-shaped array complex128 [3][MX][MZ][NY] (every mode).

    Used for operator tests where the input need not be divergence-free
    (for example dot-product tests of the adjoint). Standard normal entries.
    """
    kx, kz, mx, mz, nyy = couette_dims(nx, ny, nz)
    rng = np.random.default_rng(seed)
    r = rng.standard_normal((2, 3, mx, mz, nyy))
    return r[0] + 1j * r[1]


def pipe_random_coeffs(seed, kz, mt, kmax=2, mmax=3, npoly=4):
    """Random shapes for the seeded pipe state: (streak, pol).

    streak[m'] for m' = 1..3: real standard normal amplitudes of the k = 0
    axial streaks; pol[p, m', n]: complex standard-normal coefficients, damped by
    2**-n, of the poloidal potentials of the modes 1 <= |kz| <= kmax,
    m' <= mmax (zero elsewhere), Hermitian-consistent in the m' = 0 plane.
    Layout: p in FFT order over 2 kz + 1 axial wavenumbers, m' in 0..mt.
    """
    rng = np.random.default_rng(seed)
    mk = 2 * kz + 1
    streak = np.zeros(mt + 1)
    streak[1:min(4, mt + 1)] = rng.standard_normal(min(3, mt))
    pol = np.zeros((mk, mt + 1, npoly), np.complex128)
    decay = 2.0 ** -np.arange(npoly)
    for q in range(0, min(mmax, mt) + 1):
        for kk in range(-min(kmax, kz), min(kmax, kz) + 1):
            if kk == 0 or (q == 0 and kk < 0):
                continue
            p = kk if kk >= 0 else kk + mk
            rr = rng.standard_normal((2, npoly))
            pol[p, q] = (rr[0] + 1j * rr[1]) * decay
            if q == 0:
                pm = (-kk) if -kk >= 0 else -kk + mk
                pol[pm, 0] = np.conj(pol[p, 0])
    return streak, pol


def idr_shadow(s: int, nx: int, ny: int, nz: int, seed: int = 77):
    """``s`` state-shaped standard-normal arrays complex128 [3][MX][MZ][NY]: the raw
    shadow vectors of IDR(s) (and, with s = 1, a BiCGSTAB shadow residual). The
    solver's caller projects and orthonormalises them in its own inner product."""
    kx, kz, mx, mz, nyy = couette_dims(nx, ny, nz)
    rng = np.random.default_rng(seed)
    r = rng.standard_normal((s, 2, 3, mx, mz, nyy))
    return [r[i, 0] + 1j * r[i, 1] for i in range(s)]
