"""FP64 oracle: one BEFE step for pipe flow in a frame moving with speed c.

TEST INFRASTRUCTURE ONLY (see the package docstring).

What it computes (paper: Sec. 2 Eqs. befe, Gstokes and the traveling-wave
paragraph; Sec. 3.1 pipe flow; Sec. 3.2 Openpipeflow's discretisation classes):
    G(u, c) = B_dt(u; c) - u,  B_dt = (I - dt L)^-1 (I + dt N_c),
    N_c(u) = U_tot x Omega_tot + c d/dz u,
for the deviation u = U - (1 - r^2) e_z from Hagen-Poiseuille flow in a pipe of
radius 1 (velocity scale: centreline speed; Re = U_c R / nu, which equals the
paper's bulk-velocity x diameter number, Sec. 3.1). In deviation form the
driving pressure gradient and the laminar viscous term cancel, so laminar flow
is an exact fixed point for every dt and every c.

Discretisation (readings; the paper only names the classes, Sec. 3.2):
  * Fourier in theta (m = Ms m', rotational symmetry Ms) and z (k = alpha kz);
    stored modes 0 <= m' <= Mt and |kz| <= Kz, physical grid Nt x Nz over
    theta in [0, 2 pi/Ms), z in [0, 2 pi/alpha), products on the grid;
  * radial points r_j = cos(pi j / (2 Nr - 1)), j = 0..Nr-1 (r_0 = 1 the
    wall, the axis excluded); derivatives by 9-point finite differences whose
    weights come from the plain definition (a Vandermonde solve), with
    mirror points -r_j carrying the parity f(-r) = (-1)^q f(r) of the field
    (q = m for u_z and p, m +- 1 for u+- = u_r +- i u_theta);
  * per mode the coupled system for u+, u-, u_z, p (4 Nr unknowns):
    momentum (lam - nu L_q) u + grad p = f at the interior points j >= 1 with
    the decoupled vector Laplacian L_q = D2 + D1/r - q^2/r^2 - k^2
    (q = m+1, m-1, m); no-slip at r = 1; the pressure Poisson equation
    L_m p = div_h f at the interior points (the divergence of momentum with
    div u = 0); continuity div_h u = 0 at the wall, with
    div_h u = (1/2)[(D1 + (1+m)/r) u+ + (D1 + (1-m)/r) u-] + i k u_z.
    (Continuity at every point instead, the other natural reading, gives a
    system with one singular value near 1e-13 of the largest at Nr = 64: not
    usable.) Mode (0,0): Helmholtz for u_theta (L_1) and u_z (L_0), u_r = 0,
    pressure dropped. Solved by dense LU (nothing clever).

Layout: complex128 [3][2Kz+1][Mt+1][Nr] (components u_r, u_theta, u_z; kz in
FFT order 0..Kz, -Kz..-1; m' = 0..Mt; radial index j), plus the speed c.
The m' = 0 plane is stored for both kz and -kz and projected on Hermitian
states. Inner product: sum over stored values of w(m') Re(conj a b), w(0) = 1,
w(m' > 0) = 2, plus c_a c_b.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla


def fd_weights(x0, xs, order):
    """Weights w with sum_k w_k f(xs_k) = f^(order)(x0) exactly for polynomials
    of degree < len(xs): the plain definition, a Vandermonde solve in scaled
    coordinates."""
    xs = np.asarray(xs, float)
    h = np.max(np.abs(xs - x0))
    t = (xs - x0) / h
    n = len(xs)
    V = np.vander(t, n, increasing=True).T           # V[p, k] = t_k^p
    rhs = np.zeros(n)
    rhs[order] = math.factorial(order)
    w = np.linalg.solve(V, rhs)
    return w / h ** order


class Pipe:
    def __init__(self, nr=64, mt=12, kz=24, nt=48, nz=96, ms=2, alpha=1.25, re=2500.0, dt=50.0, stencil=9):
        self.nr, self.mt, self.kzmax, self.nt, self.nz = nr, mt, kz, nt, nz
        self.ms, self.alpha, self.re, self.dt = ms, float(alpha), float(re), float(dt)
        self.nu = 1.0 / self.re
        self.MK = 2 * kz + 1
        self.MT = mt + 1
        self.kzs = np.array([p if p <= kz else p - self.MK for p in range(self.MK)])
        self.k = self.alpha * self.kzs                      # [MK]
        self.m = self.ms * np.arange(self.MT)                # [MT]
        j = np.arange(nr)
        self.r = np.cos(np.pi * j / (2 * nr - 1))
        self.w = np.where(np.arange(self.MT) == 0, 1.0, 2.0)
        self.stencil = stencil
        self.D = {}
        for par in (0, 1):
            self.D[par] = (self._fd_matrix(1, par), self._fd_matrix(2, par))
        th = np.arange(nt) * (2 * np.pi / ms) / nt
        zz = np.arange(nz) * (2 * np.pi / alpha) / nz
        self.Et = np.exp(1j * np.outer(th, self.m))         # [i, m']
        self.Ez = np.exp(1j * np.outer(zz, self.k))         # [l, kz]
        self._lu = {}

    # ------------------------------------------------------------ radial FD
    def _fd_matrix(self, order, par):
        """Derivative matrix on r_j for fields of parity (-1)^par under r -> -r."""
        r = self.r
        nr = self.nr
        pts = np.concatenate([r, -r])
        sgn = np.concatenate([np.ones(nr), (-1.0) ** par * np.ones(nr)])
        idx = np.concatenate([np.arange(nr), np.arange(nr)])
        M = np.zeros((nr, nr))
        for i in range(nr):
            near = np.argsort(np.abs(pts - r[i]), kind="stable")[: self.stencil]
            wts = fd_weights(r[i], pts[near], order)
            for wv, q in zip(wts, near):
                M[i, idx[q]] += wv * sgn[q]
        return M

    def parity(self, mm):
        return int(mm) % 2

    # ------------------------------------------------------------------ basics
    def zeros(self):
        return np.zeros((3, self.MK, self.MT, self.nr), np.complex128), 0.0

    def inner(self, a, b):
        ua, ca = a
        ub, cb = b
        return float(np.sum(self.w[None, None, :, None] * (np.conj(ua) * ub).real)) + ca * cb

    def norm(self, a):
        return math.sqrt(self.inner(a, a))

    def sym(self, u):
        out = u.copy()
        p0 = u[..., :, 0, :]
        mirror = np.conj(p0[..., [(-p) % self.MK for p in range(self.MK)], :])
        out[..., :, 0, :] = 0.5 * (p0 + mirror)
        return out

    # --------------------------------------------------------------- transforms
    def to_physical(self, s):
        """[.., MK, MT, Nr] -> real [.., Nr, Nz, Nt]."""
        t = np.einsum('...pqj,lp->...qjl', s * self.w[:, None], self.Ez)
        return np.einsum('...qjl,iq->...jli', t, self.Et).real

    def to_spectral(self, f):
        t = np.einsum('...jli,iq->...qjl', f, np.conj(self.Et))
        return np.einsum('...qjl,lp->...pqj', t, np.conj(self.Ez)) / (self.nt * self.nz)

    # --------------------------------------------------------------- operators
    def d1(self, f, mm, comp):
        """Radial derivative of component comp (0 u_r, 1 u_theta, 2 u_z / scalar) of mode m."""
        par = self.parity(mm + (1 if comp in (0, 1) else 0))
        return self.D[par][0] @ f

    def fields(self, u):
        """Physical u_r, u_theta, u_z, omega_r, omega_theta, omega_z (no laminar part)."""
        ur, ut, uz = u
        r = self.r
        out = np.zeros((6, self.MK, self.MT, self.nr), np.complex128)
        out[0], out[1], out[2] = ur, ut, uz
        for p in range(self.MK):
            for q in range(self.MT):
                m, k = self.m[q], self.k[p]
                dz = self.d1(uz[p, q], m, 2)
                dt_ = self.d1(ut[p, q], m, 1)
                out[3, p, q] = 1j * m / r * uz[p, q] - 1j * k * ut[p, q]
                out[4, p, q] = 1j * k * ur[p, q] - dz
                out[5, p, q] = dt_ + ut[p, q] / r - 1j * m / r * ur[p, q]
        return self.to_physical(out)

    def total_fields(self, u):
        f = self.fields(u)
        r = self.r[:, None, None]
        f[2] += 1.0 - r ** 2
        f[4] += 2.0 * r
        return f

    @staticmethod
    def cross(a, b):
        return np.stack([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])

    def nonlinear(self, u):
        f = self.total_fields(u)
        return self.to_spectral(self.cross(f[0:3], f[3:6]))

    def nonlinear_tangent(self, base, du):
        g = self.fields(du)
        n = self.cross(base[0:3], g[3:6]) + self.cross(g[0:3], base[3:6])
        return self.to_spectral(n)

    def ddz(self, u):
        return 1j * self.k[None, :, None, None] * u

    # --------------------------------------------------------------- the solve
    def lap(self, q, par, k):
        D1, D2 = self.D[par]
        r = self.r
        return D2 + D1 / r[:, None] - np.diag(q * q / r ** 2) - k * k * np.eye(self.nr)

    def assemble_mode(self, m, k, lam):
        """Dense system for u+, u-, u_z, p (4 Nr unknowns) of mode (m, k) != (0, 0).

        Rows: momentum at j >= 1 (three blocks), no-slip at j = 0, pressure
        Poisson at j >= 1, continuity at j = 0. The RHS is built by rhs_mode."""
        nr = self.nr
        nu = self.nu
        r = self.r
        pe = self.parity(m + 1)      # u+-
        pz = self.parity(m)          # u_z, p
        I = np.eye(nr)
        A = np.zeros((4 * nr, 4 * nr), np.complex128)
        Dp1 = self.D[pz][0]
        Du1 = self.D[pe][0]
        blocks = [(0, lam * I - nu * self.lap(m + 1, pe, k), Dp1 - np.diag(m / r)),
                  (1, lam * I - nu * self.lap(m - 1, pe, k), Dp1 + np.diag(m / r)),
                  (2, lam * I - nu * self.lap(m, pz, k), 1j * k * I)]
        for c, H, G in blocks:
            rows = slice(c * nr + 1, (c + 1) * nr)
            A[rows, c * nr:(c + 1) * nr] = H[1:]
            A[rows, 3 * nr:4 * nr] = G[1:]
            A[c * nr, c * nr] = 1.0                            # no-slip at r = 1
        A[3 * nr + 1:, 3 * nr:] = self.lap(m, pz, k)[1:]     # pressure Poisson
        div = self.div_rows(m, k)
        A[3 * nr, :3 * nr] = div[0]                          # continuity at the wall
        return A

    def div_rows(self, m, k):
        """[Nr, 3 Nr] matrix of div_h acting on (u+, u-, u_z)."""
        nr = self.nr
        r = self.r
        Du1 = self.D[self.parity(m + 1)][0]
        C = np.zeros((nr, 3 * nr), np.complex128)
        C[:, :nr] = 0.5 * (Du1 + np.diag((1 + m) / r))
        C[:, nr:2 * nr] = 0.5 * (Du1 + np.diag((1 - m) / r))
        C[:, 2 * nr:] = 1j * k * np.eye(nr)
        return C

    def rhs_mode(self, m, k, fp, fm, fz):
        nr = self.nr
        rhs = np.zeros(4 * nr, np.complex128)
        rhs[1:nr] = fp[1:]
        rhs[nr + 1:2 * nr] = fm[1:]
        rhs[2 * nr + 1:3 * nr] = fz[1:]
        rhs[3 * nr + 1:] = (self.div_rows(m, k) @ np.concatenate([fp, fm, fz]))[1:]
        return rhs

    def _factor(self, p, q):
        key = (p, q)
        if key not in self._lu:
            m, k = self.m[q], self.k[p]
            lam = 1.0 / self.dt
            if p == 0 and q == 0:
                nr = self.nr
                out = []
                for qq, par in ((1, 1), (0, 0)):   # u_theta with L_1 (odd), u_z with L_0 (even)
                    A = lam * np.eye(nr) - self.nu * self.lap(qq, par, 0.0)
                    A[0] = 0.0
                    A[0, 0] = 1.0
                    out.append(sla.lu_factor(A))
                self._lu[key] = out
            else:
                self._lu[key] = sla.lu_factor(self.assemble_mode(m, k, lam))
        return self._lu[key]

    def solve(self, f):
        """Velocity (u_r, u_theta, u_z) of the per-mode Stokes problems with RHS f."""
        nr = self.nr
        out = np.zeros_like(f)
        for p in range(self.MK):
            for q in range(self.MT):
                lu = self._factor(p, q)
                fr, ft, fz = f[0, p, q], f[1, p, q], f[2, p, q]
                if p == 0 and q == 0:
                    for comp, (lu1, src) in zip((1, 2), zip(lu, (ft, fz))):
                        rhs = src.copy()
                        rhs[0] = 0.0
                        out[comp, 0, 0] = sla.lu_solve(lu1, rhs.real) + 1j * sla.lu_solve(lu1, rhs.imag)
                    continue
                fp = fr + 1j * ft
                fm = fr - 1j * ft
                rhs = self.rhs_mode(self.m[q], self.k[p], fp, fm, fz)
                x = sla.lu_solve(lu, rhs)
                up, um, uz = x[:nr], x[nr:2 * nr], x[2 * nr:3 * nr]
                out[0, p, q] = 0.5 * (up + um)
                out[1, p, q] = (up - um) / 2j
                out[2, p, q] = uz
        return out

    # ---------------------------------------------------------------- the maps
    def step(self, state):
        """G(u, c) = (B_dt(u; c) - u, 0): the speed has no equation of its own."""
        u, c = state
        us = self.sym(u)
        f = us / self.dt + self.nonlinear(us) + c * self.ddz(us)
        return self.sym(self.solve(f) - us), 0.0

    def base(self, state):
        u, c = state
        us = self.sym(u)
        return self.total_fields(us), us, c

    def jvp(self, base, dstate):
        """(G_u du + G_c dc, <d/dz U, du>): tangent plus the phase condition."""
        bf, us, c = base
        du, dc = dstate
        ds = self.sym(du)
        f = ds / self.dt + self.nonlinear_tangent(bf, ds) + c * self.ddz(ds) + dc * self.ddz(us)
        dzU = self.ddz(us)
        phase = self.inner((dzU, 0.0), (ds, 0.0))
        return self.sym(self.solve(f) - ds), phase

    # -------------------------------------------------------------- diagnostics
    def divergence(self, u):
        ur, ut, uz = u
        r = self.r
        out = np.zeros((self.MK, self.MT, self.nr), np.complex128)
        for p in range(self.MK):
            for q in range(self.MT):
                m, k = self.m[q], self.k[p]
                out[p, q] = self.d1(ur[p, q], m, 0) + ur[p, q] / r + 1j * m / r * ut[p, q] + 1j * k * uz[p, q]
        return out


# ---------------------------------------------------------------------- seeding
def poloidal_fields(r, m, k, coef):
    """u = curl curl (phi e_z) for phi = (1 - r^2)^3 r^m sum_n coef_n r^(2n):
    u_r = i k phi', u_theta = -(m k / r) phi, u_z = -(phi'' + phi'/r - m^2 phi / r^2).
    Divergence-free, no-slip at r = 1 (phi, phi', phi'' vanish there), regular at
    the axis. Polynomials evaluated exactly with numpy.polynomial."""
    P = np.polynomial.polynomial
    q = np.zeros(2 * len(coef) + 1, complex)
    q[0:2 * len(coef):2] = coef
    phi = P.polymul(P.polymul(P.polypow([1.0, 0.0, -1.0], 3), np.concatenate([np.zeros(m), [1.0]])), q)
    d1 = P.polyder(phi)
    d2 = P.polyder(d1)
    ph, p1, p2 = P.polyval(r, phi), P.polyval(r, d1), P.polyval(r, d2)
    ur = 1j * k * p1
    ut = -(m * k / r) * ph
    uz = -(p2 + p1 / r - m * m * ph / (r * r))
    return ur, ut, uz


def seed_state(pipe, streak, pol, amp_streak=0.05, frac=0.1, c0=0.5):
    """Hagen-Poiseuille + streaks + a divergence-free k != 0 part (recipe of the
    seeded pipe workload). ``streak[m']`` (m' = 1, 2, 3) are the axial-velocity
    streak amplitudes u_z = a (1 - r^2) r^m (k = 0); ``pol[p, m', n]`` the
    coefficients of the poloidal potentials of the k != 0 modes."""
    u = np.zeros((3, pipe.MK, pipe.MT, pipe.nr), complex)
    r = pipe.r
    for q in range(1, min(4, pipe.MT)):
        m = pipe.m[q]
        u[2, 0, q] = streak[q] * (1 - r * r) * r ** m
    nrm = math.sqrt(float(np.sum(pipe.w[None, None, :, None] * np.abs(u) ** 2)))
    if nrm > 0:
        u *= amp_streak / nrm
    v = np.zeros_like(u)
    for p in range(pipe.MK):
        if pipe.kzs[p] == 0:
            continue
        for q in range(pipe.MT):
            if not np.any(pol[p, q]):
                continue
            ur, ut, uz = poloidal_fields(r, int(pipe.m[q]), pipe.k[p], pol[p, q])
            v[0, p, q], v[1, p, q], v[2, p, q] = ur, ut, uz
    v = pipe.sym(v)
    nv = math.sqrt(float(np.sum(pipe.w[None, None, :, None] * np.abs(v) ** 2)))
    if nv > 0:
        v *= frac * amp_streak / nv
    return pipe.sym(u + v), c0
