"""FP64 oracle: one Backwards-Euler/Forwards-Euler step for plane Couette flow.

TEST INFRASTRUCTURE ONLY (see the package docstring): a plain, slow, readable
CPU restatement of what the method computes, used to check the CUDA library.

What it computes (paper: Sec. 2, Eqs. befe, mycalc, Gstokes; Sec. 3.2):
    G(u) = B_dt(u) - u,   B_dt = (I - dt L)^-1 (I + dt N)
for the deviation u = U - y e_x from laminar plane Couette flow, where
    L u = nu lap(u) - grad p  (with no-slip walls and div u = 0),
    N(u) = U_tot x Omega_tot,  U_tot = u + y e_x, Omega_tot = curl(u) - e_z
(rotational form; the gradient part of the advection goes into the pressure).
One BEFE step is therefore the Stokes problem
    (1/dt - nu lap) u_new + grad p = u/dt + N(u),  div u_new = 0,  u_new(+-1) = 0,
and G = u_new - u (Sec. 2: a single step with dt = T).

Discretisation (Sec. 3.2 names the classes; the concrete choices below are the
readings this library adopts where the paper is silent):
  * Fourier in x and z, Chebyshev in y on Gauss-Lobatto points y_j = cos(pi j/N);
  * retained modes |ix| <= (Nx-1)//3, 0 <= iz <= (Nz-1)//3 (2/3 rule), all
    others zeroed after every product;
  * products at the collocation points (pseudospectral, Sec. 3.2);
  * per Fourier mode (kx,kz) != (0,0) the coupled Chebyshev-tau system with
    unknowns u,v,w,p in P_N: momentum rows n = 0..N-2, no-slip rows at y=+-1,
    continuity for every coefficient n = 0..N (square, 4N+4);
  * the (0,0) mode: Helmholtz for the mean u and w, v = 0, pressure dropped.
Here it is solved by a dense LU per mode: nothing clever.

Spectral layout: complex128 [3][MX][MZ][NY] with x-index ix in FFT order
(0..Kx, -Kx..-1), iz in 0..Kz and Chebyshev degree n fastest. The kz = 0 plane
is stored twice (ix and -ix); every map first projects onto the Hermitian
subspace (``sym``), which is what a real field requires.

Inner product (used for norms, GMRES and the adjoint):
    <a, b> = sum over stored coefficients of w(iz) Re(conj(a) b),
    w(0) = 1, w(iz > 0) = 2.

Laminar advection in L (``lam_adv=True``; Sec. 3.6, the closing proposal, and
Eq. modelgen): the linearisation of the advection about laminar flow,
    M u = (U_lam . grad) u + (u . grad) U_lam = y du/dx + v e_x,
moves from N to L: L' = L - M, N' = N + M, so that the step is
    (1/dt - nu lap + M) u_new + grad p = u/dt + N(u) + M u.
Per mode M is i kx Y (Y: multiplication by y in Chebyshev coefficients) on
every component plus v in the x-momentum rows; the fixed points of B' are
those of B (both steps leave u_new = u where L u + N(u) = 0).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla


class Couette:
    """Grid, operators and per-mode factorisations for one configuration."""

    def __init__(self, nx, ny, nz, lx=2 * math.pi / 1.14, lz=2 * math.pi / 2.5,
                 re=400.0, dt=100.0, lam_adv=False):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.lam_adv = bool(lam_adv)
        self.lx, self.lz, self.re, self.dt = float(lx), float(lz), float(re), float(dt)
        self.nu = 1.0 / self.re
        self.N = ny - 1
        self.Kx = (nx - 1) // 3
        self.Kz = (nz - 1) // 3
        self.MX = 2 * self.Kx + 1
        self.MZ = self.Kz + 1
        self.NY = ny
        N = self.N
        alpha = 2 * math.pi / self.lx
        beta = 2 * math.pi / self.lz
        ixs = np.array([p if p <= self.Kx else p - self.MX for p in range(self.MX)])
        self.ixs = ixs
        self.kx = alpha * ixs                       # [MX]
        self.kz = beta * np.arange(self.MZ)         # [MZ]
        # Chebyshev: Gauss-Lobatto points and T_n(y_j) = cos(pi j n / N)
        j = np.arange(N + 1)
        self.y = np.cos(np.pi * j / N)
        self.T = np.cos(np.pi * np.outer(j, j) / N)          # [j, n]
        cbar = np.ones(N + 1)
        cbar[0] = cbar[N] = 2.0
        # forward transform a_n = 2/(N cbar_n) sum_j u_j T_n(y_j)/cbar_j
        self.Cf = (2.0 / (N * cbar))[:, None] * self.T.T / cbar[None, :]   # [n, j]
        # coefficient-space derivative: (Du)_n = (2/c_n) sum_{p>n, p+n odd} p u_p
        c = np.ones(N + 1)
        c[0] = 2.0
        D = np.zeros((N + 1, N + 1))
        for n in range(N + 1):
            for p in range(n + 1, N + 1):
                if (p + n) % 2 == 1:
                    D[n, p] = 2.0 * p / c[n]
        self.D = D
        self.D2 = D @ D
        # multiplication by y: y T_0 = T_1, y T_m = (T_(m+1) + T_(m-1))/2 (degree N+1 dropped)
        Y = np.zeros((N + 1, N + 1))
        for m in range(N + 1):
            if m == 0:
                Y[1, 0] = 1.0
                continue
            Y[m - 1, m] += 0.5
            if m + 1 <= N:
                Y[m + 1, m] += 0.5
        self.Y = Y
        # Fourier: physical points and the explicit exponentials
        xg = np.arange(nx) * self.lx / nx
        zg = np.arange(nz) * self.lz / nz
        self.Ex = np.exp(1j * np.outer(xg, self.kx))           # [i, pos]
        self.Ez = np.exp(1j * np.outer(zg, self.kz))           # [k, iz]
        self.wz = np.where(np.arange(self.MZ) == 0, 1.0, 2.0)  # weights w(iz)
        self._lu = {}

    # ------------------------------------------------------------------ basics
    def zeros(self):
        return np.zeros((3, self.MX, self.MZ, self.NY), np.complex128)

    def inner(self, a, b):
        """<a,b> = sum w(iz) Re(conj(a) b) over all stored coefficients."""
        return float(np.sum(self.wz[None, None, :, None] * (np.conj(a) * b).real))

    def norm(self, a):
        return math.sqrt(self.inner(a, a))

    def sym(self, a):
        """Projection onto Hermitian-consistent states (kz = 0 plane)."""
        out = a.copy()
        p0 = a[..., :, 0, :]
        mirror = np.conj(p0[..., [(-p) % self.MX for p in range(self.MX)], :])
        out[..., :, 0, :] = 0.5 * (p0 + mirror)
        return out

    # ------------------------------------------------------- transforms (plain)
    def cheb_values(self, coef):
        """Chebyshev coefficients -> values at y_j (last axis)."""
        return coef @ self.T.T

    def cheb_coeffs(self, vals):
        """Values at y_j -> Chebyshev coefficients (last axis)."""
        return vals @ self.Cf.T

    def to_physical(self, spec_vals):
        """[.., MX, MZ, NY] Fourier coefficients at y_j -> real [.., NY, Nx, Nz].

        u(x_i, y_j, z_k) = Re( sum_{ix, iz>=0} w'(iz) c[ix,iz,j] e^{i(kx x_i + kz z_k)} )
        with w'(0) = 1 and w'(iz>0) = 2 (the iz < 0 half is the conjugate).
        """
        wz = self.wz
        t = np.einsum('...pzj,ip->...zji', spec_vals * wz[:, None], self.Ex)
        return np.einsum('...zji,kz->...jik', t, self.Ez).real

    def to_spectral(self, phys):
        """Real [.., NY, Nx, Nz] -> retained Fourier coefficients [.., MX, MZ, NY]."""
        t = np.einsum('...jik,kz->...zji', phys, np.conj(self.Ez))
        return np.einsum('...zji,ip->...pzj', t, np.conj(self.Ex)) / (self.nx * self.nz)

    # -------------------------------------------------------------- derivatives
    def curl(self, c):
        """Coefficients of (u,v,w) -> coefficients of the six fields u,v,w,wx,wy,wz."""
        u, v, w = c[0], c[1], c[2]
        ikx = 1j * self.kx[:, None, None]
        ikz = 1j * self.kz[None, :, None]
        Du = u @ self.D.T
        Dw = w @ self.D.T
        ox = Dw - ikz * v
        oy = ikz * u - ikx * w
        oz = ikx * v - Du
        return np.stack([u, v, w, ox, oy, oz])

    def fields(self, c):
        """Six physical fields (u, v, w, omega) of the spectral state c (no laminar part)."""
        return self.to_physical(self.cheb_values(self.curl(c)))

    def total_fields(self, c):
        """U_tot = u + y e_x and Omega_tot = curl u - e_z on the grid, [6][NY][Nx][Nz]."""
        f = self.fields(c)
        f[0] += self.y[:, None, None]
        f[5] -= 1.0
        return f

    # ----------------------------------------------------- nonlinear term N(u)
    @staticmethod
    def cross(a, b):
        return np.stack([a[1] * b[2] - a[2] * b[1],
                         a[2] * b[0] - a[0] * b[2],
                         a[0] * b[1] - a[1] * b[0]])

    def nonlinear(self, c):
        """Spectral coefficients of N(u) = U_tot x Omega_tot (retained modes)."""
        f = self.total_fields(c)
        n = self.cross(f[0:3], f[3:6])
        return self.cheb_coeffs(self.to_spectral(n))

    def nonlinear_tangent(self, base_fields, dc):
        """Coefficients of U_tot x omega(du) + du x Omega_tot (linearised N, Sec. 2)."""
        g = self.fields(dc)
        n = self.cross(base_fields[0:3], g[3:6]) + self.cross(g[0:3], base_fields[3:6])
        return self.cheb_coeffs(self.to_spectral(n))

    def laminar_advection(self, c):
        """M u = y du/dx + v e_x per mode (Sec. 3.6): i kx Y on every component, + v in x."""
        ikx = 1j * self.kx[:, None, None]
        m = ikx * (c @ self.Y.T)
        m[0] = m[0] + c[1]
        return m

    # -------------------------------------------------------- per-mode Stokes
    def assemble_mode(self, kx, kz, lam):
        """Dense coupled Chebyshev-tau matrix for one mode (kx,kz) != (0,0).

        Unknown order [u(0..N), v(0..N), w(0..N), p(0..N)]. Rows: x-, y-, z-
        momentum for n = 0..N-2; no-slip at y = +1 and y = -1 for u, v, w;
        continuity i kx u + Dv + i kz w = 0 for n = 0..N. ``lam`` multiplies
        the identity in the momentum rows (lam = 1/dt + nu (kx^2 + kz^2)).
        With laminar advection in L the momentum rows also carry i kx Y on
        every component and v in the x-momentum rows.
        """
        N = self.N
        n1 = N + 1
        nu = self.nu
        A = np.zeros((4 * n1, 4 * n1), np.complex128)
        I = np.eye(n1)
        H = lam * I - nu * self.D2
        r = 0
        for comp in range(3):
            for n in range(N - 1):
                A[r, comp * n1:(comp + 1) * n1] = H[n]
                if self.lam_adv:
                    A[r, comp * n1:(comp + 1) * n1] += 1j * kx * self.Y[n]
                    if comp == 0:
                        A[r, n1 + n] += 1.0
                if comp == 0:
                    A[r, 3 * n1 + n] = 1j * kx
                elif comp == 1:
                    A[r, 3 * n1:4 * n1] = self.D[n]
                else:
                    A[r, 3 * n1 + n] = 1j * kz
                r += 1
        plus = np.ones(n1)
        minus = (-1.0) ** np.arange(n1)
        for comp in range(3):
            A[r, comp * n1:(comp + 1) * n1] = plus
            r += 1
            A[r, comp * n1:(comp + 1) * n1] = minus
            r += 1
        for n in range(n1):
            A[r, 0 * n1 + n] = 1j * kx
            A[r, 1 * n1:2 * n1] = self.D[n]
            A[r, 2 * n1 + n] = 1j * kz
            r += 1
        assert r == 4 * n1
        return A

    def assemble_mean(self):
        """Dense tau matrix for the mean flow: (1/dt - nu D^2) on rows 0..N-2 + two walls."""
        N = self.N
        n1 = N + 1
        A = np.zeros((n1, n1))
        H = (1.0 / self.dt) * np.eye(n1) - self.nu * self.D2
        A[:N - 1] = H[:N - 1]
        A[N - 1] = 1.0
        A[N] = (-1.0) ** np.arange(n1)
        return A

    def _factor(self, p, iz):
        key = (p, iz)
        if key not in self._lu:
            kx, kz = self.kx[p], self.kz[iz]
            if p == 0 and iz == 0:
                self._lu[key] = sla.lu_factor(self.assemble_mean())
            else:
                lam = 1.0 / self.dt + self.nu * (kx * kx + kz * kz)
                self._lu[key] = sla.lu_factor(self.assemble_mode(kx, kz, lam))
        return self._lu[key]

    def solve(self, f):
        """Velocity coefficients solving the per-mode Stokes systems for RHS f."""
        N = self.N
        n1 = N + 1
        out = self.zeros()
        for p in range(self.MX):
            for iz in range(self.MZ):
                lu = self._factor(p, iz)
                if p == 0 and iz == 0:
                    for comp in (0, 2):
                        rhs = np.zeros(n1, np.complex128)
                        rhs[:N - 1] = f[comp, 0, 0, :N - 1]
                        out[comp, 0, 0] = (sla.lu_solve(lu, rhs.real)
                                           + 1j * sla.lu_solve(lu, rhs.imag))
                    continue
                rhs = np.zeros(4 * n1, np.complex128)
                for comp in range(3):
                    rhs[comp * (N - 1):(comp + 1) * (N - 1)] = f[comp, p, iz, :N - 1]
                x = sla.lu_solve(lu, rhs)
                for comp in range(3):
                    out[comp, p, iz] = x[comp * n1:(comp + 1) * n1]
        return out

    def solve_adjoint(self, g):
        """Plain real transpose of ``solve`` (conjugate transpose per mode)."""
        N = self.N
        n1 = N + 1
        out = self.zeros()
        for p in range(self.MX):
            for iz in range(self.MZ):
                lu = self._factor(p, iz)
                if p == 0 and iz == 0:
                    for comp in (0, 2):
                        gr = g[comp, 0, 0]
                        z = (sla.lu_solve(lu, gr.real, trans=1)
                             + 1j * sla.lu_solve(lu, gr.imag, trans=1))
                        out[comp, 0, 0, :N - 1] = z[:N - 1]
                    continue
                rhs = np.zeros(4 * n1, np.complex128)
                for comp in range(3):
                    rhs[comp * n1:(comp + 1) * n1] = g[comp, p, iz]
                z = sla.lu_solve(lu, rhs, trans=2)
                for comp in range(3):
                    out[comp, p, iz, :N - 1] = z[comp * (N - 1):(comp + 1) * (N - 1)]
        return out

    # ---------------------------------------------------------------- the maps
    def _rhs(self, cs, n):
        """u/dt + N(u) (+ M u with laminar advection in L) from the nonlinear part n."""
        f = cs / self.dt + n
        if self.lam_adv:
            f = f + self.laminar_advection(cs)
        return f

    def step(self, c):
        """G(u) = B_dt(u) - u (Eqs. befe, Gstokes) for the spectral state c."""
        cs = self.sym(c)
        return self.sym(self.solve(self._rhs(cs, self.nonlinear(cs))) - cs)

    def befe(self, c):
        """B_dt(u) itself (Eq. befe)."""
        cs = self.sym(c)
        return self.sym(self.solve(self._rhs(cs, self.nonlinear(cs))))

    def base(self, c):
        """Total fields U_tot, Omega_tot on the grid: the linearisation point."""
        return self.total_fields(self.sym(c))

    def jvp(self, base_fields, dc):
        """Tangent G_U du: N -> N_U with homogeneous boundary data (Sec. 2)."""
        ds = self.sym(dc)
        f = self._rhs(ds, self.nonlinear_tangent(base_fields, ds))
        return self.sym(self.solve(f) - ds)

    def jvp_fd(self, c, dc, eps=None, g0=None):
        """Finite-difference action [G(U + eps du) - G(U)]/eps (Eq. finitediff)."""
        if eps is None:
            eps = 1e-7 * (1.0 + self.norm(c)) / max(self.norm(dc), 1e-300)
        if g0 is None:
            g0 = self.step(c)
        return (self.step(c + eps * dc) - g0) / eps

    # ----------------------------------------------------------------- adjoint
    def _curl_T(self, g6):
        """Plain real transpose of ``curl`` (conjugate transpose per mode)."""
        gu, gv, gw, gx, gy, gz = g6
        ikx = 1j * self.kx[:, None, None]
        ikz = 1j * self.kz[None, :, None]
        u = gu - ikz * gy - gz @ self.D
        v = gv + ikz * gx - ikx * gz
        w = gw + gx @ self.D + ikx * gy
        return np.stack([u, v, w])

    def _to_physical_T(self, g):
        """Plain real transpose of ``to_physical``: real grid -> spectral."""
        t = np.einsum('...jik,kz->...zji', g, np.conj(self.Ez))
        out = np.einsum('...zji,ip->...pzj', t, np.conj(self.Ex))
        return out * self.wz[:, None]

    def _to_spectral_T(self, a):
        """Plain real transpose of ``to_spectral``: spectral -> real grid."""
        t = np.einsum('...pzj,ip->...zji', a, self.Ex)
        return np.einsum('...zji,kz->...jik', t, self.Ez).real / (self.nx * self.nz)

    def vjp(self, base_fields, r):
        """Adjoint G_U^* r with respect to the weighted inner product <.,.>."""
        if self.lam_adv:
            raise NotImplementedError("the adjoint is defined for the Stokes step only")
        W = self.wz[None, None, :, None]
        rw = self.sym(r * W)
        # J = sym o S o (sym/dt + M o sym) - sym, M = to_spec o prod o to_phys
        gs = self.solve_adjoint(rw)
        a = self._to_spectral_T(gs @ self.Cf)                  # [3][NY][Nx][Nz]
        Ub, Ob = base_fields[0:3], base_fields[3:6]
        g_vel = self.cross(Ob, a)                              # Omega x a
        g_vort = self.cross(a, Ub)                             # a x U
        g6 = np.concatenate([g_vel, g_vort])
        m_t = self._curl_T(self._to_physical_T(g6) @ self.T)
        out = self.sym(gs / self.dt + m_t) - rw
        return out / W

    # ------------------------------------------------------------ diagnostics
    def divergence(self, c):
        """Coefficients of i kx u + Dv + i kz w for every mode (all n)."""
        ikx = 1j * self.kx[:, None, None]
        ikz = 1j * self.kz[None, :, None]
        return ikx * c[0] + c[1] @ self.D.T + ikz * c[2]

    def wall_values(self, c):
        """Values at y = +1 and y = -1 of every component and mode."""
        plus = c.sum(axis=-1)
        minus = (c * (-1.0) ** np.arange(self.NY)).sum(axis=-1)
        return plus, minus

    def laplacian_part(self, c):
        """nu (D^2 - k^2) u per mode (the viscous part of L, without pressure)."""
        k2 = self.kx[:, None, None] ** 2 + self.kz[None, :, None] ** 2
        return self.nu * (c @ self.D2.T - k2 * c)

    # ---------------------------------------------------------------- seeding
    def seed_state(self, a, b, cmean, amp):
        """Divergence-free, no-slip state from the random shapes of seeded_inputs.

        Per mode: v = (1-y^2)^2 sum a_n T_n, eta = (1-y^2) sum b_n T_n, and
        u = i (kx Dv - kz eta)/k^2, w = i (kz Dv + kx eta)/k^2 (so that
        i kx u + Dv + i kz w = 0 and eta = i kz u - i kx w). Mean mode:
        u00 = (1-y^2) sum b_n T_n, w00 = (1-y^2) sum c_n T_n, v00 = 0.
        Scaled so that the weighted coefficient norm equals ``amp``.
        """
        y = self.y
        bump = 1.0 - y * y
        v = self.cheb_coeffs(bump ** 2 * self.cheb_values(a))
        eta = self.cheb_coeffs(bump * self.cheb_values(b))
        Dv = v @ self.D.T
        kx = self.kx[:, None, None]
        kz = self.kz[None, :, None]
        k2 = kx * kx + kz * kz
        k2s = np.where(k2 == 0.0, 1.0, k2)
        u = 1j * (kx * Dv - kz * eta) / k2s
        w = 1j * (kz * Dv + kx * eta) / k2s
        st = np.stack([u, v, w])
        st[:, 0, 0, :] = 0.0
        st[0, 0, 0] = self.cheb_coeffs(bump * self.cheb_values(b[0, 0])).real
        st[2, 0, 0] = self.cheb_coeffs(bump * self.cheb_values(cmean[0, 0])).real
        nrm = self.norm(st)
        return st * (amp / nrm) if nrm > 0 else st
