"""FP64 oracle: the multi-step time-integration operator G^int (Eq. Gint).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper compares Stokes preconditioning, G^Stokes_T = B_T - I with one BEFE
step of size T (Eq. Gstokes), with the time-integration operator
    G^int_T = (B_dt)^(T/dt) - I                                     (Eq. Gint)
built from the same BEFE step with a small dt (Sec. 2). Its Jacobian follows
from the chain rule along the trajectory U_k = B^k(U):
    d_0 = du,  d_(k+1) = B'(U_k) d_k = d_k + G'(U_k) d_k,  G^int_U du = d_n - d_0,
where G'(U_k) is the single step's tangent (``Couette.jvp``). Everything here is
a plain loop over the single-step oracle.
"""
from __future__ import annotations


def trajectory(orc, u, n):
    """The states U_0 = u, ..., U_n = B^n(u) (n + 1 arrays)."""
    states = [u]
    for _ in range(n):
        x = states[-1]
        states.append(x + orc.step(x))
    return states


def step_n(orc, u, n):
    """G^int(u) = B^n(u) - u."""
    return trajectory(orc, u, n)[-1] - u


def jvp_n(orc, u, n, du):
    """G^int_U du by the chain rule along the trajectory of u."""
    states = trajectory(orc, u, n)
    d = du
    for k in range(n):
        d = d + orc.jvp(orc.base(states[k]), d)
    return d - du
