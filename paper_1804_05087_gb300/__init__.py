"""Python binding of the stokesprec C ABI (include/stokesprec.h).

Argument marshalling only: every step of the BEFE map, its tangent, adjoint
and the Newton-GMRES vector work runs in the CUDA library
``_lib/libstokesprec.so``. PyTorch provides device memory and streams.
There is no CPU fallback: importing the binding without the built library
raises immediately.

States are complex128 CUDA tensors of shape [..., 3, MX, MZ, NY] (component,
x-wavenumber in FFT order, z-wavenumber 0..Kz, Chebyshev degree), contiguous.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libstokesprec.so")

SP_FP64 = 0
SP_MIXED = 1
_STATUS = {0: "SP_OK", 1: "SP_EINVAL", 2: "SP_ENOMEM", 3: "SP_ECUDA", 4: "SP_ENOTCONV",
           5: "SP_ETIMEOUT", 6: "SP_ENAN"}


class SpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("lz", ctypes.c_double), ("re", ctypes.c_double),
                ("dt", ctypes.c_double), ("prec", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("lam_adv", ctypes.c_int)]


class _PipeConfig(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int), ("mt", ctypes.c_int), ("kz", ctypes.c_int), ("ntheta", ctypes.c_int),
                ("nz", ctypes.c_int), ("sym", ctypes.c_int), ("alpha", ctypes.c_double), ("re", ctypes.c_double),
                ("dt", ctypes.c_double), ("prec", ctypes.c_int), ("max_batch", ctypes.c_int)]


class _NewtonOpts(ctypes.Structure):
    _fields_ = [("max_newton", ctypes.c_int), ("max_krylov", ctypes.c_int), ("tol", ctypes.c_double),
                ("eta", ctypes.c_double), ("delta0", ctypes.c_double), ("use_fd", ctypes.c_int),
                ("use_gradient", ctypes.c_int), ("int_steps", ctypes.c_int), ("krylov", ctypes.c_int),
                ("ell", ctypes.c_int), ("use_graphs", ctypes.c_int)]


class _TuneReport(ctypes.Structure):
    _fields_ = [("n_shapes", ctypes.c_int), ("tile", ctypes.c_int * 8), ("threads", ctypes.c_int * 8),
                ("ms_tangent", ctypes.c_double * 8), ("ms_step", ctypes.c_double * 8),
                ("chosen_tangent", ctypes.c_int), ("chosen_step", ctypes.c_int)]


class _NewtonReport(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("total_jvps", ctypes.c_int), ("total_steps", ctypes.c_int),
                ("norm_F", ctypes.c_double), ("norm_F0", ctypes.c_double), ("t_action_ms", ctypes.c_double),
                ("t_orth_ms", ctypes.c_double), ("t_total_ms", ctypes.c_double), ("spec_jvps", ctypes.c_int),
                ("hook_trials", ctypes.c_int), ("delta", ctypes.c_double), ("lin_rel", ctypes.c_double),
                ("newton_len", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"stokesprec library not built ({LIB_PATH} missing); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, D, I, V = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p
    sig = {
        "sp_create": ([ctypes.POINTER(_Config), ctypes.POINTER(ctypes.c_void_p)], I),
        "sp_pipe_create": ([ctypes.POINTER(_PipeConfig), ctypes.POINTER(ctypes.c_void_p)], I),
        "sp_pipe_seed_state": ([P, P, P, I, D, D, D, P, V], I),
        "sp_destroy": ([P], I),
        "sp_last_error": ([P], ctypes.c_char_p),
        "sp_state_len": ([P], ctypes.c_size_t),
        "sp_dims": ([P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "sp_seed_state": ([P, P, P, P, D, P, V], I),
        "sp_step": ([P, P, P, V], I),
        "sp_set_base": ([P, P, V], I),
        "sp_jvp": ([P, P, P, I, V], I),
        "sp_vjp": ([P, P, P, I, V], I),
        "sp_jvp_fd": ([P, P, P, I, V], I),
        "sp_inner": ([P, P, P, I, ctypes.POINTER(D), V], I),
        "sp_newton_gmres": ([P, P, ctypes.POINTER(_NewtonOpts), ctypes.POINTER(_NewtonReport), V], I),
        "sp_krylov_solve": ([P, P, P, I, I, I, D, P, ctypes.POINTER(D), I, ctypes.POINTER(I), ctypes.POINTER(I), V],
                            I),
        "sp_jvp_static": ([P, P, P, V], I),
        "sp_probe_fp64_fma": ([P, I, I, V], I),
        "sp_vjp_euclid": ([P, P, P, I, V], I),
        "sp_trace_enable": ([P, I], I),
        "sp_trace_read": ([P, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_longlong), I], I),
        "sp_autotune": ([P, I, ctypes.POINTER(_TuneReport), V], I),
        "sp_set_tensor_cores": ([P, I, I], I),
        "sp_step_n": ([P, P, P, I, V], I),
        "sp_jvp_host": ([P, P, P, I, I, V], I),
        "sp_set_base_n": ([P, P, I, V], I),
        "sp_jvp_n": ([P, P, P, I, V], I),
        "sp_set_solve_shape": ([P, I, I], I),
        "sp_group_create": ([ctypes.POINTER(_Config), I, ctypes.POINTER(ctypes.c_void_p)], I),
        "sp_group_destroy": ([P], I),
        "sp_group_last_error": ([P], ctypes.c_char_p),
        "sp_group_size": ([P], I),
        "sp_group_state_len": ([P], ctypes.c_size_t),
        "sp_group_offset": ([P, I], ctypes.c_size_t),
        "sp_group_member": ([P, I], ctypes.c_void_p),
        "sp_group_step": ([P, P, P, V], I),
        "sp_group_set_base": ([P, P, V], I),
        "sp_group_jvp": ([P, P, P, V], I),
        "sp_group_inner": ([P, P, P, ctypes.POINTER(D), V], I),
        "sp_group_newton_gmres": ([P, P, ctypes.POINTER(_NewtonOpts), I, ctypes.POINTER(_NewtonReport), V], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()

#: names every build must export (the declarations of include/stokesprec.h)
EXPORTS = ("sp_create", "sp_destroy", "sp_last_error", "sp_state_len", "sp_dims", "sp_seed_state",
           "sp_step", "sp_set_base", "sp_jvp", "sp_vjp", "sp_jvp_fd", "sp_inner", "sp_newton_gmres",
           "sp_trace_enable", "sp_trace_read", "sp_jvp_static", "sp_vjp_euclid", "sp_pipe_create",
           "sp_pipe_seed_state", "sp_group_create", "sp_group_destroy", "sp_group_last_error", "sp_group_size",
           "sp_group_state_len", "sp_group_offset", "sp_group_member", "sp_group_step", "sp_group_set_base",
           "sp_group_jvp", "sp_group_inner", "sp_group_newton_gmres", "sp_autotune",
           "sp_set_solve_shape", "sp_step_n", "sp_set_base_n", "sp_jvp_n",
           "sp_jvp_host", "sp_krylov_solve", "sp_probe_fp64_fma", "sp_set_tensor_cores")
STAGES = ("k_yinv", "k_xz", "k_solve", "step", "vector", "k_rhs")


@dataclass
class Config:
    nx: int
    ny: int
    nz: int
    lx: float = 2 * 3.141592653589793 / 1.14
    lz: float = 2 * 3.141592653589793 / 2.5
    re: float = 400.0
    dt: float = 100.0
    prec: int = SP_FP64
    max_batch: int = 1
    lam_adv: int = 0


@dataclass
class PipeConfig:
    """Pipe flow in a frame moving with the wave speed (sp_pipe_config)."""
    nr: int = 64
    mt: int = 12
    kz: int = 24
    ntheta: int = 48
    nz: int = 96
    sym: int = 2
    alpha: float = 1.25
    re: float = 2500.0
    dt: float = 50.0
    prec: int = SP_FP64
    max_batch: int = 1


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Context:
    """One configuration: plans, operators and workspaces on the current GPU."""

    def __init__(self, cfg, _borrowed=None):
        self.cfg = cfg
        h = ctypes.c_void_p()
        self.pipe = isinstance(cfg, PipeConfig)
        self._owned = _borrowed is None
        if _borrowed is not None:  # a group member: the group owns the handle
            h = ctypes.c_void_p(_borrowed)
            st = 0
        elif self.pipe:
            c = _PipeConfig(cfg.nr, cfg.mt, cfg.kz, cfg.ntheta, cfg.nz, cfg.sym, cfg.alpha, cfg.re, cfg.dt,
                            cfg.prec, cfg.max_batch)
            st = _lib.sp_pipe_create(ctypes.byref(c), ctypes.byref(h))
        else:
            c = _Config(cfg.nx, cfg.ny, cfg.nz, cfg.lx, cfg.lz, cfg.re, cfg.dt, cfg.prec, cfg.max_batch,
                        int(cfg.lam_adv))
            st = _lib.sp_create(ctypes.byref(c), ctypes.byref(h))
        if st != 0:
            raise SpError(st, _lib.sp_last_error(None).decode())
        self._h = h
        kx, kz, ny = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _lib.sp_dims(h, ctypes.byref(kx), ctypes.byref(kz), ctypes.byref(ny))
        self.Kx, self.Kz, self.NY = kx.value, kz.value, ny.value
        self.MX, self.MZ = 2 * self.Kx + 1, self.Kz + 1
        self.state_len = int(_lib.sp_state_len(h))
        self.field_shape = (3, self.MX, self.MZ, self.NY)
        # pipe states are flat: the field followed by one complex slot (speed, 0)
        self.shape = (self.state_len // 2,) if self.pipe else self.field_shape

    def close(self):
        if getattr(self, "_h", None):
            if self._owned:
                _lib.sp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            raise SpError(st, _lib.sp_last_error(self._h).decode())

    def _ptr(self, t: torch.Tensor, count: int = None):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError("expected a CUDA tensor")
        if t.dtype != torch.complex128 or not t.is_contiguous():
            raise TypeError("expected a contiguous complex128 tensor")
        if t.is_conj() or t.is_neg():
            raise TypeError("tensor carries a lazy conjugate/negative bit; call resolve_conj()/resolve_neg()")
        n = t.numel() * 2
        if n % self.state_len:
            raise ValueError(f"tensor size {t.numel()} is not a whole number of states")
        if count is not None and n != count * self.state_len:
            raise ValueError("tensor holds the wrong number of states")
        return ctypes.c_void_p(t.data_ptr()), n // self.state_len

    def zeros(self, n=None, device="cuda"):
        shape = self.shape if n is None else (n,) + self.shape
        return torch.zeros(shape, dtype=torch.complex128, device=device)

    # ------------------------------------------------------------ pipe states
    def pipe_join(self, u, c):
        """Flat pipe state from a field [3, 2kz+1, mt+1, nr] (complex) and a speed."""
        flat = torch.zeros(self.shape, dtype=torch.complex128, device=u.device)
        flat[:-1] = u.reshape(-1)
        flat[-1] = complex(c, 0.0)
        return flat

    def pipe_split(self, s):
        """(field view [3, 2kz+1, mt+1, nr], speed) of a flat pipe state."""
        return s[:-1].reshape(self.field_shape), float(s[-1].real)

    def sp_pipe_seed_state(self, streak, pol, amp, frac, c0, U, stream=None):
        import numpy as np
        streak = np.ascontiguousarray(streak, dtype=np.float64)
        pol = np.ascontiguousarray(pol, dtype=np.complex128)
        npoly = pol.shape[-1]
        pu, _ = self._ptr(U, 1)
        self._check(_lib.sp_pipe_seed_state(self._h, streak.ctypes.data_as(ctypes.c_void_p),
                                            pol.ctypes.data_as(ctypes.c_void_p), npoly, float(amp), float(frac),
                                            float(c0), pu, _stream(stream)))
        return U

    # ------------------------------------------------------------ the ABI
    def sp_seed_state(self, ra, rb, rc, amp, U, stream=None):
        for t in (ra, rb, rc):
            if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous() \
                    or t.numel() * 6 != self.state_len:
                raise ValueError("random shapes must be complex128 [MX][MZ][NY] CUDA tensors")
        pu, _ = self._ptr(U, 1)
        self._check(_lib.sp_seed_state(self._h, ctypes.c_void_p(ra.data_ptr()), ctypes.c_void_p(rb.data_ptr()),
                                       ctypes.c_void_p(rc.data_ptr()), float(amp), pu, _stream(stream)))
        return U

    def sp_step(self, U, G, stream=None):
        pu, _ = self._ptr(U, 1)
        pg, _ = self._ptr(G, 1)
        self._check(_lib.sp_step(self._h, pu, pg, _stream(stream)))
        return G

    def sp_set_base(self, U, stream=None):
        pu, _ = self._ptr(U, 1)
        self._check(_lib.sp_set_base(self._h, pu, _stream(stream)))

    def sp_jvp(self, du, out, stream=None):
        pd, n = self._ptr(du)
        po, _ = self._ptr(out, n)
        self._check(_lib.sp_jvp(self._h, pd, po, n, _stream(stream)))
        return out

    def sp_step_n(self, U, G, n, stream=None):
        """G = B^n(U) - U: n steps of the context's dt (Eq. Gint)."""
        pu, _ = self._ptr(U, 1)
        pg, _ = self._ptr(G, 1)
        self._check(_lib.sp_step_n(self._h, pu, pg, int(n), _stream(stream)))
        return G

    def sp_set_base_n(self, U, n, stream=None):
        pu, _ = self._ptr(U, 1)
        self._check(_lib.sp_set_base_n(self._h, pu, int(n), _stream(stream)))

    def sp_jvp_n(self, du, out, stream=None):
        pd, n = self._ptr(du)
        po, _ = self._ptr(out, n)
        self._check(_lib.sp_jvp_n(self._h, pd, po, n, _stream(stream)))
        return out

    def sp_jvp_host(self, du, out, chunk=0, stream=None):
        """sp_jvp on host tensors (pinned CPU complex128): copies overlap the computation.
        Asynchronous on `stream`: synchronise it before reading `out`."""
        for t in (du, out):
            if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.complex128 or not t.is_contiguous():
                raise TypeError("expected contiguous complex128 host tensors")
        n = du.numel() * 2 // self.state_len
        if du.numel() * 2 != n * self.state_len or out.numel() != du.numel():
            raise ValueError("tensor sizes are not whole, equal numbers of states")
        self._check(_lib.sp_jvp_host(self._h, ctypes.c_void_p(du.data_ptr()), ctypes.c_void_p(out.data_ptr()), n,
                                     int(chunk), _stream(stream)))
        return out

    def sp_jvp_static(self, du, out, stream=None):
        """One tangent action that allocates nothing (see include/stokesprec.h)."""
        pd, _ = self._ptr(du, 1)
        po, _ = self._ptr(out, 1)
        self._check(_lib.sp_jvp_static(self._h, pd, po, _stream(stream)))
        return out

    def sp_vjp(self, r, out, stream=None):
        pr, n = self._ptr(r)
        po, _ = self._ptr(out, n)
        self._check(_lib.sp_vjp(self._h, pr, po, n, _stream(stream)))
        return out

    def sp_vjp_euclid(self, g, out, stream=None):
        pg, n = self._ptr(g)
        po, _ = self._ptr(out, n)
        self._check(_lib.sp_vjp_euclid(self._h, pg, po, n, _stream(stream)))
        return out

    def sp_jvp_fd(self, du, out, stream=None):
        pd, n = self._ptr(du)
        po, _ = self._ptr(out, n)
        self._check(_lib.sp_jvp_fd(self._h, pd, po, n, _stream(stream)))
        return out

    def sp_inner(self, a, b, stream=None):
        pa, n = self._ptr(a)
        pb, _ = self._ptr(b, n)
        out = (ctypes.c_double * n)()
        self._check(_lib.sp_inner(self._h, pa, pb, n, out, _stream(stream)))
        return list(out)

    def sp_set_tensor_cores(self, inverse=True, forward=False):
        """Choose the tensor-core forms of the mixed tangent's Chebyshev transforms (see the header)."""
        self._check(_lib.sp_set_tensor_cores(self._h, int(bool(inverse)), int(bool(forward))))

    def sp_autotune(self, n_dir=1, stream=None):
        """Time the solve kernel's tile shapes and keep the fastest (see include/stokesprec.h)."""
        r = _TuneReport()
        self._check(_lib.sp_autotune(self._h, int(n_dir), ctypes.byref(r), _stream(stream)))
        n = r.n_shapes
        return {"shapes": [(r.tile[i], r.threads[i]) for i in range(n)],
                "ms_tangent": [r.ms_tangent[i] for i in range(n)], "ms_step": [r.ms_step[i] for i in range(n)],
                "tangent": (r.tile[r.chosen_tangent], r.threads[r.chosen_tangent]),
                "step": (r.tile[r.chosen_step], r.threads[r.chosen_step])}

    def sp_set_solve_shape(self, tangent=-1, step=-1):
        self._check(_lib.sp_set_solve_shape(self._h, int(tangent), int(step)))

    def sp_trace_enable(self, on=True):
        self._check(_lib.sp_trace_enable(self._h, 1 if on else 0))

    def sp_trace_read(self):
        """{stage: (total ms, launches)} accumulated since sp_trace_enable."""
        n = len(STAGES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_longlong * n)()
        self._check(_lib.sp_trace_read(self._h, ms, cnt, n))
        return {STAGES[i]: (ms[i], cnt[i]) for i in range(n)}

    def sp_newton_gmres(self, U, max_newton=20, max_krylov=30, tol=1e-10, eta=1e-3, delta0=0.0,
                        use_fd=False, use_gradient=False, int_steps=1, krylov="gmres", ell=2, use_graphs=True,
                        stream=None):
        pu, _ = self._ptr(U, 1)
        o = _opts(max_newton, max_krylov, tol, eta, delta0, use_fd, use_gradient, int_steps, krylov, ell, use_graphs)
        r = _NewtonReport()
        st = _lib.sp_newton_gmres(self._h, pu, ctypes.byref(o), ctypes.byref(r), _stream(stream))
        rep = {k: getattr(r, k) for k, _ in _NewtonReport._fields_}
        rep["converged"] = st == 0
        if st not in (0, 4):
            self._check(st)
        return rep


    def sp_krylov_solve(self, F, X, krylov="bicgstab", param=2, max_act=1000, eta=1e-3, shadow=None,
                        max_hist=4096, stream=None):
        """Solve G_U X = F at the linearisation point with BiCGSTAB(l) or IDR(s).
        shadow: None, or 1 (BiCGSTAB) / s (IDR) states. Returns (|r| history, actions)."""
        pf, _ = self._ptr(F, 1)
        px, _ = self._ptr(X, 1)
        ps = None
        if shadow is not None:
            ps, n = self._ptr(shadow, 1 if krylov == "bicgstab" else int(param))
        h = (ctypes.c_double * max_hist)()
        nh, na = ctypes.c_int(0), ctypes.c_int(0)
        self._check(_lib.sp_krylov_solve(self._h, pf, px, KRYLOV[krylov], int(param), int(max_act), float(eta), ps,
                                         h, max_hist, ctypes.byref(nh), ctypes.byref(na), _stream(stream)))
        return [h[i] for i in range(min(nh.value, max_hist))], na.value


KRYLOV = {"gmres": 0, "bicgstab": 1, "idr": 2}


def probe_fp64_fma(out, blocks, iters, stream=None):
    """Launch the FP64 FMA-rate probe (4096 x blocks x iters flops) on `stream`.
    out: float64 CUDA tensor of at least blocks x 256 elements."""
    if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64
            and out.is_contiguous() and out.numel() >= blocks * 256):
        raise TypeError("expected a contiguous float64 CUDA tensor of blocks x 256 elements")
    st = _lib.sp_probe_fp64_fma(ctypes.c_void_p(out.data_ptr()), int(blocks), int(iters), _stream(stream))
    if st != 0:
        raise SpError(st, "sp_probe_fp64_fma")


def _opts(max_newton, max_krylov, tol, eta, delta0, use_fd, use_gradient, int_steps=1, krylov="gmres", ell=2,
          use_graphs=False):
    return _NewtonOpts(max_newton, max_krylov, tol, eta, delta0, 1 if use_fd else 0, 1 if use_gradient else 0,
                       int(int_steps), KRYLOV[krylov], int(ell), 1 if use_graphs else 0)


class Group:
    """Many independent plane Couette problems stepped together (sp_group_*).

    A group vector is a flat complex128 CUDA tensor of state_len // 2 values;
    member i's state is ``member_view(x, i)`` (shape [3, MX, MZ, NY])."""

    def __init__(self, cfgs):
        cfgs = list(cfgs)
        arr = (_Config * len(cfgs))(*[_Config(c.nx, c.ny, c.nz, c.lx, c.lz, c.re, c.dt, c.prec, 1, int(c.lam_adv))
                                       for c in cfgs])
        h = ctypes.c_void_p()
        st = _lib.sp_group_create(arr, len(cfgs), ctypes.byref(h))
        if st != 0:
            raise SpError(st, _lib.sp_group_last_error(None).decode())
        self._h = h
        self.cfgs = cfgs
        self.n = int(_lib.sp_group_size(h))
        self.state_len = int(_lib.sp_group_state_len(h))
        self.offsets = [int(_lib.sp_group_offset(h, i)) for i in range(self.n)]
        self.members = [Context(cfgs[i], _borrowed=_lib.sp_group_member(h, i)) for i in range(self.n)]

    def close(self):
        if getattr(self, "_h", None):
            for m in self.members:
                m._h = None
            _lib.sp_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            raise SpError(st, _lib.sp_group_last_error(self._h).decode())

    def _ptr(self, t):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.complex128 \
                or not t.is_contiguous() or t.numel() * 2 != self.state_len:
            raise TypeError("expected a contiguous complex128 CUDA group vector")
        if t.is_conj() or t.is_neg():
            raise TypeError("tensor carries a lazy conjugate/negative bit")
        return ctypes.c_void_p(t.data_ptr())

    def zeros(self, device="cuda"):
        return torch.zeros(self.state_len // 2, dtype=torch.complex128, device=device)

    def member_view(self, x, i):
        m = self.members[i]
        o = self.offsets[i] // 2
        return x[o:o + m.state_len // 2].view(m.shape)

    def sp_group_step(self, U, G, stream=None):
        self._check(_lib.sp_group_step(self._h, self._ptr(U), self._ptr(G), _stream(stream)))
        return G

    def sp_group_set_base(self, U, stream=None):
        self._check(_lib.sp_group_set_base(self._h, self._ptr(U), _stream(stream)))

    def sp_group_jvp(self, du, out, stream=None):
        self._check(_lib.sp_group_jvp(self._h, self._ptr(du), self._ptr(out), _stream(stream)))
        return out

    def sp_group_inner(self, a, b, stream=None):
        out = (ctypes.c_double * self.n)()
        self._check(_lib.sp_group_inner(self._h, self._ptr(a), self._ptr(b), out, _stream(stream)))
        return list(out)

    def sp_group_newton_gmres(self, U, max_newton=20, max_krylov=40, tol=1e-10, eta=1e-3, delta0=0.0,
                              use_graphs=True, stream=None):
        """Lock-step Newton-GMRES-hookstep on every member; returns (all converged, [reports])."""
        o = _opts(max_newton, max_krylov, tol, eta, delta0, False, False)
        reps = (_NewtonReport * self.n)()
        st = _lib.sp_group_newton_gmres(self._h, self._ptr(U), ctypes.byref(o), 1 if use_graphs else 0, reps,
                                        _stream(stream))
        if st not in (0, 4):
            self._check(st)
        out = []
        for r in reps:
            d = {k: getattr(r, k) for k, _ in _NewtonReport._fields_}
            d["converged"] = d["norm_F"] < tol
            out.append(d)
        return st == 0, out


class StokesStep(torch.autograd.Function):
    """G = B_dt(U) - U as a differentiable function of the spectral state.

    forward  -> sp_step (FP64); the linearisation point is set with sp_set_base.
    backward -> sp_vjp_euclid: G_U^T applied to the incoming gradient (the
                hand-written adjoint step, in the Euclidean inner product of
                the stored real and imaginary parts that torch uses).
    jvp      -> sp_jvp: the hand-written tangent step (forward-mode AD).
    Usage: G = StokesStep.apply(U, ctx) with U a complex128 CUDA tensor.
    """

    @staticmethod
    def forward(fctx, U, ctx):
        G = ctx.zeros()
        ctx.sp_step(U.detach().resolve_conj().resolve_neg().contiguous(), G)
        fctx.sp = ctx
        fctx.save_for_backward(U.detach().clone())
        fctx.U_fw = U.detach().clone()
        return G

    @staticmethod
    def backward(fctx, grad):
        ctx = fctx.sp
        (U,) = fctx.saved_tensors
        ctx.sp_set_base(U)
        out = ctx.zeros()
        ctx.sp_vjp_euclid(grad.resolve_conj().resolve_neg().contiguous(), out)
        return out, None

    @staticmethod
    def jvp(fctx, dU, _):
        ctx = fctx.sp
        ctx.sp_set_base(fctx.U_fw)
        out = ctx.zeros()
        ctx.sp_jvp(dU.resolve_conj().resolve_neg().contiguous(), out)
        return out
