#!/usr/bin/env python
"""Throughput of the Stokes-preconditioned Newton hot path on one GB300.

Metric: Jacobian-vector products per second of the BEFE step + tangent at
48 x 65 x 48 (plane Couette, Re = 400, dt = 100, box 2pi/1.14 x 2 x 2pi/2.5).
One timed step = one pass of the hot path over one batch: set the
linearisation point (one full FP64 BEFE step plus the total fields on the
grid) and apply the tangent step to 256 seeded unit directions (batched).
Inputs are larger than L2 (256 directions x 1.55 MB), so no flush is needed.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the comparison arm; it is deliberately slow).
Under torchrun every rank runs its own 256 directions (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NY, NZ = 48, 65, 48
RE, DT = 400.0, 100.0
LX, LZ = 2 * math.pi / 1.14, 2 * math.pi / 2.5
BASE_SEED, DIR_SEED0 = 1001, 2000
LAM_ADV = False  # the throughput run with laminar advection in L (--lam-adv)
METRIC = "JVPs/s (BEFE step+tangent) at 48x65x48"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--prec", default="fp64", choices=["mixed", "fp64"],
                   help="precision of the headline value; the other one is reported beside it")
    p.add_argument("--single-prec", action="store_true", help="time only the --prec precision")
    p.add_argument("--no-newton", action="store_true", help="skip the time-to-converge block")
    p.add_argument("--ndir", type=int, default=256)
    p.add_argument("--pipe-ndir", type=int, default=64, help="directions per tangent launch of --config3")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--newton", action="store_true",
                   help="time-to-converge comparison (Newton-GMRES-hookstep) instead of the JVP throughput")
    p.add_argument("--grid", default="16x33x16", help="grid of the --newton run")
    p.add_argument("--krylov", type=int, default=300)
    p.add_argument("--config2", action="store_true",
                   help="64 plane Couette instances (Re ~ U[200,1000], four grids) in lock-step group Newton")
    p.add_argument("--gint", action="store_true",
                   help="Newton with G^Stokes_T (one step of size T) vs G^int_T (T/dt steps of dt = 1/32)")
    p.add_argument("--spectra", action="store_true",
                   help="dense Jacobian spectra of G^Stokes_T and G^int_T at laminar flow, Re 500 and 1750")
    p.add_argument("--config3", action="store_true",
                   help="pipe flow, Re 2500, Nr 64, m<=24, |k|<=24: tangent throughput and traveling-wave Newton")
    p.add_argument("--config4", action="store_true",
                   help="96x97x96, Re 1000, doubled box: adjoint gradient check and Newton-hookstep with J^T F")
    p.add_argument("--eq", action="store_true",
                   help="continuation from a nontrivial equilibrium (48x35x48, Re 400 -> 380): G^Stokes_T vs G^int_T")
    p.add_argument("--eq-spectra", action="store_true",
                   help="spectra of G^Stokes_T and G^int_T at a nontrivial equilibrium (Re 500) and its leading "
                        "eigenvalue")
    p.add_argument("--lam-adv", action="store_true",
                   help="the default throughput run with laminar advection folded into L")
    p.add_argument("--convergence", action="store_true",
                   help="Newton to |F| < 1e-10 on every workload (configs 0, 1, 2, 4)")
    p.add_argument("--lamadv", action="store_true",
                   help="laminar advection folded into L vs the Stokes step: Krylov actions, Newton time, "
                        "tangent throughput")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ----------------------------------------------------------------- replicas (one process per GPU)
# The path has no exchange step: every rank processes its own units and the ranks meet only
# to time the slowest one.
def rank_direction_seeds(rank, nd):
    """Seeds of one rank's nd tangent directions: disjoint across ranks (weak scaling)."""
    return [DIR_SEED0 + rank * nd + i for i in range(nd)]


def shard(units, rank, world):
    """Round-robin share of independent units (directions, group members) for one rank."""
    return list(units)[rank::world]


def max_over_ranks(ms, world, device="cuda"):
    """The slowest rank's time: one all-reduce of a scalar, the only collective."""
    if world == 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, units_per_rank, steps, ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank * steps / (ms * 1e-3)


# ----------------------------------------------------------------- workload sizes
def dims():
    kx, kz = (NX - 1) // 3, (NZ - 1) // 3
    mx, mz = 2 * kx + 1, kz + 1
    return kx, kz, mx, mz, NY


def n_unique():
    kx, kz, mx, mz, ny = dims()
    return (kx + 1) * mz + kx * (mz - 1)


CHAIN_MIN_BATCH = 32  # contexts with max_batch >= this solve the tangent by O(N) chains


def chain(n_dir):
    """The batched tangent's per-mode solve is k_rhs + the O(N) chain kernel (k_solve stage)."""
    return n_dir >= CHAIN_MIN_BATCH and not LAM_ADV


def chain_record_doubles():
    """Doubles of one mode's chain records: per parity the two sweep records (6 per unknown),
    the influence vectors (2 per unknown) and 8 scalars."""
    nh = (NY - 1) // 2 + 1
    return 2 * (14 * nh + 8)


def kernel_bytes(stage, n_dir, esz):
    """Algorithmic HBM bytes of one launch (each datum read or written once)."""
    kx, kz, mx, mz, ny = dims()
    mm = mx * mz
    state = 3 * mm * ny * 16
    rhs = 3 * (ny - 2) * n_unique() * 16  # the chains' right-hand sides, FP64
    if stage == "k_yinv":
        return n_dir * (state + 6 * ny * mm * esz)
    if stage == "k_xz":
        return n_dir * 9 * ny * mm * esz + 6 * ny * NX * NZ * esz // 2
    if stage == "k_rhs":
        return n_dir * (3 * ny * mm * esz + state + rhs)
    if stage == "k_solve":
        if chain(n_dir):
            return n_dir * (rhs + 2 * state) + n_unique() * chain_record_doubles() * 8
        ops = n_unique() * (la_op_entries() * 16 if LAM_ADV else op_entries() * 8)
        return n_dir * (3 * ny * mm * esz + 2 * state) + ops
    return 0


def op_entries():
    """Entries of the per-mode operators V_0, V_1, H_0, H_1 (each nv_P x rb_P, real)."""
    n = NY - 1
    nv0, nv1, rb0, rb1 = n // 2 + 1, n // 2, n // 2, n // 2 - 1
    return 2 * (nv0 * rb0 + nv1 * rb1)


def la_op_entries():
    """Complex entries of the per-mode operators V' and H' with laminar advection in L
    ((N - 1) columns of N + 1 rows each)."""
    n = NY - 1
    return 2 * (n - 1) * NY


def kernel_flops(stage, n_dir, prec="mixed"):
    """Algorithmic floating-point operations of one launch (FFT: 5 n log2 n)."""
    kx, kz, mx, mz, ny = dims()
    mm = mx * mz
    nh = (ny - 1) // 2 + 1
    if stage == "k_yinv":
        return n_dir * mm * 5 * nh * ny * 4
    if stage == "k_xz":
        fx = 5 * NX * math.log2(NX)
        fz = 5 * NZ * math.log2(NZ)
        per_plane = (6 + 3) * mz * fx + (6 + 3) * (NX // 2) * fz + NX * NZ * 30
        return n_dir * ny * per_plane
    if stage == "k_rhs":
        # forward Chebyshev transform of the three product components: per row a real
        # even/odd half-length dot product with complex values (4 flops per term) after one
        # pairing pass (4 flops per value), plus du/dt (4 per row); FP64 in FP64 mode, only
        # du/dt in FP64 in mixed mode (the transform is float there and not counted)
        n = ny - 1
        per = 3 * (n - 1) * 4
        if prec == "fp64":
            per += 3 * ((n - 1) * nh * 4 + ny * 4)
        return n_dir * n_unique() * per
    if stage == "k_solve" and chain(n_dir):
        # O(N) chains, FP64, per (mode, parity) thread and coefficient: the w_A sweep with the
        # reduced right-hand side (38 flops), the v_A sweep (22), the influence correction,
        # G_v and the continuity suffix sum (20), the b sweep with the back-rotation and
        # G_u, G_w (44): 124 flops per coefficient, NH coefficients per parity. A sweep step
        # is 18 flops (the row weights folded into the records) and a substitution step 4.
        return n_dir * n_unique() * 2 * nh * 124
    if stage == "k_solve":
        # FP64 work: the per-mode operators (real matrices on complex right-hand sides,
        # 4 flops per entry), the reduced right-hand side g (one complex FMA and one complex
        # update per momentum row) and the continuity/rotation epilogue (16 per point).
        # With laminar advection in L: complex operators on complex right-hand sides (8 flops
        # per entry), plus the M du right-hand-side term and the v -> b coupling (10 per row).
        # In FP64 mode the forward Chebyshev transform of the three product components is FP64
        # too: per row, a real even/odd half-length dot product with complex values (4 flops
        # per term), after one pairing pass (4 flops per value); in mixed mode it is float
        # and not counted here.
        n = ny - 1
        if LAM_ADV:
            per = la_op_entries() * 8 + (n - 1) * 18 + ny * 16
        else:
            per = op_entries() * 4 + (n - 1) * 8 + ny * 16
        if prec == "fp64":
            per += 3 * ((n - 1) * nh * 4 + ny * 4)
        return n_dir * n_unique() * per
    return 0


FP64_NOMINAL = 1.25  # TFLOP/s, the recipe's nominal GB300 FP64 rate (replaced by the measured probe)


def kernel_traffic(stage, n_dir, prec, lam_adv):
    """DRAM bytes of one launch from an ncu capture of the current kernel, or None."""
    if stage == "k_solve" and prec == "mixed" and not lam_adv and not chain(n_dir):
        return solve_traffic(n_dir)
    if stage == "k_xz" and prec == "fp64" and not lam_adv and (NX, NY, NZ) == (48, 65, 48):
        rd, wr = K_XZ64_DRAM_64  # every byte scales with the directions (one plane per block)
        return (rd + wr) * n_dir / 64
    return None


# DRAM bytes of one FP64 tangent launch of the register plane stage k_xz_reg64<48, 48> at
# 48x65x48 with 64 directions (dram__bytes_read.sum, dram__bytes_write.sum of that launch;
# the kernel with the packed row pairs of phase 1 and the quarter-turn twiddles)
K_XZ64_DRAM_64 = (205629696, 68856832)


# DRAM bytes of one mixed-precision k_solve tangent launch at 48x65x48 with 64 directions, from
# one ncu capture of that launch (dram__bytes_read.sum, dram__bytes_write.sum). The
# reads are 64 x (values + state) plus the per-mode operators once; both scale with the
# directions except the operators.
K_SOLVE_DRAM_64 = (164997632, 72500224)


def solve_traffic(n_dir):
    ops = n_unique() * op_entries() * 8
    rd, wr = K_SOLVE_DRAM_64
    return (rd - ops) * n_dir / 64 + ops + wr * n_dir / 64


# ----------------------------------------------------------------- clocks
class Clocks:
    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "20"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- oracle arm
def oracle_jvps(budget_s, max_jvps=None):
    """Time the FP64 oracle's tangent step on host cores: (JVPs/s, count, seconds)."""
    import seeded_inputs as si
    from oracle.couette import Couette
    g = Couette(NX, NY, NZ, lx=LX, lz=LZ, re=RE, dt=DT)
    u = g.seed_state(*si.couette_random_coeffs(BASE_SEED, NX, NY, NZ), 0.1)
    base = g.base(u)
    d0 = g.seed_state(*si.couette_random_coeffs(DIR_SEED0, NX, NY, NZ), 1.0)
    g.jvp(base, d0)  # factor the per-mode systems once (setup, untimed)
    n, t0 = 0, time.perf_counter()
    while True:
        d = g.seed_state(*si.couette_random_coeffs(DIR_SEED0 + n, NX, NY, NZ), 1.0)
        g.jvp(base, d)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_jvps and n >= max_jvps):
            return n / el, n, el


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cores = os.cpu_count()
    per_step = 2
    times = []
    for i in range(args.warmup + args.steps):
        rate, n, el = oracle_jvps(0.0, max_jvps=per_step)
        if i >= args.warmup:
            times.append(el)
    tot = sum(times)
    value = per_step * args.steps / tot
    out = {"metric": METRIC, "value": value, "unit": "JVP/s", "impl": "reference", "n_gpus": 0,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "plane Couette 48x65x48 Re=400 dt=100, FP64 oracle tangent", "ndir_per_step": per_step},
           "cpu_baseline": {"value": value, "unit": "JVP/s", "cores": cores, "kind": "oracle",
                            "sample": f"{per_step} tangent steps per timed step at 48x65x48 (one base state)"},
           "e2e": {"value": value, "unit": "JVP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ----------------------------------------------------------------- our arm
def run_newton(args):
    """Time to |G(U)| < 1e-10 from a seeded perturbed-laminar state (Newton-GMRES-hookstep):
    mixed tangent JVPs versus the plain FP64 finite-difference JVPs, same kernels."""
    import torch
    torch.cuda.set_device(0)
    import paper_1804_05087_gb300 as sp
    import seeded_inputs as si
    nx, ny, nz = (int(t) for t in args.grid.split("x"))
    res = {}
    for name, prec, fd, kry, ell in (("mixed_tangent", sp.SP_MIXED, False, "gmres", 0),
                                     ("fp64_tangent", sp.SP_FP64, False, "gmres", 0),
                                     ("fp64_fd", sp.SP_FP64, True, "gmres", 0),
                                     ("mixed_bicgstab2", sp.SP_MIXED, False, "bicgstab", 2),
                                     ("mixed_bicgstab4", sp.SP_MIXED, False, "bicgstab", 4),
                                     ("mixed_idr4", sp.SP_MIXED, False, "idr", 4),
                                     ("mixed_idr8", sp.SP_MIXED, False, "idr", 8)):
        ctx = sp.Context(sp.Config(nx, ny, nz, lx=LX, lz=LZ, re=RE, dt=DT, prec=prec))
        ctx.sp_autotune(1)
        a, b, c = si.couette_random_coeffs(1000, nx, ny, nz)
        U = ctx.zeros()
        ctx.sp_seed_state(*[torch.from_numpy(x).cuda() for x in (a, b, c)], 0.1, U)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        kmax = args.krylov if kry == "gmres" else 20 * args.krylov  # BiCGSTAB: actions per Newton step
        rep = ctx.sp_newton_gmres(U, max_newton=30, max_krylov=kmax, tol=1e-10, eta=1e-3, use_fd=fd,
                                  krylov=kry, ell=max(ell, 1))
        torch.cuda.synchronize()
        rep["wall_s"] = time.perf_counter() - t0
        res[name] = rep
    out = {"metric": "time to |F|<1e-10 (Newton-GMRES-hookstep)", "unit": "s", "higher_is_better": False,
           "config": {"workload": f"plane Couette {args.grid}, Re=400, dt=100, seed 1000, amplitude 0.1",
                      "max_krylov": args.krylov, "eta": 1e-3},
           "runs": res,
           "speedup_mixed_vs_fp64_fd": res["fp64_fd"]["wall_s"] / res["mixed_tangent"]["wall_s"]}
    print(json.dumps(out))


def run_config4(args):
    """96x97x96 plane Couette, Re 1000, box 4pi/1.14 x 2 x 4pi/2.5, mixed precision:
    (1) J^T F from the adjoint step against central differences of |F|^2/2 (h = 1e-7) on
    32 seeded directions (FP64 steps); (2) 8 Newton-hookstep iterations whose trust-region
    space includes J^* F."""
    import torch
    torch.cuda.set_device(0)
    import paper_1804_05087_gb300 as sp
    import seeded_inputs as si
    nx, ny, nz = 96, 97, 96
    lx, lz = 4 * math.pi / 1.14, 4 * math.pi / 2.5
    ctx = sp.Context(sp.Config(nx, ny, nz, lx=lx, lz=lz, re=1000.0, dt=DT, prec=sp.SP_MIXED))
    ctx64 = sp.Context(sp.Config(nx, ny, nz, lx=lx, lz=lz, re=1000.0, dt=DT, prec=sp.SP_FP64))
    ctx.sp_autotune(1)
    ctx64.sp_autotune(1)

    def seeded(c, seed, amp):
        a, b, cc = si.couette_random_coeffs(seed, nx, ny, nz)
        U = c.zeros()
        return c.sp_seed_state(*[torch.from_numpy(x).cuda() for x in (a, b, cc)], amp, U)

    def wdot(c, a, b):
        return c.sp_inner(a, b)[0]

    U = seeded(ctx64, 6000, 0.1)
    F = ctx64.zeros()
    ctx64.sp_step(U, F)
    ctx64.sp_set_base(U)
    g = ctx64.zeros()
    t0 = time.perf_counter()
    ctx64.sp_vjp(F, g)
    torch.cuda.synchronize()
    t_vjp = time.perf_counter() - t0
    errs = []
    h = 1e-7
    for s in range(32):
        d = seeded(ctx64, 5000 + s, 1.0)
        Fp, Fm = ctx64.zeros(), ctx64.zeros()
        ctx64.sp_step(U + h * d, Fp)
        ctx64.sp_step(U - h * d, Fm)
        fd = (0.5 * wdot(ctx64, Fp, Fp) - 0.5 * wdot(ctx64, Fm, Fm)) / (2 * h)
        an = wdot(ctx64, g, d)
        errs.append(abs(fd - an) / max(abs(an), 1e-30))
    # Newton-hookstep with the gradient direction, mixed tangents, FP64 residual
    U2 = seeded(ctx, 6000, 0.1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep = ctx.sp_newton_gmres(U2, max_newton=8, max_krylov=40, tol=1e-10, eta=1e-3, use_gradient=True)
    torch.cuda.synchronize()
    rep["wall_s"] = time.perf_counter() - t0
    # beyond the stated budget: larger Krylov spaces, up to 20 Newton steps
    U3 = seeded(ctx, 6000, 0.1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep2 = ctx.sp_newton_gmres(U3, max_newton=20, max_krylov=300, tol=1e-10, eta=1e-3, use_gradient=True)
    torch.cuda.synchronize()
    rep2["wall_s"] = time.perf_counter() - t0
    # the same guess with laminar advection folded into L (Sec. 3.6; no adjoint, so no gradient
    # direction): plain Newton-GMRES-hookstep
    ctx_la = sp.Context(sp.Config(nx, ny, nz, lx=lx, lz=lz, re=1000.0, dt=DT, prec=sp.SP_MIXED, lam_adv=1))
    U4 = seeded(ctx_la, 6000, 0.1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep3 = ctx_la.sp_newton_gmres(U4, max_newton=40, max_krylov=300, tol=1e-10, eta=1e-3)
    torch.cuda.synchronize()
    rep3["wall_s"] = time.perf_counter() - t0
    rep3["norm_U"] = math.sqrt(ctx_la.sp_inner(U4, U4)[0])
    ctx_la.close()
    out = {"metric": "config 4: adjoint gradient check and Newton-hookstep with J^T F",
           "config": {"workload": "plane Couette 96x97x96, Re=1000, dt=100, box 4pi/1.14 x 2 x 4pi/2.5"},
           "gradient_check": {"directions": 32, "h": h, "max_rel_err": max(errs), "median_rel_err": statistics.median(errs),
                              "vjp_ms": 1e3 * t_vjp},
           "newton": rep, "newton_to_convergence": dict(rep2, max_newton=20, max_krylov=300),
           "newton_laminar_advection_in_L": dict(rep3, max_newton=40, max_krylov=300)}
    print(json.dumps(out))


def config2_members(seed=3000, n=64):
    """The 64 instances: Re ~ U[200, 1000] and grids drawn uniformly from four sizes."""
    import numpy as np
    rng = np.random.default_rng(seed)
    grids = [(24, 33, 24), (32, 49, 32), (48, 65, 48), (64, 65, 64)]
    res = rng.uniform(200.0, 1000.0, n)
    gi = rng.integers(0, len(grids), n)
    return [(grids[int(k)], float(r)) for k, r in zip(gi, res)]


def run_config2(args):
    """Batched continuation: 64 plane Couette instances with their own Re and grid, mixed
    precision, Newton-GMRES-hookstep with a budget of 3 Newton steps x 40 Krylov vectors.
    The group runs every member in lock step (one launch per stage over all members,
    optionally graph-replayed Arnoldi steps); the baselines solve the members one after
    another through their own contexts: mixed tangent, and the plain FP64 GPU path
    (finite-difference actions, no batching, no graphs)."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    import paper_1804_05087_gb300 as sp
    import seeded_inputs as si
    members = config2_members()
    budget = dict(max_newton=3, max_krylov=40, tol=1e-10, eta=1e-3)

    def cfg(g, re, prec):
        return sp.Config(*g, lx=LX, lz=LZ, re=re, dt=DT, prec=prec)

    def seed_into(ctx, i, U):
        a, b, c = si.couette_random_coeffs(3001 + i, ctx.cfg.nx, ctx.cfg.ny, ctx.cfg.nz)
        ctx.sp_seed_state(*[torch.from_numpy(x).cuda() for x in (a, b, c)], 0.1, U)

    def summary(reps, wall):
        red = [r["norm_F"] / r["norm_F0"] for r in reps]
        return {"wall_s": wall, "converged": int(sum(r["norm_F"] < 1e-10 for r in reps)),
                "median_F_over_F0": float(np.median(red)), "max_F_over_F0": float(np.max(red)),
                "total_jvps": int(sum(r["total_jvps"] for r in reps)),
                "newton_iters": int(sum(r["newton_iters"] for r in reps))}

    grp = sp.Group([cfg(g, re, sp.SP_MIXED) for g, re in members])
    U0 = grp.zeros()
    for i, m in enumerate(grp.members):
        seed_into(m, i, grp.member_view(U0, i))
    out = {"metric": "config 2: batched continuation, 64 instances, 3 Newton x 40 GMRES (mixed)",
           "unit": "s", "higher_is_better": False,
           "config": {"workload": "64 plane Couette instances, Re ~ U[200,1000], grids from "
                                  "{24x33x24, 32x49x32, 48x65x48, 64x65x64} (seed 3000), dt=100, amplitude 0.1",
                      "group_state_MB": grp.state_len * 8 / 1e6,
                      "grids": {f"{g[0]}x{g[1]}x{g[2]}": sum(1 for gg, _ in members if gg == g)
                                for g in sorted(set(g for g, _ in members))}},
           "runs": {}}
    for graphs in (True, False):
        for rep_i in range(2):  # the first call builds the graphs and the Krylov basis
            U = U0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ok, reps = grp.sp_group_newton_gmres(U, use_graphs=graphs, **budget)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        run = summary(reps, wall)
        run["t_action_ms"] = reps[0]["t_action_ms"]
        run["t_orth_ms"] = reps[0]["t_orth_ms"]
        out["runs"]["group_graphs" if graphs else "group_launches"] = run
    for name, prec, fd in (("sequential_mixed_tangent", sp.SP_MIXED, False), ("sequential_fp64_fd", sp.SP_FP64, True)):
        reps, wall = [], 0.0
        for i, (g, re) in enumerate(members):
            ctx = sp.Context(cfg(g, re, prec))
            ctx.sp_autotune(1)
            U = ctx.zeros()
            seed_into(ctx, i, U)
            ctx.sp_newton_gmres(U.clone(), max_newton=1, max_krylov=2, tol=1e-10)  # warm the context
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = ctx.sp_newton_gmres(U, use_fd=fd, **budget)
            torch.cuda.synchronize()
            wall += time.perf_counter() - t0
            reps.append(rep)
            ctx.close()
        out["runs"][name] = summary(reps, wall)
    r = out["runs"]
    out["speedup_group_vs_sequential_fp64_fd"] = r["sequential_fp64_fd"]["wall_s"] / r["group_graphs"]["wall_s"]
    out["speedup_group_vs_sequential_mixed"] = r["sequential_mixed_tangent"]["wall_s"] / r["group_graphs"]["wall_s"]
    # beyond the budget: how many members reach |F| < 1e-10
    U = U0.clone()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ok, reps = grp.sp_group_newton_gmres(U, max_newton=20, max_krylov=args.krylov, tol=1e-10, eta=1e-3,
                                         use_graphs=True)
    torch.cuda.synchronize()
    conv = summary(reps, time.perf_counter() - t0)
    conv["max_newton"], conv["max_krylov"] = 20, args.krylov
    out["to_convergence"] = conv
    grp.close()
    # laminar advection folded into L (Sec. 3.6): the same members and initial guesses
    gla = sp.Group([sp.Config(*g, lx=LX, lz=LZ, re=re, dt=DT, prec=sp.SP_MIXED, lam_adv=1) for g, re in members])
    U0 = gla.zeros()
    for i, m in enumerate(gla.members):
        seed_into(m, i, gla.member_view(U0, i))
    for rep_i in range(2):
        U = U0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ok, reps = gla.sp_group_newton_gmres(U, use_graphs=True, **budget)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    out["runs"]["group_graphs_lam_adv"] = summary(reps, wall)
    U = U0.clone()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ok, reps = gla.sp_group_newton_gmres(U, max_newton=20, max_krylov=args.krylov, tol=1e-10, eta=1e-3,
                                         use_graphs=True)
    torch.cuda.synchronize()
    conv = summary(reps, time.perf_counter() - t0)
    conv["max_newton"], conv["max_krylov"] = 20, args.krylov
    out["to_convergence_lam_adv"] = conv
    gla.close()
    print(json.dumps(out))


def run_convergence(args):
    """Newton to |G(U)| < 1e-10 on every workload, each from its seeded guess: config 0
    (16x33x16), config 1's grid (48x65x48), the 64 members of config 2 (lock-step group), the pipe
    of config 3 and config 4 (96x97x96, Re 1000, doubled box). The Stokes step first; at high Re,
    where its Krylov spaces exceed the budget (Sec. 3.3: K grows with Re), the step with laminar
    advection folded into L (Sec. 3.6). Every run that stops short reports what stopped it: the
    trust radius, the relative residual of the last linear solve and the length of the last
    unconstrained Newton step."""
    import torch
    torch.cuda.set_device(0)
    import paper_1804_05087_gb300 as sp
    import seeded_inputs as si
    out = {"metric": "Newton to |F| < 1e-10 on every workload", "unit": "s", "runs": {}}
    keep = ("newton_iters", "total_jvps", "total_steps", "norm_F0", "norm_F", "converged", "wall_s", "t_action_ms",
            "t_orth_ms", "delta", "lin_rel", "newton_len", "hook_trials")

    def single(name, grid, re, seed, lx=LX, lz=LZ, lam_adv=0, krylov=300, max_newton=30, use_gradient=False):
        ctx = sp.Context(sp.Config(*grid, lx=lx, lz=lz, re=re, dt=DT, prec=sp.SP_MIXED, lam_adv=lam_adv))
        ctx.sp_autotune(1)
        a, b, c = si.couette_random_coeffs(seed, *grid)
        U = ctx.zeros()
        ctx.sp_seed_state(*[torch.from_numpy(x).cuda() for x in (a, b, c)], 0.1, U)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = ctx.sp_newton_gmres(U, max_newton=max_newton, max_krylov=krylov, tol=1e-10, eta=1e-3,
                                  use_gradient=use_gradient)
        torch.cuda.synchronize()
        rep["wall_s"] = time.perf_counter() - t0
        r = {k: rep[k] for k in keep}
        r["norm_U"] = math.sqrt(ctx.sp_inner(U, U)[0])
        r.update({"grid": list(grid), "re": re, "lam_adv": lam_adv, "max_krylov": krylov, "max_newton": max_newton,
                  "seed": seed, "use_gradient": use_gradient})
        out["runs"][name] = r
        ctx.close()

    single("config0_16x33x16_re400", (16, 33, 16), RE, 1000)
    single("config1_48x65x48_re400", (NX, NY, NZ), RE, BASE_SEED)
    # config 2: the 64 members in lock step, laminar advection in L
    members = config2_members()
    grp = sp.Group([sp.Config(*g, lx=LX, lz=LZ, re=re, dt=DT, prec=sp.SP_MIXED, lam_adv=1) for g, re in members])
    U = grp.zeros()
    for i, m in enumerate(grp.members):
        a, b, c = si.couette_random_coeffs(3001 + i, m.cfg.nx, m.cfg.ny, m.cfg.nz)
        m.sp_seed_state(*[torch.from_numpy(x).cuda() for x in (a, b, c)], 0.1, grp.member_view(U, i))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ok, reps = grp.sp_group_newton_gmres(U, max_newton=60, max_krylov=300, tol=1e-10, eta=1e-3, use_graphs=True)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    conv = [r["norm_F"] < 1e-10 for r in reps]
    out["runs"]["config2_64_members_lam_adv_K300_N60"] = {
        "wall_s": wall, "converged": int(sum(conv)), "members": len(reps),
        "newton_iters_max": int(max(r["newton_iters"] for r in reps)),
        "total_jvps": int(sum(r["total_jvps"] for r in reps)),
        "not_converged": [{"member": i, "grid": list(members[i][0]), "re": members[i][1],
                           "norm_F": reps[i]["norm_F"], "delta": reps[i]["delta"], "lin_rel": reps[i]["lin_rel"],
                           "newton_len": reps[i]["newton_len"]} for i in range(len(reps)) if not conv[i]]}
    grp.close()
    # config 3: pipe, Hagen-Poiseuille plus seeded streaks, the speed c an unknown
    ctx = sp.Context(sp.PipeConfig(prec=sp.SP_MIXED, max_batch=1))
    st, pol = si.pipe_random_coeffs(4000, ctx.cfg.kz, ctx.cfg.mt)
    U = ctx.zeros()
    ctx.sp_pipe_seed_state(st, pol, 0.05, 0.1, 0.5, U)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep = ctx.sp_newton_gmres(U, max_newton=20, max_krylov=300, tol=1e-10, eta=1e-3)
    torch.cuda.synchronize()
    r = {k: rep[k] for k in keep if k in rep}
    r["wall_s"] = time.perf_counter() - t0
    u, c = ctx.pipe_split(U)
    r.update({"speed_c": c, "deviation_norm": float(torch.linalg.vector_norm(u)), "seed": 4000})
    out["runs"]["config3_pipe_re2500"] = r
    ctx.close()
    # config 4: the Stokes step with the gradient direction (K-limited at Re 1000), then laminar
    # advection in L with a longer Newton budget
    lx4, lz4 = 4 * math.pi / 1.14, 4 * math.pi / 2.5
    single("config4_96x97x96_re1000_gradient_K300", (96, 97, 96), 1000.0, 6000, lx=lx4, lz=lz4, krylov=300,
           max_newton=20, use_gradient=True)
    single("config4_96x97x96_re1000_lam_adv_K300", (96, 97, 96), 1000.0, 6000, lx=lx4, lz=lz4, lam_adv=1,
           krylov=300, max_newton=60)
    print(json.dumps(out))


def run_gint(args):
    """The paper's comparison (Sec. 3.3, Fig. 2 and the K-vs-T figure) on a synthetic stand-in:
    Newton-GMRES-hookstep on G^Stokes_T = B_T - I (one BEFE step of size T) and on
    G^int_T = (B_dt)^(T/dt) - I with dt = 1/32, for several T, at the paper's resolution
    48 x 35 x 48 and Re = 380, from a seeded perturbed-laminar state (amplitude 0.1; the
    paper's EQ1 field is not available). Reported per run: Newton steps, actions (GMRES
    iterations), timesteps (residual and trajectory steps plus T/dt per action) and wall time."""
    import torch
    torch.cuda.set_device(0)
    import paper_1804_05087_gb300 as sp
    import seeded_inputs as si
    nx, ny, nz, re, dt_int = 48, 35, 48, 380.0, 1.0 / 32
    runs = []
    for kind, T in (("stokes", 1.0), ("stokes", 10.0), ("stokes", 100.0), ("int", 0.125), ("int", 0.25),
                    ("int", 1.0)):
        dt = T if kind == "stokes" else dt_int
        n = 1 if kind == "stokes" else int(round(T / dt_int))
        ctx = sp.Context(sp.Config(nx, ny, nz, lx=LX, lz=LZ, re=re, dt=dt, prec=sp.SP_MIXED))
        ctx.sp_autotune(1)
        a, b, c = si.couette_random_coeffs(1000, nx, ny, nz)
        U = ctx.zeros()
        ctx.sp_seed_state(*[torch.from_numpy(x).cuda() for x in (a, b, c)], 0.1, U)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = ctx.sp_newton_gmres(U, max_newton=30, max_krylov=args.krylov, tol=1e-10, eta=1e-3, int_steps=n)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        steps = rep["total_steps"] + rep["total_jvps"] * n
        runs.append({"operator": "G^Stokes" if kind == "stokes" else "G^int", "T": T, "dt": dt,
                     "steps_per_action": n, "converged": rep["converged"], "newton_iters": rep["newton_iters"],
                     "actions": rep["total_jvps"],
                     "K_per_newton": rep["total_jvps"] / max(rep["newton_iters"], 1), "timesteps": steps,
                     "norm_F": rep["norm_F"], "wall_s": wall})
        ctx.close()
    best = {op: min((r for r in runs if r["operator"] == op and r["converged"]), key=lambda r: r["timesteps"],
                    default=None) for op in ("G^Stokes", "G^int")}
    out = {"metric": "timesteps and time to |G|<1e-10: G^Stokes_T vs G^int_T (dt = 1/32)", "unit": "timesteps",
           "higher_is_better": False,
           "config": {"workload": "plane Couette 48x35x48, Re=380, box 2pi/1.14 x 2 x 2pi/2.5, mixed precision, "
                                  "seeded perturbed-laminar state (amplitude 0.1, seed 1000)",
                      "max_krylov": args.krylov, "eta": 1e-3},
           "runs": runs}
    if best["G^Stokes"] and best["G^int"]:
        out["timestep_ratio_best_int_over_best_stokes"] = best["G^int"]["timesteps"] / best["G^Stokes"]["timesteps"]
        out["time_ratio_best_int_over_best_stokes"] = best["G^int"]["wall_s"] / best["G^Stokes"]["wall_s"]
    print(json.dumps(out))


def dense_jacobian(ctx, n_steps, batch=256):
    """Real Jacobian (state_len x state_len) of G (n_steps = 1: G^Stokes, > 1: G^int) at the
    linearisation point already set, one batched tangent launch per block of unit vectors."""
    import numpy as np
    import torch
    L = ctx.state_len
    J = np.empty((L, L))
    for i0 in range(0, L, batch):
        nb = min(batch, L - i0)
        D = ctx.zeros(nb)
        Dr = torch.view_as_real(D).reshape(nb, L)
        Dr[torch.arange(nb), torch.arange(i0, i0 + nb)] = 1.0
        out = ctx.zeros(nb)
        if n_steps > 1:
            ctx.sp_jvp_n(D, out)
        else:
            ctx.sp_jvp(D, out)
        J[:, i0:i0 + nb] = torch.view_as_real(out).reshape(nb, L).cpu().numpy().T
    return J


def hermitian_projection(ctx):
    """Matrix (real coordinates) of the projection onto Hermitian-consistent states that every
    map of the library applies to its input: in the kz = 0 plane, (a(ix) + conj a(-ix)) / 2.
    The tangent is J = P S P - P, so B_U = J + P and G_U vanishes on the range of I - P."""
    import numpy as np
    mx, mz, ny = ctx.MX, ctx.MZ, ctx.NY
    L = ctx.state_len
    P = np.eye(L)
    def idx(c, pos, iz, n):
        return 2 * (((c * mx + pos) * mz + iz) * ny + n)
    for c in range(3):
        for pos in range(mx):
            mpos = (mx - pos) % mx
            for n in range(ny):
                i, j = idx(c, pos, 0, n), idx(c, mpos, 0, n)
                P[i, i] = P[i + 1, i + 1] = 0.0
                P[i, i] += 0.5
                P[i, j] += 0.5          # Re: (a_re + b_re) / 2
                P[i + 1, i + 1] += 0.5
                P[i + 1, j + 1] -= 0.5  # Im: (a_im - b_im) / 2
    return P


def run_spectra(args):
    """Spectra of the Jacobians G_U (Sec. 3.3, the spectra figures and Eqs. beaumescale, lims,
    model, TRe) at laminar plane Couette flow on a 12 x 17 x 12 grid, FP64, Re 500 and 1750.
    Each Jacobian is built column by column from batched tangent actions on unit vectors and
    restricted to the physical subspace S (divergence-free, no-slip, Hermitian states: the range
    of one BEFE step), where G_U acts invariantly; outside S, G_U = -I. Eigenvalues on the host.
    Checks of the paper's model lambda_k = -k^2/Re +- i k U:
      * the most negative real eigenvalue of G^Stokes_(T = 1e-4), rescaled by (1 + T)/T, scales as
        1/Re;
      * the largest imaginary part of G^Stokes_100 (rescaled) scales as Re;
      * the radius r around -1 holding 95 % of the eigenvalues of G^int_T (dt = 1/32) obeys
        T/Re = ln(1/r)/k*^2: ln(1/r) ratios equal T ratios at fixed Re and inverse Re ratios at
        fixed T."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    import paper_1804_05087_gb300 as sp
    nx, ny, nz = 12, 17, 12
    dt_int = 1.0 / 32
    Q = None
    res = {}
    for re in (500.0, 1750.0):
        specs = {}
        for kind, T in (("stokes", 1e-4), ("stokes", 0.1), ("stokes", 100.0), ("int", 1.0), ("int", 10.0)):
            dt = T if kind == "stokes" else dt_int
            n = 1 if kind == "stokes" else int(round(T / dt_int))
            ctx = sp.Context(sp.Config(nx, ny, nz, lx=LX, lz=LZ, re=re, dt=dt, prec=sp.SP_FP64, max_batch=256))
            U = ctx.zeros()  # laminar flow
            ctx.sp_set_base_n(U, n)
            J = dense_jacobian(ctx, n)
            if Q is None:  # S = range of B_U = J + P (the same subspace for every T and Re)
                u_, sv, _ = np.linalg.svd(J + hermitian_projection(ctx))
                d = int(np.sum(sv > 1e-10 * sv[0]))
                Q = u_[:, :d]
            A = Q.T @ J @ Q
            inv = float(np.linalg.norm(J @ Q - Q @ A) / np.linalg.norm(J @ Q))
            ev = np.linalg.eigvals(A)
            if kind == "stokes":
                ev = ev * (1 + T) / T  # Eq. beaumescale
            specs[(kind, T)] = (ev, inv)
            ctx.close()
        st4, st100 = specs[("stokes", 1e-4)][0], specs[("stokes", 100.0)][0]
        r95 = {}
        for T in (1.0, 10.0):
            dist = np.sort(np.abs(specs[("int", T)][0] + 1.0))
            r95[T] = float(dist[int(np.ceil(0.95 * len(dist))) - 1])
        res[re] = {"subspace_dim": int(Q.shape[1]),
                   "invariance_residual_max": max(v[1] for v in specs.values()),
                   "stokes_1e-4_most_negative_real": float(st4.real.min()),
                   "stokes_0.1_real_range": [float(specs[("stokes", 0.1)][0].real.min()),
                                             float(specs[("stokes", 0.1)][0].real.max())],
                   "stokes_100_max_imag": float(np.abs(st100.imag).max()),
                   "stokes_100_frac_real_within_0.2_of_-1": float(np.mean(np.abs(st100.real + 1) < 0.2)),
                   "int_r95": r95}
    # laminar advection folded into L (Sec. 3.6): spectra of G^Stokes_100 and G'^Stokes_100 at
    # laminar flow and at a seeded perturbed state (amplitude 0.1), on the same subspace S
    import seeded_inputs as si
    for re in (500.0, 1750.0):
        la = {}
        for lam_adv in (0, 1):
            for amp in (0.0, 0.1):
                ctx = sp.Context(sp.Config(nx, ny, nz, lx=LX, lz=LZ, re=re, dt=100.0, prec=sp.SP_FP64,
                                           max_batch=256, lam_adv=lam_adv))
                U = ctx.zeros()
                if amp > 0:
                    a_, b_, c_ = si.couette_random_coeffs(1000, nx, ny, nz)
                    ctx.sp_seed_state(*[torch.from_numpy(x).cuda() for x in (a_, b_, c_)], amp, U)
                ctx.sp_set_base(U)
                J = dense_jacobian(ctx, 1)
                ev = np.linalg.eigvals(Q.T @ J @ Q) * (1 + 100.0) / 100.0
                dist = np.sort(np.abs(ev + 1.0))
                la[f"{'lam_adv' if lam_adv else 'stokes'}_amp{amp}"] = {
                    "max_imag": float(np.abs(ev.imag).max()), "max_dist_from_-1": float(dist[-1]),
                    "r95_around_-1": float(dist[int(np.ceil(0.95 * len(dist))) - 1])}
                ctx.close()
        res[re]["laminar_advection_in_L"] = la
    a, b = res[500.0], res[1750.0]
    out = {"metric": "Jacobian spectra: model scalings (Sec. 3.3)", "config": {
        "workload": "laminar plane Couette flow, 12x17x12, box 2pi/1.14 x 2 x 2pi/2.5, FP64; G^Stokes_T for "
                    "T = 1e-4, 0.1, 100 (rescaled by (1+T)/T), G^int_T for T = 1, 10 with dt = 1/32"},
        "Re500": a, "Re1750": b,
        "checks": {
            "most_negative_ratio_500_over_1750 (model: 3.5)": a["stokes_1e-4_most_negative_real"]
            / b["stokes_1e-4_most_negative_real"],
            "max_imag_ratio_1750_over_500 (model: 3.5)": b["stokes_100_max_imag"] / a["stokes_100_max_imag"],
            "ln(1/r95) ratio T=10 over T=1 at Re 500 (model: 10)": math.log(1 / a["int_r95"][10.0])
            / math.log(1 / a["int_r95"][1.0]),
            "ln(1/r95) ratio Re 500 over 1750 at T=10 (model: 3.5)": math.log(1 / a["int_r95"][10.0])
            / math.log(1 / b["int_r95"][10.0])}}
    print(json.dumps(out))


def run_config3(args):
    """Pipe flow in the frame moving with the wave (config 3): Re 2500, alpha 1.25, 2-fold
    symmetry, Nr 64, m' <= 12 (m <= 24), |kz| <= 24, 48 x 96 physical grid, dt 50.
    (1) tangent throughput (set_base + 64 directions) in mixed and FP64 precision;
    (2) Newton-GMRES-hookstep from Hagen-Poiseuille plus seeded streaks (amplitude 0.05 and a
    10 % divergence-free k != 0 part, c0 = 0.5) with the speed as an unknown."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    import paper_1804_05087_gb300 as sp
    import seeded_inputs as si
    nd = args.pipe_ndir
    out = {"metric": "config 3: pipe traveling-wave tangent throughput and Newton", "unit": "JVP/s",
           "config": {"workload": "pipe Re=2500, alpha=1.25, sym 2, Nr=64, m'<=12, |kz|<=24, 48x96, dt=50",
                      "directions": nd}, "throughput": {}}
    for name, prec in (("mixed", sp.SP_MIXED), ("fp64", sp.SP_FP64)):
        ctx = sp.Context(sp.PipeConfig(prec=prec, max_batch=nd))
        def seeded(seed, amp, frac, c0):
            st, pol = si.pipe_random_coeffs(seed, ctx.cfg.kz, ctx.cfg.mt)
            U = ctx.zeros()
            return ctx.sp_pipe_seed_state(st, pol, amp, frac, c0, U)
        U = seeded(4000, 0.05, 0.1, 0.5)
        D = ctx.zeros(nd)
        for i in range(nd):
            D[i].copy_(seeded(4100 + i, 1.0, 1.0, 0.1))
        J = ctx.zeros(nd)
        for _ in range(3):
            ctx.sp_set_base(U)
            ctx.sp_jvp(D, J)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        e0.record()
        for _ in range(reps):
            ctx.sp_set_base(U)
            ctx.sp_jvp(D, J)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out["throughput"][name] = {"ms_per_step": ms, "jvp_per_s": nd / (ms * 1e-3)}
        if prec == sp.SP_MIXED and not args.no_newton:
            U0 = U.clone()
            G = ctx.zeros()
            ctx.sp_step(U0, G)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = ctx.sp_newton_gmres(U, max_newton=20, max_krylov=args.krylov, tol=1e-10, eta=1e-3)
            torch.cuda.synchronize()
            rep["wall_s"] = time.perf_counter() - t0
            u, c = ctx.pipe_split(U)
            rep["speed_c"] = c
            rep["deviation_norm"] = float(torch.linalg.vector_norm(u))
            out["newton"] = rep
        ctx.close()
    print(json.dumps(out))


def run_lamadv(args):
    """Laminar advection folded into L (Sec. 3.6, the closing proposal) against the Stokes
    step: Krylov actions of one linear solve at fixed states, Newton-GMRES-hookstep to
    |F| < 1e-10 from perturbed-laminar guesses, and the tangent throughput at 48x65x48."""
    import torch
    torch.cuda.set_device(0)
    import paper_1804_05087_gb300 as sp
    import seeded_inputs as si

    def context(grid, re, lam_adv, max_batch=1):
        nx, ny, nz = grid
        ctx = sp.Context(sp.Config(nx, ny, nz, lx=LX, lz=LZ, re=re, dt=DT, prec=sp.SP_MIXED,
                                   max_batch=max_batch, lam_adv=lam_adv))
        return ctx

    def seeded(ctx, grid, seed, amp):
        a, b, c = si.couette_random_coeffs(seed, *grid)
        U = ctx.zeros()
        return ctx.sp_seed_state(*[torch.from_numpy(x).cuda() for x in (a, b, c)], amp, U)

    first_solve, newton = [], []
    for grid, re in (((16, 33, 16), 400.0), ((48, 35, 48), 380.0), ((32, 33, 32), 1000.0)):
        g = "x".join(map(str, grid))
        for lam_adv in (0, 1):
            ctx = context(grid, re, lam_adv)
            ctx.sp_autotune(1)
            # one Newton step: the Krylov dimension GMRES needs for eta = 1e-3 at the guess
            for amp in (0.1, 0.3):
                U = seeded(ctx, grid, 1000, amp)
                rep = ctx.sp_newton_gmres(U, max_newton=1, max_krylov=max(args.krylov, 1200), tol=1e-30)
                first_solve.append({"grid": g, "re": re, "amplitude": amp, "lam_adv": lam_adv,
                                    "actions": rep["total_jvps"]})
            U = seeded(ctx, grid, 1000, 0.1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = ctx.sp_newton_gmres(U, max_newton=30, max_krylov=args.krylov, tol=1e-10)
            torch.cuda.synchronize()
            newton.append({"grid": g, "re": re, "lam_adv": lam_adv, "converged": rep["converged"],
                           "newton_iters": rep["newton_iters"], "actions": rep["total_jvps"],
                           "norm_F": rep["norm_F"], "wall_s": time.perf_counter() - t0})
            ctx.close()

    # the short-recurrence solvers of Sec. 3.6 with and without laminar advection in L
    short = []
    grid = (16, 33, 16)
    for krylov, ell in (("bicgstab", 4), ("idr", 8)):
        for lam_adv in (0, 1):
            ctx = context(grid, 400.0, lam_adv)
            U = seeded(ctx, grid, 1000, 0.1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = ctx.sp_newton_gmres(U, max_newton=20, max_krylov=4000, tol=1e-10, krylov=krylov, ell=ell)
            torch.cuda.synchronize()
            short.append({"solver": f"{krylov}({ell})", "lam_adv": lam_adv, "converged": rep["converged"],
                          "newton_iters": rep["newton_iters"], "actions": rep["total_jvps"],
                          "norm_F": rep["norm_F"], "wall_s": time.perf_counter() - t0})
            ctx.close()

    # tangent throughput with the complex per-mode operators (48x65x48, 256 directions)
    grid, nd = (NX, NY, NZ), args.ndir
    thr = {}
    for lam_adv in (0, 1):
        ctx = context(grid, RE, lam_adv, max_batch=nd)
        U = seeded(ctx, grid, BASE_SEED, 0.1)
        D = ctx.zeros(nd)
        for i in range(nd):
            D[i].copy_(seeded(ctx, grid, DIR_SEED0 + i, 1.0))
        OUT = ctx.zeros(nd)
        tune = ctx.sp_autotune(nd)
        for _ in range(max(args.warmup, 3)):
            ctx.sp_set_base(U)
            ctx.sp_jvp(D, OUT)
        torch.cuda.synchronize()
        ctx.sp_trace_enable(True)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            ctx.sp_set_base(U)
            ctx.sp_jvp(D, OUT)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        tr = ctx.sp_trace_read()
        ctx.sp_trace_enable(False)
        solve_ms = tr["k_solve"][0] / tr["k_solve"][1]
        n = NY - 1
        flops = (nd * n_unique() * (la_op_entries() * 8 + (n - 1) * 18 + NY * 16) if lam_adv
                 else nd * n_unique() * (op_entries() * 4 + (n - 1) * 8 + NY * 16))
        thr["lam_adv" if lam_adv else "stokes"] = {
            "jvp_per_s": nd * args.steps / (ms * 1e-3), "k_solve_ms": solve_ms,
            "k_solve_tflops": flops / (solve_ms * 1e-3) / 1e12, "tile": tune["tangent"],
            "kernel_ms_per_step": {k: v[0] / args.steps for k, v in tr.items()}}
        ctx.close()
    out = {"metric": "Krylov actions and time to |F|<1e-10: laminar advection in L vs the Stokes step",
           "unit": "actions", "higher_is_better": False,
           "config": {"workload": "plane Couette, dt=100, seed 1000 perturbed-laminar guesses; tangent "
                                  f"throughput {NX}x{NY}x{NZ} Re {RE} {nd} directions, mixed",
                      "max_krylov": args.krylov, "eta": 1e-3},
           "first_solve": first_solve, "newton": newton, "short_recurrence_16x33x16_re400": short,
           "throughput": thr}
    print(json.dumps(out))


# seeded guesses (seed, amplitude, perturbed modes |ix|, |iz| <= mmax) from which Newton with
# laminar advection in L reached the spanwise-fundamental equilibrium at 48 x 35 x 48, Re 400
EQ_SEEDS = ((7123, 0.3, 1), (7143, 0.3, 1), (7159, 0.3, 1), (7156, 0.05, 1), (7207, 0.3, 2), (7220, 0.05, 2))


def find_equilibrium(sp, si, torch, grid=(48, 35, 48), re=400.0):
    """A nontrivial plane Couette equilibrium: Newton-GMRES-hookstep with laminar advection in
    L from seeded perturbed-laminar guesses, keeping the first root with weighted norm above
    0.2: the state with the box's fundamental spanwise streak pair and a mean-flow correction
    (norm 0.2243, energy input 1.43 times the laminar one at 48 x 35 x 48, Re 400). The other
    roots these guesses reach have norms 0.11 to 0.15. Which root a guess reaches depends on
    rounding along the Newton path, hence the list."""
    ctx = sp.Context(sp.Config(*grid, lx=LX, lz=LZ, re=re, dt=DT, prec=sp.SP_MIXED, lam_adv=1))
    tried = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for seed, amp, mmax in EQ_SEEDS:
        a, b, c = si.couette_random_coeffs(seed, *grid, mmax=mmax)
        U = ctx.zeros()
        ctx.sp_seed_state(*[torch.from_numpy(x).cuda() for x in (a, b, c)], amp, U)
        rep = ctx.sp_newton_gmres(U, max_newton=40, max_krylov=300, tol=1e-10)
        rep["norm_U"] = math.sqrt(ctx.sp_inner(U, U)[0])
        tried.append({"seed": seed, "amplitude": amp, "mmax": mmax, "converged": rep["converged"],
                      "norm_U": rep["norm_U"]})
        if rep["converged"] and rep["norm_U"] > 0.2:
            break
    torch.cuda.synchronize()
    rep["wall_s"] = time.perf_counter() - t0
    rep["tried"] = tried
    ctx.close()
    if not (rep["converged"] and rep["norm_U"] > 0.2):
        raise RuntimeError(f"no seeded guess reached the equilibrium: {tried}")
    return U, rep


def run_eq(args):
    """The Newton-performance experiment of Sec. 3.3 (figures on G^Stokes_T and G^int_T) from a
    nontrivial equilibrium instead of laminar flow: the equilibrium at Re 400 (48 x 35 x 48, the
    paper's box) is the initial guess at Re 380. G^Stokes_T = B_T - I for T = 1, 10, 100 (and
    with laminar advection in L); G^int_T = (B_dt)^(T/dt) - I with the same BEFE step at
    dt = 1/32 (the paper's dt; the explicit advection of this first-order step is unstable there
    for the largest kx, so only short T converge) and at dt = 1/256 (stable). Timesteps =
    residual steps + (actions x T/dt)."""
    import torch
    torch.cuda.set_device(0)
    import paper_1804_05087_gb300 as sp
    import seeded_inputs as si
    grid = (48, 35, 48)
    U400, rep0 = find_equilibrium(sp, si, torch)
    eq = {k: rep0[k] for k in ("converged", "newton_iters", "total_jvps", "norm_F", "wall_s", "norm_U", "tried")}
    runs = []
    cases = [("stokes", 100.0, None, 0, 30, 300), ("stokes", 10.0, None, 0, 30, 300), ("stokes", 1.0, None, 0, 30, 300),
             ("stokes", 100.0, None, 1, 30, 300), ("int", 0.25, 1 / 32, 0, 30, 300),
             ("int", 0.25, 1 / 256, 0, 12, 150), ("int", 1.0, 1 / 256, 0, 12, 150), ("int", 4.0, 1 / 256, 0, 8, 100)]
    for kind, T, dti, la, max_newton, max_krylov in cases:
        dt = T if kind == "stokes" else dti
        ns = 1 if kind == "stokes" else int(round(T / dti))
        ctx = sp.Context(sp.Config(*grid, lx=LX, lz=LZ, re=380.0, dt=dt, prec=sp.SP_MIXED, lam_adv=la))
        U = U400.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = ctx.sp_newton_gmres(U, max_newton=max_newton, max_krylov=max_krylov, tol=1e-10, int_steps=ns)
        torch.cuda.synchronize()
        it = max(rep["newton_iters"], 1)
        runs.append({"operator": "G^Stokes_T" if kind == "stokes" else "G^int_T", "T": T, "dt": dt,
                     "laminar_advection_in_L": bool(la), "converged": rep["converged"],
                     "newton_iters": rep["newton_iters"], "actions": rep["total_jvps"],
                     "K_per_newton_step": rep["total_jvps"] / it,
                     "timesteps": rep["total_steps"] + rep["total_jvps"] * ns,
                     "wall_s": time.perf_counter() - t0, "norm_F": rep["norm_F"],
                     "norm_U": math.sqrt(ctx.sp_inner(U, U)[0]), "caps": [max_newton, max_krylov]})
        ctx.close()
    out = {"metric": "timesteps and time to |F|<1e-10, continuation from an equilibrium (Re 400 -> 380)",
           "unit": "timesteps", "higher_is_better": False,
           "config": {"workload": "plane Couette 48x35x48, box 2pi/1.14 x 2 x 2pi/2.5, mixed tangent; initial "
                                  "guess: the equilibrium at Re 400 found from the seeded guesses of EQ_SEEDS; target Re 380", "eta": 1e-3},
           "equilibrium_search": eq, "runs": runs}
    st = [r for r in runs if r["operator"] == "G^Stokes_T" and r["T"] == 100.0 and not r["laminar_advection_in_L"]][0]
    conv_int = [r for r in runs if r["operator"] == "G^int_T" and r["converged"]]
    if conv_int and st["converged"]:
        fastest = min(conv_int, key=lambda r: r["timesteps"])
        out["ratio_timesteps_int_over_stokes"] = fastest["timesteps"] / st["timesteps"]
        out["ratio_time_int_over_stokes"] = fastest["wall_s"] / st["wall_s"]
        out["fastest_int"] = {"T": fastest["T"], "dt": fastest["dt"]}
    print(json.dumps(out))


def truncate_state(ctx_to, U, Kx_from):
    """Copy the retained modes of a plane Couette state onto a coarser grid (Fourier modes
    |ix| <= Kx, iz <= Kz of the target, Chebyshev degrees < NY of the target)."""
    out = ctx_to.zeros()
    MXf = 2 * Kx_from + 1
    for ix in range(-ctx_to.Kx, ctx_to.Kx + 1):
        out[:, ix % ctx_to.MX, :, :] = U[:, ix % MXf, :ctx_to.MZ, :ctx_to.NY]
    return out


def continue_in_re(sp, torch, grid, U, res, lam_adv=1):
    """Newton continuation of an equilibrium through the Reynolds numbers ``res``."""
    reps = []
    for re in res:
        ctx = sp.Context(sp.Config(*grid, lx=LX, lz=LZ, re=re, dt=DT, prec=sp.SP_MIXED, lam_adv=lam_adv))
        rep = ctx.sp_newton_gmres(U, max_newton=30, max_krylov=300, tol=1e-11)
        reps.append({"re": re, "converged": rep["converged"], "newton_iters": rep["newton_iters"],
                     "norm_F": rep["norm_F"], "norm_U": math.sqrt(ctx.sp_inner(U, U)[0])})
        ctx.close()
    return reps


def run_eq_spectra(args):
    """Spectra of the Jacobians at a nontrivial equilibrium (Sec. 3.5, the spectra figures at
    EQ1, Re 500): the equilibrium of --eq is continued from Re 400 to 500 at 48 x 35 x 48; its
    leading eigenvalue (the paper quotes 0.06 for EQ1 at Re 500) comes from power iteration on
    the tangent of the propagator B_dt^n (dt = 1/256, T = n dt = 5: mu = exp(lambda T)). The
    same equilibrium, truncated to 12 x 25 x 12 and re-converged, gives dense Jacobians of
    G^Stokes_T (T = 1e-4, 0.1, 100; rescaled by (1 + T)/T) and G^int_10 (dt = 1/256),
    restricted to the physical subspace; eigenvalues on the host."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    import paper_1804_05087_gb300 as sp
    import seeded_inputs as si
    big = (48, 35, 48)
    U, rep0 = find_equilibrium(sp, si, torch)
    cont = continue_in_re(sp, torch, big, U, (450.0, 500.0))
    # leading eigenvalue at 48 x 35 x 48, Re 500: power iteration on (B^n)_U
    dt, n = 1.0 / 256, 1280
    ctx = sp.Context(sp.Config(*big, lx=LX, lz=LZ, re=500.0, dt=dt, prec=sp.SP_MIXED))
    ctx.sp_set_base_n(U, n)
    v = ctx.zeros()
    a, b, c = si.couette_random_coeffs(4242, *big)
    ctx.sp_seed_state(*[torch.from_numpy(x).cuda() for x in (a, b, c)], 1.0, v)
    w = ctx.zeros()
    mus = []
    for _ in range(40):
        ctx.sp_jvp_n(v, w)
        w += v                                    # (B^n)_U v = G^int_U v + v
        mu = math.sqrt(ctx.sp_inner(w, w)[0] / ctx.sp_inner(v, v)[0])
        mus.append(mu)
        v = w / math.sqrt(ctx.sp_inner(w, w)[0])
    lead = {"mu": mus[-1], "lambda": math.log(mus[-1]) / (n * dt), "T": n * dt, "dt": dt,
            "mu_change_last": abs(mus[-1] - mus[-2]) / mus[-1]}
    ctx.close()
    # dense spectra on 12 x 25 x 12
    small = (12, 25, 12)
    cs = sp.Context(sp.Config(*small, lx=LX, lz=LZ, re=500.0, dt=DT, prec=sp.SP_MIXED, lam_adv=1))
    Us = truncate_state(cs, U, 15)
    cs.close()
    cont_small = continue_in_re(sp, torch, small, Us, (500.0,))
    specs = {}
    Q = None
    for kind, T in (("stokes", 1e-4), ("stokes", 0.1), ("stokes", 100.0), ("int", 10.0)):
        dts = T if kind == "stokes" else 1.0 / 256
        ns = 1 if kind == "stokes" else int(round(T / dts))
        ctx = sp.Context(sp.Config(*small, lx=LX, lz=LZ, re=500.0, dt=dts, prec=sp.SP_FP64, max_batch=256))
        ctx.sp_set_base_n(Us, ns)
        J = dense_jacobian(ctx, ns)
        if Q is None:
            u_, sv, _ = np.linalg.svd(J + hermitian_projection(ctx))
            d = int(np.sum(sv > 1e-10 * sv[0]))
            Q = u_[:, :d]
        ev = np.linalg.eigvals(Q.T @ J @ Q)
        if kind == "stokes":
            ev = ev * (1 + T) / T
        dist = np.sort(np.abs(ev + 1.0))
        specs[f"{kind}_{T:g}"] = {
            "most_negative_real": float(ev.real.min()), "max_real": float(ev.real.max()),
            "max_imag": float(np.abs(ev.imag).max()),
            "frac_real_within_0.2_of_-1": float(np.mean(np.abs(ev.real + 1) < 0.2)),
            "r95_around_-1": float(dist[int(np.ceil(0.95 * len(dist))) - 1]),
            "largest_real_parts": [float(x) for x in np.sort(ev.real)[::-1][:3]]}
        ctx.close()
    out = {"metric": "Jacobian spectra at a nontrivial equilibrium (Re 500)", "config": {
        "workload": "equilibrium of --eq continued to Re 500 (48x35x48; leading eigenvalue by power iteration "
                    "on the propagator, dt = 1/256, T = 5); dense spectra on 12x25x12 (re-converged there), "
                    "FP64 tangent, restricted to the physical subspace"},
        "equilibrium_search": {k: rep0[k] for k in ("converged", "newton_iters", "norm_F", "norm_U", "tried")},
        "continuation_48x35x48": cont, "leading_eigenvalue_48x35x48": lead,
        "continuation_12x25x12": cont_small, "subspace_dim": int(Q.shape[1]), "spectra_12x25x12": specs}
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.newton:
        return run_newton(args)
    if args.config2:
        return run_config2(args)
    if args.config3:
        return run_config3(args)
    if args.gint:
        return run_gint(args)
    if args.spectra:
        return run_spectra(args)
    if args.config4:
        return run_config4(args)
    if args.lamadv:
        return run_lamadv(args)
    if args.eq:
        return run_eq(args)
    if args.eq_spectra:
        return run_eq_spectra(args)
    if args.convergence:
        return run_convergence(args)
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import paper_1804_05087_gb300 as sp

    global LAM_ADV
    LAM_ADV = bool(args.lam_adv)
    head = throughput(args, args.prec, rank, world, local, keep_out=True)
    other = None
    if not args.single_prec:
        # the other precision on the same inputs, with its per-field error against FP64
        oth = "mixed" if args.prec == "fp64" else "fp64"
        o = throughput(args, oth, rank, world, local, keep_out=True, e2e=False)
        f64, mix = (head, o) if args.prec == "fp64" else (o, head)
        err = field_errors(f64["out"], mix["out"])
        other = {k: o[k] for k in ("value", "unit", "ms_per_step", "dtype", "roofline", "gpu_launches")}
        other["precision"] = oth
        other["per_field_rel_err_vs_fp64"] = err
    peak = None
    if rank == 0:
        peak = measure_fp64_peak(sp, torch, local)
        for r in (head, other):
            if r is not None:
                attach_fp64_peak(r["roofline"], peak)
    ttc = None
    if rank == 0 and world == 1 and not args.no_newton:
        ttc = time_to_converge(args)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, n, el = oracle_jvps(12.0)
        cpu = {"value": rate, "unit": "JVP/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n} FP64 oracle tangent steps at 48x65x48 in {el:.1f} s (after its one-time LU setup)"}

    if rank == 0:
        nd = args.ndir
        out = {"metric": METRIC, "value": head["value"], "unit": "JVP/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": head["dtype"], "data": "synthetic",
               "config": {"workload": f"plane Couette 48x65x48, Re=400, dt=100, box 2pi/1.14 x 2 x 2pi/2.5; "
                                      f"per step: set_base + tangent on {nd} seeded unit directions",
                          "grid": [NX, NY, NZ], "ndir_per_gpu": nd, "precision": args.prec,
                          "laminar_advection_in_L": bool(args.lam_adv),
                          "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}",
                          "solve_tile": head["solve_tile"]},
               "roofline": head["roofline"], "cpu_baseline": cpu, "e2e": head["e2e"],
               "gpu_launches": head["gpu_launches"], "clocks": head["clocks"]}
        if other is not None:
            out["mixed" if other["precision"] == "mixed" else "fp64"] = other
        if peak is not None:
            out["fp64_peak_probe"] = peak
        if ttc is not None:
            out["time_to_converge"] = ttc
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def throughput(args, prec_name, rank, world, local, keep_out=False, e2e=True):
    """The timed step (set_base + tangent on the batch) in one precision."""
    import torch
    import paper_1804_05087_gb300 as sp
    import seeded_inputs as si
    prec = sp.SP_MIXED if prec_name == "mixed" else sp.SP_FP64
    esz = 8 if prec_name == "mixed" else 16
    nd = args.ndir
    ctx = sp.Context(sp.Config(NX, NY, NZ, lx=LX, lz=LZ, re=RE, dt=DT, prec=prec, max_batch=nd,
                               lam_adv=1 if args.lam_adv else 0))

    def seeded(seed, amp):
        a, b, c = si.couette_random_coeffs(seed, NX, NY, NZ)
        U = ctx.zeros()
        tr = [torch.from_numpy(x).cuda() for x in (a, b, c)]
        return ctx.sp_seed_state(*tr, amp, U)
    U = seeded(BASE_SEED, 0.1)
    D = ctx.zeros(nd)
    dir_seeds = rank_direction_seeds(rank, nd)
    for i in range(nd):
        D[i].copy_(seeded(dir_seeds[i], 1.0))
    OUT = ctx.zeros(nd)
    stream = torch.cuda.current_stream()
    tune = ctx.sp_autotune(nd)  # tile shapes of the solve kernel, before any timing

    def step():
        ctx.sp_set_base(U)
        ctx.sp_jvp(D, OUT)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(local)
    ctx.sp_trace_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    trace = ctx.sp_trace_read()
    ctx.sp_trace_enable(False)
    clk = clocks.stop()
    ms = max_over_ranks(ms, world)
    value = aggregate_rate(world, nd, args.steps, ms)
    launches = int(sum(v[1] for v in trace.values()))

    # end to end through the public API with host buffers (pinned), copies timed
    e2e_rec = None
    if e2e and not args.no_e2e:
        hD = D.cpu().pin_memory()
        hU = U.cpu().pin_memory()
        hO = torch.empty_like(hD).pin_memory()
        dU = torch.empty_like(U)

        def step_e2e():
            # the base state from host memory, then the directions through the host-buffer
            # tangent (copies in and out overlap the computation of neighbouring chunks)
            dU.copy_(hU, non_blocking=True)
            ctx.sp_set_base(dU)
            ctx.sp_jvp_host(hD, hO)
        for _ in range(3):
            step_e2e()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step_e2e()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_e = e0.elapsed_time(e1)
        ms_e = max_over_ranks(ms_e, world)
        e2e_rec = {"value": aggregate_rate(world, nd, args.steps, ms_e), "unit": "JVP/s",
                   "h2d_bytes_per_step": hD.numel() * 16 + hU.numel() * 16, "d2h_bytes_per_step": hO.numel() * 16}

    # roofline of the dominant kernel (live CUDA-event durations on the launching stream)
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        peaks = json.load(f)
    dom = max(("k_yinv", "k_xz", "k_rhs", "k_solve"), key=lambda k: trace[k][0] if trace[k][1] else -1.0)
    dom_ms, dom_n = trace[dom]
    avg_s = dom_ms / dom_n * 1e-3
    bytes_l = kernel_bytes(dom, nd, esz)  # every tangent launch processes the whole batch
    flops_l = kernel_flops(dom, nd, prec_name)
    gbs = bytes_l / avg_s / 1e9
    tfs = flops_l / avg_s / 1e12
    hbm = peaks["hbm_gbs"]
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FP32 lanes x FMA x max clock
    fp64_bound = prec_name == "fp64" or dom == "k_solve"  # the solve is FP64 in both modes
    alu_peak = FP64_NOMINAL if fp64_bound else fp32_peak
    if gbs / hbm >= tfs / alu_peak:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    else:
        roof = {"bound": "alu", "achieved": tfs, "peak": alu_peak, "unit": "TFLOP/s", "frac": tfs / alu_peak,
                "peak_source": f"nominal FP64 {FP64_NOMINAL} TFLOP/s" if fp64_bound
                else "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz", "fp64": fp64_bound}
    roof.update({"kernel": dom, "traffic": kernel_traffic(dom, nd, prec_name, bool(args.lam_adv)),
                 "avg_launch_ms": dom_ms / dom_n,
                 "algorithmic_bytes_per_launch": bytes_l, "algorithmic_flops_per_launch": flops_l,
                 "kernel_ms_per_step": {k: v[0] / args.steps for k, v in trace.items()}})
    rec = {"value": value, "unit": "JVP/s", "ms_per_step": ms / args.steps, "dtype": "f64" if prec_name == "fp64"
           else "f32+f64", "roofline": roof, "e2e": e2e_rec, "gpu_launches": launches, "clocks": clk,
           "solve_tile": {"tangent": list(tune["tangent"]), "step": list(tune["step"])}}
    if keep_out:
        rec["out"] = OUT.cpu().numpy()
    return rec


def field_errors(ref, got):
    """Per velocity component: max |got - ref| / max |ref| over the batch."""
    import numpy as np
    out = {}
    for c, name in enumerate(("u", "v", "w")):
        r = ref[:, c]
        out[name] = float(np.max(np.abs(got[:, c] - r)) / np.max(np.abs(r)))
    return out


def measure_fp64_peak(sp, torch, local, blocks=152 * 8, iters=2048, reps=5):
    """FP64 FMA rate of this device (the library's probe), timed with CUDA events on the
    launching stream, clocks sampled meanwhile. TFLOP/s = 4096 blocks iters / time."""
    buf = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):
        sp.probe_fp64_fma(buf, blocks, iters)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        sp.probe_fp64_fma(buf, blocks, iters)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    clk = clocks.stop()
    return {"tflops": 4096.0 * blocks * iters / (ms * 1e-3) / 1e12, "ms_per_launch": ms, "clocks": clk,
            "how": f"sp_probe_fp64_fma: {blocks} blocks x 256 threads x 8 chains x {iters} FMAs, mean of {reps}"}


def attach_fp64_peak(roof, peak):
    """Use the measured FP64 rate as the ALU denominator of an FP64-bound roofline."""
    if roof.get("bound") != "alu" or not roof.get("fp64"):
        return
    roof["peak"] = peak["tflops"]
    roof["frac"] = roof["achieved"] / peak["tflops"]
    roof["peak_source"] = "measured FP64 FMA rate (fp64_peak_probe)"


def time_to_converge(args):
    """Secondary metric: time to |G(U)| < 1e-10 (Newton-GMRES-hookstep) at 16x33x16, Re 400,
    from the seeded amplitude-0.1 state: the mixed tangent (graph-replayed Arnoldi steps)
    against the plain FP64 GPU path (finite-difference actions, no graphs) and the FP64
    tangent."""
    import torch
    import paper_1804_05087_gb300 as sp
    import seeded_inputs as si
    nx, ny, nz = 16, 33, 16
    res = {}
    for name, prec, fd, graphs in (("mixed_tangent", sp.SP_MIXED, False, True),
                                   ("fp64_tangent", sp.SP_FP64, False, True),
                                   ("plain_fp64_fd", sp.SP_FP64, True, False)):
        ctx = sp.Context(sp.Config(nx, ny, nz, lx=LX, lz=LZ, re=RE, dt=DT, prec=prec))
        ctx.sp_autotune(1)
        a, b, c = si.couette_random_coeffs(1000, nx, ny, nz)
        U = ctx.zeros()
        ctx.sp_seed_state(*[torch.from_numpy(x).cuda() for x in (a, b, c)], 0.1, U)
        if graphs:  # capture the Arnoldi graphs outside the timing (a warm start from the same guess)
            W = U.clone()
            ctx.sp_newton_gmres(W, max_newton=1, max_krylov=args.krylov, tol=1e-10, eta=1e-3, use_fd=fd,
                                use_graphs=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = ctx.sp_newton_gmres(U, max_newton=30, max_krylov=args.krylov, tol=1e-10, eta=1e-3, use_fd=fd,
                                  use_graphs=graphs)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        res[name] = {"seconds": wall, "converged": bool(rep["converged"]), "newton_steps": rep["newton_iters"],
                     "actions": rep["total_jvps"], "norm_F": rep["norm_F"], "t_action_ms": rep["t_action_ms"],
                     "t_orth_ms": rep["t_orth_ms"]}
    return {"metric": "time to |F|<1e-10 vs plain FP64 GPU", "unit": "s", "higher_is_better": False,
            "workload": f"plane Couette 16x33x16, Re=400, dt=100, seed 1000, amplitude 0.1, K <= {args.krylov}, "
                        "eta 1e-3",
            "runs": res, "speedup_mixed_vs_plain_fp64": res["plain_fp64_fd"]["seconds"] / res["mixed_tangent"]["seconds"]}


if __name__ == "__main__":
    main()
