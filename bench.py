#!/usr/bin/env python
"""Benchmark of the FEM-PIC particle step on GB300 (one JSON line on rank 0).

A step is one pass of the hot path over one batch of synthetic input: the periodic
cell sort (every --sort-every steps), the particle push with gather, tet walk and
charge-conserving deposit for every species, the implicit field step (Newmark,
Gauss-law projection, Faraday) and the FP64 invariant residuals (continuity and
magnetic Gauss law, logged every timed step).  Default workload (the largest that fits
one GPU): cube 96^3 x 6 tets with +-10% jitter, 50M electrons + 50M ions (mass ratio
1836), Bx = 0.2 T, dt = 0.2 electron gyro-periods, FP32 particle path, 50 timed steps.
The 32^3 / 2M-electron workload is measured after it in the same run (--also) and
reported under "workloads".

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run, one independent replica per GPU (weak scaling, no collective
on the data path; timing uses a barrier and the max over ranks).
--impl reference times the FP64 CPU oracle on host cores on the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/sec at stated FP32 error; field-solve ms/step learned vs plain CG"
UNIT = "particle-steps/s"
# nominal HBM3e bandwidth of one GB300, for fractions quoted beside the measured copy peak
NOMINAL_HBM_GBS = 7900.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", type=int, default=5, choices=[1, 2, 3, 5])
    ap.add_argument("--also", default="2",
                    help="further workloads measured after the headline one in the same run (timed steps and "
                         "per-kernel times only), comma-separated; empty: none")
    ap.add_argument("--scale", type=float, default=1.0, help="particle-count scale (tests only)")
    ap.add_argument("--mesh", type=int, default=0,
                    help="mesh resolution n of the workload's n^3 x 6 cube instead of its own, with the same "
                         "particles per tet and displacement per step in cells (profiling cases)")
    ap.add_argument("--deposits", default="change", choices=["change", "change64", "fp32", "fp64"],
                    help="deposit arrays: change (float dG, double Q carried from step to step by each "
                         "particle's charge change, FP_CHARGE_CHANGE; at 96^3 with Chebyshev-Jacobi solves it "
                         "cut the Gauss-law projection from 32.7 to 17.9 inner iterations, 6.1 -> 3.4 ms, for "
                         "0.16 ms more push and walk), fp32 (float dG and Q, the end-point charge) or fp64 "
                         "(double dG and Q: 121 -> 104 learned projection iterations, push and walk 0.6 ms "
                         "slower); change64 is change with a double dG as well")
    ap.add_argument("--sort-every", type=int, default=0,
                    help="steps between cell sorts (0: the workload's own: 2 for the drifting beam, whose cell "
                         "order decays fastest, 10 otherwise; negative: never)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-field", action="store_true", help="skip timing the oracle's field step")
    ap.add_argument("--no-graphs", action="store_true", help="launch eagerly instead of replaying CUDA graphs")
    ap.add_argument("--no-field", action="store_true", help="particle step only (no implicit field solve)")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--max-iter", type=int, default=2000)
    ap.add_argument("--solver", default="mixed,mixed",
                    help="field CG for the Newmark and Gauss systems: mixed (refinement) or fp64, e.g. mixed,fp64")
    ap.add_argument("--inner-tol", type=float, default=1e-5)
    ap.add_argument("--poly", default="3,8",
                    help="Chebyshev degree of the inner preconditioner, Newmark and Gauss systems (1 = Jacobi)")
    ap.add_argument("--poly-ratio", default="15,100",
                    help="lambda_max / lambda_low of the Chebyshev interval, Newmark and Gauss systems")
    ap.add_argument("--learned", default="auto", choices=["auto", "off", "on"],
                    help="learned preconditioners of the Newmark and Gauss-law solves: trained by the protocol on "
                         "the 4^3 and 32^3 workloads, each used in the timed steps if it beats plain CG and the "
                         "configured polynomial (auto)")
    ap.add_argument("--learned-systems", default="newmark,gauss",
                    help="systems whose learned correction is trained and compared with plain CG (newmark, gauss)")
    ap.add_argument("--proto-systems", type=int, default=1000,
                    help="field systems collected per workload (4^3 and 32^3) for the learned preconditioner; "
                         "a tenth of them are held out")
    ap.add_argument("--proto-rounds", type=int, default=6,
                    help="training rounds; each trains a few epochs on each workload in turn")
    ap.add_argument("--proto-epochs", type=int, default=3, help="epochs per workload per round")
    ap.add_argument("--compare-steps", type=int, default=20)
    ap.add_argument("--tune-systems", type=int, default=64,
                    help="systems of the measured workload's own steps the learned preconditioners are fine-tuned "
                         "on (96^3 Newmark: 32 systems x 8 epochs 36.8 inner iterations, 32 x 24 and 64 x 16 35.0)")
    ap.add_argument("--tune-epochs", type=int, default=16)
    ap.add_argument("--tune-seeds", type=int, default=2,
                    help="fine-tunes of the learned preconditioner from the protocol's weights, one per training "
                         "seed, each timed on the comparison steps; the fastest is kept (the iteration count "
                         "of one fine-tune varied from 35 to 40 between runs)")
    ap.add_argument("--fp64-steps", type=int, default=10,
                    help="timed particle steps of the FP64 mode in a context of its own (0: skip)")
    ap.add_argument("--neumann-steps", type=int, default=10,
                    help="timed field steps with the natural (Neumann) field boundary (0: skip)")
    ap.add_argument("--adams-steps", type=int, default=20,
                    help="timed calls of the fourth-order Adams particle step (0: skip that measurement)")
    ap.add_argument("--drift-steps", type=int, default=-1,
                    help="steps of the Gauss-law comparison of the projected step with the unprojected "
                         "first-order mixed FEM and wave-equation FEM (0: skip; -1: 200 on the 32^3 and "
                         "smaller workloads, 0 on the larger ones)")
    ap.add_argument("--drift-tol", type=float, default=1e-6,
                    help="second run of the Gauss-law comparison with this solver tolerance for the two "
                         "unprojected systems (the projected step keeps --tol; 0: skip)")
    ap.add_argument("--min-warmup-s", type=float, default=1.5,
                    help="keep warming up at least this long (clock sampling under load)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time (the whole job's), on every rank; ms itself for one rank."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(units: float, world: int, device) -> float:
    """The units all ranks processed, on every rank."""
    if world <= 1:
        return float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_all_ranks: float, ms_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_all_ranks / (ms_max * 1e-3)


# ------------------------------------------------------------------ clocks

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def clocks_start(gpu_index: int):
    path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
    try:
        f = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={CLOCK_FIELDS}",
                              "--format=csv,noheader,nounits", "-lms", "200"], stdout=f,
                             stderr=subprocess.DEVNULL)
        return p, f, path
    except Exception:
        return None, None, path


def clocks_stop(handle) -> dict:
    p, f, path = handle
    if p is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    f.close()
    sm, smax, reasons, busy = [], [], set(), []
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        c = [x.strip() for x in line.split(",")]
        if len(c) < 10:
            continue
        try:
            mhz, mx, util = float(c[1]), float(c[2]), float(c[4])
        except ValueError:
            continue
        smax.append(mx)
        if util >= 50:
            busy.append(mhz)
            for k, nm in enumerate(names):
                if c[6 + k].lower().startswith("active"):
                    reasons.add(nm)
        sm.append(mhz)
    os.unlink(path)
    use = busy if busy else sm
    return {"sm_mhz": statistics.median(use) if use else None, "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm), "samples_busy": len(busy)}


# ------------------------------------------------------------------ workload

def build_workload(args):
    from paper_2103_06737_gb300 import inputs as I
    return I.config(args.workload, args.scale, mesh_n=args.mesh)


def algorithmic_bytes(n_particles, sizes, real_bytes=4):
    """Minimal DRAM bytes of one push_deposit launch over all species (stated reading):
    particle state read+write (cell + 3 off + 3 vel), each tet's tables once (96 B FP64
    geometry + 80 B topology), each e and b DOF once (FP64), dG and Q read-modify-write."""
    state = n_particles * 2 * (4 + 6 * real_bytes)
    tets = sizes["n_tets"] * (96 + 80)
    dofs = 8 * (sizes["n_edges"] + sizes["n_faces"])
    dep = 2 * real_bytes * (sizes["n_edges"] + sizes["n_nodes"])
    return state + tets + dofs + dep


def fast_kernel_bytes(n_particles, sizes, dep_bytes=4, q_bytes=None):
    """Minimal DRAM bytes of one fast-push launch (k_push_run32): cell + off + vel read (28 B) and
    off + vel written (24 B) per particle, each tet's 128-byte record once, dG and Q
    read-modify-write once (dep_bytes per element: 4 for float, 8 for double deposit arrays)."""
    q_bytes = dep_bytes if q_bytes is None else q_bytes
    return n_particles * 52 + sizes["n_tets"] * 128 + 2 * (dep_bytes * sizes["n_edges"] + q_bytes * sizes["n_nodes"])


def adams_kernel_bytes(n_particles, sizes):
    """Minimal DRAM bytes of one fourth-order Adams fast-push launch: the fast
    Boris launch's bytes plus the derivative history, 3 slots x (v, a) read (72 B) and the new
    slot written (24 B) per particle."""
    return fast_kernel_bytes(n_particles, sizes) + 96 * n_particles


def cg_iter_bytes(n_rows, nnz):
    """Algorithmic DRAM bytes of one Jacobi-PCG iteration as the hot-path table states them:
    the FP64 SpMV (8 B value + 4 B column per nonzero; per row 8 B in, 8 B out, 4 B row
    pointer) and the PCG vector traffic (7 FP64 passes), 12 B per nonzero + 76 B per row."""
    return 12 * nnz + 76 * n_rows


def push_call_bytes(n_particles, n_tets):
    """Algorithmic DRAM bytes of one push call (FP32) as the hot-path table states them: 56 B
    of particle state per particle (28 B read, 28 B written) and about 230 B per tet (its
    record, its e and b values and the read-modify-write of its 10 deposit targets)."""
    return 56 * n_particles + 230 * n_tets


L2_BYTES = 129e6


def pcg_bytes_per_iter(n_rows, nnz, val_bytes=8):
    """Minimal DRAM bytes of one FP64 Jacobi-PCG iteration (two barriers per iteration): the
    operator once (value + column index per nonzero) and 13 passes over n-vectors
    (update: x, r read+write, p, q, diag^-1 read, z write; search: z, p, q read, p, q write)."""
    return nnz * (val_bytes + 4) + 13 * 8 * n_rows


def mixed_solve_bytes(n_rows, nnz, inner_iters, outer, deg=1):
    """Minimal DRAM bytes of one mixed-precision solve: per FP32 inner PCG iteration the FP32
    operator once (4 B value + 4 B column per nonzero) and 13 FP32 vector passes (update: c,
    r read+write, p, q, diag^-1 read, z written; search: z, p, q read, p, q written); with a
    Chebyshev preconditioner of degree deg > 1, per application 5 vector passes to start it (r,
    diag^-1 read; d, z, s written) and deg - 1 further products with 7 vector passes each (d,
    s, diag^-1, z read; s, d, z written); per refinement the start of the inner solve (one
    preconditioner application, one FP32 product, r64 and diag^-1 read, r, z, p, q written)
    and the FP64 update x += |r| c; outer + 1 FP64 residuals b - A x (12 B per nonzero, b and x
    read, r64 written, c cleared)."""
    prec = 0 if deg <= 1 else 5 * 4 * n_rows + (deg - 1) * (nnz * 8 + 7 * 4 * n_rows)
    inner = inner_iters * (nnz * 8 + 13 * 4 * n_rows + prec)
    start = outer * (prec + nnz * 8 + (8 + 4 + 4 * 4) * n_rows + (8 + 8 + 4) * n_rows)
    resid = (outer + 1) * (nnz * 12 + (8 + 8 + 8 + 4) * n_rows)
    return inner + start + resid


def measured_traffic(kernel: str, workload: str, iterations=None):
    """DRAM bytes per launch (read + write) of `kernel` from the ncu capture recorded in
    profiles/traffic.json (key kernel@workload), or None when there is none for this workload
    or any source file the kernel is built from has changed since the capture (sha256 recorded
    with it).  A solver
    record holds bytes per inner iteration (its launches' bytes over their iterations), scaled
    here by this run's iterations per launch."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[f"{kernel}@{workload}"]
    except Exception:
        return None
    for path, digest in rec.get("sources", {}).items():
        try:
            with open(os.path.join(ROOT, path), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != digest:
                    return None
        except OSError:
            return None
    if "dram_bytes_per_iteration" in rec:
        return None if iterations is None else float(rec["dram_bytes_per_iteration"]) * float(iterations)
    return float(rec["dram_bytes_per_launch"])


def peak_hbm():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def set_deposits(args, lib, F):
    """The deposit arrays' element types for the --deposits choice."""
    if args.deposits in ("fp64", "change64"):
        lib.set_deposit_precision(F.FP_FP64)
    elif args.deposits == "change":
        lib.set_charge_precision(F.FP_FP64)


def learned_protocol(args, dev):
    """Training and evaluation protocol of the learned preconditioner (the FP_LEARNED_PRECOND
    network) on both field systems, Newmark (edge graph) and Gauss-law projection (node graph).
    Field systems come from PIC runs of the 4^3 / 1,000-electron and the 32^3 / 2M-electron
    workloads: the residual of each solve's start, one per system per step, args.proto_systems
    steps per workload, the last tenth held out.  One network per system is trained on both
    workloads' training systems (rounds of a few epochs on each workload in turn, the weights
    carried from one to the other).  The held-out steps are then run again from the same state
    with plain Jacobi-CG and with the learned preconditioner, both in the mixed solver to
    args.tol: iterations and CUDA-event time per solve.  Returns the report and the weights."""
    import torch
    import paper_2103_06737_gb300.fem_pic as F
    from paper_2103_06737_gb300 import inputs as I
    t0 = time.time()
    n_sys = max(20, args.proto_systems)
    n_hold = max(2, n_sys // 10)
    n_train = n_sys - n_hold
    systems = ((F.FP_SYS_NEWMARK, F.FP_PC_LEARNED, "newmark", "cg_newmark"),
               (F.FP_SYS_GAUSS, F.FP_PC_LEARNED_GAUSS, "gauss", "cg_gauss"))
    runs = []
    for idx in (1, 2):
        wl = I.config(idx)
        lib = F.FemPic(wl.mesh.xyz, wl.mesh.tets, F.FP_FP32)
        set_deposits(args, lib, F)
        cflag = F.FP_CHARGE_CHANGE if args.deposits.startswith("change") else 0
        sizes = lib.sizes
        sps = []
        for s_ in wl.species:
            d0 = lib.species(s_.cell, s_.X, s_.V, s_.q, s_.m, s_.w, device=dev)
            d1 = d0.empty_like()
            lib.sort(d0, d1)
            sps.append(d1)
        e, b = lib.fields_uniform((0.0, 0.0, 0.0), wl.B0, device=dev)
        ne, nn = sizes["n_edges"], sizes["n_nodes"]
        dG = torch.zeros(ne, dtype=lib.deposit_dtype, device=dev)
        dGp = torch.zeros_like(dG)
        Qn = torch.zeros(nn, dtype=lib.charge_dtype, device=dev)
        Qo = torch.zeros_like(Qn)
        Q_ion = torch.zeros_like(Qn)
        if wl.background_ions:
            alpha = F.fem_pic_whitney0_integrals(lib.h)
            qtot = sum(s_.q * s_.w * s_.n for s_ in sps)
            Q_ion.copy_(torch.as_tensor(-qtot * alpha / alpha.sum(), device=dev))
        Ep = torch.zeros(ne, dtype=torch.float64, device=dev)
        En = torch.zeros_like(Ep)
        F.fem_pic_field_setup(lib.h, wl.dt)
        F.fem_pic_field_options(lib.h, F.FP_PC_JACOBI, F.FP_PC_JACOBI, args.inner_tol)
        for sys_id, _, _, _ in systems:
            F.fem_pic_field_poly(lib.h, sys_id, 1, 30.0)       # plain Jacobi inner preconditioner
            F.fem_pic_learned_select(lib.h, sys_id)
            F.fem_pic_learned_init_model(lib.h, seed=7 + sys_id, sample_capacity=n_sys, model=F.FP_LEARNED_PRECOND)
            F.fem_pic_learned_mode(lib.h, collect=True, active=False)
        Qo.copy_(Q_ion)
        for k, s_ in enumerate(sps):
            lib.deposit_charge(s_, Qo, flags=F.FP_ACCUMULATE)
        st0, inf0 = F.fem_pic_field_initial(lib.h, Qo, e, tol=args.tol)
        Ep.copy_(e)

        def step(pc, lib=lib, sps=sps, e=e, b=b, dG=dG, dGp=dGp, Qn=Qn, Qo=Qo, Q_ion=Q_ion, Ep=Ep, En=En, wl=wl,
                 cflag=cflag):
            dG.zero_()
            Qn.copy_(Qo if cflag else Q_ion)     # the charge change is added onto Q^n
            for k, s_ in enumerate(sps):
                lib.push_deposit(e, b, s_, wl.dt, dG, Qn,
                                 flags=F.FP_ACCUMULATE | cflag | (F.FP_SAME_FIELDS if k else 0))
            F.fem_pic_field_step(lib.h, Ep, e, En, b, dG, dGp, Qn, tol=args.tol, max_iter=args.max_iter,
                                 precond=pc, info=False)
            Qo.copy_(Qn)
            dGp.copy_(dG)
            Ep.copy_(e)
            e.copy_(En)
        for k in range(n_train):
            step(F.FP_PC_JACOBI)
        torch.cuda.synchronize()
        snap = [t_.clone() for t_ in (e, b, Ep, dGp, Qo)] + [(s_.cell.clone(), s_.off.clone(), s_.vel.clone())
                                                             for s_ in sps]
        for k in range(n_hold):
            step(F.FP_PC_JACOBI)
        torch.cuda.synchronize()
        for sys_id, _, _, _ in systems:
            F.fem_pic_learned_select(lib.h, sys_id)
            F.fem_pic_learned_mode(lib.h, collect=False, active=False)
        st = lib.status()
        if st != F.FP_OK:
            raise RuntimeError(f"learned protocol, workload {wl.name}: status {st}: {F.fem_pic_last_error(lib.h)}")

        def restore(snap=snap, e=e, b=b, Ep=Ep, dGp=dGp, Qo=Qo, sps=sps):
            for t_, c_ in zip((e, b, Ep, dGp, Qo), snap[:5]):
                t_.copy_(c_)
            for s_, (c_, o_, v_) in zip(sps, snap[5:]):
                s_.cell.copy_(c_)
                s_.off.copy_(o_)
                s_.vel.copy_(v_)
        runs.append({"wl": wl, "lib": lib, "step": step, "restore": restore,
                     "alive": sum(int((s_.cell >= 0).sum()) for s_ in sps)})
    t_collect = time.time() - t0
    # training: one network per system on both workloads' training systems
    params, report = {}, {"workloads": [r["wl"].name for r in runs], "systems_per_workload": n_sys,
                          "held_out_per_workload": n_hold, "train_per_workload": n_train,
                          "collect_s": t_collect}
    for sys_id, bit, name, ph in systems:
        t1 = time.time()
        P = None
        before, losses = {}, []
        for r in runs:
            F.fem_pic_learned_select(r["lib"].h, sys_id)
            before[r["wl"].name] = float(np.mean(F.fem_pic_learned_eval(r["lib"].h, n_train, n_hold)))
        for rd in range(args.proto_rounds):
            lr = 2e-3 * (1.0 - rd / max(1, args.proto_rounds)) + 1e-4
            for r in runs:
                F.fem_pic_learned_select(r["lib"].h, sys_id)
                if P is not None:
                    F.fem_pic_learned_params(r["lib"].h, P)
                ls = F.fem_pic_learned_train(r["lib"].h, 0, n_train, args.proto_epochs, lr=lr, seed=rd)
                losses.append(float(ls[-1]))
                P = F.fem_pic_learned_params(r["lib"].h)
        params[sys_id] = P
        rep = {"train_s": time.time() - t1, "train_loss_first": losses[0], "train_loss_last": losses[-1],
               "model": "3-layer message passing on the " + ("edge" if sys_id == F.FP_SYS_NEWMARK else "node") +
                        " graph, 64 features, BF16 weights with FP32 accumulation (tensor cores), static input; "
                        "head: a symmetric sparse correction of the Jacobi preconditioner on the operator's pattern"}
        for r in runs:
            lib = r["lib"]
            F.fem_pic_learned_select(lib.h, sys_id)
            F.fem_pic_learned_params(lib.h, P)
            after = float(np.mean(F.fem_pic_learned_eval(lib.h, n_train, n_hold)))
            F.fem_pic_learned_build(lib.h)

            def run(pc, lib=lib, r=r):
                r["restore"]()
                torch.cuda.synchronize()
                F.fem_pic_profile_read(lib.h, reset=True)
                F.fem_pic_profile_enable(lib.h, True)
                its, fb = [], 0
                for k in range(n_hold):
                    r["step"](pc)
                    fi = F.fem_pic_field_last_info(lib.h)
                    its.append(fi[sys_id]["iters"])
                    fb += fi[sys_id]["fell_back"]
                torch.cuda.synchronize()
                F.fem_pic_profile_enable(lib.h, False)
                phs = F.fem_pic_profile_read(lib.h, reset=True)
                return {"iters_mean": statistics.mean(its), "ms_per_solve": phs.get(ph, (0.0, 1))[0] / n_hold,
                        "fell_back": fb}
            plain = run(F.FP_PC_JACOBI)
            learn = run(bit)
            rep[r["wl"].name] = {"held_out_ratio_before": before[r["wl"].name], "held_out_ratio_after": after,
                                 "plain_jacobi_cg": plain, "learned": learn,
                                 "iters_ratio": learn["iters_mean"] / max(1e-9, plain["iters_mean"]),
                                 "time_ratio": learn["ms_per_solve"] / max(1e-9, plain["ms_per_solve"])}
        report[name] = rep
    for r in runs:
        r["lib"].close()
    report["total_s"] = time.time() - t0
    return {"report": report, "params": params}


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_2103_06737_gb300.fem_pic as F
    from paper_2103_06737_gb300 import build as B

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    proto = None
    if not args.no_field and args.learned != "off":
        proto = learned_protocol(args, torch.device("cuda", local))
        torch.cuda.empty_cache()
    wl = build_workload(args)
    if args.sort_every == 0:
        # the beam's cell order decays fastest (0.1c drift along the axis); measured on it, sort +
        # fast push per step: every 2 steps 0.55 ms, 3: 0.54, 5: 0.59, 10: 0.69; the thermal
        # workloads gain nothing below 10
        args.sort_every = 2 if args.workload == 3 else 10
    if args.drift_steps < 0:
        args.drift_steps = 200 if wl.mesh.n <= 32 else 0
    lib = F.FemPic(wl.mesh.xyz, wl.mesh.tets, F.FP_FP32)
    sizes = lib.sizes
    dev = torch.device("cuda", local)
    species = [lib.species(s.cell, s.X, s.V, s.q, s.m, s.w, device=dev) for s in wl.species]
    n_part = sum(s.n for s in species)
    e, b = lib.fields_uniform((0.0, 0.0, 0.0), wl.B0, device=dev)
    if wl.E_amp > 0:
        # seeded random edge field: e_k = amp * l_k * U(-1,1) on interior edges, 0 on PEC edges
        from paper_2103_06737_gb300 import inputs as I
        topo = F.fem_pic_topology(lib.h)
        rp, col, val = F.fem_pic_incidence(lib.h, 0)
        ij = col.reshape(-1, 2)
        length = np.linalg.norm(wl.mesh.xyz[ij[:, 1]] - wl.mesh.xyz[ij[:, 0]], axis=1)
        u = I.random_dofs(sizes["n_edges"], 31, 1.0)
        nb = topo["tet_neigh"]
        bt = np.nonzero((nb < 0).any(axis=1))[0]
        wall = np.zeros(sizes["n_edges"], bool)
        faces_of = {0: (1, 2, 3), 1: (0, 2, 3), 2: (0, 1, 3), 3: (0, 1, 2)}
        le = {(0, 1): 0, (0, 2): 1, (0, 3): 2, (1, 2): 3, (1, 3): 4, (2, 3): 5}
        for t in bt:
            for k in range(4):
                if nb[t, k] < 0:
                    f = faces_of[k]
                    for a in range(3):
                        for c in range(a + 1, 3):
                            wall[topo["tet_edges"][t, le[(f[a], f[c])]]] = True
        ev = wl.E_amp * length * u
        ev[wall] = 0.0
        e.copy_(torch.as_tensor(ev, device=dev))
    set_deposits(args, lib, F)
    cflag = F.FP_CHARGE_CHANGE if args.deposits.startswith("change") else 0
    DEP, DQ = lib.deposit_dtype, lib.charge_dtype
    dG = torch.zeros(sizes["n_edges"], dtype=DEP, device=dev)       # dG^{n+1/2}
    dG_prev = torch.zeros(sizes["n_edges"], dtype=DEP, device=dev)  # dG^{n-1/2}
    Qn = torch.zeros(sizes["n_nodes"], dtype=DQ, device=dev)
    Qo = torch.zeros(sizes["n_nodes"], dtype=DQ, device=dev)
    res = torch.zeros(6, dtype=torch.float64, device=dev)
    # uniform immobile neutralising ion background where the workload has one:
    # Q_ion,n = -(total electron charge) alpha^0_n / V, alpha^0_n = integral of W0_n
    Q_ion = torch.zeros(sizes["n_nodes"], dtype=DQ, device=dev)
    if wl.background_ions:
        alpha = F.fem_pic_whitney0_integrals(lib.h)
        qtot = sum(s_.q * s_.w * s_.n for s_ in species)
        Q_ion.copy_(torch.as_tensor(-qtot * alpha / alpha.sum(), device=dev))
    field = not args.no_field
    solv = (args.solver.split(",") + args.solver.split(","))[:2]
    code = {"mixed": F.FP_PC_JACOBI, "fp64": F.FP_PC_JACOBI_FP64}
    precond = F.FP_PC_JACOBI
    if field:
        F.fem_pic_field_setup(lib.h, wl.dt)
        F.fem_pic_field_options(lib.h, code[solv[0]], code[solv[1]], args.inner_tol)
        pdeg = [int(x) for x in (args.poly.split(",") + args.poly.split(","))[:2]]
        pdeg_cfg = list(pdeg)     # as configured (the learned comparison may set a system to 1)
        prat = [float(x) for x in (args.poly_ratio.split(",") + args.poly_ratio.split(","))[:2]]
        F.fem_pic_field_poly(lib.h, F.FP_SYS_NEWMARK, pdeg[0], prat[0])
        F.fem_pic_field_poly(lib.h, F.FP_SYS_GAUSS, pdeg[1], prat[1])
    E_prev = torch.zeros(sizes["n_edges"], dtype=torch.float64, device=dev)
    E_next = torch.zeros_like(E_prev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    flush_rd = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def flush_l2(k):
        # write a buffer larger than L2, then read another one so the dirty lines of the
        # write are written back here and not inside the next timed step
        flush.fill_(float(k))
        return flush_rd.sum()
    stream = torch.cuda.current_stream()

    # initial sort and charge
    bufs = [[s_, s_.empty_like()] for s_ in species]     # double buffers for the sort
    cur = [0] * len(species)
    for k in range(len(species)):
        lib.sort(bufs[k][0], bufs[k][1])
        cur[k] = 1
    Qo.copy_(Q_ion)
    for k in range(len(species)):
        lib.deposit_charge(bufs[k][cur[k]], Qo, flags=F.FP_ACCUMULATE)
    if field:   # E^0 from the Gauss law of the initial charge; E^{-1} = E^0, dG^{-1/2} = 0
        st0, inf0 = F.fem_pic_field_initial(lib.h, Qo, e, tol=args.tol)
        if st0 != F.FP_OK:
            raise RuntimeError(f"initial field: {inf0}")
        E_prev.copy_(e)
    st = lib.status()
    if st != F.FP_OK:
        raise RuntimeError(f"setup status {st}: {F.fem_pic_last_error(lib.h)}")

    # The measured regions start from this initial state (particles and fields): electrons
    # stream along B0 and are absorbed by the PEC walls, so a long warm-up would otherwise
    # leave fewer live particles in the timed steps.  Only live particles are counted.
    snap_cur = list(cur)
    snap_sp = [(bufs[k][cur[k]].cell.clone(), bufs[k][cur[k]].off.clone(), bufs[k][cur[k]].vel.clone())
               for k in range(len(species))]
    snap_f = [(t_, t_.clone()) for t_ in (e, b, E_prev, dG_prev, Qo)]

    def alive():
        return sum(int((bufs[k][cur[k]].cell >= 0).sum()) for k in range(len(species)))

    def plan(i):
        """(sort now?, buffer index per species before the step) of step i"""
        sort_now = args.sort_every > 0 and i > 0 and i % args.sort_every == 0
        return sort_now, tuple(cur)

    def enqueue_push_part(pl, k):
        """Species k's share of the step's particle part on the current stream (its periodic
        sort, its push and deposits; species 0 also clears dG and starts Q^{n+1} from the ion
        background): returns (library kernels launched, the buffer it used)."""
        sort_now, before = pl
        n_k = 0
        b_ = before[k]
        if sort_now:
            lib.sort(bufs[k][b_], bufs[k][1 - b_])
            b_ = 1 - b_
            n_k += 5
        s_ = bufs[k][b_]
        if k == 0:
            dG.zero_()
            Qn.copy_(Qo if cflag else Q_ion)     # the charge change is added onto Q^n
        # particles: gather at E^n, push, walk, deposit dG^{n+1/2}, Q^{n+1}; the field records
        # are made once per step (the first species' call)
        lib.push_deposit(e, b, s_, wl.dt, dG, Qn, flags=F.FP_ACCUMULATE | cflag | (F.FP_SAME_FIELDS if k else 0))
        n_k += 3 if k == 0 else 2     # field prep (first species), fast push, FP64 walk of the queue
        return n_k, s_

    def enqueue_push(pl):
        """The step's particle part on the current stream (periodic sort, push, deposits):
        returns (library kernels launched, the species' buffers it used)."""
        n_k, use = 0, []
        for k in range(len(species)):
            m_, s_ = enqueue_push_part(pl, k)
            n_k += m_
            use.append(s_)
        return n_k, use

    def enqueue_field():
        """The step's field part on the current stream (field step, residuals, leapfrog state);
        it does not touch the particle state.  Returns the library kernels launched."""
        n_k = 0
        if field:                 # fields: Newmark, Gauss-law projection, Faraday -> E^{n+1}, b^{n+1}
            F.fem_pic_field_step(lib.h, E_prev, e, E_next, b, dG, dG_prev, Qn, tol=args.tol,
                                 max_iter=args.max_iter, precond=state["precond"], info=False)
            # Newmark right-hand side (2) and solve (mixed: gather into its row order, solve,
            # scatter out with A E^N: 3; FP64: the solve, then M E^N: 2), Gauss right-hand side
            # (1), solve (1), projection and Faraday update (2)
            n_k += 9 if solv[0] == "mixed" else 8     # (a learned preconditioner acts inside the solver)
        lib.residuals(dG, Qn, Qo, b, res)
        n_k += 1
        Qo.copy_(Qn)
        if field:
            dG_prev.copy_(dG)
            E_prev.copy_(e)
            e.copy_(E_next)
        return n_k

    def enqueue(pl):
        """One PIC step on the current stream; returns the number of library kernels launched."""
        n_k, _ = enqueue_push(pl)
        return n_k + enqueue_field()

    def advance(pl):
        if pl[0]:
            for k in range(len(species)):
                cur[k] = 1 - cur[k]

    state = {"i": 0, "precond": precond}

    def restore():
        for k in range(len(species)):
            cur[k] = snap_cur[k]
            c_, o_, v_ = snap_sp[k]
            bufs[k][cur[k]].cell.copy_(c_)
            bufs[k][cur[k]].off.copy_(o_)
            bufs[k][cur[k]].vel.copy_(v_)
        for t_, c_ in snap_f:
            t_.copy_(c_)
        state["i"] = 0

    def eager_step():
        pl = plan(state["i"])
        n_k = enqueue(pl)
        advance(pl)
        state["i"] += 1
        return n_k

    # warm-up (eager): allocates the library's scratch before any capture
    clk = clocks_start(local)
    t0 = time.time()
    w = 0
    while w < max(args.warmup, 2 * args.sort_every + 2) or time.time() - t0 < args.min_warmup_s:
        eager_step()
        if w % 20 == 0:
            torch.cuda.synchronize()
        w += 1
    torch.cuda.synchronize()
    st = lib.status()
    if st != F.FP_OK:
        raise RuntimeError(f"warm-up status {st}: {F.fem_pic_last_error(lib.h)}")

    # learned preconditioner, per system (Newmark edge system, Gauss-law node system): the
    # network trained by the protocol on the 4^3 and 32^3 workloads' systems, fine-tuned on
    # args.tune_systems systems of this workload's own steps, then timed against plain
    # Jacobi-CG (the reference solver) and the configured Chebyshev polynomial on the same steps.  The
    # timed steps use the fastest of the three for each system.
    def learned_pick(sys_id, params0, n_compare, flush_base=0):
        """Fine-tune the learned preconditioner of one system (starting from params0) on
        args.tune_systems systems of this workload's own steps, then time plain Jacobi-CG, the
        learned preconditioner and the configured polynomial on the same steps from the initial
        state; set up the fastest for the system.  Returns (report, choice, tuned weights)."""
        bit = F.FP_PC_LEARNED if sys_id == F.FP_SYS_NEWMARK else F.FP_PC_LEARNED_GAUSS
        ph_cg = "cg_newmark" if sys_id == F.FP_SYS_NEWMARK else "cg_gauss"
        sysname = "newmark" if sys_id == F.FP_SYS_NEWMARK else "gauss"
        t_l0 = time.time()
        keep = state["precond"]
        state["precond"] = keep & ~bit
        F.fem_pic_learned_select(lib.h, sys_id)
        F.fem_pic_learned_init_model(lib.h, seed=0, sample_capacity=max(1, args.tune_systems),
                                     model=F.FP_LEARNED_PRECOND)
        F.fem_pic_learned_params(lib.h, params0)
        tune = None
        if args.tune_systems > 0:
            restore()
            F.fem_pic_learned_mode(lib.h, collect=True, active=False)
            for _ in range(args.tune_systems):
                eager_step()
            torch.cuda.synchronize()
            F.fem_pic_learned_mode(lib.h, collect=False, active=False)
            n_t = F.fem_pic_learned_samples(lib.h)
            r_before = float(np.mean(F.fem_pic_learned_eval(lib.h, 0, n_t)))
            ls = F.fem_pic_learned_train(lib.h, 0, n_t, args.tune_epochs, lr=5e-4, seed=1)
            r_after = float(np.mean(F.fem_pic_learned_eval(lib.h, 0, n_t)))
            tune = {"systems": n_t, "epochs": args.tune_epochs, "ratio_before": r_before,
                    "ratio_after": r_after, "loss_last": float(ls[-1])}
        F.fem_pic_learned_build(lib.h)
        torch.cuda.synchronize()
        t_prep = time.time() - t_l0

        def compare(pc, deg):
            F.fem_pic_field_poly(lib.h, sys_id, deg, prat[sys_id])
            state["precond"] = pc
            restore()
            F.fem_pic_profile_read(lib.h, reset=True)
            F.fem_pic_profile_enable(lib.h, True)
            its, fb = [], 0
            for k in range(n_compare):
                flush_l2(flush_base + k)
                eager_step()
                fi = F.fem_pic_field_last_info(lib.h)
                its.append(fi[sys_id]["iters"])
                fb += fi[sys_id]["fell_back"]
            torch.cuda.synchronize()
            F.fem_pic_profile_enable(lib.h, False)
            ph = F.fem_pic_profile_read(lib.h, reset=True)
            tot = sum(ph.get(k, (0.0, 1))[0] for k in ("field_other", "cg_newmark", "cg_gauss", "learned"))
            return {"field_ms_per_step": tot / n_compare,
                    ph_cg + "_ms_per_step": ph.get(ph_cg, (0.0, 1))[0] / n_compare,
                    "iters_mean": statistics.mean(its), "fell_back": fb}
        base = keep & ~bit
        plain = compare(base, 1)             # plain Jacobi-CG
        learn = compare(base | bit, 1)       # the learned preconditioner (replaces the polynomial)
        untuned = None
        if learn["fell_back"] and tune is not None:
            # the tuned correction made the preconditioner indefinite on some residual (the
            # solver fell back to Jacobi): the protocol's weights, as trained on the 4^3 and
            # 32^3 systems, are timed too and kept if they do better
            tuned_params = F.fem_pic_learned_params(lib.h)
            F.fem_pic_learned_params(lib.h, params0)
            F.fem_pic_learned_build(lib.h)
            untuned = compare(base | bit, 1)
            if untuned[ph_cg + "_ms_per_step"] >= learn[ph_cg + "_ms_per_step"]:
                F.fem_pic_learned_params(lib.h, tuned_params)
                F.fem_pic_learned_build(lib.h)
            else:
                learn, untuned = untuned, learn
                tune["kept"] = "protocol weights (the tuned ones fell back to Jacobi and were slower)"
        if tune is not None and args.tune_seeds > 1:
            # further fine-tunes from the same start weights on the same systems with other training
            # seeds (the optimiser's moments carry over from the previous fine-tune: setting weights
            # leaves them), each timed on the same steps; the fastest weights are kept
            best_params = F.fem_pic_learned_params(lib.h)
            tune["seeds"] = [{"seed": 1, "iters_mean": learn["iters_mean"],
                              "ms": learn[ph_cg + "_ms_per_step"]}]
            for sd in range(2, args.tune_seeds + 1):
                F.fem_pic_learned_params(lib.h, params0)
                F.fem_pic_learned_train(lib.h, 0, tune["systems"], args.tune_epochs, lr=5e-4, seed=sd)
                F.fem_pic_learned_build(lib.h)
                alt = compare(base | bit, 1)
                tune["seeds"].append({"seed": sd, "iters_mean": alt["iters_mean"],
                                      "ms": alt[ph_cg + "_ms_per_step"]})
                if alt[ph_cg + "_ms_per_step"] < learn[ph_cg + "_ms_per_step"]:
                    learn = alt
                    best_params = F.fem_pic_learned_params(lib.h)
            F.fem_pic_learned_params(lib.h, best_params)
            F.fem_pic_learned_build(lib.h)
            torch.cuda.synchronize()
        poly = compare(base, pdeg_cfg[sys_id]) if pdeg_cfg[sys_id] > 1 else None
        ms = {"plain": plain[ph_cg + "_ms_per_step"], "learned": learn[ph_cg + "_ms_per_step"]}
        if poly is not None:
            ms["chebyshev"] = poly[ph_cg + "_ms_per_step"]
        best = min(ms, key=ms.get) if args.learned == "auto" else "learned"
        pdeg[sys_id] = pdeg_cfg[sys_id] if best == "chebyshev" else 1
        F.fem_pic_field_poly(lib.h, sys_id, pdeg[sys_id], prat[sys_id])
        state["precond"] = base | (bit if best == "learned" else 0)
        rep = {"plain": plain, "learned": learn, "chebyshev": poly, "fine_tune": tune, "prepare_s": t_prep,
               "learned_other_weights": untuned,
               "learned_vs_plain_ms": ms["learned"] / ms["plain"],
               "learned_beats_plain_cg": bool(ms["learned"] < ms["plain"]),
               "timed_steps_use": best, "used_in_timed_steps": best == "learned",
               "compared_against": f"plain Jacobi-CG (Jacobi inner preconditioner on the {sysname} system) and the "
                                   f"Chebyshev-Jacobi polynomial of degree {pdeg_cfg[sys_id]}, same steps, "
                                   f"same {args.tol}"}
        return rep, best, F.fem_pic_learned_params(lib.h)

    # learned preconditioner, per system (Newmark edge system, Gauss-law node system): the
    # network trained by the protocol on the 4^3 and 32^3 workloads' systems, fine-tuned on
    # this workload's own steps, then timed against plain Jacobi-CG (the reference solver) and the
    # configured Chebyshev polynomial on the same steps; the timed steps use the fastest.
    learned = None
    tuned = {}
    if field and proto is not None:
        learned = {"protocol": proto["report"]}
        for sysname in [x for x in args.learned_systems.split(",") if x]:
            sys_id = F.FP_SYS_NEWMARK if sysname == "newmark" else F.FP_SYS_GAUSS
            rep, best, tuned[sys_id] = learned_pick(sys_id, proto["params"][sys_id], args.compare_steps)
            rep["weights"] = "trained by the protocol on the 4^3 and 32^3 workloads, fine-tuned on this workload's " \
                             "own systems"
            learned[sysname] = rep

    # one CUDA graph per distinct step shape (sort or not, buffers, Q parity)
    graphs = {}
    use_graphs = not args.no_graphs

    def graph_step():
        pl = plan(state["i"])
        key = (pl, state["precond"])
        if key not in graphs:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                n_k = enqueue(pl)
            graphs[key] = (g, n_k)
            torch.cuda.synchronize()
        g, n_k = graphs[key]
        g.replay()
        advance(pl)
        state["i"] += 1
        return n_k

    step = graph_step if use_graphs else eager_step
    if use_graphs:                       # capture every shape once, outside the timed region
        restore()
        for _ in range(2 * args.sort_every + 2):
            step()
        torch.cuda.synchronize()
    restore()
    torch.cuda.synchronize()
    alive0 = alive()

    # timed: K steps, each bracketed by events; L2 flushed between steps (outside the events);
    # each step's FP64 residuals (continuity, D2 b) are kept, copied after its end event
    launches = 0
    evs = []
    res_log = torch.zeros((args.steps, 6), dtype=torch.float64, device=dev)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    th0 = time.perf_counter()
    for k in range(args.steps):
        flush_l2(k)
        a = torch.cuda.Event(enable_timing=True)
        z = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed_step")      # marks the timed steps for profilers
        a.record(stream)
        launches += step()
        z.record(stream)
        torch.cuda.nvtx.range_pop()
        res_log[k].copy_(res)
        evs.append((a, z))
    th1 = time.perf_counter()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = clocks_stop(clk)
    step_ms = [a.elapsed_time(z) for a, z in evs]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    st = lib.status()
    r = res.cpu().numpy()
    rlog = res_log.cpu().numpy()
    alive1 = alive()
    alive_timed = 0.5 * (alive0 + alive1)          # absorption is gradual: mean of start and end
    units_all = sum_over_ranks(alive_timed * args.steps, world, dev)
    restore()

    # per-kernel durations: an eager pass of the same steps with the library's event profiler
    F.fem_pic_profile_read(lib.h, reset=True)
    F.fem_pic_profile_enable(lib.h, True)
    push_ms = []
    iters_n, iters_g, relres, outer_n, outer_g = [], [], [], [], []
    for k in range(args.steps):
        flush_l2(k)
        a = torch.cuda.Event(enable_timing=True)
        z = torch.cuda.Event(enable_timing=True)
        pl = plan(state["i"])
        torch.cuda.nvtx.range_push("eager_step")      # the per-kernel pass, for profilers
        a.record(stream)
        enqueue(pl)
        z.record(stream)
        torch.cuda.nvtx.range_pop()
        advance(pl)
        state["i"] += 1
        push_ms.append((a, z))
        if field:
            fi = F.fem_pic_field_last_info(lib.h)
            iters_n.append(fi[0]["iters"])
            iters_g.append(fi[1]["iters"])
            outer_n.append(fi[0]["outer"])
            outer_g.append(fi[1]["outer"])
            relres.append(max(fi[0]["rel_res"], fi[1]["rel_res"]))
    torch.cuda.synchronize()
    F.fem_pic_profile_enable(lib.h, False)
    phases = F.fem_pic_profile_read(lib.h, reset=True)
    push_ms = [a.elapsed_time(z) for a, z in push_ms]
    alive_eager = 0.5 * (alive0 + alive())
    push_call = (phases.get("prep", (0, 1))[0] + phases.get("push_fast", (0, 1))[0] +
                 phases.get("walk", (0, 1))[0]) / max(1, phases.get("push_fast", (0, 1))[1])

    # e2e through the public API with host buffers: H2D of the step's inputs (particle
    # state + fields) from pinned memory, the step, D2H of the results (state + deposits)
    e2e = None
    if not args.no_e2e:
        restore()
        species = [bufs[k][cur[k]] for k in range(len(species))]
        hs = [(torch.empty_like(s.cell, device="cpu").pin_memory(), torch.empty_like(s.off, device="cpu").pin_memory(),
               torch.empty_like(s.vel, device="cpu").pin_memory()) for s in species]
        for (hc, ho, hv), s in zip(hs, species):
            hc.copy_(s.cell)
            ho.copy_(s.off)
            hv.copy_(s.vel)
        # results go to pinned buffers of their own: a device-to-host copy into the pinned pages a
        # host-to-device copy of the same step has just read ran at less than half the rate
        hs_out = [tuple(torch.empty_like(x).pin_memory() for x in tr) for tr in hs]
        # the step's inputs: particle state, fields E^n, E^{n-1}, b, dG^{n-1/2}, Q^n
        fin = [(e, e.cpu().pin_memory()), (b, b.cpu().pin_memory()), (E_prev, E_prev.cpu().pin_memory()),
               (dG_prev, dG_prev.cpu().pin_memory()), (Qo, Qo.cpu().pin_memory())]
        hdG = torch.empty_like(dG, device="cpu").pin_memory()
        hQ = torch.empty_like(Qn, device="cpu").pin_memory()
        hE = torch.empty_like(e, device="cpu").pin_memory()
        bi = sum(x.numel() * x.element_size() for tr in hs for x in tr) + \
            sum(h_.numel() * h_.element_size() for _, h_ in fin)
        bo = sum(x.numel() * x.element_size() for tr in hs_out for x in tr) + hdG.numel() * hdG.element_size() + \
            hQ.numel() * hQ.element_size() + \
            (hE.numel() * 8 if field else 0)
        # Pipelined by species and across steps: each species is pushed (one CUDA graph per species
        # and step shape) as soon as its state has been copied in, and its new state goes back on an
        # output stream (into pinned buffers of its own) during the next push and the field step
        # (a second graph), which does not touch the particles; the next step's particle state is
        # copied in on an input stream during this step's field step, once this step's copies out
        # of the same device buffers are done.  The fields' copies in and the results' copies out
        # (deposits, E) stay on the compute stream.  One timed region over all steps, from the
        # first copy in to the last copy out; every step's inputs (3 GB at the largest workload)
        # are larger than L2, so no flush is needed between steps.
        in_stream = torch.cuda.Stream(device=dev)
        out_stream = torch.cuda.Stream(device=dev)
        e2e_graphs = {}
        nsp = len(species)

        def e2e_graph(pl):
            key = (pl, state["precond"])
            if key not in e2e_graphs:
                gps, use = [], []
                for k in range(nsp):
                    g_ = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(g_):
                        _, s_ = enqueue_push_part(pl, k)
                    gps.append(g_)
                    use.append(s_)
                gb = torch.cuda.CUDAGraph()
                with torch.cuda.graph(gb):
                    enqueue_field()
                e2e_graphs[key] = (gps, gb, use)
                torch.cuda.synchronize()
            return e2e_graphs[key]
        restore()
        for k in range(args.steps):      # capture every shape of the run first (not timed)
            pl = plan(k)
            e2e_graph(pl)
            advance(pl)
        restore()
        species = [bufs[k][cur[k]] for k in range(nsp)]
        flush_l2(0)
        torch.cuda.synchronize()

        def copy_in(dst, after):
            evs = []
            with torch.cuda.stream(in_stream):
                for j, ((hc, ho, hv), s) in enumerate(zip(hs, dst)):
                    if after[j] is not None:
                        in_stream.wait_event(after[j])
                    s.cell.copy_(hc, non_blocking=True)
                    s.off.copy_(ho, non_blocking=True)
                    s.vel.copy_(hv, non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(in_stream)
                    evs.append(ev)
            return evs
        # the fields' copies in and the results' copies out go through device staging buffers:
        # the next step's fields are copied from host memory into staging on the input stream
        # during this step, and this step's results are copied to staging on the compute stream
        # (device-to-device) and from there to host memory on the output stream, so only the
        # device-to-device copies sit on the compute stream
        stg_in = [torch.empty_like(d_) for d_, _ in fin]
        res_dev = [dG, Qn] + ([e] if field else [])
        res_host = [hdG, hQ] + ([hE] if field else [])
        stg_out = [torch.empty_like(x) for x in res_dev]

        def fields_in(after):
            with torch.cuda.stream(in_stream):
                if after is not None:
                    in_stream.wait_event(after)
                for (_, h_), g_ in zip(fin, stg_in):
                    g_.copy_(h_, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(in_stream)
            return ev
        t_a = torch.cuda.Event(enable_timing=True)
        t_z = torch.cuda.Event(enable_timing=True)
        t_a.record(stream)
        in_stream.wait_event(t_a)
        out_stream.wait_event(t_a)
        ev_f = fields_in(None)
        ev_in = copy_in(species, [None] * nsp)
        out_done = [None] * nsp
        res_done = None
        for k in range(args.steps):
            pl = plan(state["i"])
            gps, gb, use = e2e_graph(pl)
            stream.wait_event(ev_f)
            for (d_, _), g_ in zip(fin, stg_in):
                d_.copy_(g_, non_blocking=True)
            if k + 1 < args.steps:
                staged = torch.cuda.Event()
                staged.record(stream)
                ev_f = fields_in(staged)
            for j in range(nsp):
                stream.wait_event(ev_in[j])
                gps[j].replay()
                pushed = torch.cuda.Event()
                pushed.record(stream)
                out_stream.wait_event(pushed)
                with torch.cuda.stream(out_stream):
                    hc, ho, hv = hs_out[j]
                    hc.copy_(use[j].cell, non_blocking=True)
                    ho.copy_(use[j].off, non_blocking=True)
                    hv.copy_(use[j].vel, non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(out_stream)
                    out_done[j] = ev
            gb.replay()
            if res_done is not None:
                stream.wait_event(res_done)   # the previous step's results have left staging
            for x, g_ in zip(res_dev, stg_out):
                g_.copy_(x, non_blocking=True)
            copied = torch.cuda.Event()
            copied.record(stream)
            out_stream.wait_event(copied)
            with torch.cuda.stream(out_stream):
                for g_, h_ in zip(stg_out, res_host):
                    h_.copy_(g_, non_blocking=True)
                res_done = torch.cuda.Event()
                res_done.record(out_stream)
            advance(pl)
            state["i"] += 1
            species = [bufs[j][cur[j]] for j in range(nsp)]
            if k + 1 < args.steps:
                ev_in = copy_in(species, out_done)
        for ev in out_done + [res_done]:
            stream.wait_event(ev)
        t_z.record(stream)
        torch.cuda.synchronize()
        e2e_ms = t_a.elapsed_time(t_z)
        e2e_max = max_over_ranks(e2e_ms, world, dev)
        e2e = {"value": whole_job_rate(sum_over_ranks(alive0 * args.steps, world, dev), e2e_max), "unit": UNIT,
               "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo),
               "ms_per_step": e2e_ms / args.steps,
               "l2": "not flushed between steps: each step copies its inputs in from host memory "
                     f"({bi / 1e9:.2f} GB, larger than L2)",
               "overlap": "pipelined by species and across steps: species k pushed once its state is in while "
                          "species k+1's state is copied in, species k's new state copied back on an output stream "
                          "(into pinned buffers of its own) during the next push and the field step, the next "
                          "step's particle state and fields copied in during this step (the fields through device "
                          "staging buffers), deposits and E copied out through staging on the output stream; one "
                          "timed region over all steps"}

    # the main measurement's preconditioners (the side legs below choose their own)
    main_pc, main_pdeg = state["precond"], list(pdeg)
    fp64 = None if args.fp64_steps <= 0 else measure_fp64(args, F, wl, dev, flush_l2, stream)
    adams = None if args.adams_steps <= 0 else measure_adams(args, lib, F, species, restore, bufs, cur, e, b, dG,
                                                             Qn, flush_l2, stream, sizes, wl, dev)
    def measure_neumann():
        """The PIC step with the natural (Neumann) field boundary and the zero-mean constrained
        Gauss-law projection: fields set up again with FP_BC_NEUMANN (this replaces the PEC
        setup, so it runs last), the initial state restored, E^0 from its charge, then
        args.neumann_steps timed eager steps (L2 flushed between them) with the per-phase
        profiler on."""
        F.fem_pic_field_setup(lib.h, wl.dt, bc=F.FP_BC_NEUMANN)
        F.fem_pic_field_options(lib.h, code[solv[0]], code[solv[1]], args.inner_tol)
        F.fem_pic_field_poly(lib.h, F.FP_SYS_NEWMARK, pdeg_cfg[0], prat[0])
        F.fem_pic_field_poly(lib.h, F.FP_SYS_GAUSS, pdeg_cfg[1], prat[1])
        pdeg[0], pdeg[1] = pdeg_cfg[0], pdeg_cfg[1]
        state["precond"] = precond
        restore()
        st0, inf0 = F.fem_pic_field_initial(lib.h, Qo, e, tol=args.tol)
        E_prev.copy_(e)
        snap_f[2] = (E_prev, E_prev.clone())   # this boundary's E^0 is the restored start
        snap_f[0] = (e, e.clone())
        # the new setup discarded the PEC networks: the same weights (tuned on the PEC systems of
        # this mesh) are tuned again on this boundary's systems and compared the same way
        nlearn = {}
        for sys_id, prm in tuned.items():
            rep, best, _ = learned_pick(sys_id, prm, args.neumann_steps, flush_base=4000)
            nlearn["newmark" if sys_id == F.FP_SYS_NEWMARK else "gauss"] = rep
        restore()
        E_prev.copy_(e)
        for _ in range(3):
            eager_step()
        torch.cuda.synchronize()
        F.fem_pic_profile_read(lib.h, reset=True)
        F.fem_pic_profile_enable(lib.h, True)
        ev, its, outs, rr, live = [], [], [], [], []
        for k in range(args.neumann_steps):
            live.append(alive())
            flush_l2(2000 + k)
            a = torch.cuda.Event(enable_timing=True)
            z = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            eager_step()
            z.record(stream)
            ev.append((a, z))
            fi = F.fem_pic_field_last_info(lib.h)
            its.append((fi[0]["iters"], fi[1]["iters"]))
            outs.append((fi[0]["outer"], fi[1]["outer"]))
            rr.append(max(fi[0]["rel_res"], fi[1]["rel_res"]))
        torch.cuda.synchronize()
        F.fem_pic_profile_enable(lib.h, False)
        ph = F.fem_pic_profile_read(lib.h, reset=True)
        ms = sum(a.elapsed_time(z) for a, z in ev) / len(ev)
        nsteps = len(ev)
        return {"ms_per_step": ms, "particle_steps_per_s": sum(live) / (ms * nsteps * 1e-3),
                "timed_steps": nsteps, "initial_status": int(st0), "launches": "eager",
                "field_ms_per_step": sum(ph.get(k, (0.0, 1))[0] for k in ("field_other", "cg_newmark", "cg_gauss"))
                / nsteps,
                "ms_newmark_cg": ph.get("cg_newmark", (0.0, 1))[0] / nsteps,
                "ms_gauss_cg": ph.get("cg_gauss", (0.0, 1))[0] / nsteps,
                "newmark_iters_mean": float(np.mean([i[0] for i in its])),
                "gauss_iters_mean": float(np.mean([i[1] for i in its])), "max_rel_res": max(rr),
                "newmark_refinements_mean": float(np.mean([o[0] for o in outs])),
                "gauss_refinements_mean": float(np.mean([o[1] for o in outs])),
                "status": int(lib.status()),
                "learned_vs_plain": nlearn or None,
                "precond": {nm: ("learned preconditioner" if state["precond"] & bit else
                                 (f"Chebyshev-Jacobi degree {pdeg[k_]}" if pdeg[k_] > 1 else "jacobi"))
                            for k_, (nm, bit) in enumerate((("newmark", F.FP_PC_LEARNED),
                                                            ("gauss", F.FP_PC_LEARNED_GAUSS)))},
                "what": "PIC step with the natural field boundary: Newmark over all edges, Gauss-law projection "
                        "with the zero-mean constraint (a net charge spread as alpha), Faraday"}
    def measure_gauss_drift():
        """The Gauss-law comparison of Sec. V and VI.B on this workload: the projected step (the
        product path) against the first-order mixed FEM and the wave-equation FEM without the
        projection.  All three are fed the deposits of the same particle steps, pushed with the
        projected step's fields, from the same initial state (E^0 from the Gauss law, b^0 the
        uniform B0, which drives no interior edge).  Per step: max |D0^T [*eps] E + Q| over
        interior nodes divided by its scale, for each; the two comparison steps are timed with
        CUDA events, L2 flushed before each step (outside the events).  Run once with every
        solve at --tol, and once with the unprojected systems' solves at --drift-tol: the
        excitation of their gradient null space follows the solves' errors (Sec. V)."""
        mh = F.fem_pic_mfem_create(lib.h)
        names = ("projected", "mfem", "wave")
        solver = code[solv[0]]

        def run(tol_cmp):
            state["precond"] = precond
            restore()
            torch.cuda.synchronize()
            E_m, E_m2, b_m = e.clone(), torch.empty_like(e), b.clone()
            E_wp, E_w, E_w2, b_w = e.clone(), e.clone(), torch.empty_like(e), b.clone()
            K = args.drift_steps
            hist = torch.zeros(K, 3, 2, dtype=torch.float64, device=dev)
            ev = []
            for k in range(K):
                pl = plan(state["i"])
                flush_l2(3000 + k)
                enqueue_push(pl)
                ta, tb, tc = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                ta.record(stream)
                F.fem_pic_mfem_step(lib.h, mh, E_m, E_m2, b_m, dG, tol=tol_cmp, max_iter=args.max_iter,
                                    precond=solver, info=False)
                tb.record(stream)
                F.fem_pic_wave_step(lib.h, mh, E_wp, E_w, E_w2, b_w, dG, dG_prev, tol=tol_cmp,
                                    max_iter=args.max_iter, precond=solver, info=False)
                tc.record(stream)
                ev.append((ta, tb, tc))
                enqueue_field()          # the projected step: e <- E^{n+1}, dG_prev <- dG, Qo <- Qn
                F.fem_pic_mfem_gauss_residual(lib.h, mh, e, Qn, hist[k, 0])
                F.fem_pic_mfem_gauss_residual(lib.h, mh, E_m2, Qn, hist[k, 1])
                F.fem_pic_mfem_gauss_residual(lib.h, mh, E_w2, Qn, hist[k, 2])
                E_m, E_m2 = E_m2, E_m
                E_wp, E_w, E_w2 = E_w, E_w2, E_wp
                advance(pl)
                state["i"] += 1
            torch.cuda.synchronize()
            h = hist.cpu().numpy()
            rel = h[:, :, 0] / np.maximum(h[:, :, 1], 1e-300)
            at = [n for n in (1, 2, 5, 10, 20, 50, 100, 200, 500, 1000) if n <= K]

            def slope(j):
                # least-squares exponent of the relative residual against the step number (second half)
                n = np.arange(1, K + 1)[K // 2:]
                y = np.maximum(rel[K // 2:, j], 1e-300)
                return float(np.polyfit(np.log(n), np.log(y), 1)[0]) if K >= 8 else None
            return {
                "tol_projected": args.tol, "tol_unprojected": tol_cmp, "steps": K, "status": int(lib.status()),
                "rel_residual_at_step": {nm: {str(n): float(rel[n - 1, j]) for n in at} for j, nm in enumerate(names)},
                "rel_residual_max": {nm: float(rel[:, j].max()) for j, nm in enumerate(names)},
                "growth_exponent_second_half": {nm: slope(j) for j, nm in enumerate(names)},
                "ms_mfem_step": float(np.mean([a.elapsed_time(b_) for a, b_, _ in ev])),
                "ms_wave_step": float(np.mean([b_.elapsed_time(c) for _, b_, c in ev])),
            }
        try:
            out = {"what": "Gauss-law residual max|D0^T M E + Q| / scale over interior nodes: the projected step "
                           "against the first-order mixed FEM (trapezoidal Newmark on the E-b system) and Newmark "
                           "on the wave equation, both without the projection, fed the same deposits",
                   "solver": solv[0], "same_tol": run(args.tol)}
            if args.drift_tol > 0:
                out["loose_unprojected"] = run(args.drift_tol)
            return out
        finally:
            F.fem_pic_mfem_destroy(mh)

    drift = None
    if args.drift_steps > 0 and field:
        try:
            drift = measure_gauss_drift()
        except Exception as ex:   # the comparison never takes the main measurement down with it
            drift = {"error": f"{type(ex).__name__}: {ex}"}
    neumann = None if (args.neumann_steps <= 0 or not field) else measure_neumann()

    out = None
    if rank == 0:
        value = whole_job_rate(units_all, total_ms)
        avg_push = push_call
        abytes = push_call_bytes(alive_eager / len(species), sizes["n_tets"])   # one push call (one species)
        peak, peak_kind = peak_hbm()
        achieved = abytes / (avg_push * 1e-3) / 1e9
        fast_ms, fast_n = phases.get("push_fast", (float("nan"), 1))
        fast_avg = fast_ms / max(1, fast_n)
        # bytes of one launch: one species' live particles (alive_eager counts all species),
        # its tet records and deposits
        fbytes = fast_kernel_bytes(alive_eager / len(species), sizes, torch.empty(0, dtype=DEP).element_size(),
                                   torch.empty(0, dtype=DQ).element_size())
        fast_achieved = fbytes / (fast_avg * 1e-3) / 1e9
        roof_push = {"kernel": "k_push_run32", "bound": "hbm", "achieved": fast_achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": fast_achieved / peak,
                     "frac_of_nominal": fast_achieved / NOMINAL_HBM_GBS,
                     "algorithmic_bytes_per_launch": fbytes, "avg_launch_ms": fast_avg,
                     "traffic": measured_traffic("k_push_run32", wl.name)}
        roof = roof_push
        if field:
            nnz = np.zeros(2, dtype=np.int64)
            F.lib().fem_pic_field_nnz(lib.h, nnz.ctypes.data_as(F.ctypes.c_void_p))
            cand = []
            for k_sys, (ph, rows, nz, its, outs) in enumerate(
                    (("cg_newmark", sizes["n_edges"], int(nnz[0]), statistics.mean(iters_n), statistics.mean(outer_n)),
                     ("cg_gauss", sizes["n_nodes"], int(nnz[1]), statistics.mean(iters_g), statistics.mean(outer_g)))):
                t_ms, cnt = phases.get(ph, (0.0, 1))
                if cnt and t_ms > 0:
                    avg = t_ms / cnt
                    mixed = solv[k_sys] == "mixed"
                    # algorithmic bytes: 12 B per nonzero + 76 B per row per CG iteration, times the
                    # solve's (inner) CG iterations
                    byt = cg_iter_bytes(rows, nz) * max(its, 1)
                    lrn = bool(main_pc & (F.FP_PC_LEARNED if k_sys == 0 else F.FP_PC_LEARNED_GAUSS))
                    model = (mixed_solve_bytes(rows, nz, its, outs, 1 if lrn else main_pdeg[k_sys]) if mixed else
                             pcg_bytes_per_iter(rows, nz) * max(its, 1))
                    if lrn:   # one product with the BF16 learned correction per inner iteration
                        model += its * nz * 6
                    op_bytes = nz * 8 * 1.2          # FP32 SELL operator (value + column), ~1.2x padding
                    on_chip = op_bytes < L2_BYTES
                    traffic = measured_traffic(("k_pcg_mixed/" if mixed else "k_pcg/") + ph +
                                               ("/learned" if lrn else ""), wl.name, its)
                    pc_name = ("learned preconditioner" if lrn else
                               f"Chebyshev-Jacobi degree {main_pdeg[k_sys]}" if main_pdeg[k_sys] > 1 else "Jacobi")
                    name = ("k_pcg_mixed (" + ph.split("_")[1] + f" system, FP32 inner PCG, {pc_name}, FP64 residual)"
                            if mixed else "k_pcg (" + ph.split("_")[1] + " system, FP64)")
                    ach = byt / (avg * 1e-3) / 1e9
                    cand.append((avg, {
                        "kernel": name,
                        "bound": "latency" if on_chip else "hbm",
                        "achieved": ach, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": ach / peak,
                        "frac_of_nominal": ach / NOMINAL_HBM_GBS,
                        "algorithmic_bytes_per_launch": byt,
                        "algorithmic_bytes_rule": "12 B per nonzero + 76 B per row per CG iteration (FP64 SpMV + "
                                                  "PCG vectors) x CG iterations per launch",
                        "avg_launch_ms": avg, "iterations_per_launch": its, "refinements_per_launch": outs,
                        "rows": rows, "nnz": nz,
                        "model_bytes_per_launch": model,
                        "model_frac": model / (avg * 1e-3) / 1e9 / peak,
                        "model_rule": ("what the mixed solver moves: the FP32 operator (8 B per nonzero) once per "
                                       "product, deg products per inner iteration, FP32 vector passes, FP64 "
                                       "residuals per refinement" if mixed else "FP64 PCG, 12 B per nonzero + "
                                       "13 FP64 vector passes per iteration"),
                        "traffic": traffic,
                        "traffic_frac": None if traffic is None else traffic / (avg * 1e-3) / 1e9 / peak,
                        "note": ("the FP32 operator fits on chip (shared memory / L2): DRAM traffic is about one "
                                 "read of it per launch and the kernel is bound by its grid barriers and gather "
                                 "latency, not by HBM" if on_chip else
                                 "the FP32 operator is larger than L2: every product streams it from HBM")}))
            cand.append((fast_avg, roof_push))
            roof = max(cand, key=lambda c: c[0])[1]
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "mesh": f"cube {wl.mesh.n}^3 x 6 tets, +-10% jitter" if wl.mesh.n > 4
                       else f"cube {wl.mesh.n}^3 x 6 tets", "n_tets": sizes["n_tets"], "n_edges": sizes["n_edges"],
                       "particles": n_part, "alive_in_timed_steps": alive_timed,
                       "counted": "particle-steps of live particles only; every measured region starts from the "
                                  "initial state (particles absorbed by the PEC walls are not counted)",
                       "species": len(species), "dt_s": wl.dt, "B0_T": list(wl.B0),
                       "sort_every": args.sort_every, "precision": "fp32 particle path, fp64 walk test",
                       "deposits": {"fp64": "double dG and Q (FP32 contributions added with FP64 atomics)",
                                    "change": "float dG (FP32 atomics); double Q carried from step to step, each "
                                              "particle's FP32 charge change added with FP64 atomics",
                                    "change64": "double dG (FP64 atomics); double Q carried from step to step, "
                                                "each particle's FP32 charge change added with FP64 atomics",
                                    "fp32": "float dG and Q (FP32 atomics)"}[args.deposits],
                       "l2": "flushed between timed steps: 256 MB written, then another 256 MB read (outside the step events)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "step": "sort (periodic) + push/gather/walk/deposit + implicit field step "
                               "(Newmark + Gauss-law projection + Faraday, Jacobi-CG to 1e-10 relative residual in FP64) "
                               "+ fp64 residuals"},
            "roofline": roof,
            "roofline_push": roof_push,
            "roofline_push_call": {"kernels": "k_field_prep32 + k_push_run32 + k_walk32 (sum of kernel times)",
                                   "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                   "frac": achieved / peak, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                                   "algorithmic_bytes_per_launch": abytes,
                                   "algorithmic_bytes_rule": "56 B per particle + 230 B per tet",
                                   "avg_call_ms": avg_push},
            "timing": ("timed steps replay one CUDA graph per step shape" if use_graphs else "eager launches") +
                      "; per-kernel times from an eager pass of the same steps with the library's CUDA-event profiler",
            "phases_ms_per_step": {k: v[0] / args.steps for k, v in phases.items()},
            "host_ms_per_step": (th1 - th0) * 1e3 / args.steps,
            "push_deposit_particle_steps_per_s": alive_eager / len(species) / (avg_push * 1e-3),
            "field_solve": None if not field else {
                "ms_per_step": sum(phases.get(k, (0.0, 1))[0] for k in ("field_other", "cg_newmark", "cg_gauss",
                                                                          "learned")) / args.steps,
                "precond": {nm: ("learned preconditioner" if main_pc & bit else
                                 (f"Chebyshev-Jacobi degree {main_pdeg[k_]}" if main_pdeg[k_] > 1 else "jacobi"))
                            for k_, (nm, bit) in enumerate((("newmark", F.FP_PC_LEARNED),
                                                            ("gauss", F.FP_PC_LEARNED_GAUSS)))},
                "learned_vs_plain": learned,
                "solver": {"newmark": solv[0], "gauss": solv[1], "mixed": "refinement: FP64 residual, FP32 "
                           "inner Jacobi-PCG (FP32 products, dot products and grid sums)", "fp64": "plain FP64 Jacobi-PCG",
                           "inner_tol": args.inner_tol,
                           "inner_precond_degree": {"newmark": main_pdeg[0], "gauss": main_pdeg[1]},
                           "chebyshev_ratio": {"newmark": prat[0], "gauss": prat[1]}},
                "ms_newmark_cg": phases.get("cg_newmark", (0.0, 1))[0] / args.steps,
                "ms_gauss_cg": phases.get("cg_gauss", (0.0, 1))[0] / args.steps,
                "initial_guess": "2E^n - E^(n-1) (Newmark), 0 (Gauss)",
                "tol": args.tol, "newmark_iters": iters_n, "gauss_iters": iters_g,
                "newmark_iters_mean": statistics.mean(iters_n),
                "gauss_iters_mean": statistics.mean(iters_g), "max_rel_res": max(relres),
                "newmark_refinements_mean": statistics.mean(outer_n), "gauss_refinements_mean": statistics.mean(outer_g),
                "n_edges": sizes["n_edges"], "n_nodes": sizes["n_nodes"]},
            "eager_ms_per_step": statistics.mean(push_ms),
            "residuals": {"continuity_interior_max": float(r[4]), "continuity_interior_scale": float(r[5]),
                          "continuity_all_nodes_max": float(r[0]), "continuity_all_nodes_scale": float(r[1]),
                          "divB_max": float(r[2]), "divB_scale": float(r[3]),
                          "per_step": {
                              "what": "every timed step: max|D0^T dG - (Q^{n+1} - Q^n)| over interior nodes and "
                                      "max|D2 b| over tets, each over its scale (FP64 residual kernel)",
                              "continuity_interior_rel_max": float(np.max(rlog[:, 4] / np.maximum(rlog[:, 5], 1e-300))),
                              "divB_rel_max": float(np.max(rlog[:, 2] / np.maximum(rlog[:, 3], 1e-300))),
                              "continuity_interior_rel": [float(f"{x:.3e}") for x in
                                                          rlog[:, 4] / np.maximum(rlog[:, 5], 1e-300)],
                              "divB_rel": [float(f"{x:.3e}") for x in rlog[:, 2] / np.maximum(rlog[:, 3], 1e-300)]}},
            "status": int(st),
            "clocks": clocks,
            "gpu_launches": launches,
            "e2e": e2e,
            "adams": adams,
            "neumann": neumann,
            "gauss_drift": drift,
            "fp64_mode": fp64,
        }
    del lib
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return out, wl


def measure_adams(args, lib, F, species, restore, bufs, cur, e, b, dG, Qn, flush_l2, stream, sizes, wl, dev):
    """The particle step with the fourth-order Adams mover (fem_pic_push_deposit_adams) on the
    same particles and fields, from the initial state: three start-up steps (orders 1-3), one
    more warm-up step, then args.adams_steps timed calls at order 4 (L2 flushed between them).
    dt is a quarter of the workload's (omega_c dt = 0.1 pi), inside the explicit method's
    stability interval for gyration.  Particles are not re-sorted inside this short run."""
    import torch
    restore()
    sps = [bufs[k][cur[k]] for k in range(len(species))]
    hist = [torch.zeros((18, s_.n), dtype=torch.float32, device=dev) for s_ in sps]
    dt = wl.dt / 4
    step = 0

    # the Adams mover takes FP32 deposits: arrays of its own while it runs, the context's setting
    # restored after
    dep_keep = F.fem_pic_deposit_precision(lib.h), F.fem_pic_charge_precision(lib.h)
    lib.set_deposit_precision(F.FP_FP32)
    dG = torch.zeros(sizes["n_edges"], dtype=torch.float32, device=dev)
    Qn = torch.zeros(sizes["n_nodes"], dtype=torch.float32, device=dev)
    def call():
        nonlocal step
        dG.zero_()
        Qn.zero_()
        for k, (s_, h_) in enumerate(zip(sps, hist)):
            lib.push_deposit_adams(e, b, s_, h_, step, dt, dG, Qn,
                                   flags=F.FP_ACCUMULATE | (F.FP_SAME_FIELDS if k else 0))
        step += 1

    for _ in range(4):
        call()
    torch.cuda.synchronize()
    F.fem_pic_profile_read(lib.h, reset=True)
    F.fem_pic_profile_enable(lib.h, True)
    ev, live = [], []
    for k in range(args.adams_steps):
        live.append(sum(int((s_.cell >= 0).sum()) for s_ in sps))
        flush_l2(1000 + k)
        a = torch.cuda.Event(enable_timing=True)
        z = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        call()
        z.record(stream)
        ev.append((a, z))
    torch.cuda.synchronize()
    F.fem_pic_profile_enable(lib.h, False)
    ph = F.fem_pic_profile_read(lib.h, reset=True)
    st = lib.status()
    lib.set_deposit_precision(dep_keep[0])
    lib.set_charge_precision(dep_keep[1])
    ms = sum(a.elapsed_time(z) for a, z in ev)
    n_live = sum(live) / len(live)
    f_ms, f_n = ph.get("adams_push", (float("nan"), 1))
    w_ms, _ = ph.get("adams_walk", (0.0, 1))
    p_ms, _ = ph.get("prep", (0.0, 1))
    f_avg = f_ms / max(1, f_n)
    byt = adams_kernel_bytes(n_live / len(sps), sizes)
    peak, peak_kind = peak_hbm()
    ach = byt / (f_avg * 1e-3) / 1e9
    return {"particle_steps_per_s": sum(live) / (ms * 1e-3), "ms_per_call": ms / args.adams_steps,
            "order": 4, "dt_s": dt, "timed_calls": args.adams_steps, "alive_mean": n_live, "status": int(st),
            "kernel_ms_per_call": {"k_field_prep32": p_ms / args.adams_steps, "fast_push": f_avg,
                                   "k_walk_adams32": w_ms / args.adams_steps},
            "roofline": {"kernel": "k_push_ws32<AdamsStep<float>> (warp-specialised push with the Adams mover; "
                                   "k_push_adams32 when the state is not 16-byte aligned)",
                         "bound": "hbm", "achieved": ach, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": ach / peak,
                         "frac_of_nominal": ach / NOMINAL_HBM_GBS,
                         "algorithmic_bytes_per_launch": byt, "avg_launch_ms": f_avg,
                         "traffic": measured_traffic("k_push_ws32/adams", wl.name)}}


def measure_fp64(args, F, wl, dev, flush_l2, stream):
    """The particle step in FP64 mode (FP64 state, fields, Boris, walk and deposits: the per-tet
    field records, then k_push_deposit<double>) on the same particles and B0, in a context of its own: cell-sorted
    state, 3 warm-up calls, then args.fp64_steps timed calls (L2 flushed between them)."""
    import torch
    lib = F.FemPic(wl.mesh.xyz, wl.mesh.tets, F.FP_FP64)
    sizes = lib.sizes
    sps = []
    for s in wl.species:
        d0 = lib.species(s.cell, s.X, s.V, s.q, s.m, s.w, device=dev)
        d1 = d0.empty_like()
        lib.sort(d0, d1)
        sps.append(d1)
    e, b = lib.fields_uniform((0.0, 0.0, 0.0), wl.B0, device=dev)
    dG = torch.zeros(sizes["n_edges"], dtype=torch.float64, device=dev)
    Q = torch.zeros(sizes["n_nodes"], dtype=torch.float64, device=dev)

    def call():
        dG.zero_()
        Q.zero_()
        for k, s_ in enumerate(sps):
            lib.push_deposit(e, b, s_, wl.dt, dG, Q, flags=F.FP_ACCUMULATE | (F.FP_SAME_FIELDS if k else 0))
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    F.fem_pic_profile_read(lib.h, reset=True)
    F.fem_pic_profile_enable(lib.h, True)
    ev, live = [], []
    for k in range(args.fp64_steps):
        live.append(sum(int((s_.cell >= 0).sum()) for s_ in sps))
        flush_l2(3000 + k)
        a = torch.cuda.Event(enable_timing=True)
        z = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        call()
        z.record(stream)
        ev.append((a, z))
    torch.cuda.synchronize()
    F.fem_pic_profile_enable(lib.h, False)
    ph = F.fem_pic_profile_read(lib.h, reset=True)
    st = lib.status()
    ms = sum(a.elapsed_time(z) for a, z in ev) / len(ev)
    k_ms, k_n = ph.get("push_fp64", (float("nan"), 1))
    k_avg = k_ms / max(1, k_n)
    n_live = sum(live) / len(live)
    byt = algorithmic_bytes(n_live / len(sps), sizes, 8)
    peak, peak_kind = peak_hbm()
    ach = byt / (k_avg * 1e-3) / 1e9
    lib.close()
    return {"particle_steps_per_s": sum(live) / (ms * 1e-3 * len(ev)), "ms_per_call": ms, "status": int(st),
            "timed_calls": len(ev), "alive_mean": n_live,
            "kernel": "k_push_deposit<double>", "avg_launch_ms": k_avg,
            "bound": "FP64 pipe: every particle takes the FP64 fields (per-tet affine records), push, exit test "
                     "and walk (GB300 issues 2 FP64 operations per clock per SM), not HBM",
            "algorithmic_bytes_per_launch": byt, "hbm_achieved_gbs": ach, "hbm_frac": ach / peak,
            "hbm_peak_gbs": peak, "hbm_peak_kind": peak_kind}


def oracle_sample_size(orc, sp, e, b, dt, threads, step_s, cap=8_000_000):
    """Particles per oracle call such that one call takes about step_s seconds.  Each call pays a
    fixed cost per mesh entity (its thread-private deposit arrays, first touched by the first
    call) besides its cost per particle: after one untimed call, calls of n1 and 16 n1 particles
    give the two, and the sample is sized from them (at most cap particles)."""
    def call(n):
        t = time.perf_counter()
        orc.step(sp.cell[:n], sp.X[:n], sp.V[:n], e, b, sp.q, sp.m, sp.w, dt, nthreads=threads)
        return time.perf_counter() - t
    n1 = min(sp.n, 20000)
    call(min(sp.n, 1000))
    t1 = call(n1)
    n2 = min(sp.n, 16 * n1)
    if n2 <= n1:
        return n1
    t2 = call(n2)
    per = max((t2 - t1) / (n2 - n1), 1e-12)
    fixed = max(t1 - per * n1, 0.0)
    return int(min(sp.n, cap, max(n2, (step_s - fixed) / per)))


def cpu_baseline(args, wl, budget_s):
    """The FP64 oracle as it stands, on the host cores, over a bounded sample of the workload."""
    import oracle as O
    orc = O.Oracle(wl.mesh.xyz, wl.mesh.tets)
    e, b = orc.project_uniform((0.0, 0.0, 0.0), wl.B0)
    sp = wl.species[0]
    threads = O.nproc_threads()
    n2 = oracle_sample_size(orc, sp, e, b, wl.dt, threads, 0.25 * budget_s)
    done, el = 0, 0.0
    while el < 0.5 * budget_s or done == 0:
        t = time.perf_counter()
        orc.step(sp.cell[:n2], sp.X[:n2], sp.V[:n2], e, b, sp.q, sp.m, sp.w, wl.dt, nthreads=threads)
        el += time.perf_counter() - t
        done += n2
    # the field step of the oracle (scipy: direct solve of the Gauss-law projection, CG on the
    # Newmark system to 1e-13), one step on the same mesh with a continuity-respecting current
    field = None
    if wl.mesh.n > 32 and not args.no_field:
        field = {"skipped": "the oracle's scipy field step is timed on the 32^3 and smaller meshes only (at this "
                            "size one step takes minutes on one host thread)"}
    elif not args.no_field and not args.no_cpu_field:
        import numpy as np
        from oracle import fields as OF
        t = time.perf_counter()
        fo = OF.FieldOracle(orc.cx, wl.dt)
        t_setup = time.perf_counter() - t
        rng = np.random.default_rng(0)
        cx = orc.cx
        E0 = 1e3 * rng.uniform(-1.0, 1.0, cx.n_edges)
        E0[cx.boundary_edge] = 0.0
        dG = 1e-12 * rng.uniform(-1.0, 1.0, cx.n_edges)
        dG[cx.boundary_edge] = 0.0
        Q = cx.D0().T @ dG
        t = time.perf_counter()
        fo.step(E0, E0, b, dG, np.zeros_like(dG), Q)
        field = {"ms_per_field_step": (time.perf_counter() - t) * 1e3, "setup_s": t_setup, "threads": 1,
                 "what": "oracle field step (Newmark CG + Gauss-law projection by a direct solve + Faraday), "
                         "scipy on one host thread"}
    # the same oracle on one host thread, over a smaller sample
    n1 = min(sp.n, 20000)
    t = time.perf_counter()
    orc.step(sp.cell[:n1], sp.X[:n1], sp.V[:n1], e, b, sp.q, sp.m, sp.w, wl.dt, nthreads=1)
    el1 = time.perf_counter() - t
    return {"value": done / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n2} of {sp.n} particles of species 0, {done // n2} step(s), FP64 oracle (C, OpenMP), "
                      f"{el:.1f} s",
            "value_1_thread": n1 / max(el1, 1e-9), "sample_1_thread": f"{n1} particles, 1 step, 1 thread",
            "field_step": field}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    wl = build_workload(args)
    import oracle as O
    orc = O.Oracle(wl.mesh.xyz, wl.mesh.tets)
    e, b = orc.project_uniform((0.0, 0.0, 0.0), wl.B0)
    threads = O.nproc_threads()
    sp = wl.species[0]
    # each step is a bounded sample sized so the whole run stays within a few minutes
    per_step_s = min(4.0, 150.0 / max(1, args.steps + args.warmup))
    ns = oracle_sample_size(orc, sp, e, b, wl.dt, threads, per_step_s)
    cell, X, V = sp.cell[:ns].copy(), sp.X[:ns].copy(), sp.V[:ns].copy()
    for _ in range(args.warmup):
        r = orc.step(cell, X, V, e, b, sp.q, sp.m, sp.w, wl.dt, nthreads=threads)
        cell, X, V = r["cell"], r["X"], r["V"]
    t = time.perf_counter()
    for _ in range(args.steps):
        r = orc.step(cell, X, V, e, b, sp.q, sp.m, sp.w, wl.dt, nthreads=threads)
        cell, X, V = r["cell"], r["X"], r["V"]
    el = time.perf_counter() - t
    value = ns * args.steps / el
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": wl.name, "particles_per_step_sample": ns, "particles_full": sp.n,
                      "step": "FP64 oracle particle step (gather, Boris, walk, deposit) on host cores"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": f"{ns} of {sp.n} particles per step"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_also(args):
    """The further workloads of --also: the same timed PIC steps (and per-kernel pass), without
    the side measurements; returns {workload name: its main numbers}."""
    import copy
    import gc
    import torch
    res = {}
    for tok in [x for x in args.also.split(",") if x.strip()]:
        idx = int(tok)
        if idx == args.workload:
            continue
        a = copy.copy(args)
        a.workload, a.also, a.learned = idx, "", "off"
        a.no_e2e, a.fp64_steps, a.adams_steps, a.neumann_steps, a.drift_steps = True, 0, 0, 0, 0
        a.steps = max(args.steps, 20)
        o, wl2 = run_gpu(a)
        gc.collect()
        torch.cuda.empty_cache()
        if o is None:
            continue
        fs = o.get("field_solve") or {}
        res[wl2.name] = {k: o[k] for k in ("value", "unit", "ms_per_step", "steps", "roofline", "roofline_push",
                                           "roofline_push_call", "phases_ms_per_step", "residuals", "clocks",
                                           "gpu_launches", "status")}
        res[wl2.name]["config"] = o["config"]
        res[wl2.name]["field_solve"] = {k: fs.get(k) for k in ("ms_per_step", "newmark_iters_mean",
                                                                 "gauss_iters_mean", "max_rel_res")}
    return res


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    out, wl = run_gpu(args)
    rank, world, _ = dist_env()
    also = run_also(args) if world == 1 and args.also else None
    if rank == 0 and out is not None:
        if also:
            out["workloads"] = also
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args, wl, args.cpu_seconds)
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
