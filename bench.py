#!/usr/bin/env python
"""Throughput of the fermion part of the many-flavour HMC MD step on GB300.

One step = one pass of the hot path on the 12^4 SF workload with 5
pseudo-fermion fields (N_f = 10): link preparation for the current gauge
field (SU(3) check, FP64/FP32/FP16 kernel copies), the blocked solves of
Alg. 2 (X = Dhat^-1 Phi, Y = Dhat^-dag X to true relative residual 1e-10, FP32
BiCGStab inner / FP64 defect-correction outer), odd-site reconstruction and
the force F = sum_i f[x_i, y_i] of Eq. (3) with the FP64 momentum update.
The metric is 5-RHS solves per second (a solve = X and Y for all 5 fields,
plus the force), summed over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the same workload (full
steps, measured, on the host cores).  Under torchrun every rank runs its own
replica of the workload (the path has no exchange step); the time is the
maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "5-RHS SF Wilson solves/s at true rel. residual 1e-10"
UNIT = "solves/s"
L2_FLUSH_BYTES = 512 << 20


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_hash():
    h = hashlib.sha256()
    for f in ("hop.cuh", "sf_device.cuh"):
        with open(os.path.join(ROOT, "paper_1009_5169_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(key, TS, NR, pipe=0):
    """Per-launch DRAM bytes of the dslash kernel at this tiling from the
    committed ncu summary, if it was taken on the current kernel source."""
    try:
        with open(os.path.join(ROOT, "profiles", "dslash_traffic.json")) as f:
            d = json.load(f)
        e = d.get(f"{key}:TS{TS}NR{NR}" + (f":pipe{pipe}" if pipe else ""))
        if e and e.get("kernel_hash") == _kernel_hash():
            return e
    except Exception:
        pass
    return None


def max_over_ranks(x: float, device=None) -> float:
    """The maximum of x over all ranks of the initialised process group (x on
    a single process); every rank gets the result."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"sf_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# --------------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1009_5169_gb300 import binding as sf
    from paper_1009_5169_gb300 import inputs

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    w = inputs.workload(args.workload)
    lt = w.lattices[0]
    nrhs, tol = w.nrhs, w.tol
    U = lt.make_links()
    phi = lt.make_sources(nrhs)
    stream = torch.cuda.current_stream(dev)
    U_d = torch.from_numpy(U).to(dev)
    phi_d = torch.from_numpy(phi).to(dev)
    X_d = torch.empty_like(phi_d)
    Y_d = torch.empty_like(phi_d)
    fshape = ((lt.T + 1) * lt.L ** 3, 4, 8)
    F_d = torch.zeros(fshape, dtype=torch.float64, device=dev)
    mom_d = torch.zeros(fshape, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    lat = sf.Lattice(lt.L, lt.T, lt.theta, lt.kappa, lt.beta, U_d, device=local_rank)
    # the precision of the inner solve (its hop is the kernel the roofline reports)
    prec = "fp32" if args.algo in ("mixed_dc", "cg_normal") else ("fp16" if args.algo == "mixed_dc_half" else "fp64")
    if args.solve_tiling:  # fixed inner-solve tiling instead of the autotuner's (for reproducible profiles)
        lat.set_tuning(prec, *args.solve_tiling)
    eps_md = 0.01

    def step(Ub, ph, X, Y, F, mom):
        # the links of this MD step, then Alg. 2: X, Y and the force (the odd
        # sites of X, Y come from the final residuals' hops)
        lat.set_links(Ub)
        return sf.md_force_step(lat, args.algo, ph, X, Y, F, mom, eps=eps_md, tol=tol, maxiter=args.maxiter)

    # launches per step outside md_force_step's own count: SU(3) check + link prep
    fixed_launches = 2
    for _ in range(args.warmup):
        info = step(U_d, phi_d, X_d, Y_d, F_d, mom_d)
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches = 0
    infos = []
    for k in range(args.steps):
        flush.zero_()                      # L2 flushed between steps (outside the timed step)
        starts[k].record(stream)
        info = step(U_d, phi_d, X_d, Y_d, F_d, mom_d)
        ends[k].record(stream)
        infos.append(info)
        launches += info["kernel_launches"] + fixed_launches
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), dev)
    ms_per_step = ms / args.steps
    value = world * args.steps / (ms / 1e3)

    # accuracy of the last step, from the library's FP64 recomputation
    last = infos[-1]
    resid = max(max(last["true_resid"]), max(last["true_resid_y"]))

    # ---------------- end to end through the public API with host buffers
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    U_h, phi_h = pin(U), pin(phi)
    X_h, Y_h = torch.empty_like(phi_h).pin_memory(), torch.empty_like(phi_h).pin_memory()
    F_h = torch.zeros(fshape, dtype=torch.float64).pin_memory()
    mom_h = torch.zeros(fshape, dtype=torch.float64).pin_memory()
    step(U_h, phi_h, X_h, Y_h, F_h, mom_h)
    e2e_s = 0.0
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(U_h, phi_h, X_h, Y_h, F_h, mom_h)
        torch.cuda.synchronize()
        e2e_s += time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dev)
    nb = lambda a: a.numel() * a.element_size()
    h2d = nb(U_h) + nb(phi_h) + nb(mom_h)   # links, phi, mom (md_force_step only writes X, Y, F)
    d2h = nb(X_h) + nb(Y_h) + nb(F_h) + nb(mom_h)
    e2e = {"value": world * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # ---------------- accuracy re-check outside the timed region: solve_block
    # recomputes the FP64 true residual |Phi - Dhat X| / |Phi| of every RHS.
    # With the normal-equation route X is formed as Dhat^dag Y by the FP64
    # kernel, so |X - Dhat^dag Y| is zero by construction and Y's accuracy is
    # that of |Phi - Dhat Dhat^dag Y| = |Phi - Dhat X|; the oracle's own
    # residuals of the final X and Y (both equations of Alg. 2) are in
    # cpu_baseline.oracle_check.
    chk = sf.solve_block(lat, args.algo, phi_d, X_d, Y_d, tol=tol, maxiter=args.maxiter)
    recheck = {"max_true_rel_resid_x": max(chk["true_resid"]),
               "max_true_rel_resid_y": max(chk["true_resid_y"]),
               "note": ("cg_normal: X = Dhat^dag Y by construction, so the Y line is |X - Dhat^dag Y| = 0; "
                        "the oracle's residuals of both are under cpu_baseline.oracle_check")
               if args.algo == "cg_normal" else "library FP64 recomputation"}
    host_solution = {"X": X_d.cpu().numpy(), "Y": Y_d.cpu().numpy()}

    # ---------------- the 16^4 kappa 0.134 workload: FP32- and FP16-inner
    # solves (their per-RHS error against the oracle is measured in the
    # cpu_baseline leg)
    acc_cfg = None
    if not args.no_accuracy_configs and rank == 0:
        acc_cfg = accuracy_config_solves(args, sf, inputs, dev, local_rank)

    # ---------------- roofline of the dominant kernel: the FP32 dslash (hop)
    peak, peak_kind = _peaks()
    TS, NR, PIPE = lat.get_tuning(prec, nrhs)
    Vh = lt.Vh
    site_bytes = {"fp32": nrhs * 96 * 2 + 8 * 48, "fp16": nrhs * 52 * 2 + 8 * 24,
                  "fp64": nrhs * 192 * 2 + 8 * 144}[prec]
    alg_bytes = Vh * site_bytes
    sf.wilson_hop_resident(lat, prec, nrhs, 1)
    reps = 50
    cold = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sf.wilson_hop_resident(lat, prec, nrhs, 1)
        b.record(stream)
        cold.append((a, b))
    torch.cuda.synchronize()
    t_cold = statistics.mean(a.elapsed_time(b) for a, b in cold) * 1e-3
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        sf.wilson_hop_resident(lat, prec, nrhs, 1)
    b.record(stream)
    torch.cuda.synchronize()
    t_warm = a.elapsed_time(b) * 1e-3 / reps
    achieved = alg_bytes / t_cold / 1e9
    tr = _ncu_traffic(f"{args.workload}:{prec}", TS, NR, PIPE)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": tr["dram_bytes_per_launch"] if tr else None,
                "kernel": f"k_hop<{prec}> (dslash H_oe), TS={TS}, NR={NR}, pipelined={PIPE}, "
                          "L2 flushed before each launch",
                "algorithmic_bytes_per_launch": alg_bytes, "launch_us": round(t_cold * 1e6, 2),
                "l2_warm_launch_us": round(t_warm * 1e6, 2), "peak_kind": peak_kind}

    # ---------------- the FP64 kernels of the step against the FP64 pipe: the
    # hop of the true residuals and the force (both bound by FP64 arithmetic on
    # this GPU, whose FP64 rate is 1/64 of FP32's)
    fp64 = fp64_roofline(sf, lat, lt, nrhs, stream, flush, dev)

    # ---------------- dslash on a lattice larger than L2 (HBM-bound case)
    hbm = None
    if not args.no_hbm_case and rank == 0:
        Lh, Th = 32, 32
        Ub = inputs.links(Lh, Th, 0.2, inputs.SEED_BASE + 32)
        big = sf.Lattice(Lh, Th, 0.5, 0.13, 4.52, torch.from_numpy(Ub).to(dev), device=local_rank)
        del Ub
        res = {}
        for p in ("fp32", "fp16"):
            TSb, NRb, PIPEb = big.get_tuning(p, nrhs)
            sf.wilson_hop_resident(big, p, nrhs, 1)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(20):
                sf.wilson_hop_resident(big, p, nrhs, 1)
            b.record(stream)
            torch.cuda.synchronize()
            t = a.elapsed_time(b) * 1e-3 / 20
            cold = []
            for _ in range(20):
                flush.zero_()
                c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                c0.record(stream)
                sf.wilson_hop_resident(big, p, nrhs, 1)
                c1.record(stream)
                cold.append((c0, c1))
            torch.cuda.synchronize()
            tc = statistics.mean(c0.elapsed_time(c1) for c0, c1 in cold) * 1e-3
            Vhb = Lh ** 3 * (Th - 1) // 2
            sb = {"fp32": nrhs * 96 * 2 + 8 * 48, "fp16": nrhs * 52 * 2 + 8 * 24}[p]
            ab = Vhb * sb
            trb = _ncu_traffic(f"sf32:{p}", TSb, NRb, PIPEb)
            res[p] = {"achieved": round(ab / t / 1e9, 1), "frac": round(ab / t / 1e9 / peak, 4),
                      "launch_us": round(t * 1e6, 2), "achieved_l2_flushed": round(ab / tc / 1e9, 1),
                      "launch_us_l2_flushed": round(tc * 1e6, 2), "algorithmic_bytes_per_launch": ab,
                      "TS": TSb, "NR": NRb, "pipelined": PIPEb,
                      "traffic": trb["dram_bytes_per_launch"] if trb else None}
        big.close()
        hbm = {"lattice": f"{Lh}^3x{Th} SF, 5 RHS (working set per launch larger than L2)", "unit": "GB/s",
               "peak": peak, **res}

    # ---------------- solver comparators on the same workload (X and Y, no force)
    comparators = None
    if not args.no_comparators:
        def time_solve(algo, ph, Xo, Yo, reps=3):
            sf.solve_block(lat, algo, ph, Xo, Yo, tol=tol, maxiter=args.maxiter)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                inf = sf.solve_block(lat, algo, ph, Xo, Yo, tol=tol, maxiter=args.maxiter)
            torch.cuda.synchronize()
            return (time.perf_counter() - t0) / reps, inf
        comparators = {}
        for algo in ("bicgstab", "mixed_dc", "mixed_dc_half", "cg_normal", "gl_bicgstab", "bl_bicgstab"):
            # gl_bicgstab: the paper's D1 solver, its "sweeps" are preconditioner calls;
            # bl_bicgstab: the paper's case C, its "inner_iters" are block iterations
            t, inf = time_solve(algo, phi_d, X_d, Y_d)
            comparators[f"{algo}_block{nrhs}"] = {
                "ms": round(t * 1e3, 3), "sweeps": [inf["iters_outer"], inf["iters_outer_y"]],
                "inner_iters": [inf["iters_inner"], inf["iters_inner_y"]],
                "max_true_rel_resid": max(max(inf["true_resid"]), max(inf["true_resid_y"]))}
        # the plain FP64 single-RHS solver run once per field, in sequence
        one = [phi_d[i:i + 1].contiguous() for i in range(nrhs)]
        X1, Y1 = torch.empty_like(one[0]), torch.empty_like(one[0])
        sf.solve_block(lat, "bicgstab", one[0], X1, Y1, tol=tol, maxiter=args.maxiter)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        worst = 0.0
        for i in range(nrhs):
            inf = sf.solve_block(lat, "bicgstab", one[i], X1, Y1, tol=tol, maxiter=args.maxiter)
            worst = max(worst, inf["true_resid"][0], inf["true_resid_y"][0])
        torch.cuda.synchronize()
        t_seq = time.perf_counter() - t0
        comparators["bicgstab_fp64_single_rhs_x5"] = {"ms": round(t_seq * 1e3, 3), "max_true_rel_resid": worst}
        best = min(v["ms"] for k, v in comparators.items() if k.startswith("mixed"))
        comparators["speedup_best_vs_fp64_single_rhs_x5"] = round(t_seq * 1e3 / best, 2)
        lat.get_tuning("fp64", nrhs)  # restore the 5-RHS workspace

    # ---------------- batched uneven workload: 24 lattices in one launch per kernel
    batched = None
    if not args.no_batched and rank == 0:
        wb = inputs.workload("batched_uneven")
        blats = [sf.Lattice(b.L, b.T, b.theta, b.kappa, b.beta, torch.from_numpy(b.make_links()).to(dev),
                            device=local_rank) for b in wb.lattices]
        bphi = [torch.from_numpy(b.make_sources(wb.nrhs)).to(dev) for b in wb.lattices]
        bX = [torch.empty_like(p) for p in bphi]
        bY = [torch.empty_like(p) for p in bphi]
        batch = sf.Batch(blats, wb.nrhs)
        balgo = args.algo if args.algo in ("bicgstab", "mixed_dc", "mixed_dc_half", "cg_normal") else "mixed_dc"
        batch.solve(balgo, bphi, bX, bY, tol=wb.tol, maxiter=args.maxiter)
        torch.cuda.synchronize()
        reps = 3
        t0 = time.perf_counter()
        for _ in range(reps):
            binfo = batch.solve(balgo, bphi, bX, bY, tol=wb.tol, maxiter=args.maxiter)
        torch.cuda.synchronize()
        tb = (time.perf_counter() - t0) / reps
        for l, bl in enumerate(blats):
            sf.solve_block(bl, balgo, bphi[l], bX[l], bY[l], tol=wb.tol, maxiter=args.maxiter)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for l, bl in enumerate(blats):
            sf.solve_block(bl, balgo, bphi[l], bX[l], bY[l], tol=wb.tol, maxiter=args.maxiter)
        torch.cuda.synchronize()
        ts = time.perf_counter() - t0
        batched = {"workload": "24 SF fields: 8 each of 8^4, 12^4, 16^4; eps 0.15/0.25/0.35; kappa 0.13; 5 RHS; "
                               "X and Y to 1e-10, FP32 inner / FP64 outer", "algo": balgo,
                   "batched_solves_per_s": round(len(blats) / tb, 2), "batch_ms": round(tb * 1e3, 2),
                   "one_lattice_at_a_time_ms": round(ts * 1e3, 2), "speedup": round(ts / tb, 2),
                   "groups": batch.num_groups,
                   "max_true_rel_resid": max(max(max(i["true_resid"]), max(i["true_resid_y"])) for i in binfo)}
        batch.close()
        for bl in blats:
            bl.close()

    # ---------------- HMC trajectories around the MD step (same lattice and pseudo-fermion count)
    hmc = None
    if not args.no_hmc and rank == 0:
        hmc = hmc_section(args, sf, inputs, lt, U_d, nrhs, tol, fshape, dev, local_rank)

    learned, learned_check = None, None
    if not args.no_learned and rank == 0:
        learned_check, learned = learned_section(args, dev, local_rank, stream)

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner / f64 outer" if prec == "fp32" else prec,
        "data": "synthetic (seeded SF gauge field exp(i eps H) and Gaussian pseudo-fermions)",
        "config": {"workload": _workload_desc(args.workload, lt, nrhs, tol),
                   "algo": args.algo, "l2": "flushed between steps", "parallelism": f"replicas x{world}",
                   "tiling": {"fp64": lat.get_tuning("fp64", nrhs), prec: (TS, NR, PIPE)}},
        "accuracy": {"max_true_rel_resid": resid, "sweeps_x": last["iters_outer"], "inner_iters_x": last["iters_inner"],
                     "sweeps_y": last["iters_outer_y"], "inner_iters_y": last["iters_inner_y"],
                     "solve_block_recheck": recheck},
        "roofline": roofline, "fp64_roofline": fp64, "dslash_hbm": hbm, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
        "comparators": comparators, "batched": batched, "hmc_trajectory": hmc, "learned": learned,
        "accuracy_configs": acc_cfg["summary"] if acc_cfg else None,
    }
    lat.close()
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, host_solution, acc_cfg, learned_check)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# --------------------------------------------------------------------- oracle
def _oracle_full_step(w, U, phi):
    """One full step of the FP64 oracle on the workload: X = Dhat^-1 Phi and
    Y = Dhat^-dag X for every pseudo-fermion field to the workload's true
    residual (textbook BiCGStab, one field after the other), then the force of
    Eq. (3).  Returns (seconds, X, Y, info)."""
    import oracle
    lt = w.lattices[0]
    t0 = time.perf_counter()
    X, Y, info = oracle.solve_pair(U, phi, lt.L, lt.T, lt.theta, lt.kappa, tol=w.tol, maxiter=20000)
    oracle.force(U, X, Y, lt.L, lt.T, lt.theta, lt.kappa)
    return time.perf_counter() - t0, X, Y, info


def _workload_desc(name, lt, nrhs, tol):
    """The workload as both arms name it in `config`."""
    return (f"{name}: {lt.L}^3x{lt.T} SF, eps {lt.eps}, kappa {lt.kappa}, theta {lt.theta}, {nrhs} RHS, "
            f"tol {tol}, X and Y solves + force")


def _host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _per_rhs_relerr(a, b):
    n = a.shape[0]
    return (np.linalg.norm((a - b).reshape(n, -1), axis=1) / np.linalg.norm(b.reshape(n, -1), axis=1)).tolist()


def cpu_baseline(args, host_solution=None, acc_cfg=None, learned_check=None):
    """The FP64 oracle as it stands, timed on the host cores: full steps of
    the bench workload (every field's X and Y to the workload's residual and
    the force), once with OpenMP on every core this process may run on and
    once single-threaded.  The same leg checks the GPU's results with the
    oracle: its true residuals of the bench step's X and Y, and on the 16^4
    kappa 0.134 workload every RHS's error of the FP32- and FP16-inner
    solutions against the oracle's own solutions (solved to 1e-12), and the
    oracle's residuals of every solver's X and Y on the first held-out 24^4
    field of the learned-preconditioner comparison."""
    import oracle
    from paper_1009_5169_gb300 import inputs
    w = inputs.workload(args.workload)
    lt = w.lattices[0]
    U = lt.make_links()
    phi = lt.make_sources(w.nrhs)
    cores = _host_cores()
    oracle.set_num_threads(cores)
    t_all, Xo, Yo, info = _oracle_full_step(w, U, phi)
    out = {"value": round(1.0 / t_all, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"one full step of the workload, measured: {w.nrhs} fields, X and Y by FP64 BiCGStab to "
                     f"{w.tol} ({int(np.sum(info['iters_x']))}+{int(np.sum(info['iters_y']))} iterations) and "
                     f"the force, OpenMP on {cores} cores",
           "seconds_per_step": round(t_all, 3)}
    if not args.no_cpu_single:
        oracle.set_num_threads(1)
        t_one, _, _, _ = _oracle_full_step(w, U, phi)
        oracle.set_num_threads(cores)
        out["single_thread"] = {"value": round(1.0 / t_one, 6), "unit": UNIT, "cores": 1,
                                "seconds_per_step": round(t_one, 3), "sample": "the same full step, one thread"}
    if host_solution is not None:
        X, Y = host_solution["X"], host_solution["Y"]
        rx = oracle.true_residual(U, phi, X, lt.L, lt.T, lt.theta, lt.kappa)
        ry = oracle.true_residual(U, X, Y, lt.L, lt.T, lt.theta, lt.kappa, dagger=True)
        out["oracle_check"] = {
            "what": "the bench step's final X, Y: the oracle's true residuals |Phi - Dhat X|/|Phi| and "
                    "|X - Dhat^dag Y|/|X| per RHS, and the error against the oracle's X, Y (solved to the same "
                    "1e-10, so that difference is bounded by both solutions' errors)",
            "resid_x": [float(v) for v in rx], "resid_y": [float(v) for v in ry],
            "err_x_vs_oracle_1e-10": _per_rhs_relerr(X, Xo), "err_y_vs_oracle_1e-10": _per_rhs_relerr(Y, Yo)}
    if acc_cfg is not None:
        out["oracle_check_sf16"] = _oracle_check_sf16(acc_cfg, cores)
    if learned_check is not None and learned_check.get("solutions"):
        lc = learned_check["lattice"]
        chk = {"workload": f"held-out field 0 of the learned comparison ({lc.L}^3x{lc.T}, kappa {lc.kappa}, "
                           f"eps {lc.eps}): the oracle's true residuals |Phi - Dhat X|/|Phi| and |X - Dhat^dag Y|/|X| "
                           f"per RHS of each solver's X, Y"}
        for algo, (X, Y) in learned_check["solutions"].items():
            rx = oracle.true_residual(learned_check["U"], learned_check["phi"], X, lc.L, lc.T, lc.theta, lc.kappa)
            ry = oracle.true_residual(learned_check["U"], X, Y, lc.L, lc.T, lc.theta, lc.kappa, dagger=True)
            chk[algo] = {"oracle_resid_x": [float(v) for v in rx], "oracle_resid_y": [float(v) for v in ry]}
        out["oracle_check_learned"] = chk
    out["configs"] = _oracle_configs(cores, acc_cfg, learned_check)
    return out


def _oracle_configs(cores, acc_cfg, learned_check):
    """The oracle's time on the other workloads: the 8^4 FP64 1-RHS step in
    full; the 16^4 solves from the oracle check above; the 24^4 field from a
    measured cost per BiCGStab iteration times iteration counts (a full
    oracle solve there takes minutes)."""
    import oracle
    from paper_1009_5169_gb300 import inputs
    res = {}
    w = inputs.workload("sf8_plain_1rhs")
    lt = w.lattices[0]
    U = lt.make_links()
    phi = lt.make_sources(w.nrhs)
    t, _, _, info = _oracle_full_step(w, U, phi)
    res[w.name] = {"seconds_per_step": round(t, 3), "cores": cores, "kind": "measured",
                   "sample": f"X and Y by FP64 BiCGStab to {w.tol} ({int(info['iters_x'][0])}+"
                             f"{int(info['iters_y'][0])} iterations) and the force"}
    if acc_cfg is not None:
        res["sf16_mixed"] = {"kind": "measured", "sample": "X and Y of the 5 RHS to 1e-12 (no force): "
                                                          "cpu_baseline.oracle_check_sf16.oracle.seconds"}
    if learned_check is not None and "U" in learned_check:
        lc = learned_check["lattice"]
        n_it = 10
        t0 = time.perf_counter()
        oracle.bicgstab(learned_check["U"], learned_check["phi"][:1], lc.L, lc.T, lc.theta, lc.kappa, tol=1e-30,
                        maxiter=n_it)
        per_it = (time.perf_counter() - t0) / n_it
        e = {"seconds_per_bicgstab_iteration": round(per_it, 4), "cores": cores, "kind": "extrapolated",
             "sample": f"{n_it} oracle BiCGStab iterations on one RHS of a {lc.L}^3x{lc.T} field, timed"}
        its = learned_check.get("iters", {}).get("bicgstab")
        if its is not None:
            ix, iy = its
            total = int(sum(ix)) + 5 * int(iy)
            e["seconds_per_solve_pair"] = round(per_it * total, 1)
            e["sample"] += (f"; times {total} iterations: the library's FP64 BiCGStab on the same field, X per RHS "
                            f"{ix} and 5 x the largest Y count {iy} (no force)")
        res["sf24_cnn"] = e
    return res


def _oracle_check_sf16(acc_cfg, cores):
    """The oracle's X, Y of the 16^4 kappa 0.134 workload at 1e-12, and the
    GPU solutions' per-RHS errors against them and oracle residuals."""
    import oracle
    w, lt, U, phi = acc_cfg["workload"]
    t0 = time.perf_counter()
    Xo, Yo, info = oracle.solve_pair(U, phi, lt.L, lt.T, lt.theta, lt.kappa, tol=1e-12, maxiter=20000)
    t_or = time.perf_counter() - t0
    res = {"workload": acc_cfg["summary"]["workload"],
           "oracle": {"tol": 1e-12, "seconds": round(t_or, 2), "cores": cores,
                      "iters_x": [int(v) for v in info["iters_x"]], "iters_y": [int(v) for v in info["iters_y"]]}}
    for algo, (X, Y) in acc_cfg["solutions"].items():
        rx = oracle.true_residual(U, phi, X, lt.L, lt.T, lt.theta, lt.kappa)
        ry = oracle.true_residual(U, X, Y, lt.L, lt.T, lt.theta, lt.kappa, dagger=True)
        res[algo] = {"inner": acc_cfg["summary"]["solves"][algo]["inner"],
                     "err_x": _per_rhs_relerr(X, Xo), "err_y": _per_rhs_relerr(Y, Yo),
                     "oracle_resid_x": [float(v) for v in rx], "oracle_resid_y": [float(v) for v in ry]}
    return res


def accuracy_config_solves(args, sf, inputs, dev, local_rank):
    """The 16^4 SF workload (eps 0.2, kappa 0.134, 5 RHS, 1e-10) solved on the
    GPU with the FP32-inner and the FP16-inner defect correction and with the
    normal-equation CG route: time, sweeps and inner iterations; the solutions
    go to the oracle check of the cpu_baseline leg."""
    import torch
    w = inputs.workload("sf16_mixed")
    lt = w.lattices[0]
    U = lt.make_links()
    phi = lt.make_sources(w.nrhs)
    lat = sf.Lattice(lt.L, lt.T, lt.theta, lt.kappa, lt.beta, torch.from_numpy(U).to(dev), device=local_rank)
    phid = torch.from_numpy(phi).to(dev)
    X, Y = torch.empty_like(phid), torch.empty_like(phid)
    solves, sols = {}, {}
    inner = {"mixed_dc": "FP32 BiCGStab", "mixed_dc_half": "FP16-operand BiCGStab", "cg_normal": "FP32 CG on Dhat Dhat^dag"}
    for algo in ("mixed_dc", "mixed_dc_half", "cg_normal"):
        sf.solve_block(lat, algo, phid, X, Y, tol=w.tol, maxiter=args.maxiter)   # autotune, graph capture
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = sf.solve_block(lat, algo, phid, X, Y, tol=w.tol, maxiter=args.maxiter)
        torch.cuda.synchronize()
        solves[algo] = {"inner": inner[algo], "ms": round((time.perf_counter() - t0) * 1e3, 2),
                        "sweeps": [info["iters_outer"], info["iters_outer_y"]],
                        "inner_iters": [info["iters_inner"], info["iters_inner_y"]],
                        "library_resid_x": [float(v) for v in info["true_resid"]]}
        sols[algo] = (X.cpu().numpy(), Y.cpu().numpy())
    lat.close()
    summary = {"workload": "sf16_mixed: 16^3x16 SF, eps 0.2, kappa 0.134, theta 0.5, 5 RHS, tol 1e-10 "
                           "(per-RHS errors against the oracle: cpu_baseline.oracle_check_sf16)",
               "solves": solves}
    return {"summary": summary, "solutions": sols, "workload": (w, lt, U, phi)}


def hmc_section(args, sf, inputs, lt, U_d, nrhs, tol, fshape, dev, local_rank):
    """HMC on the bench lattice: the synthetic field is first brought towards
    equilibrium by MD trajectories accepted unconditionally (untimed), then
    trajectories with fresh momenta and pseudo-fermions and the Metropolis
    test are timed; reports dH, the acceptance and the time per trajectory
    and per accepted trajectory, for the leapfrog, the Omelyan integrator over
    the same trajectory length at the same force count, and the leapfrog with
    the gauge force on 4 substeps per step."""
    import torch
    hlat = sf.Lattice(lt.L, lt.T, lt.theta, lt.kappa, lt.beta, U_d, device=local_rank)
    nst, dt = args.hmc_steps, args.hmc_dt

    def draws(k):
        seed = inputs.SEED_BASE + 600 + k
        P = torch.from_numpy(inputs.su3_directions(fshape[:2], seed)).to(dev)
        eta = torch.from_numpy(inputs.sources(lt.L, lt.T, nrhs, seed)).to(dev)
        u = float(inputs.rng(seed, inputs.FIELD_AUX + 1).random())
        return P, eta, u

    plaq = [sf.plaquette_action(hlat)]
    dh_therm = []
    for k in range(args.hmc_therm):
        P, eta, _ = draws(k)
        d = sf.hmc_trajectory(hlat, args.algo, eta, P, -1.0, nst, dt, tol=tol, maxiter=args.maxiter)
        dh_therm.append(round(d["dH"], 4))
        plaq.append(sf.plaquette_action(hlat))
    torch.cuda.synchronize()
    dhs, acc, ms, iters, launches = [], [], [], 0, 0
    for k in range(args.hmc_traj):
        P, eta, u = draws(1000 + k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d = sf.hmc_trajectory(hlat, args.algo, eta, P, u, nst, dt, tol=tol, maxiter=args.maxiter)
        torch.cuda.synchronize()
        ms.append(round((time.perf_counter() - t0) * 1e3, 2))
        dhs.append(round(d["dH"], 5))
        acc.append(bool(d["accepted"]))
        iters += d["inner_iters"]
        launches += d["kernel_launches"]
    # the same trajectory length with the Omelyan integrator at half the
    # steps (two force evaluations per step: the same force count, +1)
    nst_o = max(1, nst // 2)
    dt_o = dt * nst / nst_o
    dho, acco, mso = [], [], []
    for k in range(args.hmc_traj):
        P, eta, u = draws(2000 + k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d = sf.hmc_trajectory(hlat, args.algo, eta, P, u, nst_o, dt_o, tol=tol, maxiter=args.maxiter,
                              integrator="omelyan")
        torch.cuda.synchronize()
        mso.append(round((time.perf_counter() - t0) * 1e3, 2))
        dho.append(round(d["dH"], 5))
        acco.append(bool(d["accepted"]))
    # the leapfrog again with the gauge force on 4 substeps of each step
    # (two time scales: the same fermion force count)
    dhm, accm, msm = [], [], []
    for k in range(args.hmc_traj):
        P, eta, u = draws(3000 + k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d = sf.hmc_trajectory(hlat, args.algo, eta, P, u, nst, dt, tol=tol, maxiter=args.maxiter, gauge_substeps=4)
        torch.cuda.synchronize()
        msm.append(round((time.perf_counter() - t0) * 1e3, 2))
        dhm.append(round(d["dH"], 5))
        accm.append(bool(d["accepted"]))
    hlat.close()
    n_accm = sum(accm)
    two_scales = {"integrator": "leapfrog, gauge force on 4 substeps per step (Sexton-Weingarten)", "steps": nst,
                  "dt": dt, "force_evals_per_trajectory": nst + 1, "dH": dhm, "accepted": accm,
                  "acceptance": round(n_accm / max(1, len(accm)), 3),
                  "mean_min_1_exp_minus_dH": round(statistics.mean(min(1.0, math.exp(-x)) for x in dhm), 3) if dhm else None,
                  "ms_per_trajectory": round(statistics.mean(msm), 2) if msm else None,
                  "ms_per_accepted_trajectory": round(sum(msm) / n_accm, 2) if n_accm else None}
    n_acco = sum(acco)
    omelyan = {"integrator": f"Omelyan, Mryglod and Folk second-order minimum-norm, lambda {sf.OMELYAN_LAMBDA}",
               "steps": nst_o, "dt": dt_o, "force_evals_per_trajectory": 2 * nst_o + 1, "dH": dho, "accepted": acco,
               "acceptance": round(n_acco / max(1, len(acco)), 3),
               "mean_min_1_exp_minus_dH": round(statistics.mean(min(1.0, math.exp(-x)) for x in dho), 3) if dho else None,
               "ms_per_trajectory": round(statistics.mean(mso), 2) if mso else None,
               "ms_per_accepted_trajectory": round(sum(mso) / n_acco, 2) if n_acco else None}
    n_acc = sum(acc)
    V4 = lt.L ** 3 * lt.T * 6
    return {"workload": f"{lt.L}^3x{lt.T} SF, beta {lt.beta}, {nrhs} pseudo-fermions phi = Dhat eta, Gaussian "
                        f"momenta, leapfrog {nst} x dt {dt} (trajectory length {nst * dt:g}), {args.algo} to {tol}",
            "thermalisation": {"trajectories": args.hmc_therm, "accepted": "all (MD only, untimed)",
                               "dH": dh_therm,
                               "plaquette_action_per_plaquette": [round(p / (lt.beta * V4), 5) for p in plaq[::max(1, len(plaq) // 8)]]},
            "trajectories": args.hmc_traj, "dH": dhs, "accepted": acc, "acceptance": round(n_acc / max(1, len(acc)), 3),
            "mean_min_1_exp_minus_dH": round(statistics.mean(min(1.0, math.exp(-x)) for x in dhs), 3) if dhs else None,
            "ms": ms, "ms_per_trajectory": round(statistics.mean(ms), 2) if ms else None,
            "ms_per_accepted_trajectory": round(sum(ms) / n_acc, 2) if n_acc else None,
            "force_evals_per_trajectory": nst + 1, "inner_iters": iters, "kernel_launches": launches,
            "omelyan": omelyan, "two_time_scales": two_scales}


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle as it stands, full steps of the bench
    workload (every field's X and Y to 1e-10 and the force) on the host
    cores, W untimed and K timed."""
    if rank != 0:
        return
    import oracle
    from paper_1009_5169_gb300 import inputs
    w = inputs.workload(args.workload)
    lt = w.lattices[0]
    U = lt.make_links()
    phi = lt.make_sources(w.nrhs)
    cores = _host_cores()
    oracle.set_num_threads(cores)
    for _ in range(args.warmup):
        _oracle_full_step(w, U, phi)
    times = []
    info = None
    for _ in range(args.steps):
        t, _, _, info = _oracle_full_step(w, U, phi)
        times.append(t)
    sps = args.steps / sum(times)
    out = {"impl": "reference", "metric": METRIC, "value": round(sps, 6), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sum(times) / args.steps * 1e3, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": _workload_desc(args.workload, lt, w.nrhs, w.tol)},
           "cpu_baseline": {"kind": "oracle", "cores": cores, "value": round(sps, 6), "unit": UNIT,
                            "sample": f"{args.steps} full steps, measured: {w.nrhs} fields, X and Y by FP64 BiCGStab "
                                      f"to {w.tol} ({int(np.sum(info['iters_x']))}+{int(np.sum(info['iters_y']))} "
                                      f"iterations per step) and the force"},
           "e2e": {"value": round(sps, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def _fp64_gemm_tflops(dev):
    """Measured FP64 denominator: cuBLAS DGEMM (torch.matmul, 4096^3) timed
    with CUDA events, TFLOP/s."""
    import torch
    n = 4096
    g = torch.Generator(device=dev).manual_seed(7)
    a = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g)
    b = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g)
    torch.matmul(a, b)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        torch.matmul(a, b)
    e1.record()
    torch.cuda.synchronize()
    return 2.0 * n ** 3 * 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12


def fp64_roofline(sf, lat, lt, nrhs, stream, flush, dev):
    """FLOP-based roofline of the FP64 hop (the true residuals' Dhat) and the
    force kernel on the bench lattice, each launch timed alone with CUDA
    events after an L2 flush.  Algorithmic FLOPs: the hop 1320 per site and
    rhs (8 directions of projection, two SU(3) products and accumulation);
    the force 336 per link and rhs (four spin projections, two 3 x 3 outer
    products) + 470 per link (V M1 - M2 V^dag, the eight traces, the
    scaling), on the (4T - 5) L^3 dynamic links that carry a fermion force."""
    import torch
    peak = _fp64_gemm_tflops(dev)
    fshape = ((lt.T + 1) * lt.L ** 3, 4, 8)
    F = torch.zeros(fshape, dtype=torch.float64, device=dev)

    def timed(fn, reps=20):
        fn()
        torch.cuda.synchronize()
        ev = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            ev.append((a, b))
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in ev) * 1e-3

    t_hop = timed(lambda: sf.wilson_hop_resident(lat, "fp64", nrhs, 1))
    t_force = timed(lambda: sf.fermion_force_resident(lat, nrhs, F))
    hop_flops = 1320.0 * lt.Vh * nrhs
    links = (4 * lt.T - 5) * lt.L ** 3
    force_flops = links * (336.0 * nrhs + 470.0)
    out = {"unit": "TFLOP/s", "peak": round(peak, 3), "peak_kind": "measured cuBLAS DGEMM (4096^3) in this run",
           "nominal_peak": 1.25}
    for name, fl, t in (("k_hop<P64> (dslash H_oe)", hop_flops, t_hop), ("k_force", force_flops, t_force)):
        ach = fl / t / 1e12
        out[name] = {"bound": "alu", "achieved": round(ach, 3), "frac": round(ach / peak, 4),
                     "frac_of_nominal": round(ach / 1.25, 4), "flops_per_launch": fl,
                     "launch_us": round(t * 1e6, 2)}
    return out


def learned_section(args, dev, local_rank, stream):
    """The learned preconditioner on the 24^4 workload (kappa 0.134, eps 0.2,
    5 RHS, 1e-10).  The network is trained on the GPU by the library's own
    forward and backward kernels on the residual norm |r - Dhat M(r)|^2 / |r|^2,
    with residuals from this library's own solves on seeded 12^4 fields of the
    same kappa / eps (the network is translation invariant; the smaller volume
    keeps training short): for each field phi and gamma5 X of the solves of
    Alg. 2, 5 RHS each.  On held-out 24^4 fields its mixed-
    precision form (FP32 flexible GCR under FP64 defect correction) is timed
    against the same solver without the network, plain FP64 BiCGStab on the
    5-RHS block, and the FP32-inner mixed solves; every answer is judged by
    the library's FP64 true residual.  Returns (the first held-out field's
    links, sources and every solver's X, Y for the oracle check of the
    cpu_baseline leg; the section's summary)."""
    import torch
    from paper_1009_5169_gb300 import binding as sf
    from paper_1009_5169_gb300 import inputs
    w = inputs.workload("sf24_cnn")
    big = w.lattices[0]
    hidden = 16
    t0 = time.perf_counter()
    net = sf.Cnn(hidden, inputs.cnn_init_params(hidden, inputs.SEED_BASE + 40), device=local_rank)
    train_lats = []
    samples = []
    g5 = torch.tensor([1, 1, -1, -1], dtype=torch.float64, device=dev).view(1, 1, 4, 1)
    for f in range(args.learned_train_fields):
        lt = inputs.Lattice(12, 12, big.eps, big.kappa, inputs.SEED_BASE + 4000 + f)
        lat = sf.Lattice(lt.L, lt.T, lt.theta, lt.kappa, lt.beta, torch.from_numpy(lt.make_links()).to(dev),
                         device=local_rank)
        phi = torch.from_numpy(inputs.sources(lt.L, lt.T, 5, inputs.SEED_BASE + 4000 + f)).to(dev)
        X, Y = torch.empty_like(phi), torch.empty_like(phi)
        sf.solve_block(lat, "mixed_dc", phi, X, Y, tol=1e-8, maxiter=args.maxiter)
        samples.append((lat, phi))
        samples.append((lat, (X * g5).contiguous()))   # smoother residuals: Dhat (g5 Y) = g5 X
        train_lats.append(lat)
    losses = []
    for epoch in range(args.learned_epochs):
        for lat, r in samples:
            losses.append(net.train_step(lat, r, None, 1e-3))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    for lat in train_lats:
        lat.close()
    # one application of the network at 24^4 (5 RHS, both signs): tcgen05 and mma.sync convolutions
    lt = inputs.Lattice(big.L, big.T, big.eps, big.kappa, inputs.SEED_BASE + 1000)
    lat = sf.Lattice(lt.L, lt.T, lt.theta, lt.kappa, lt.beta, torch.from_numpy(lt.make_links()).to(dev),
                     device=local_rank)
    r = torch.from_numpy(inputs.sources(lt.L, lt.T, w.nrhs, inputs.SEED_BASE + 1000)).to(dev)
    out = torch.empty_like(r)
    apply_ms = {}
    for impl in ("mma_sync", "tcgen05"):
        net.set_conv_impl(impl)
        net.forward(lat, r, out)
        torch.cuda.synchronize()
        a = time.perf_counter()
        for _ in range(5):
            net.forward(lat, r, out)
        torch.cuda.synchronize()
        apply_ms[impl] = round((time.perf_counter() - a) / 5 * 1e3, 3)
    net.set_conv_impl("tcgen05")
    lat.close()
    flops = 2.0 * 81 * sum(ci * co for ci, co in zip(inputs.cnn_widths(hidden)[:-1], inputs.cnn_widths(hidden)[1:]))
    rows = 2 * w.nrhs * big.V
    res = {}
    slow = ("bicgstab", "fgcr_mixed")
    # the first held-out field's solutions go to the oracle check of the cpu_baseline leg
    check = {"solutions": {}}
    for h in range(args.learned_heldout):
        lt = inputs.Lattice(big.L, big.T, big.eps, big.kappa, inputs.SEED_BASE + 1000 + h)
        Uh = lt.make_links()
        lat = sf.Lattice(lt.L, lt.T, lt.theta, lt.kappa, lt.beta, torch.from_numpy(Uh).to(dev),
                         device=local_rank)
        sf.set_preconditioner(lat, net)
        phin = inputs.sources(lt.L, lt.T, w.nrhs, inputs.SEED_BASE + 1000 + h)
        phi = torch.from_numpy(phin).to(dev)
        if h == 0:
            check.update(lattice=lt, U=Uh, phi=phin)
        del Uh
        X, Y = torch.empty_like(phi), torch.empty_like(phi)
        for algo in ("fgcr_cnn_mixed", "fgcr_mixed", "bicgstab", "mixed_dc", "cg_normal"):
            if algo in slow and h >= args.learned_slow_fields:
                continue
            # first use: autotuning, graph capture, workspace (a short solve, not timed)
            sf.solve_block(lat, algo, phi, X, Y, tol=1e-4, maxiter=args.maxiter)
            torch.cuda.synchronize()
            a = time.perf_counter()
            info = sf.solve_block(lat, algo, phi, X, Y, tol=w.tol, maxiter=args.maxiter)
            torch.cuda.synchronize()
            e = res.setdefault(algo, {"ms": [], "iters_x": [], "iters_y": [], "max_true_rel_resid": 0.0})
            e["ms"].append(round((time.perf_counter() - a) * 1e3, 2))
            e["iters_x"].append(info["iters_inner"])
            e["iters_y"].append(info["iters_inner_y"])
            e["max_true_rel_resid"] = max(e["max_true_rel_resid"], max(info["true_resid"]), max(info["true_resid_y"]))
            if h == 0:
                check["solutions"][algo] = (X.cpu().numpy(), Y.cpu().numpy())
                check.setdefault("iters", {})[algo] = (list(info["iters_inner_rhs"][:w.nrhs]), info["iters_inner_y"])
        sf.set_preconditioner(lat, None)
        lat.close()
    net.close()
    mean = lambda v: statistics.mean(v) if v else None
    summary = {k: {"mean_ms": round(mean(v["ms"]), 1), "fields": len(v["ms"]),
                   "mean_iters": [round(mean(v["iters_x"]), 1), round(mean(v["iters_y"]), 1)]}
               for k, v in res.items()}
    learned = summary["fgcr_cnn_mixed"]["mean_ms"]
    return check, {"workload": f"{big.L}^3x{big.T} SF, kappa {big.kappa}, eps {big.eps}, {w.nrhs} RHS, tol {w.tol}; "
                        f"{args.learned_heldout} held-out fields (plain FP64 BiCGStab and FGCR without the network "
                        f"on the first {args.learned_slow_fields})",
            "network": f"4 x 3^4 conv, widths {inputs.cnn_widths(hidden)}, BF16 operands, FP32 accumulation, "
                       f"tcgen05 (TMEM accumulators); residual-norm loss",
            "training": {"fields": f"{args.learned_train_fields} seeded 12^4 fields (eps {big.eps}, kappa {big.kappa}); "
                                   f"residuals phi and g5 X of each field's own solves, 5 RHS each",
                         "residual_fields_per_epoch": len(samples) * 5, "epochs": args.learned_epochs,
                         "steps": len(losses), "residual_fields_seen": len(losses) * 5,
                         "loss_first": round(float(np.mean(losses[:len(samples)])), 4),
                         "loss_last": round(float(np.mean(losses[-len(samples):])), 4),
                         "seconds": round(t_train, 1)},
            "network_application_ms": apply_ms,
            "network_tflops_tcgen05": round(flops * rows / (apply_ms["tcgen05"] * 1e-3) / 1e12, 1),
            "solves": res, "summary": summary,
            "speedup_vs_fp64_bicgstab": round(summary["bicgstab"]["mean_ms"] / learned, 2) if "bicgstab" in summary else None,
            "speedup_vs_fgcr_without_network": round(summary["fgcr_mixed"]["mean_ms"] / learned, 2)
            if "fgcr_mixed" in summary else None,
            "ratio_vs_mixed_dc": round(summary["mixed_dc"]["mean_ms"] / learned, 3),
            "ratio_vs_cg_normal": round(summary["cg_normal"]["mean_ms"] / learned, 3),
            "fgcr_iteration_gain_from_network": round(
                summary["fgcr_mixed"]["mean_iters"][0] / max(1e-9, statistics.mean(res["fgcr_cnn_mixed"]["iters_x"][:args.learned_slow_fields])), 2)
            if "fgcr_mixed" in summary else None}


def run_dslash_only(args, local_rank):
    """Hop kernels alone on an L^3 x T lattice with a fixed tiling (for
    profiler captures): one launch per precision, then `reps` timed ones."""
    import torch
    from paper_1009_5169_gb300 import binding as sf
    from paper_1009_5169_gb300 import inputs
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    L, T = args.dslash_lattice
    U = inputs.links(L, T, 0.2, inputs.SEED_BASE + 32)
    lat = sf.Lattice(L, T, 0.5, 0.13, 4.52, torch.from_numpy(U).to(dev), device=local_rank)
    del U
    stream = torch.cuda.current_stream(dev)
    peak, _ = _peaks()
    res = {}
    Vh = L ** 3 * (T - 1) // 2
    for p in args.dslash_precs.split(","):
        TS, NR, PIPE = (list(args.tiling) + [0])[:3]
        lat.set_tuning(p, TS, NR, PIPE if p != "fp64" else 0)
        sf.wilson_hop_resident(lat, p, 5, 1)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.reps):
            sf.wilson_hop_resident(lat, p, 5, 1)
        b.record(stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(b) * 1e-3 / args.reps
        sb = {"fp64": 5 * 192 * 2 + 8 * 144, "fp32": 5 * 96 * 2 + 8 * 48, "fp16": 5 * 52 * 2 + 8 * 24}[p]
        res[p] = {"launch_us": round(t * 1e6, 2), "achieved_GBs": round(Vh * sb / t / 1e9, 1),
                  "frac": round(Vh * sb / t / 1e9 / peak, 4), "algorithmic_bytes_per_launch": Vh * sb}
    lat.close()
    print(json.dumps({"dslash_only": f"{L}^3x{T}", "tiling": args.tiling, "reps": args.reps, **res}), flush=True)


def run_network_only(args, local_rank):
    """The learned preconditioner's forward pass alone on an L^4 lattice
    with 5 RHS and seeded, untrained weights (for profiler captures): one
    application per convolution implementation, then `reps` timed ones."""
    import torch
    from paper_1009_5169_gb300 import binding as sf
    from paper_1009_5169_gb300 import inputs
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    L = args.network_lattice
    hidden = 16
    lt = inputs.Lattice(L, L, 0.2, 0.134, inputs.SEED_BASE + 1000)
    lat = sf.Lattice(lt.L, lt.T, lt.theta, lt.kappa, lt.beta, torch.from_numpy(lt.make_links()).to(dev),
                     device=local_rank)
    r = torch.from_numpy(inputs.sources(lt.L, lt.T, 5, inputs.SEED_BASE + 1000)).to(dev)
    out = torch.empty_like(r)
    net = sf.Cnn(hidden, inputs.cnn_init_params(hidden, inputs.SEED_BASE + 40), device=local_rank)
    stream = torch.cuda.current_stream(dev)
    widths = inputs.cnn_widths(hidden)
    flops = 2.0 * 81 * sum(ci * co for ci, co in zip(widths[:-1], widths[1:])) * 2 * 5 * L ** 3 * L
    res = {}
    for impl in args.network_impls.split(","):
        net.set_conv_impl(impl)
        net.forward(lat, r, out)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.reps):
            net.forward(lat, r, out)
        b.record(stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(b) * 1e-3 / args.reps
        res[impl] = {"forward_ms": round(t * 1e3, 3), "conv_tflops": round(flops / t / 1e12, 1)}
    net.close()
    lat.close()
    print(json.dumps({"network_only": f"{L}^4", "widths": widths, "reps": args.reps, **res}), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sf12_nf10")
    ap.add_argument("--algo", default="cg_normal", choices=["bicgstab", "mixed_dc", "mixed_dc_half", "cg_normal"])
    ap.add_argument("--maxiter", type=int, default=5000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-hbm-case", action="store_true")
    ap.add_argument("--no-comparators", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-hmc", action="store_true")
    ap.add_argument("--solve-tiling", type=int, nargs=3, default=None, metavar=("TS", "NR", "PIPE"),
                    help="fix the inner solve's tiling of the timed step instead of autotuning it")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--learned-train-fields", type=int, default=40)
    ap.add_argument("--learned-epochs", type=int, default=50)
    ap.add_argument("--learned-heldout", type=int, default=10)
    ap.add_argument("--learned-slow-fields", type=int, default=2,
                    help="held-out fields the slow comparators (FP64 BiCGStab, FGCR without the network) run on")
    ap.add_argument("--no-cpu-single", action="store_true", help="skip the single-threaded oracle step")
    ap.add_argument("--no-accuracy-configs", action="store_true")
    ap.add_argument("--hmc-steps", type=int, default=10)
    ap.add_argument("--hmc-dt", type=float, default=0.02)
    ap.add_argument("--hmc-therm", type=int, default=20)
    ap.add_argument("--hmc-traj", type=int, default=6)
    ap.add_argument("--dslash-only", action="store_true", help="time the hop kernel alone (profiling aid)")
    ap.add_argument("--dslash-lattice", type=int, nargs=2, default=(32, 24), metavar=("L", "T"))
    ap.add_argument("--dslash-precs", default="fp32,fp16")
    ap.add_argument("--tiling", type=int, nargs="+", default=(64, 1), metavar="N",
                    help="TS NR [pipe]: sites per tile, rhs per thread, pipelined hop (0/1)")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--network-only", action="store_true",
                    help="time the learned preconditioner's forward pass alone (profiling aid)")
    ap.add_argument("--network-lattice", type=int, default=24, metavar="L")
    ap.add_argument("--network-impls", default="tcgen05,mma_sync")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 0)
    rank, world, local_rank = _env_rank()
    if args.network_only:
        run_network_only(args, local_rank)
        return
    if args.dslash_only:
        run_dslash_only(args, local_rank)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
