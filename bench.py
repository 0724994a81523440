"""Benchmark: interacting pairs per second of one force evaluation.

One evaluation = the whole hot path through the C ABI: lattice evolution and
remap, grid + stencil, fractional wrap + counting-sort binning, cell-pair
force/energy/virial and the float64 reductions (nemd_set_state ->
nemd_build_cells -> nemd_compute_forces).  One step = the evaluations at S
evenly spaced strains of one period of the general 3D flow on the
N = 1,048,576 perturbed-FCC LJ system (rc = 2.5).  Every strain has its own
24 MB position array, so a step streams inputs far larger than L2.

Printed as one JSON line (rank 0):
  value        pairs/s of the tuned form (per-step variant choice, tuned kernel)
  plain        pairs/s of the plain fixed-variant cell lists on the same steps
  e2e          pairs/s through the C ABI with pinned host buffers, copies timed
  roofline     force kernel: algorithmic FP32 instructions / launch time against
               the FP32 issue peak (bound "alu")
  cpu_baseline the FP64 oracle on a bounded sample, on the host cores

--impl reference times the oracle (the reference arm of this project) on the
same workload, one strain per step.
"""
from __future__ import annotations

import argparse
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

WORKLOADS = {
    # name: (k for N = 4k^3, strains per period)
    "general_n1m": (64, 128),
    "general_n256k": (40, 128),
    "general_n2m": (80, 256),
}
C_TEST = 7     # FP32 instructions per candidate test: 3 FADD, 1 FMUL, 2 FFMA, 1 FSETP
C_PAIR = 24    # FP32 instructions per interacting pair (force, energy, virial, both sides)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="general_n1m", choices=sorted(WORKLOADS))
    p.add_argument("--strains", type=int, default=0, help="strains per step (default: the workload's)")
    p.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle sample")
    p.add_argument("--e2e-strains", type=int, default=16)
    p.add_argument("--kernel", type=int, default=1, help="force kernel of the tuned form (0 plain, 1 grouped)")
    p.add_argument("--group", type=int, default=16, help="lanes per group of the grouped kernel")
    p.add_argument("--kfac", type=int, default=1, help="cell-size factor of the tuned form")
    return p.parse_args()


def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class Clocks:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.idx = device_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def fp32_issue_peak(sms, mhz):
    """FP32 lanes per SM (128) x SMs x clock: FP32 instructions (lane-ops) per second."""
    return 128.0 * sms * mhz * 1e6


def run_reference(args, rank, world):
    """The oracle as the reference arm: one strain per step, dynamic size cell list."""
    if rank != 0:
        return
    import oracle
    from paper_1412_3784_gb300 import workloads as W
    k, nstrain = WORKLOADS[args.workload]
    ser = W.general_series(k=k)
    ts = [i / nstrain for i in range(nstrain)]
    pairs = 0
    elapsed = 0.0
    for step in range(args.warmup + args.steps):
        t = ts[(step * 37) % nstrain]
        w = ser.workload(t)
        t0 = time.perf_counter()
        r = oracle.evaluate(w, "ds")
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            pairs += r.npairs
            elapsed += dt
    value = pairs / elapsed
    line = {
        "impl": "reference", "metric": "interacting pairs/s per force eval", "value": value,
        "unit": "pairs/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: general 3D flow, N={ser.n}, LJ rc=2.5, "
                               f"one strain per step (dynamic size cell list)"},
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": 1, "kind": "oracle",
                         "sample": f"one force evaluation per step of the N={ser.n} system"},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_sample(ser, t):
    import oracle
    w = ser.workload(t)
    t0 = time.perf_counter()
    r = oracle.evaluate(w, "ds")
    dt = time.perf_counter() - t0
    return {"value": r.npairs / dt, "unit": "pairs/s", "cores": 1, "kind": "oracle",
            "sample": f"one force evaluation (dynamic size cell list, FP64) of the N={ser.n} "
                      f"general-flow system at t={t:.4f}: {r.npairs} pairs in {dt:.2f} s"}


def main():
    args = parse()
    rank, world, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
        barrier(world)
        return

    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1412_3784_gb300 import nemd
    from paper_1412_3784_gb300 import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    k, nstrain = WORKLOADS[args.workload]
    S = args.strains or nstrain
    ser = W.general_series(k=k)
    n = ser.n
    ts = [i / S for i in range(S)]
    q_all = torch.empty((S, n, 3), dtype=torch.float64, device=dev)
    for i, t in enumerate(ts):
        q_all[i].copy_(torch.from_numpy(ser.positions(t)))
    F = torch.empty((n, 3), dtype=torch.float32, device=dev)
    U = torch.zeros(1, dtype=torch.float64, device=dev)
    Wv = torch.zeros(9, dtype=torch.float64, device=dev)

    ctx = nemd.Context(local)
    ctx.set_flow(ser.A, ser.L0, ser.M, ser.period)
    ctx.set_potential(nemd.NEMD_LJ, 1.0, 1.0, 1)

    def configure(kind):
        if kind == "plain_ds" or kind == "plain_do":
            ctx.set_option(nemd.NEMD_OPT_KERNEL, 0)
            ctx.set_option(nemd.NEMD_OPT_CELL_FACTOR, 1)
            return nemd.NEMD_DS if kind == "plain_ds" else nemd.NEMD_DO
        ctx.set_option(nemd.NEMD_OPT_KERNEL, args.kernel)
        ctx.set_option(nemd.NEMD_OPT_GROUP, args.group)
        ctx.set_option(nemd.NEMD_OPT_CELL_FACTOR, args.kfac)
        return nemd.NEMD_AUTO_HEURISTIC

    def one_step(variant):
        for i in range(S):
            ctx.set_state(q_all[i], ts[i])
            ctx.build_cells(variant, ser.rc)
            ctx.compute_forces(F, U, Wv)

    # untimed pass: pairs and candidates per strain for each form
    per = {}
    for kind in ("plain_ds", "plain_do", "tuned"):
        variant = configure(kind)
        pairs, cands, variants, rech = [], [], [], []
        for i in range(S):
            ctx.set_state(q_all[i], ts[i])
            ctx.build_cells(variant, ser.rc)
            ctx.compute_forces(F, U, Wv)
            ctx.sync()
            st = ctx.stats()
            pairs.append(st["pairs"])
            cands.append(st["candidates"])
            variants.append(st["variant"])
            rech.append(st["rechecks"])
        per[kind] = {"pairs": pairs, "cands": cands, "variants": variants, "rechecks": rech}
    pairs_per_step = sum(per["tuned"]["pairs"])
    assert pairs_per_step == sum(per["plain_ds"]["pairs"]) == sum(per["plain_do"]["pairs"])
    # algorithmic FP32 instructions of the tuned step, per the k = 1 stencil of the
    # variant chosen at each strain: 7 per unordered candidate + 24 per pair
    ops_step = 0.0
    for i in range(S):
        v = per["tuned"]["variants"][i]
        cand_k1 = (per["plain_do"] if v == 1 else per["plain_ds"])["cands"][i]
        ops_step += 0.5 * C_TEST * cand_k1 + C_PAIR * per["tuned"]["pairs"][i]

    def timed(kind, steps, warmup, timing=False):
        variant = configure(kind)
        for _ in range(warmup):
            one_step(variant)
        ctx.sync()
        if timing:
            ctx.set_option(nemd.NEMD_OPT_TIMING, 1)
        launches0 = ctx.stats()["launches"]
        barrier(world)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            one_step(variant)
        e1.record()
        torch.cuda.synchronize(dev)
        barrier(world)
        ms = e0.elapsed_time(e1)
        launches = ctx.stats()["launches"] - launches0
        ctx.sync()
        kt = None
        if timing:
            kt = ctx.kernel_time()
            ctx.set_option(nemd.NEMD_OPT_TIMING, 0)
        return ms, launches, kt

    clocks = Clocks(local)
    clocks.start()
    ms_tuned, launches, ktime = timed("tuned", args.steps, args.warmup, timing=True)
    clk = clocks.stop()
    ms_ds, _, _ = timed("plain_ds", args.steps, 1)
    ms_do, _, _ = timed("plain_do", args.steps, 1)

    ms_tuned_max = max_over_ranks(ms_tuned, world, dev)
    total_pairs = sum_over_ranks(float(pairs_per_step * args.steps), world, dev)
    value = total_pairs / (ms_tuned_max * 1e-3)
    plain_ds = sum_over_ranks(float(pairs_per_step * args.steps), world, dev) / (max_over_ranks(ms_ds, world, dev) * 1e-3)
    plain_do = sum_over_ranks(float(pairs_per_step * args.steps), world, dev) / (max_over_ranks(ms_do, world, dev) * 1e-3)

    # roofline of the force kernel (FP32 issue bound)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peak_mhz = 2070.0
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak_mhz = float(mp.get("sm_max_mhz", peak_mhz))
    except (OSError, ValueError):
        pass
    peak = fp32_issue_peak(sms, peak_mhz)
    k_ms, k_n = ktime
    avg_launch_s = (k_ms / k_n) * 1e-3
    ops_per_launch = ops_step / S
    achieved = ops_per_launch / avg_launch_s
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "k_force_chunk" if args.kernel == 1 else "k_force_plain", "ops_per_launch": ops_per_launch,
                "avg_launch_ms": avg_launch_s * 1e3,
                "peak_basis": f"{sms} SMs x 128 FP32 lanes x {peak_mhz:.0f} MHz (FP32 instruction lane-ops/s)"}

    # end to end through the C ABI with pinned host buffers
    Se = min(args.e2e_strains, S)
    qh = [torch.from_numpy(ser.positions(ts[i])).pin_memory() for i in range(Se)]
    Fh = torch.empty((n, 3), dtype=torch.float32).pin_memory()
    Uh = torch.zeros(1, dtype=torch.float64).pin_memory()
    Wh = torch.zeros(9, dtype=torch.float64).pin_memory()
    variant = configure("tuned")
    for i in range(min(3, Se)):
        ctx.set_state(qh[i], ts[i])
        ctx.build_cells(variant, ser.rc)
        ctx.compute_forces(Fh, Uh, Wh)
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for i in range(Se):
        ctx.set_state(qh[i], ts[i])
        ctx.build_cells(variant, ser.rc)
        ctx.compute_forces(Fh, Uh, Wh)   # host outputs: returns after the copy back
    torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e_pairs = sum_over_ranks(float(sum(per["tuned"]["pairs"][:Se])), world, dev)
    e2e = {"value": e2e_pairs / e2e_s, "unit": "pairs/s",
           "h2d_bytes_per_step": int(S * n * 3 * 8), "d2h_bytes_per_step": int(S * (n * 3 * 4 + 80)),
           "strains_timed": Se}

    cpu = None
    if rank == 0 and world == 1 and not args.no_baseline:
        cpu = cpu_baseline_sample(ser, ts[S // 3])

    eta_ds = 2 * sum(per["plain_ds"]["pairs"]) / sum(per["plain_ds"]["cands"])
    eta_do = 2 * sum(per["plain_do"]["pairs"]) / sum(per["plain_do"]["cands"])
    if rank == 0:
        line = {
            "metric": "interacting pairs/s per force eval", "value": value, "unit": "pairs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_tuned_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 pair math, f64 lattice/wrap/reductions",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: general 3D flow M=[[3,2,1],[2,2,1],[1,1,1]], "
                                   f"perturbed FCC N={n}, rho=0.8442, LJ rc=2.5, {S} strains per step "
                                   f"(one period), one force evaluation per strain",
                       "n": n, "strains_per_step": S, "pairs_per_step": pairs_per_step,
                       "tuned": f"per-strain variant by neighbourhood volume, kernel {args.kernel} "
                                f"(group {args.group}), cell factor {args.kfac}",
                       "coarse_band_candidates_per_step": int(sum(per["tuned"]["rechecks"])),
                       "l2": "inputs larger than L2: a distinct 24 MB position array per strain",
                       "parallelism": f"replicas x{world}"},
            "plain": {"dynamic_size_pairs_per_s": plain_ds, "dynamic_offset_pairs_per_s": plain_do,
                      "search_efficiency_ds": eta_ds, "search_efficiency_do": eta_do},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    barrier(world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
