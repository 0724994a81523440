"""Benchmark: interacting pairs per second of one force evaluation.

One evaluation = the whole hot path through the C ABI: lattice evolution and
remap, grid + stencil, fractional wrap + counting-sort binning, cell-pair
force/energy/virial and the float64 reductions (nemd_set_state ->
nemd_build_cells -> nemd_compute_forces).  One step = the evaluations at S
evenly spaced strains of one period of the general 3D flow on the
N = 1,048,576 perturbed-FCC LJ system (rc = 2.5).  Every strain has its own
24 MB position array, so a step streams inputs far larger than L2.

Printed as one JSON line (rank 0):
  value        pairs/s of the tuned form: the library's autotuner picks the
               force kernel, lanes per group and cell factor; the cell list of
               each strain is the paper's neighbourhood-volume choice
  plain        pairs/s of the plain fixed-variant cell lists on the same steps
  e2e          pairs/s through the C ABI with pinned host buffers, copies timed
  roofline     force kernel: algorithmic FP32 instructions / launch time against
               the FP32 issue peak (bound "alu")
  cpu_baseline the FP64 oracle on a bounded sample, on the host cores
  batched      256 independent systems (N ~ U[1000, 20000], planar or general
               flow, WCA or LJ) as one batch: one launch per stage, replayed
               CUDA graph, autotuned cell factor and tile; against a loop of
               per-system contexts with the plain kernel
  learned      the learned cell-list selector, trained on timings of the
               N = 32000 planar, N = 256000 and 2^20 general and 256 batched
               systems, driving the N = 2,097,152 general-flow system: regret
               against the exhaustive choice, pairs/s against the plain variants
  shear        Lees-Edwards shear remapped half way through the period, N = 2^20:
               tuned against plain cell lists
  equilibrium  the N = 2^20 system at rest (A = 0), 16 perturbed cubes per step
  integrate    time integration under the flow (nemd_integrate): 1728 WCA
               particles for 10,000 steps (the paper's runtime comparison of the
               two cell lists) and the N = 2^20 LJ system for 50 steps

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
    "general_n2m": (0, 256),   # N = 2^21: FCC 81^3 with vacancies
}
C_TEST = 7     # FP32 instructions per candidate test: 3 FADD, 1 FMUL, 2 FFMA, 1 FSETP
C_PAIR = 24    # FP32 instructions per interacting pair (force, energy, virial, both sides)

# DRAM bytes (read + write) of one k_force_row launch on the N = 2^20 general-flow
# system at t = T/2, from one ncu capture of that launch (dram__bytes_read.sum +
# dram__bytes_write.sum; bench.py --sections kernel, third of three back-to-back
# launches, so that no earlier kernel's output is written back during it); valid
# only while the kernel's sources are the ones captured (sha1 prefixes).
ROW_TRAFFIC = {"bytes": 40.376832e6 + 1.360128e6,
               "sha1": {"paper_1412_3784_gb300/csrc/force_row.cu": "de5d4de416f6",
                        "paper_1412_3784_gb300/csrc/force_common.cuh": "7add2c4a0360"}}


def row_traffic():
    import hashlib
    for rel, prefix in ROW_TRAFFIC["sha1"].items():
        with open(os.path.join(ROOT, rel), "rb") as f:
            if not hashlib.sha1(f.read()).hexdigest().startswith(prefix):
                return None
    return ROW_TRAFFIC["bytes"]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="general_n1m", choices=sorted(WORKLOADS))
    p.add_argument("--strains", type=int, default=0, help="strains per step (default: the workload's)")
    p.add_argument("--no-baseline", action="store_true", help="skip the CPU oracle sample")
    p.add_argument("--e2e-strains", type=int, default=32)
    p.add_argument("--no-autotune", action="store_true",
                   help="tuned form with --kernel/--group/--kfac instead of the autotuner's choice")
    p.add_argument("--kernel", type=int, default=4,
                   help="force kernel without autotuning (0 plain, 1 grouped, 2 warp, 3 warp half, 4 row)")
    p.add_argument("--group", type=int, default=16, help="lanes per group of the grouped kernel")
    p.add_argument("--kfac", type=int, default=1, help="cell-size factor without autotuning")
    p.add_argument("--streams", type=int, default=5,
                   help="contexts (each on its own CUDA stream) that take the strains of the tuned step in turn")
    p.add_argument("--sections", default="main,batched,learned,shear,equilibrium,integrate",
                   help="comma list of main, batched, learned, shear, equilibrium, integrate; or "
                        "'kernel' alone: one strain's forces evaluated three times back to back "
                        "(the force kernel of the default options, for a counter capture)")
    p.add_argument("--batch-steps", type=int, default=10)
    p.add_argument("--batch-streams", type=int, default=4,
                   help="batches of the same systems (each on its own CUDA stream) that take the batched "
                        "section's steps in turn")
    p.add_argument("--learned-strains", type=int, default=64,
                   help="strains of the N = 2^21 system in the learned section (256 = one per period step)")
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
    ser = series_for(W, k)
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
                         "sample": f"one force evaluation per step (a strain of the period) of the N={ser.n} "
                                   f"system, dynamic size cell list, FP64, one core",
                         "host": dict(zip(("nproc", "model"), host_cpu()))},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def series_for(W, k):
    return W.general_series_2m() if k == 0 else W.general_series(k=k)


def host_cpu():
    """(threads the host offers, CPU model name) of the machine the bench runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return os.cpu_count() or 1, model


def _oracle_eval_worker(args):
    """One oracle evaluation in a fresh process (all-cores leg): returns (pairs, seconds)."""
    k, t, method = args
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1412_3784_gb300 import workloads as W
    w = series_for(W, k).workload(t)
    t0 = time.perf_counter()
    r = oracle.evaluate(w, method)
    return r.npairs, time.perf_counter() - t0


def cpu_baseline_sample(ser, k, ts, reps=3):
    """The FP64 oracle on the host cores, on a bounded sample of the benchmark
    workload: each cell list (dynamic size, dynamic offset) evaluated `reps`
    times on one core at one strain (median), then one evaluation per core at
    as many strains, run as independent processes (the oracle itself stays
    single-threaded)."""
    import multiprocessing as mp
    import oracle
    nproc, model = host_cpu()
    t = ts[len(ts) // 3]
    w = ser.workload(t)
    single = {}
    for method in ("ds", "do"):
        rates = []
        for _ in range(reps):
            t0 = time.perf_counter()
            r = oracle.evaluate(w, method)
            rates.append(r.npairs / (time.perf_counter() - t0))
        single[method] = statistics.median(rates)
    jobs = [(k, ts[(j * len(ts)) // nproc], "ds") for j in range(nproc)]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(nproc) as pool:
        res = pool.map(_oracle_eval_worker, jobs)
    wall = time.perf_counter() - t0
    # the evaluations run side by side: the slowest one bounds the time they took
    all_cores = sum(p for p, _ in res) / max(dt for _, dt in res)
    best = max(single.values())
    return {"value": best, "unit": "pairs/s", "cores": 1, "kind": "oracle",
            "sample": f"FP64 oracle cell lists on the N={ser.n} general-flow system at t={t:.4f}: median of "
                      f"{reps} evaluations per variant on one core (value = the faster variant); then one "
                      f"dynamic size evaluation per core at {nproc} strains as independent processes",
            "single_core": {"ds": single["ds"], "do": single["do"]},
            "all_cores": {"value": all_cores, "cores": nproc, "processes": nproc, "wall_s": wall,
                          "basis": "pairs of all processes / the slowest process's evaluation time"},
            "host": {"nproc": nproc, "model": model}}


def timed_loop(torch, dev, world, fn, steps, warmup, nvtx=None):
    """CUDA-event time (ms) of `steps` calls of fn after `warmup` untimed ones,
    bracketed by a barrier and a device synchronise on both sides (inside an
    NVTX range named nvtx, when given, for profilers)."""
    for _ in range(warmup):
        fn()
    barrier(world)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if nvtx:
        torch.cuda.nvtx.range_push(nvtx)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    if nvtx:
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(dev)
    barrier(world)
    return e0.elapsed_time(e1)


def section_kernel(args, dev, torch, nemd, W):
    """The workload's strain at t = T/2: cell list once, then the forces three
    times back to back with the default kernel options (no autotuning), so that
    a counter capture of the third force launch sees only that kernel's own
    memory traffic (no binning output waiting in L2).  Prints one JSON line."""
    k, _ = WORKLOADS[args.workload]
    ser = series_for(W, k)
    t = 0.5 * ser.period
    q = torch.from_numpy(ser.positions(t)).to(dev)
    F = torch.empty((ser.n, 3), dtype=torch.float32, device=dev)
    U = torch.zeros(1, dtype=torch.float64, device=dev)
    Wv = torch.zeros(9, dtype=torch.float64, device=dev)
    ctx = nemd.Context(dev.index)
    ctx.set_flow(ser.A, ser.L0, ser.M, ser.period)
    ctx.set_potential(nemd.NEMD_LJ, 1.0, 1.0, 1)
    ctx.set_option(nemd.NEMD_OPT_KERNEL, args.kernel)
    ctx.set_option(nemd.NEMD_OPT_CELL_FACTOR, args.kfac)
    ctx.set_state(q, t)
    ctx.build_cells(nemd.NEMD_AUTO_HEURISTIC, ser.rc)
    for _ in range(3):
        ctx.compute_forces(F, U, Wv)
    ctx.sync()
    st = ctx.stats()
    print(json.dumps({"section": "kernel", "workload": args.workload, "t": t, "kernel": args.kernel,
                      "pairs": st["pairs"], "candidates": st["candidates"], "variant": st["variant"]}))
    ctx.close()


def section_main(args, rank, world, dev, torch, nemd, W):
    k, nstrain = WORKLOADS[args.workload]
    S = args.strains or nstrain
    ser = series_for(W, k)
    n = ser.n
    ts = [i / S * ser.period for i in range(S)]
    q_all = torch.empty((S, n, 3), dtype=torch.float64, device=dev)
    for i, t in enumerate(ts):
        q_all[i].copy_(torch.from_numpy(ser.positions(t)))
    F = torch.empty((n, 3), dtype=torch.float32, device=dev)
    U = torch.zeros(1, dtype=torch.float64, device=dev)
    Wv = torch.zeros(9, dtype=torch.float64, device=dev)

    ctx = nemd.Context(dev.index)
    ctx.set_flow(ser.A, ser.L0, ser.M, ser.period)
    ctx.set_potential(nemd.NEMD_LJ, 1.0, 1.0, 1)

    # the tuned form: the autotuner's choice on three strains (start, middle,
    # just before the remap), applied from its cache at every build
    tune = None
    if not args.no_autotune:
        ctx.set_option(nemd.NEMD_OPT_AUTOTUNED, 0)
        for t in (0.0, 0.5 * ser.period, W.NEAR_REMAP_T * ser.period):
            ctx.set_state(torch.from_numpy(ser.positions(t)).to(dev), t)
            best, times = ctx.autotune(nemd.NEMD_AUTO_HEURISTIC, ser.rc, reps=2)
        tune = {"choice": best, "last_call_ms": [[c["kernel"], c["group"], c["cell_factor"], round(ms, 4)]
                                                 for c, ms in times]}

    def configure(kind):
        ctx.set_option(nemd.NEMD_OPT_AUTOTUNED, 0)
        if kind == "plain_ds" or kind == "plain_do":
            ctx.set_option(nemd.NEMD_OPT_KERNEL, 0)
            ctx.set_option(nemd.NEMD_OPT_CELL_FACTOR, 1)
            return nemd.NEMD_DS if kind == "plain_ds" else nemd.NEMD_DO
        if tune is not None:
            ctx.set_option(nemd.NEMD_OPT_AUTOTUNED, 1)
        else:
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
        pairs, cands, variants, rech, kf = [], [], [], [], []
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
            kf.append(st["cell_factor"])
        per[kind] = {"pairs": pairs, "cands": cands, "variants": variants, "rechecks": rech, "kfac": kf}
    pairs_per_step = sum(per["tuned"]["pairs"])
    assert pairs_per_step == sum(per["plain_ds"]["pairs"]) == sum(per["plain_do"]["pairs"])
    # algorithmic FP32 instructions of the tuned step, per the k = 1 stencil of the
    # variant chosen at each strain: 7 per unordered candidate + 24 per pair
    ops_step = 0.0
    for i in range(S):
        v = per["tuned"]["variants"][i]
        cand_k1 = (per["plain_do"] if v == 1 else per["plain_ds"])["cands"][i]
        ops_step += 0.5 * C_TEST * cand_k1 + C_PAIR * per["tuned"]["pairs"][i]

    clocks = Clocks(dev.index)
    variant = configure("tuned")
    # the tuned form as one context on the bench's stream (one evaluation after
    # another) ...
    for _ in range(args.warmup):
        one_step(variant)
    ctx.sync()
    # the force kernel's launch durations for the roofline come from this loop:
    # under concurrency a launch's events also count the time it waits for SMs
    # that another context's kernels hold
    ctx.set_option(nemd.NEMD_OPT_TIMING, 1)
    ms_single = timed_loop(torch, dev, world, lambda: one_step(variant), args.steps, 0)
    ctx.sync()
    k_ms, k_n = ctx.kernel_time()
    ctx.set_option(nemd.NEMD_OPT_TIMING, 0)
    # ... and as K contexts, each on its own CUDA stream, taking the strains in
    # turn: the strains are independent evaluations, so the lattice, grid and
    # stencil kernels of one overlap the force kernel of another.  Every
    # context runs the tuned configuration (the autotuner's choice above).
    K = max(1, args.streams)
    choice = tune["choice"] if tune is not None else {"kernel": args.kernel, "group": args.group,
                                                      "cell_factor": args.kfac}
    pipe = []
    for _ in range(K):
        st = torch.cuda.Stream(dev)
        c = nemd.Context(dev.index, stream=st.cuda_stream)
        c.set_flow(ser.A, ser.L0, ser.M, ser.period)
        c.set_potential(nemd.NEMD_LJ, 1.0, 1.0, 1)
        c.set_option(nemd.NEMD_OPT_KERNEL, choice["kernel"])
        c.set_option(nemd.NEMD_OPT_GROUP, choice["group"])
        c.set_option(nemd.NEMD_OPT_CELL_FACTOR, choice["cell_factor"])
        outs = (torch.empty((n, 3), dtype=torch.float32, device=dev), torch.zeros(1, dtype=torch.float64, device=dev),
                torch.zeros(9, dtype=torch.float64, device=dev))
        pipe.append((c, st, outs))

    def pipe_step():
        for i in range(S):
            c, _, (Fk, Uk, Wk) = pipe[i % K]
            c.set_state(q_all[i], ts[i])
            c.build_cells(nemd.NEMD_AUTO_HEURISTIC, ser.rc)
            c.compute_forces(Fk, Uk, Wk)

    def pipe_timed(steps, warmup):
        for _ in range(warmup):
            pipe_step()
        barrier(world)
        torch.cuda.synchronize(dev)
        home = torch.cuda.current_stream(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed_tuned")   # marks the timed region for profilers
        e0.record(home)
        for _, st, _ in pipe:
            st.wait_event(e0)
        for _ in range(steps):
            pipe_step()
        for _, st, _ in pipe:
            home.wait_stream(st)
        e1.record(home)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize(dev)
        barrier(world)
        return e0.elapsed_time(e1)

    for _ in range(args.warmup):
        pipe_step()
    torch.cuda.synchronize(dev)
    launches0 = sum(c.stats()["launches"] for c, _, _ in pipe)
    clocks.start()
    ms_tuned = pipe_timed(args.steps, 0)
    clk = clocks.stop()
    launches = sum(c.stats()["launches"] for c, _, _ in pipe) - launches0
    # each context's last strain gave the pairs of the untimed pass
    for kc, (c, _, _) in enumerate(pipe):
        c.sync()
        last = max(i for i in range(S) if i % K == kc) if kc < S else None
        if last is not None:
            assert c.stats()["pairs"] == per["tuned"]["pairs"][last], "pipelined pairs differ"
    kernel_name = {0: "k_force_plain", 1: "k_force_chunk", 2: "k_force_warp", 3: "k_force_warp (half)",
                   4: "k_force_row"}
    tuned_kernel = tune["choice"]["kernel"] if tune is not None else args.kernel
    v_ds = configure("plain_ds")
    ms_ds = timed_loop(torch, dev, world, lambda: one_step(v_ds), args.steps, 1)
    v_do = configure("plain_do")
    ms_do = timed_loop(torch, dev, world, lambda: one_step(v_do), args.steps, 1)

    ms_tuned_max = max_over_ranks(ms_tuned, world, dev)
    total_pairs = sum_over_ranks(float(pairs_per_step * args.steps), world, dev)
    value = total_pairs / (ms_tuned_max * 1e-3)
    single_stream = total_pairs / (max_over_ranks(ms_single, world, dev) * 1e-3)
    plain_ds = total_pairs / (max_over_ranks(ms_ds, world, dev) * 1e-3)
    plain_do = total_pairs / (max_over_ranks(ms_do, world, dev) * 1e-3)

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
    avg_launch_s = (k_ms / k_n) * 1e-3
    ops_per_launch = ops_step / S
    achieved = ops_per_launch / avg_launch_s
    # the library's own FFMA microbenchmark beside the derived issue peak
    try:
        peak_measured = float(nemd.measure_peaks(dev.index)["fp32_fma_ops"]) / 1e12
    except Exception:  # noqa: BLE001 -- a context that cannot run the probe reports none
        peak_measured = None
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                "unit": "T FP32 lane-instructions/s",
                "peak_measured": peak_measured,
                "peak_measured_basis": "the library's FFMA loop (nemd_measure_peaks), T lane-ops/s",
                "frac": achieved / peak, "traffic": row_traffic() if tuned_kernel == 4 else None,
                "kernel": kernel_name.get(tuned_kernel, "?"), "ops_per_launch": ops_per_launch,
                "avg_launch_ms": avg_launch_s * 1e3,
                "peak_basis": f"{sms} SMs x 128 FP32 lanes x {peak_mhz:.0f} MHz (FP32 instruction "
                              f"lane-ops/s; derived from unit counts and the clock, not measured)",
                # the force kernel alone, and the ideal roofline that counts only the
                # pair arithmetic (C_PAIR per interacting pair, no candidate tests)
                "force_kernel_pairs_per_s": (pairs_per_step / S) / avg_launch_s,
                "pair_only_frac": (C_PAIR * pairs_per_step / S) / avg_launch_s / peak}

    # precise mode (energy and virial of every accepted pair in float-float, summed
    # per particle in float-float and across particles in float64) on the row
    # kernel, the same strains and the same per-strain cell list choice
    ctx.set_option(nemd.NEMD_OPT_AUTOTUNED, 0)
    ctx.set_option(nemd.NEMD_OPT_KERNEL, 4)
    ctx.set_option(nemd.NEMD_OPT_CELL_FACTOR, 1)
    ctx.set_option(nemd.NEMD_OPT_PRECISE, 1)
    ms_pre = timed_loop(torch, dev, world, lambda: one_step(nemd.NEMD_AUTO_HEURISTIC), args.steps, 1)
    ctx.set_option(nemd.NEMD_OPT_TIMING, 1)
    one_step(nemd.NEMD_AUTO_HEURISTIC)
    ctx.sync()
    kp_ms, kp_n = ctx.kernel_time()
    ctx.set_option(nemd.NEMD_OPT_TIMING, 0)
    ctx.set_option(nemd.NEMD_OPT_PRECISE, 0)
    pre_launch_s = (kp_ms / kp_n) * 1e-3
    precise = {"pairs_per_s": total_pairs / (max_over_ranks(ms_pre, world, dev) * 1e-3),
               "ms_per_step": ms_pre / args.steps, "kernel": "k_force_row (precise)",
               "force_kernel_ms": pre_launch_s * 1e3,
               "roofline_frac": (ops_per_launch / pre_launch_s) / peak,
               "over_fast": ms_tuned / ms_pre,
               "accuracy": "U and W within 1e-9 (relative) of the FP64 oracle in the tests "
                           "(N = 2^20 and 2^21 included); F as in fast mode"}

    # end to end through the C ABI with pinned host buffers
    # Se strains spread evenly over the period, so that the e2e workload has
    # the same mix of lattice shapes as the device-resident step
    Se = min(args.e2e_strains, S)
    e2e_idx = [j * S // Se for j in range(Se)]
    qh = [torch.from_numpy(ser.positions(ts[i])).pin_memory() for i in e2e_idx]
    # the tuned form as timed above: the K contexts take the strains in turn,
    # each with its own pinned result buffers
    outh = [(torch.empty((n, 3), dtype=torch.float32).pin_memory(), torch.zeros(1, dtype=torch.float64).pin_memory(),
             torch.zeros(9, dtype=torch.float64).pin_memory()) for _ in range(K)]
    # asynchronous host I/O: the copy of the next state's positions (and of the
    # previous result) overlaps the current evaluation; results valid after sync
    for c, _, _ in pipe:
        c.set_option(nemd.NEMD_OPT_ASYNC_HOST, 1)

    def e2e_pass(host):
        for j in range(Se):
            c, _, outd = pipe[j % K]
            c.set_state(qh[j] if host else q_all[e2e_idx[j]], ts[e2e_idx[j]])
            c.build_cells(nemd.NEMD_AUTO_HEURISTIC, ser.rc)
            c.compute_forces(*(outh[j % K] if host else outd))
        for c, _, _ in pipe:
            c.sync()                         # every copy back has landed

    # untimed passes over every host buffer first: the first device accesses of
    # freshly pinned pages are measurably slower than later ones
    for _ in range(2):
        e2e_pass(True)
    # five timed passes over the Se strains; the median pass is reported (the
    # host's copy rate varies from pass to pass on a shared machine)
    e2e_reps = []
    for _ in range(5):
        barrier(world)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e2e_pass(True)
        torch.cuda.synchronize(dev)
        e2e_reps.append(max_over_ranks(time.perf_counter() - t0, world, dev))
    e2e_s = sorted(e2e_reps)[len(e2e_reps) // 2]
    for c, _, _ in pipe:
        c.set_option(nemd.NEMD_OPT_ASYNC_HOST, 0)
    e2e_pairs = sum_over_ranks(float(sum(per["tuned"]["pairs"][i] for i in e2e_idx)), world, dev)
    # the same strains from device-resident positions, timed the same way
    e2e_pass(False)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e2e_pass(False)
    torch.cuda.synchronize(dev)
    dev_same_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    for c, _, _ in pipe:
        c.close()
    # the box's pinned host <-> device copy rate, measured beside the e2e loop
    probe_h = torch.empty(6 << 20, dtype=torch.float32).pin_memory()
    probe_d = torch.empty(6 << 20, dtype=torch.float32, device=dev)
    rates = {}
    for name, dst, src in (("h2d_gbs", probe_d, probe_h), ("d2h_gbs", probe_h, probe_d)):
        for _ in range(3):
            dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        for _ in range(10):
            dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize(dev)
        rates[name] = 10 * (24 << 20) / (time.perf_counter() - t1) / 1e9
    e2e = {"value": e2e_pairs / e2e_s, "unit": "pairs/s", "copy_rates": rates,
           "device_resident_same_strains": e2e_pairs / dev_same_s,
           "pass_ms": [round(x * 1e3, 3) for x in e2e_reps],
           "h2d_bytes_per_step": int(S * n * 3 * 8), "d2h_bytes_per_step": int(S * (n * 3 * 4 + 80)),
           "strains_timed": Se, "strains_timed_are": "evenly spaced over the period",
           "mode": f"host positions in and host F, U, W out every strain through the C ABI with "
                   f"NEMD_OPT_ASYNC_HOST (copies on a second stream of each context overlap the evaluations), "
                   f"the {K} contexts of the tuned step taking the strains in turn, one sync per context at the "
                   f"end; median of five passes"}
    ctx.close()
    del q_all

    cpu = None
    if rank == 0 and world == 1 and not args.no_baseline:
        cpu = cpu_baseline_sample(ser, k, ts)

    eta_ds = 2 * sum(per["plain_ds"]["pairs"]) / sum(per["plain_ds"]["cands"])
    eta_do = 2 * sum(per["plain_do"]["pairs"]) / sum(per["plain_do"]["cands"])
    ndo = sum(1 for v in per["tuned"]["variants"] if v == 1)
    return {
        "value": value, "ms_per_step": ms_tuned_max / args.steps,
        "config": {"workload": f"{args.workload}: general 3D flow M=[[3,2,1],[2,2,1],[1,1,1]], "
                               f"perturbed FCC N={n}, rho=0.8442, LJ rc=2.5, {S} strains per step "
                               f"(one period), one force evaluation per strain",
                   "n": n, "strains_per_step": S, "pairs_per_step": pairs_per_step,
                   "tuned": (f"autotuned: kernel {tune['choice']['kernel']}, group {tune['choice']['group']}, "
                             f"cell factor {tune['choice']['cell_factor']}" if tune is not None else
                             f"kernel {args.kernel} (group {args.group}), cell factor {args.kfac}") +
                            f"; cell list per strain by neighbourhood volume (dynamic offset at {ndo} of {S})",
                   "coarse_band_candidates_per_step": int(sum(per["tuned"]["rechecks"])),
                   "l2": "inputs larger than L2: a distinct 24 MB position array per strain",
                   "streams": K,
                   "concurrency": f"{K} contexts, each on its own CUDA stream, take the strains in turn "
                                  "(independent evaluations; one context's setup kernels overlap "
                                  "another's force kernel)",
                   "parallelism": f"replicas x{world}"},
        "single_stream": {"pairs_per_s": single_stream, "ms_per_step": max_over_ranks(ms_single, world, dev) /
                          args.steps, "streams_over_single": value / single_stream,
                          "form": "the same tuned evaluations, one context on one stream"},
        "plain": {"dynamic_size_pairs_per_s": plain_ds, "dynamic_offset_pairs_per_s": plain_do,
                  "tuned_over_best_plain": single_stream / max(plain_ds, plain_do),
                  "basis": "single-stream tuned form against the plain kernels, also one stream",
                  "search_efficiency_ds": eta_ds, "search_efficiency_do": eta_do},
        "autotune": tune,
        "roofline": roofline, "precise": precise, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
        "clocks": clk,
    }


def section_batched(args, world, dev, torch, nemd, W):
    """256 independent systems: one batch (graph replay) against per-system contexts."""
    ws = W.batched_systems()
    kinds = [nemd.NEMD_WCA if w.kind == W.POT_WCA else nemd.NEMD_LJ for w in ws]
    specs = [{"A": w.A, "L0": w.L0, "M": w.M, "T": w.T, "rc": w.rc, "n": w.n, "kind": kd,
              "variant": nemd.NEMD_AUTO_HEURISTIC} for w, kd in zip(ws, kinds)]
    t0 = time.perf_counter()
    b = nemd.Batch(specs, device=dev.index)
    t_final = time.perf_counter() - t0
    q = torch.from_numpy(np.concatenate([w.q for w in ws])).to(dev)
    ts = [w.t for w in ws]
    F = torch.zeros((b.ntot, 3), dtype=torch.float32, device=dev)
    UW = torch.zeros((b.nsys, 10), dtype=torch.float64, device=dev)
    b.set_state(q, ts)
    if args.no_autotune:  # the default options: cell factor 1, 32-particle chunks
        times = [({"cell_factor": 1, "tile": 32}, float("nan"))]
    else:
        times = b.autotune(reps=3)
    b.compute(F, UW)
    b.sync()
    st, launches = b.stats()
    pairs = sum(x["pairs"] for x in st)
    ms_one = timed_loop(torch, dev, world, lambda: b.compute(F, UW), args.batch_steps, 3) / args.batch_steps
    b.sync()
    best = min(times, key=lambda x: x[1] if x[1] == x[1] else 0.0)[0]
    b.close()
    # the steps taken in turn by batch_streams batches of the same systems, each
    # on its own CUDA stream with its own outputs (one step's setup kernels run
    # beside another step's force kernel); every step evaluates all systems
    KB = max(1, args.batch_streams)
    bstreams = [torch.cuda.Stream(dev) for _ in range(KB)]
    pipe = []
    for st in bstreams:
        bk = nemd.Batch(specs, device=dev.index, stream=st.cuda_stream)
        bk.set_option(nemd.NEMD_BATCH_OPT_CELL_FACTOR, best["cell_factor"])
        bk.set_option(nemd.NEMD_BATCH_OPT_TILE, best["tile"])
        bk.set_state(q, ts)
        pipe.append((bk, st, torch.zeros((b.ntot, 3), dtype=torch.float32, device=dev),
                     torch.zeros((b.nsys, 10), dtype=torch.float64, device=dev)))
    home = torch.cuda.current_stream(dev)

    def pipe_steps(m):
        for i in range(m):
            bk, _, Fk, UWk = pipe[i % KB]
            bk.compute(Fk, UWk)

    pipe_steps(3 * KB)
    torch.cuda.synchronize(dev)
    barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed_batched")   # marks the timed region for profilers
    e0.record(home)
    for _, st, _, _ in pipe:
        st.wait_event(e0)
    pipe_steps(args.batch_steps)
    for _, st, _, _ in pipe:
        home.wait_stream(st)
    e1.record(home)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(dev)
    barrier(world)
    ms = e0.elapsed_time(e1) / args.batch_steps
    for bk, _, _, _ in pipe:
        bk.sync()
        assert sum(x["pairs"] for x in bk.stats()[0]) == pairs, "pipelined batch pairs differ"
        bk.close()
    # the same systems through per-system contexts with the same force kernel
    # (row kernel, cell list per system by neighbourhood volume), one after another
    ctxs = []
    for w, kd in zip(ws, kinds):
        c = nemd.Context(dev.index)
        c.set_flow(w.A, w.L0, w.M, w.T)
        c.set_potential(kd, 1.0, 1.0, 1)
        c.set_option(nemd.NEMD_OPT_KERNEL, 4)
        ctxs.append(c)
    qs = [q[b.offsets[s]:b.offsets[s + 1]] for s in range(len(ws))]
    Fs = [F[b.offsets[s]:b.offsets[s + 1]] for s in range(len(ws))]

    def loop():
        for s, c in enumerate(ctxs):
            c.set_state(qs[s], ts[s])
            c.build_cells(nemd.NEMD_AUTO_HEURISTIC, ws[s].rc)
            c.compute_forces(Fs[s])
    ms_loop = timed_loop(torch, dev, world, loop, 2, 1) / 2
    pairs_loop = sum(c.stats()["pairs"] for c in ctxs)
    for c in ctxs:
        c.close()
    assert pairs_loop == pairs
    return {"workload": f"{len(ws)} systems, N ~ U[1000, 20000] (total {b.ntot}), density ~ U(0.8, 0.9), "
                        "planar or general flow at rate ~ U(0.5, 2) and random phase, WCA or LJ rc 2.5",
            "pairs_per_step": pairs, "ms_per_step": ms, "pairs_per_s": pairs / ms * 1e3,
            "streams": KB,
            "single_stream": {"ms_per_step": ms_one, "pairs_per_s": pairs / ms_one * 1e3},
            "kernel_launches_per_step": launches,
            "autotuned": {"cell_factor": best["cell_factor"], "tile": best["tile"],
                          "candidates_ms": [[c["cell_factor"], c["tile"], round(t, 4)] for c, t in times
                                            if t == t]},
            "finalize_s": t_final,
            "per_system_loop": {"ms_per_step": ms_loop, "pairs_per_s": pairs / ms_loop * 1e3,
                                "form": "one context per system, row kernel, cell list by neighbourhood volume"},
            "speedup_over_loop": ms_loop / ms}


def _option_rows(ctx, torch, dev, nemd, W, ser, m, reps=3):
    """Option timings (features, ms per option) and the volume rule's option at m strains of a series."""
    ctx.set_flow(ser.A, ser.L0, ser.M, ser.period)
    ctx.set_potential(nemd.NEMD_WCA if ser.kind == W.POT_WCA else nemd.NEMD_LJ, 1.0, 1.0, 1)
    X, T, rule = [], [], []
    for i in range(m):
        t = (i + 0.5) / m * ser.period
        ctx.set_state(torch.from_numpy(ser.positions(t)).to(dev), t)
        f, ms = ctx.time_options(ser.rc, reps=reps)
        ctx.set_option(nemd.NEMD_OPT_CELL_FACTOR, 1)
        ctx.build_cells(nemd.NEMD_AUTO_HEURISTIC, ser.rc)
        ctx.compute_forces()
        ctx.sync()
        X.append(f)
        T.append(ms)
        rule.append(ctx.stats()["variant"])          # option index of the volume rule at k = 1
    return X, T, rule


def _regrets(ctx, X, T, rule):
    T = np.array(T)
    pick = np.argmin(ctx.model_predict(np.array(X)), axis=1)
    best = T.min(axis=1)
    idx = np.arange(len(T))
    return (float((T[idx, pick] - best).sum() / best.sum()),
            float((T[idx, np.array(rule)] - best).sum() / best.sum()), pick, T)


def section_learned(args, dev, torch, nemd, W):
    """Learned selector over the row kernel's options (cell list variant x cell
    factor): trained on timing rows of LJ systems (N = 32000 planar, N = 256000
    and N = 2^20 general flow), WCA systems (N = 32000 general, N = 16384 planar)
    and the batched systems; judged on held-out systems none of whose strains or
    sites it saw: the N = 2^21 LJ general flow and a WCA mix (N = 55296 general,
    N = 6912 planar)."""
    ctx = nemd.Context(dev.index)
    ctx.set_option(nemd.NEMD_OPT_KERNEL, 4)
    X, T = [], []
    t0 = time.perf_counter()
    train = ((W.planar_series(k=20), 64), (W.general_series(k=40), 64), (W.general_series(k=64), 32),
             (W.StrainSeries(W.M_GENERAL, 20, 21, kind=W.POT_WCA), 32),
             (W.StrainSeries(W.M_PLANAR, 16, 23, kind=W.POT_WCA), 32))
    for ser, m in train:
        x, tt, _ = _option_rows(ctx, torch, dev, nemd, W, ser, m)
        X += x
        T += tt
    for w in W.batched_systems():
        ctx.set_flow(w.A, w.L0, w.M, w.T)
        ctx.set_potential(nemd.NEMD_WCA if w.kind == W.POT_WCA else nemd.NEMD_LJ, 1.0, 1.0, 1)
        ctx.set_state(torch.from_numpy(w.q).to(dev), w.t)
        try:
            f, ms = ctx.time_options(w.rc, reps=3)
        except nemd.NemdError:
            continue                  # an option whose box is too small for the cut-off
        X.append(f)
        T.append(ms)
    t_rows = time.perf_counter() - t0
    X = np.array(X)
    T = np.array(T)
    t0 = time.perf_counter()
    hist = ctx.model_train(X, T, steps=3000, batch=128, lr=3e-3, seed=0)
    t_train = time.perf_counter() - t0

    # held-out WCA mix
    wx, wt, wr = [], [], []
    for ser, m in ((W.StrainSeries(W.M_GENERAL, 24, 31, kind=W.POT_WCA), 32),
                   (W.StrainSeries(W.M_PLANAR, 12, 32, kind=W.POT_WCA), 32)):
        x, tt, rr = _option_rows(ctx, torch, dev, nemd, W, ser, m)
        wx += x
        wt += tt
        wr += rr
    reg_wl, reg_wr, pick_w, Tw = _regrets(ctx, wx, wt, wr)

    ser = W.general_series_2m()
    S4 = args.learned_strains
    ts = [i / S4 * ser.period for i in range(S4)]
    ctx.set_flow(ser.A, ser.L0, ser.M, ser.period)
    ctx.set_potential(nemd.NEMD_LJ, 1.0, 1.0, 1)
    q_all = torch.empty((S4, ser.n, 3), dtype=torch.float64, device=dev)
    for i, t in enumerate(ts):
        q_all[i].copy_(torch.from_numpy(ser.positions(t)))
    table, feats, rule = [], [], []
    for i in range(S4):
        ctx.set_state(q_all[i], ts[i])
        f, ms = ctx.time_options(ser.rc, reps=3)
        table.append(ms)
        feats.append(f)
        ctx.set_option(nemd.NEMD_OPT_CELL_FACTOR, 1)
        ctx.build_cells(nemd.NEMD_AUTO_HEURISTIC, ser.rc)
        ctx.compute_forces()
        ctx.sync()
        rule.append(ctx.stats()["variant"])
    regret_learned, regret_rule, pick, table = _regrets(ctx, feats, table, rule)

    F = torch.empty((ser.n, 3), dtype=torch.float32, device=dev)
    pairs = 0
    for i in range(S4):
        ctx.set_state(q_all[i], ts[i])
        ctx.build_cells(nemd.NEMD_DS, ser.rc)
        ctx.compute_forces(F)
        ctx.sync()
        pairs += ctx.stats()["pairs"]

    def step(variant, kernel):
        ctx.set_option(nemd.NEMD_OPT_KERNEL, kernel)
        ctx.set_option(nemd.NEMD_OPT_CELL_FACTOR, 1)

        def fn():
            for i in range(S4):
                ctx.set_state(q_all[i], ts[i])
                ctx.build_cells(variant, ser.rc)
                ctx.compute_forces(F)
        return fn
    # learned and rule alternate over three rounds (medians): their difference
    # is of the order of the timing noise of one loop
    forms = (("learned", nemd.NEMD_AUTO_LEARNED, 4), ("rule", nemd.NEMD_AUTO_HEURISTIC, 4),
             ("plain_ds", nemd.NEMD_DS, 0), ("plain_do", nemd.NEMD_DO, 0))
    runs = {name: [] for name, _, _ in forms}
    for r in range(3):
        for name, variant, kernel in forms:
            if r > 0 and name.startswith("plain"):
                continue
            runs[name].append(timed_loop(torch, dev, 1, step(variant, kernel), 2, 1) / 2)
    out = {name: pairs / statistics.median(v) * 1e3 for name, v in runs.items()}
    del q_all

    # the held-out WCA mix, where the volume rule errs most: pairs/s of the
    # learned and rule choices over its strains (alternating rounds, medians)
    mix = {"learned": [], "rule": []}
    mix_pairs = 0
    for mser, m in ((W.StrainSeries(W.M_GENERAL, 24, 31, kind=W.POT_WCA), 32),
                    (W.StrainSeries(W.M_PLANAR, 12, 32, kind=W.POT_WCA), 32)):
        ctx.set_flow(mser.A, mser.L0, mser.M, mser.period)
        ctx.set_potential(nemd.NEMD_WCA, 1.0, 1.0, 1)
        mts = [i / m * mser.period for i in range(m)]
        mq = [torch.from_numpy(mser.positions(t)).to(dev) for t in mts]
        Fm = torch.empty((mser.n, 3), dtype=torch.float32, device=dev)
        ctx.set_option(nemd.NEMD_OPT_KERNEL, 4)
        ctx.set_option(nemd.NEMD_OPT_CELL_FACTOR, 1)
        for i in range(m):
            ctx.set_state(mq[i], mts[i])
            ctx.build_cells(nemd.NEMD_AUTO_HEURISTIC, mser.rc)
            ctx.compute_forces(Fm)
            ctx.sync()
            mix_pairs += ctx.stats()["pairs"]

        def mstep(variant):
            def fn():
                for i in range(m):
                    ctx.set_state(mq[i], mts[i])
                    ctx.build_cells(variant, mser.rc)
                    ctx.compute_forces(Fm)
            return fn
        for r in range(3):
            for name, variant in (("learned", nemd.NEMD_AUTO_LEARNED), ("rule", nemd.NEMD_AUTO_HEURISTIC)):
                ms = timed_loop(torch, dev, 1, mstep(variant), 3, 1) / 3
                if len(mix[name]) <= r:
                    mix[name].append(0.0)
                mix[name][r] += ms
    mix_out = {name: mix_pairs / statistics.median(v) * 1e3 for name, v in mix.items()}
    ctx.close()
    return {"workload": f"general 3D flow, N={ser.n} (FCC 81^3 with vacancies), LJ rc 2.5, {S4} strains "
                        f"of one period; and a WCA mix (N=55296 general flow, N=6912 planar flow, 32 strains "
                        f"each); all held out from training",
            "training_rows": int(len(X)), "rows_s": t_rows, "train_s": t_train,
            "train_loss_first_last": [float(hist[:50].mean()), float(hist[-50:].mean())],
            "options": "o = (variant o & 1, cell factor 1 + (o >> 1)), row kernel",
            "regret_vs_exhaustive": {"learned": regret_learned, "volume_rule_k1": regret_rule},
            "learned_choices": np.bincount(pick, minlength=4).tolist(),
            "exhaustive_choices": np.bincount(table.argmin(axis=1), minlength=4).tolist(),
            "wca_mix": {"regret_vs_exhaustive": {"learned": reg_wl, "volume_rule_k1": reg_wr},
                        "learned_choices": np.bincount(pick_w, minlength=4).tolist(),
                        "exhaustive_choices": np.bincount(Tw.argmin(axis=1), minlength=4).tolist(),
                        "rule_choices": np.bincount(np.array(wr), minlength=4).tolist(),
                        "pairs_per_s": mix_out, "learned_over_rule": mix_out["learned"] / mix_out["rule"]},
            "pairs_per_s": out,
            "learned_over_best_plain": out["learned"] / max(out["plain_ds"], out["plain_do"]),
            "learned_over_rule": out["learned"] / out["rule"]}


def section_shear(args, world, dev, torch, nemd, W):
    """Lees-Edwards shear (Sec. 2.2), remapped half way through the period, on
    N = 1,048,576 LJ particles: 128 strains of one period, the tuned form
    (autotuned kernel, per-strain cell list by neighbourhood volume) against the
    plain fixed-variant cell lists."""
    ser = W.shear_series(k=64)
    S = 128
    ts = [(i / S - 0.5) * ser.period for i in range(S)]
    q_all = torch.empty((S, ser.n, 3), dtype=torch.float64, device=dev)
    for i, t in enumerate(ts):
        q_all[i].copy_(torch.from_numpy(ser.positions(t)))
    F = torch.empty((ser.n, 3), dtype=torch.float32, device=dev)
    ctx = nemd.Context(dev.index)
    ctx.set_flow(ser.A, ser.L0, ser.M, ser.period)
    ctx.set_potential(nemd.NEMD_LJ, 1.0, 1.0, 1)
    ctx.set_option(nemd.NEMD_OPT_REMAP, 1)
    for t in (-0.5 * ser.period, 0.0, 0.25 * ser.period):
        ctx.set_state(torch.from_numpy(ser.positions(t)).to(dev), t)
        best, _ = ctx.autotune(nemd.NEMD_AUTO_HEURISTIC, ser.rc, reps=2)

    def form(kind):
        ctx.set_option(nemd.NEMD_OPT_AUTOTUNED, 1 if kind == "tuned" else 0)
        if kind != "tuned":
            ctx.set_option(nemd.NEMD_OPT_KERNEL, 0)
            ctx.set_option(nemd.NEMD_OPT_CELL_FACTOR, 1)
        variant = {"tuned": nemd.NEMD_AUTO_HEURISTIC, "plain_ds": nemd.NEMD_DS, "plain_do": nemd.NEMD_DO}[kind]

        def step():
            for i in range(S):
                ctx.set_state(q_all[i], ts[i])
                ctx.build_cells(variant, ser.rc)
                ctx.compute_forces(F)
        return variant, step

    out, cands = {}, {}
    pairs = 0
    for kind in ("plain_ds", "plain_do", "tuned"):
        variant, step = form(kind)
        c, vs, p = [], [], 0
        for i in range(S):
            ctx.set_state(q_all[i], ts[i])
            ctx.build_cells(variant, ser.rc)
            ctx.compute_forces(F)
            ctx.sync()
            st = ctx.stats()
            c.append(st["candidates"])
            vs.append(st["variant"])
            p += st["pairs"]
        cands[kind] = (c, vs)
        pairs = p
        if kind == "tuned":
            ctx.set_option(nemd.NEMD_OPT_TIMING, 1)
        ms = timed_loop(torch, dev, world, step, 2, 1) / 2
        if kind == "tuned":
            ctx.sync()
            k_ms, k_n = ctx.kernel_time()
            ctx.set_option(nemd.NEMD_OPT_TIMING, 0)
        out[kind] = pairs / ms * 1e3
    ops = 0.0
    for i in range(S):
        v = cands["tuned"][1][i]
        ops += 0.5 * C_TEST * (cands["plain_do"] if v == 1 else cands["plain_ds"])[0][i]
    ops += C_PAIR * pairs
    props = torch.cuda.get_device_properties(dev)
    peak = fp32_issue_peak(props.multi_processor_count, 2070.0)
    frac = (ops / S) / ((k_ms / k_n) * 1e-3) / peak
    ctx.close()
    del q_all
    return {"workload": f"Lees-Edwards shear u = y e_x, perturbed FCC N={ser.n}, rho=0.8442, LJ rc=2.5, "
                        f"{S} strains of one period, remapped half way (tilt within half a spacing)",
            "pairs_per_step": pairs, "pairs_per_s": out,
            "tuned": f"autotuned: kernel {best['kernel']}, cell factor {best['cell_factor']}",
            "tuned_over_best_plain": out["tuned"] / max(out["plain_ds"], out["plain_do"]),
            "force_kernel_ms": k_ms / k_n, "roofline_frac": frac}


def section_equilibrium(args, world, dev, torch, nemd, W):
    """The N = 1,048,576 LJ system at rest (A = 0): 16 independently perturbed FCC
    cubes per step (384 MB of positions, more than L2), tuned against plain."""
    ws = W.equilibrium_set(k=64)
    S = len(ws)
    qs = [torch.from_numpy(w.q).to(dev) for w in ws]
    F = torch.empty((ws[0].n, 3), dtype=torch.float32, device=dev)
    ctx = nemd.Context(dev.index)
    ctx.set_flow(ws[0].A, ws[0].L0, ws[0].M, ws[0].T)
    ctx.set_potential(nemd.NEMD_LJ, 1.0, 1.0, 1)
    ctx.set_state(qs[0], 0.0)
    best, _ = ctx.autotune(nemd.NEMD_AUTO_HEURISTIC, ws[0].rc, reps=2)
    out, cands, pairs = {}, {}, 0
    for kind, variant in (("plain_ds", nemd.NEMD_DS), ("plain_do", nemd.NEMD_DO), ("tuned", nemd.NEMD_AUTO_HEURISTIC)):
        ctx.set_option(nemd.NEMD_OPT_AUTOTUNED, 1 if kind == "tuned" else 0)
        if kind != "tuned":
            ctx.set_option(nemd.NEMD_OPT_KERNEL, 0)
            ctx.set_option(nemd.NEMD_OPT_CELL_FACTOR, 1)
        c, vs, p = [], [], 0
        for i in range(S):
            ctx.set_state(qs[i], 0.0)
            ctx.build_cells(variant, ws[i].rc)
            ctx.compute_forces(F)
            ctx.sync()
            st = ctx.stats()
            c.append(st["candidates"])
            vs.append(st["variant"])
            p += st["pairs"]
        cands[kind] = (c, vs)
        pairs = p

        def step():
            for i in range(S):
                ctx.set_state(qs[i], 0.0)
                ctx.build_cells(variant, ws[i].rc)
                ctx.compute_forces(F)
        if kind == "tuned":
            ctx.set_option(nemd.NEMD_OPT_TIMING, 1)
        ms = timed_loop(torch, dev, world, step, 3, 1) / 3
        if kind == "tuned":
            ctx.sync()
            k_ms, k_n = ctx.kernel_time()
            ctx.set_option(nemd.NEMD_OPT_TIMING, 0)
        out[kind] = pairs / ms * 1e3
    ops = sum(0.5 * C_TEST * (cands["plain_do"] if cands["tuned"][1][i] == 1 else cands["plain_ds"])[0][i]
              for i in range(S)) + C_PAIR * pairs
    peak = fp32_issue_peak(torch.cuda.get_device_properties(dev).multi_processor_count, 2070.0)
    eta = 2 * pairs / sum(cands["plain_ds"][0])
    ctx.close()
    return {"workload": f"A = 0, {S} independently perturbed FCC cubes of N={ws[0].n} per step, LJ rc=2.5",
            "pairs_per_step": pairs, "pairs_per_s": out,
            "tuned": f"autotuned: kernel {best['kernel']}, cell factor {best['cell_factor']}",
            "tuned_over_best_plain": out["tuned"] / max(out["plain_ds"], out["plain_do"]),
            "search_efficiency_ds": eta, "force_kernel_ms": k_ms / k_n,
            "roofline_frac": (ops / S) / ((k_ms / k_n) * 1e-3) / peak}


def section_integrate(args, dev, torch, nemd, W):
    """Time integration under the flow (nemd_integrate): the runtime comparison
    of Sec. 5 (1728 WCA particles, 10,000 steps; dynamic offset against dynamic
    size) on the general KR flow, and the N = 2^20 LJ system for 50 steps."""
    stats = {}

    def run(ser, w, p0, dt, nsteps, variant, kernel, autotune=False, skin=0.0):
        ctx = nemd.Context(dev.index)
        ctx.set_flow(ser.A, ser.L0, ser.M, ser.period)
        ctx.set_potential(nemd.NEMD_WCA if w.kind == W.POT_WCA else nemd.NEMD_LJ, 1.0, 1.0, 1)
        ctx.set_verlet(skin)
        q = torch.from_numpy(np.ascontiguousarray(w.q)).to(dev)
        if autotune:
            ctx.set_state(q, w.t)
            ctx.autotune(nemd.NEMD_AUTO_HEURISTIC, w.rc, reps=2)
            ctx.set_option(nemd.NEMD_OPT_AUTOTUNED, 1)
        else:
            ctx.set_option(nemd.NEMD_OPT_KERNEL, kernel)
        # untimed warm-up run, then the timed one from the same initial state
        qw, pw = q.clone(), torch.from_numpy(p0).to(dev)
        ctx.integrate(qw, pw, w.t, dt, min(nsteps, 20), variant, w.rc, 1)
        ctx.sync()
        p = torch.from_numpy(p0).to(dev)
        st = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(st)
        ctx.set_verlet(skin)           # counts from here
        ctx.integrate(q, p, w.t, dt, nsteps, variant, w.rc, 1)
        e1.record(st)
        ctx.sync()
        torch.cuda.synchronize(dev)
        if skin > 0.0:
            b, ev, width, _ = ctx.verlet_stats()
            stats[(w.n, skin)] = {"builds": b, "evaluations": ev, "entries_per_particle": width}
        ctx.close()
        return e0.elapsed_time(e1) / nsteps

    out = {}
    small = W.StrainSeries(W.M_GENERAL, 8, 41, kind=W.POT_WCA, vacancies=4 * 8 ** 3 - 1728)
    w = small.workload(0.0)
    p0 = W.maxwell_momenta(w.n, 1.0, seed=42)
    steps = 10000
    ms = {"plain_ds": run(small, w, p0, 0.004, steps, nemd.NEMD_DS, 0),
          "plain_do": run(small, w, p0, 0.004, steps, nemd.NEMD_DO, 0),
          "tuned": run(small, w, p0, 0.004, steps, nemd.NEMD_AUTO_HEURISTIC, 2, autotune=True)}
    out["n1728"] = {"workload": f"N={w.n} WCA (FCC 8^3 with vacancies), rho=0.8442, general KR flow, dt=0.004, "
                                f"kT=1 isokinetic, {steps} steps",
                    "ms_per_step": ms, "do_over_ds_time": ms["plain_do"] / ms["plain_ds"],
                    "paper_do_over_ds_time": 0.717,
                    "note": "the paper's ratio is one CPU core on a uniaxial flow; at this size every step here "
                            "is a few dozen launches of near-empty kernels"}
    big = W.general_series(k=64)
    wb = big.workload(0.0)
    pb = W.maxwell_momenta(wb.n, 0.8, seed=43)
    msb = {"plain_ds": run(big, wb, pb, 0.002, 50, nemd.NEMD_DS, 0),
           "plain_do": run(big, wb, pb, 0.002, 50, nemd.NEMD_DO, 0),
           "tuned": run(big, wb, pb, 0.002, 50, nemd.NEMD_AUTO_HEURISTIC, 2, autotune=True),
           "verlet_skin_0.3": run(big, wb, pb, 0.002, 50, nemd.NEMD_AUTO_HEURISTIC, 4, skin=0.3)}
    out["n1m"] = {"workload": f"N={wb.n} LJ rc=2.5 general KR flow, dt=0.002, kT=0.8 isokinetic, 50 steps",
                  "ms_per_step": msb, "do_over_ds_time": msb["plain_do"] / msb["plain_ds"],
                  "tuned_speedup_over_best_plain": min(msb["plain_ds"], msb["plain_do"]) / msb["tuned"],
                  "verlet": stats.get((wb.n, 0.3)),
                  "verlet_over_tuned_cell_list": msb["tuned"] / msb["verlet_skin_0.3"],
                  "verlet_note": "the list is rebuilt (cell list at rc + skin, then the list kernel) when the "
                                 "deformation-and-displacement bound says a pair outside it could have come "
                                 "within rc, and at every remap; one host synchronisation per step decides it"}
    return out


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
    sections = set(args.sections.split(","))
    # all work (library contexts, batches, events) on one stream of our own: the
    # legacy default stream adds a per-launch cost (about 4 % of an evaluation)
    stream = torch.cuda.Stream(dev)
    if sections == {"kernel"}:
        with torch.cuda.stream(stream):
            section_kernel(args, dev, torch, nemd, W)
        return
    with torch.cuda.stream(stream):
        main_part = section_main(args, rank, world, dev, torch, nemd, W)
        batched = section_batched(args, world, dev, torch, nemd, W) if "batched" in sections else None
        learned = section_learned(args, dev, torch, nemd, W) if "learned" in sections else None
        shear = section_shear(args, world, dev, torch, nemd, W) if "shear" in sections else None
        equilibrium = section_equilibrium(args, world, dev, torch, nemd, W) if "equilibrium" in sections else None
        integ = section_integrate(args, dev, torch, nemd, W) if "integrate" in sections else None
    if rank == 0:
        line = {
            "metric": "interacting pairs/s per force eval", "value": main_part["value"], "unit": "pairs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": main_part["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 pair math, f64 lattice/guard band/reductions, float-float wrap",
            "data": "synthetic",
        }
        for key in ("config", "single_stream", "plain", "autotune", "roofline", "precise", "cpu_baseline", "e2e",
                    "gpu_launches",
                    "clocks"):
            line[key] = main_part[key]
        line["batched"] = batched
        line["learned"] = learned
        line["shear"] = shear
        line["equilibrium"] = equilibrium
        line["integrate"] = integ
        print(json.dumps(line), flush=True)
    barrier(world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
