"""Benchmark of the TT finite-volume shallow-water stage on GB300.

One step = one full SSP-RK3 step (three stages: WENO5 reconstruction by
cross, Taylor reciprocal, LLF fluxes from Hadamard products, rounding) of the
nonlinear 256 x 256 workload (3 seeded Gaussian bumps, rank cap 32, tol
1e-8), through the C ABI of libttfv.so.  Metric: equivalent cell updates per
second, N^2 x steps / s (summed over ranks).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (Oracle B, the TT algorithm in
numpy) on this machine's host cores on the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# The stage graph keeps up to 16 streams busy at once; with CUDA's default of
# 8 hardware work queues, kernels of unrelated streams would queue behind each
# other.  CUDA reads this when the context is created, so it is set before
# torch initialises the device.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "equiv. cell-updates/s per RK step at fixed L2 err vs FP64 oracle; % roofline"
UNIT = "cell-updates/s"
# arithmetic of the rounding contractions per precision form (SVDs and cores stay FP64)
DTYPES = {"fp64": "f64", "fp32": "f32", "tf32": "tf32x3", "bf16": "bf16x6"}
WORKLOAD = "nonlinear256_weno5"
# GB300 FP64: 2 FMA / clk / SM (4 flop), 152 SMs, 2070 MHz maximum SM clock
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "tf32", "bf16"],
                    help="working precision of the rounding contractions (fp64: the plain path)")
    ap.add_argument("--pivots", default="maxvol", choices=["maxvol", "learned"],
                    help="cross start: maxvol of the initial TT, or the shipped learned network")
    ap.add_argument("--compare-plain", action="store_true",
                    help="ensemble workloads: also time the one-instance-at-a-time path on the same steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=1)
    return ap.parse_args()


def max_over_ranks(x):
    """The maximum of x over the ranks of the process group (x itself when
    there is none): the job's time is its slowest replica's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank, world, total_ms):
    """Whole-job throughput of N independent replicas: the units all ranks
    processed over the slowest rank's time."""
    return units_per_rank * world / (total_ms / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def make_state(w, cap):
    from synth import initial_tt
    Q, p = initial_tt(w)
    return Q, p


def traffic_for(kernel_class):
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu
    summary, if it was taken on the current source of that kernel."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    try:
        with open(path) as f:
            tab = json.load(f)
    except (OSError, ValueError):
        return None
    ent = tab.get(kernel_class)
    if not ent:
        return None
    import hashlib
    src = os.path.join(ROOT, ent["source"])
    try:
        with open(src, "rb") as f:
            text = f.read()
    except OSError:
        return None
    # the hash covers the kernel's own section of the source file when the
    # entry names its bounding markers, else the whole file
    b, e = ent.get("begin", "").encode(), ent.get("end", "").encode()
    if b and e and b in text and e in text:
        text = text[text.index(b):text.index(e)]
    h = hashlib.sha256(text).hexdigest()[:16]
    return ent["bytes_per_launch"] if h == ent.get("source_sha256_16") else None


def cpu_baseline(w, p, Q, nsteps):
    """Oracle B (numpy TT algorithm) timed on the host cores from the initial
    state for `nsteps` RK steps; returns (result dict, oracle state)."""
    from oracle import tt_fv as TB
    t0 = time.perf_counter()
    Qo = Q
    for _ in range(nsteps):
        Qo = TB.step(Qo, w, p, seed=0)
    dt = time.perf_counter() - t0
    n = w["n"]
    cores = os.cpu_count()
    return {"value": n * n * nsteps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {nsteps} SSP-RK3 step(s) of the {w['n']}x{w['n']} {w['scheme']} workload from its "
                      f"initial "
                      f"state (ranks small, cheaper than later steps); numpy/OpenBLAS float64 on {cores} threads",
            "seconds": dt}, Qo


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from synth import workload
    from oracle import tt_fv as TB
    w = workload(args.workload)
    Q, p = make_state(w, w["cap"])
    n = w["n"]
    for _ in range(args.warmup):
        Q = TB.step(Q, w, p, seed=0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Q = TB.step(Q, w, p, seed=0)
    dt = time.perf_counter() - t0
    value = n * n * args.steps / dt
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "scheme": w["scheme"], "eqn": w["eqn"],
                       "rank_cap": w["cap"], "tol": w["tol"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"SSP-RK3 steps {args.warmup + 1}..{args.warmup + args.steps} from the "
                                       f"initial state, numpy/OpenBLAS float64"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch
    from synth import workload
    from paper_2408_03483_gb300 import api, capi

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    capi.load()
    w = workload(args.workload)
    n, cap = w["n"], w["cap"]
    Q, p = make_state(w, cap)
    stream = torch.cuda.current_stream()
    net = api.PivotNet.shipped() if args.pivots == "learned" else None

    def new_solver(state):
        q0 = [api.DevTT.from_cores(A, B, cap=cap) for A, B in state]
        s = api.Solver(q0, w["eqn"], w["scheme"], n, p["dt"], w["tol"], cap, g=p["g"], H=p["H"], f=p["f"],
                       kick=4, max_sweeps=10, max_iter=50, seed=0, precision=args.precision, pivots=args.pivots)
        if args.pivots == "learned":
            s.set_pivot_net(net)
        return s

    # ---- parity sample: first step from the initial state vs the oracle
    s0 = new_solver(Q)
    s0.step(1)
    first = s0.get()
    s0.close()

    # ---- device-timed region
    s = new_solver(Q)
    for _ in range(args.warmup):
        s.step(1)
    # the state the timed steps start from: the end-to-end run below repeats
    # the same steps from it
    host = [(torch.empty((cap, n), dtype=torch.float64).pin_memory(),
             torch.empty((cap, n), dtype=torch.float64).pin_memory()) for _ in range(3)]
    st = s.get()
    for (ha, hb), q in zip(host, st):
        ha[:q.rank].copy_(q.a[:q.rank].cpu())
        hb[:q.rank].copy_(q.b[:q.rank].cpu())
    ranks_host = [q.rank for q in st]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    sec0 = s.stats()["section_ms"]
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = api.launch_count()
    step_ms = []
    # profiler range = the timed steps (ncu --profile-from-start off records these only)
    torch.cuda.profiler.start()
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(1)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    torch.cuda.profiler.stop()
    launches = api.launch_count() - launches0
    clk = clocks.stop()
    sec1 = s.stats()["section_ms"]
    # ---- per-kernel profile: further steps with every launch event-timed and
    # the independent tasks serialised (so each time is the kernel's own)
    prof_steps = max(1, min(args.steps, 2))
    s.profile(True)
    s.kernel_profile(reset=True)
    for _ in range(prof_steps):
        s.step(1)
    prof = s.kernel_profile(reset=True)
    s.profile(False)
    st_all = s.stats()
    ranks_after = st_all["rank"]
    dev_status = st_all["device_status"]
    sections = {name: round((b - a) / args.steps, 2) for name, a, b in
                zip(("faces", "side_fluxes_and_lambda", "llf", "quadrature_difference", "forward_euler",
                     "ssp_combination"), sec0, sec1)}
    cross_info = {"calls": st_all["cross_calls"], "sweeps": st_all["cross_sweeps"],
                  "sweeps_per_call": st_all["cross_sweeps"] / max(st_all["cross_calls"], 1),
                  "learned_calls": st_all["learned_calls"], "learned_accepted": st_all["learned_accepted"],
                  "roundings": st_all["rounds"], "range_finder_attempts": st_all["qb_attempts"],
                  "range_finder_uncertified": st_all["qb_uncertified"], "svd_calls": st_all["svd_calls"],
                  "svd_mean_p": st_all["svd_p_sum"] / max(st_all["svd_calls"], 1),
                  "svd_mean_sweeps": st_all["svd_sweeps_sum"] / max(st_all["svd_calls"], 1),
                  "window": "all steps of the timed solver (warm-up, timed, profile)"}
    total_ms = sum(step_ms)
    if world > 1:
        import torch.distributed as dist
        total_ms = max_over_ranks(total_ms)
        dist.barrier()

    # ---- end-to-end through the public API from pinned host buffers: the
    # same steps as the timed region (from the state after the warm-up), each
    # step's state copied in from and out to the host
    dev_in = [api.DevTT(n, n, cap) for _ in range(3)]
    h2d = d2h = 0
    torch.cuda.synchronize()
    e2e0 = time.perf_counter()
    for _ in range(args.steps):
        for (ha, hb), d, r in zip(host, dev_in, ranks_host):
            d.a[:r].copy_(ha[:r], non_blocking=True)
            d.b[:r].copy_(hb[:r], non_blocking=True)
            d.rank = r
            h2d += 8 * 2 * n * r
        s.set(dev_in)
        s.step(1)
        out = s.get()
        for (ha, hb), q in zip(host, out):
            ha[:q.rank].copy_(q.a[:q.rank], non_blocking=True)
            hb[:q.rank].copy_(q.b[:q.rank], non_blocking=True)
            d2h += 8 * 2 * n * q.rank
        torch.cuda.synchronize()
        ranks_host = [q.rank for q in out]
    e2e_s = time.perf_counter() - e2e0
    s.close()

    if rank != 0:
        return
    value = replica_value(n * n * args.steps, world, total_ms)
    # ---- roofline of the dominant kernel class (FP64 ALU bound)
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    achieved = d["flops"] / (d["ms"] / 1e3) / 1e12 if d["ms"] > 0 else 0.0
    hbm_peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm_peak = json.load(f).get("hbm_gbs")
    except (OSError, ValueError):
        pass
    tr = traffic_for(dom)
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": tr,
                "peak_source": "derived FP64: 152 SM x 2 FMA/clk x 2 flop x 2.070 GHz (no FP64 entry in "
                               "MEASURED_PEAKS.json)",
                "launches": d["launches"], "share": d["ms"] / max(sum(v["ms"] for v in prof.values()), 1e-9),
                "window": f"{prof_steps} further step(s), launches event-timed with the stage's tasks "
                          f"serialised"}
    classes = {k: {"ms": round(v["ms"], 3), "launches": v["launches"],
                   "tflops": (v["flops"] / (v["ms"] / 1e3) / 1e12 if v["ms"] > 0 else 0.0),
                   "gbs": (v["bytes"] / (v["ms"] / 1e3) / 1e9 if v["ms"] > 0 else 0.0)}
               for k, v in prof.items() if v["launches"]}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.precision], "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "scheme": w["scheme"], "eqn": w["eqn"],
                       "precision": args.precision, "pivots": args.pivots,
                       "rank_cap": cap, "tol": w["tol"], "steps_timed": f"{args.warmup + 1}..{args.warmup + args.steps}",
                       "l2": "flushed (256 MiB write) before every timed step", "parallelism": "replicas"},
            "clocks": clk, "gpu_launches": launches, "roofline": roofline, "kernel_classes": classes,
            "ranks_after": ranks_after, "device_status": dev_status, "cross": cross_info,
            "section_host_ms_per_step": sections, "wall_s_timed": wall,
            "e2e": {"value": n * n * args.steps * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d // args.steps,
                    "d2h_bytes_per_step": d2h // args.steps}}
    # ---- CPU oracle baseline and the parity of the first step
    if not args.no_cpu_baseline and world == 1:
        from oracle import tt as T
        cb, Qo = cpu_baseline(w, p, Q, args.cpu_sample_steps)
        line["cpu_baseline"] = cb
        if args.cpu_sample_steps == 1:
            scale = np.linalg.norm(T.full(Qo[0]))
            line["l2_err_vs_oracle"] = {
                "fields": [float(np.linalg.norm(first[c].full().numpy() - T.full(Qo[c])) / scale)
                           for c in range(3)],
                "note": "first step from the initial state, relative to ||h||; bar 10 x tol"}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- batched form
def run_ensemble(args):
    """The batched form: `ensembleK` = K seeded instances of uneven grid size,
    rank cap and reconstruction advanced together (tt_fv_batch_*).  The
    warm-up steps run the autotuner; one step = one SSP-RK3 step of every
    instance; value = sum of n^2 over instances x steps / device time."""
    import torch
    from synth import ensemble, initial_tt
    from paper_2408_03483_gb300 import api, capi

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    capi.load()
    count = int(args.workload[len("ensemble"):] or 256)
    ws = ensemble(count=count)
    insts = []
    for w in ws:
        Q, p = initial_tt(w)
        q0 = [api.DevTT.from_cores(A, B, cap=w["cap"]) for A, B in Q]
        insts.append((q0, dict(eqn=w["eqn"], scheme=w["scheme"], n=w["n"], dt=p["dt"], tol=w["tol"],
                               rank_cap=w["cap"], g=p["g"], H=p["H"], f=p["f"], seed=0)))
    cells = sum(w["n"] ** 2 for w in ws)
    prec = args.precision
    b = api.Batch(insts, precision=prec, workers=8)
    stream = torch.cuda.current_stream()
    # warm-up = the autotuner's trials: one step per (workers, inner tasks)
    # candidate; workers = 1 with inner tasks is the plain one-instance path
    cands = (1, 8, 16)
    (bw, bi), rates = b.tune(workers=cands, steps_per_trial=1, with_rates=True)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = api.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    launches = api.launch_count() - launches0
    clk = clocks.stop()
    total_ms = ms
    if world > 1:
        import torch.distributed as dist
        total_ms = max_over_ranks(total_ms)
    dev = max(b.stats(i)["device_status"] for i in range(count))
    b.close()
    # the plain path on the same steps: one instance at a time with its own
    # stage tasks, advanced through the same warm-up steps first
    plain_ms = None
    if args.compare_plain:
        insts2 = []
        for w in ws:
            Q, p = initial_tt(w)
            q0 = [api.DevTT.from_cores(A, B, cap=w["cap"]) for A, B in Q]
            insts2.append((q0, dict(eqn=w["eqn"], scheme=w["scheme"], n=w["n"], dt=p["dt"], tol=w["tol"],
                                    rank_cap=w["cap"], g=p["g"], H=p["H"], f=p["f"], seed=0)))
        b2 = api.Batch(insts2, precision=prec, workers=1, inner_tasks=True)
        b2.step(2 * len(cands))
        torch.cuda.synchronize()
        e0.record(stream)
        b2.step(args.steps)
        e1.record(stream)
        e1.synchronize()
        plain_ms = e0.elapsed_time(e1)
        b2.close()
    if rank != 0:
        return
    value = replica_value(cells * args.steps, world, total_ms)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": 2 * len(cands), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[prec], "data": "synthetic",
            "config": {"workload": args.workload, "instances": count, "cells": cells, "precision": prec,
                       "schemes": {s: sum(w["scheme"] == s for w in ws) for s in ("up3", "up5", "weno5")},
                       "sizes": sorted({w["n"] for w in ws}), "caps": [min(w["cap"] for w in ws),
                                                                       max(w["cap"] for w in ws)],
                       "l2": "inputs of each step are the previous step's outputs (no flush)",
                       "parallelism": "replicas"},
            "tuned": {"workers": bw, "inner_tasks": bi,
                      "trial_rates": {f"w{w}_{'inner' if i else 'flat'}": r for (w, i), r in rates.items()}},
            "plain_same_steps": ({"ms_per_step": plain_ms / args.steps, "speedup": plain_ms / total_ms,
                                  "what": "workers=1 with stage tasks (the single-instance path), same steps"}
                                 if plain_ms else None),
            "clocks": clk, "gpu_launches": launches, "device_status": dev}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload.startswith("ensemble"):
        run_ensemble(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
