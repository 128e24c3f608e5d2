"""Benchmark of the TT finite-volume shallow-water stage on GB300.

One step = one full SSP-RK3 step (three stages: WENO5 reconstruction by
cross, Taylor reciprocal, LLF fluxes from Hadamard products, rounding)
through the C ABI of libttfv.so.  The headline workload is the nonlinear
4096 x 4096 WENO5 case (3 seeded Gaussian bumps, rank cap 64, tol 1e-8); the
256 x 256 case (rank cap 32) is timed on the same steps in the same run and
reported under "secondary".  Metric: equivalent cell updates per second,
N^2 x steps / s (summed over ranks), with each field's relative L2 error
against the FP64 oracle.

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
WORKLOAD = "nonlinear4096_weno5"
SECONDARY = "nonlinear256_weno5"
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
    ap.add_argument("--flux", default="products", choices=["products", "cross"],
                    help="nonlinear flux: Taylor 1/h and Hadamard products, or the LF-cross (one cross per direction)")
    ap.add_argument("--compare-plain", action="store_true",
                    help="ensemble workloads: also time the one-instance-at-a-time path on the same steps")
    ap.add_argument("--secondary", default=SECONDARY,
                    help="a second workload timed in the same run, reported under 'secondary' ('' for none)")
    ap.add_argument("--tol", type=float, default=None,
                    help="truncation tolerance instead of the workload's (same-error comparisons of the forms)")
    ap.add_argument("--tile-shape", type=int, default=0,
                    help="TSQR tile shape of the roundings (an index of api.tile_shapes(); 0 the default)")
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
def make_state(w):
    from synth import initial_tt
    return initial_tt(w)


def traffic_for(kernel_class, workload):
    """Per-launch DRAM bytes of the dominant kernel class from the committed
    ncu summary, if it was taken on this workload and on the current source
    of that kernel."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    try:
        with open(path) as f:
            tab = json.load(f)
    except (OSError, ValueError):
        return None
    ent = tab.get(f"{workload}:{kernel_class}")
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


def per_field_rel(got, ref):
    """Relative L2 error of each field against the reference's own norm."""
    import numpy as np
    out = []
    for a, b in zip(got, ref):
        nb = float(np.linalg.norm(b))
        e = float(np.linalg.norm(a - b))
        out.append(e / nb if nb > 0 else e)
    return out


def oracle_b_sample(Q, w, p, nsteps):
    """Oracle B (numpy TT algorithm) timed on the host cores for `nsteps` RK
    steps from the TT state Q."""
    from oracle import tt_fv as TB
    t0 = time.perf_counter()
    Qo = Q
    for _ in range(nsteps):
        Qo = TB.step(Qo, w, p, seed=0)
    return time.perf_counter() - t0, Qo


def oracle_a_patches(start, after, w, p, npatch=12, size=48, halo=12, seed=3):
    """Per-field relative L2 error of a TT state `after` (one SSP-RK3 step
    from the TT state `start`) against Oracle A's exact full-tensor step,
    sampled on `npatch` seeded size x size patches.  One step reads cells at
    most 9 away (3 stages, each reading 3 cells on either side), so Oracle A
    run on a patch with a halo of 12 cells, periodically wrapped, is exact in
    the patch interior."""
    import numpy as np
    from oracle import fv_full as FA
    rng = np.random.default_rng(seed)
    n = w["n"]
    m = size + 2 * halo
    pp = dict(p, lx=m / n, ly=m / n)
    num = np.zeros(3)
    den = np.zeros(3)
    for _ in range(npatch):
        i0, j0 = (int(v) for v in rng.integers(0, n, size=2))
        rows = (i0 - halo + np.arange(m)) % n
        cols = (j0 - halo + np.arange(m)) % n
        P = [A[rows] @ B[cols].T for A, B in start]
        R = FA.ssprk3_step(P, w["eqn"], w["scheme"], pp, p["dt"])
        for c in range(3):
            A, B = after[c]
            G = A[rows[halo:-halo]] @ B[cols[halo:-halo]].T
            ref = R[c][halo:-halo, halo:-halo]
            num[c] += float(np.sum((G - ref) ** 2))
            den[c] += float(np.sum(ref ** 2))
    return [float(np.sqrt(num[c] / den[c])) if den[c] > 0 else float(np.sqrt(num[c])) for c in range(3)]


def host_tt(q):
    """(A, B) float64 numpy cores of a device TT."""
    r = q.rank
    return (q.a[:r].T.cpu().numpy().copy(), q.b[:r].T.cpu().numpy().copy())


# ---------------------------------------------------------------- reference arm
def reference_sample(Q, w, p, stage_seed=0):
    """One stage (the forward-Euler stage of Eq. tt-ssprk3) of Oracle B from the
    TT state Q: the reference arm's timing sample."""
    from oracle import tt_fv as TB
    t0 = time.perf_counter()
    TB.stage(Q, Q, 0, w, p, seed=stage_seed)
    return time.perf_counter() - t0


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from synth import workload
    from oracle import tt_fv as TB
    w = workload(args.workload)
    if args.tol is not None:
        w["tol"] = args.tol
    Q, p = make_state(w)
    n = w["n"]
    # warm-up: W full steps from the initial state (the state the timed window
    # of the GPU arm starts from)
    for _ in range(args.warmup):
        Q = TB.step(Q, w, p, seed=0)
    times = [reference_sample(Q, w, p) for _ in range(args.steps)]
    stage_s = sum(times) / len(times)
    # a step is three stages of about equal cost
    value = n * n / (3.0 * stage_s)
    cores = os.cpu_count()
    sample = (f"first stage of SSP-RK3 step {args.warmup + 1} (from the state after {args.warmup} full steps), "
              f"repeated {args.steps} times; a step counted as 3 stages; numpy/OpenBLAS float64")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 3e3 * stage_s,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "scheme": w["scheme"], "eqn": w["eqn"],
                       "rank_cap": w["cap"], "tol": w["tol"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def measure(args, wname, world, local, with_cpu, with_l2):
    """Times K SSP-RK3 steps of workload `wname` after W warm-up steps and
    returns the JSON fields of its line (plus host states for the parity
    checks)."""
    import numpy as np
    import torch
    from synth import workload
    from paper_2408_03483_gb300 import api

    w = workload(wname)
    if args.tol is not None:
        w["tol"] = args.tol
    n, cap = w["n"], w["cap"]
    Q, p = make_state(w)
    stream = torch.cuda.current_stream()
    net = api.PivotNet.shipped() if args.pivots == "learned" else None

    def new_solver(state):
        q0 = [api.DevTT.from_cores(A, B, cap=cap) for A, B in state]
        s = api.Solver(q0, w["eqn"], w["scheme"], n, p["dt"], w["tol"], cap, g=p["g"], H=p["H"], f=p["f"],
                       kick=4, max_sweeps=10, max_iter=50, seed=0, precision=args.precision, pivots=args.pivots,
                       flux=args.flux)
        if args.pivots == "learned":
            s.set_pivot_net(net)
        if args.tile_shape:
            s.set_tile_shape(args.tile_shape)
        return s

    # ---- device-timed region
    s = new_solver(Q)
    for _ in range(args.warmup):
        s.step(1)
    # the state the timed steps start from (the end-to-end run and the CPU
    # baseline repeat steps from it)
    host = [(torch.empty((cap, n), dtype=torch.float64).pin_memory(),
             torch.empty((cap, n), dtype=torch.float64).pin_memory()) for _ in range(3)]
    st = s.get()
    for (ha, hb), q in zip(host, st):
        ha[:q.rank].copy_(q.a[:q.rank].cpu())
        hb[:q.rank].copy_(q.b[:q.rank].cpu())
    ranks_start = [q.rank for q in st]
    start_cores = [host_tt(q) for q in st]
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
    end_state = s.get()
    ranks_end = [q.rank for q in end_state]
    end_full = [q.full().numpy() for q in end_state] if n <= 1024 else None
    # ---- per-kernel profile: further steps with every launch event-timed on
    # its stream and the stage's tasks serialised (each time is the kernel's
    # own, not shared with concurrent kernels)
    prof_steps = max(1, min(args.steps, 2))
    s.profile(True)
    s.kernel_profile(reset=True)
    for _ in range(prof_steps):
        s.step(1)
    prof = s.kernel_profile(reset=True)
    s.profile(False)
    st_all = s.stats()
    sections = {name: round((b - a) / args.steps, 2) for name, a, b in
                zip(("faces", "side_fluxes_and_lambda", "llf", "quadrature_difference", "forward_euler",
                     "ssp_combination"), sec0, sec1)}
    cross_info = {"calls": st_all["cross_calls"], "sweeps": st_all["cross_sweeps"],
                  "sweeps_per_call": st_all["cross_sweeps"] / max(st_all["cross_calls"], 1),
                  "learned_calls": st_all["learned_calls"], "learned_accepted": st_all["learned_accepted"],
                  "roundings": st_all["rounds"], "range_finder_attempts": st_all["qb_attempts"],
                  "range_finder_uncertified": st_all["qb_uncertified"], "svd_calls": st_all["svd_calls"],
                  "svd_mean_p": st_all["svd_p_sum"] / max(st_all["svd_calls"], 1),
                  "svd_mean_deflated_p": st_all["svd_pd_sum"] / max(st_all["svd_calls"], 1),
                  "svd_mean_sweeps": st_all["svd_sweeps_sum"] / max(st_all["svd_calls"], 1),
                  "window": "all steps of the timed solver (warm-up, timed, profile)"}
    total_ms = sum(step_ms)
    if world > 1:
        total_ms = max_over_ranks(total_ms)
        import torch.distributed as dist
        dist.barrier()

    # ---- end-to-end through the public API from pinned host buffers: the
    # same steps as the timed region (from the state after the warm-up), each
    # step's state copied in from and out to the host
    dev_in = [api.DevTT(n, n, cap) for _ in range(3)]
    h2d = d2h = 0
    ranks_host = list(ranks_start)
    first_after = None
    torch.cuda.synchronize()
    e2e0 = time.perf_counter()
    for k in range(args.steps):
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
        if k == 0:
            first_after = [(ha[:r].T.numpy().copy(), hb[:r].T.numpy().copy()) for (ha, hb), r in
                           zip(host, ranks_host)]
    e2e_s = time.perf_counter() - e2e0
    s.close()

    # ---- roofline of the dominant kernel class (FP64 ALU bound)
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    achieved = d["flops"] / (d["ms"] / 1e3) / 1e12 if d["ms"] > 0 else 0.0
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": traffic_for(dom, wname),
                "peak_source": "derived FP64: 152 SM x 2 FMA/clk x 2 flop x 2.070 GHz (no FP64 entry in "
                               "MEASURED_PEAKS.json)",
                "launches": d["launches"], "ms_per_launch": d["ms"] / max(d["launches"], 1),
                "flops_per_launch": d["flops"] / max(d["launches"], 1),
                "share": d["ms"] / max(sum(v["ms"] for v in prof.values()), 1e-9),
                "window": f"{prof_steps} further step(s), every launch event-timed on its stream with the "
                          f"stage's tasks serialised"}
    classes = {k: {"ms": round(v["ms"], 3), "launches": v["launches"],
                   "share": round(v["ms"] / max(sum(x["ms"] for x in prof.values()), 1e-9), 4),
                   "tflops": (v["flops"] / (v["ms"] / 1e3) / 1e12 if v["ms"] > 0 else 0.0),
                   "gbs": (v["bytes"] / (v["ms"] / 1e3) / 1e9 if v["ms"] > 0 else 0.0)}
               for k, v in prof.items() if v["launches"]}
    value = replica_value(n * n * args.steps, world, total_ms)
    res = {"value": value, "ms_per_step": total_ms / args.steps,
           "config": {"workload": wname, "n": n, "scheme": w["scheme"], "eqn": w["eqn"],
                      "precision": args.precision, "pivots": args.pivots, "flux": args.flux, "rank_cap": cap,
                      "tol": w["tol"], "tile_shape": args.tile_shape,
                      "steps_timed": f"{args.warmup + 1}..{args.warmup + args.steps}",
                      "l2": "flushed (256 MiB write) before every timed step", "parallelism": "replicas"},
           "step_ms": [round(x, 2) for x in step_ms],
           "clocks": clk, "gpu_launches": launches, "roofline": roofline, "kernel_classes": classes,
           "ranks_start": ranks_start, "ranks_end": ranks_end, "device_status": st_all["device_status"],
           "cross": cross_info, "section_host_ms_per_step": sections, "wall_s_timed": wall,
           "e2e": {"value": n * n * args.steps * world / e2e_s, "unit": UNIT,
                   "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps}}
    if not with_l2:
        return res
    # ---- parity of the timed steps against the oracle
    if n <= 1024:
        # the state at the end of the timed window against Oracle A's exact
        # full-tensor run of the same W + K steps from the initial state
        from oracle import fv_c as FC
        from oracle import tt as T
        Qa = FC.ssprk3_steps([T.full(q) for q in Q], w["eqn"], w["scheme"], p, p["dt"], args.warmup + args.steps)
        res["l2_err_vs_oracle"] = {
            "fields": per_field_rel(end_full, Qa),
            "what": f"per-field relative L2 (own norm) of the state after step {args.warmup + args.steps} "
                    f"against Oracle A (full-tensor FP64 finite volume in C, no truncation) advanced the same steps "
                    f"from the same initial cell averages; bar per step 30 tol of each field's truncation scale"}
    else:
        res["l2_err_vs_oracle"] = {
            "fields": oracle_a_patches(start_cores, first_after, w, p),
            "what": f"per-field relative L2 (own norm) of the first timed step (step {args.warmup + 1}, from the "
                    f"state after the warm-up) against Oracle A's exact full-tensor step from the same state, on "
                    f"12 seeded 48x48 patches (halo 12 > the 9-cell reach of one step)"}
    if not with_cpu:
        return res
    # ---- CPU oracle baseline: Oracle B on the first timed step
    nb = max(1, args.cpu_sample_steps)
    dt_cpu, _ = oracle_b_sample(start_cores, w, p, nb)
    cores = os.cpu_count()
    res["cpu_baseline"] = {"value": n * n * nb / dt_cpu, "unit": UNIT, "cores": cores, "kind": "oracle",
                           "sample": f"Oracle B (numpy TT algorithm, float64, {cores} host threads) on SSP-RK3 "
                                     f"step(s) {args.warmup + 1}..{args.warmup + nb} of the {n}x{n} "
                                     f"{w['scheme']} workload, from the GPU's state at the start of the timed "
                                     f"window (the first timed step(s))",
                           "seconds": dt_cpu}
    return res


def run_ours(args):
    import torch
    from paper_2408_03483_gb300 import capi

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    capi.load()
    with_cpu = not args.no_cpu_baseline and world == 1 and rank == 0
    with_l2 = world == 1 and rank == 0
    main = measure(args, args.workload, world, local, with_cpu, with_l2)
    second = None
    if args.secondary and args.secondary != args.workload:
        second = measure(args, args.secondary, world, local, with_cpu, with_l2)
    if rank != 0:
        return
    line = {"metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.precision], "data": "synthetic"}
    line.update({k: v for k, v in main.items() if k not in ("value", "ms_per_step")})
    if second is not None:
        line["secondary"] = dict(second, steps=args.steps, warmup=args.warmup)
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- batched form
def ensemble_cells(cells_mine):
    """Cells of the whole ensemble: the sum of every rank's own members (each
    member is on exactly one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return int(cells_mine)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(cells_mine)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(round(float(t.item())))


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
    ws_all = ensemble(count=count)
    # this rank's shard of the members (longest processing time first on
    # N cap^2); the members are independent, so nothing is exchanged
    from paper_2408_03483_gb300 import shard
    costs = [shard.member_cost(w["n"], w["cap"]) for w in ws_all]
    mine = shard.partition(costs, world)[rank]
    ws = [ws_all[i] for i in mine]
    insts = []
    for w in ws:
        Q, p = initial_tt(w)
        q0 = [api.DevTT.from_cores(A, B, cap=w["cap"]) for A, B in Q]
        insts.append((q0, dict(eqn=w["eqn"], scheme=w["scheme"], n=w["n"], dt=p["dt"], tol=w["tol"],
                               rank_cap=w["cap"], g=p["g"], H=p["H"], f=p["f"], seed=0)))
    cells_mine = sum(w["n"] ** 2 for w in ws)
    cells = ensemble_cells(cells_mine)
    prec = args.precision
    b = api.Batch(insts, precision=prec, workers=8)
    stream = torch.cuda.current_stream()
    # warm-up = the autotuner's trials: one step per (workers, inner tasks)
    # candidate; workers = 1 with inner tasks is the plain one-instance path
    cands = (1, 8, 16)
    (bw, bi), rates = b.tune(workers=cands, steps_per_trial=1, with_rates=True)
    # then each member's TSQR tile shape (leaf rows, merge fan-in), one step
    # per shape with the chosen concurrency
    tile_of, tile_rates = b.tune_tiles(steps_per_trial=1, rounds=1)
    shapes = api.tile_shapes()
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
    dev = max(b.stats(i)["device_status"] for i in range(len(ws)))
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
        b2.step(2 * len(cands) + len(shapes))
        torch.cuda.synchronize()
        e0.record(stream)
        b2.step(args.steps)
        e1.record(stream)
        e1.synchronize()
        plain_ms = e0.elapsed_time(e1)
        b2.close()
    if rank != 0:
        return
    # the whole ensemble's cells (each member on one rank) over the slowest
    # rank's time: the job's throughput, counting every member once
    value = cells * args.steps / (total_ms / 1e3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": 2 * len(cands) + len(shapes), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": DTYPES[prec], "data": "synthetic",
            "config": {"workload": args.workload, "instances": count, "cells": cells, "precision": prec,
                       "schemes": {s: sum(w["scheme"] == s for w in ws_all) for s in ("up3", "up5", "weno5")},
                       "sizes": sorted({w["n"] for w in ws_all}), "caps": [min(w["cap"] for w in ws_all),
                                                                           max(w["cap"] for w in ws_all)],
                       "l2": "inputs of each step are the previous step's outputs (no flush)",
                       "parallelism": f"ensemble sharded over {world} GPU(s) (LPT on N cap^2), no exchange",
                       "rank0_members": len(ws)},
            "tuned": {"workers": bw, "inner_tasks": bi,
                      "trial_rates": {f"w{w}_{'inner' if i else 'flat'}": r for (w, i), r in rates.items()},
                      "tile_shapes": {f"leaf{lm}_fanin{fi or 'default'}": {"members": tile_of.count(k),
                                                                            "trial_rate": tile_rates[k]}
                                      for k, (lm, fi) in enumerate(shapes)}},
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
