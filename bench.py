"""Benchmark: half-space Spectral Ewald evaluation on GB300 (arXiv 1802.07844).

One step = one full evaluation through the C ABI (hse_eval): input check,
cell-list binning and sort, real-space sum, spreading, forward FFTs, k-space
scaling, inverse FFTs and gather, for the workload
  stokeslet + rotlet, N = 1M sources = targets, x, y uniform in [0,1),
  z ~ Exponential(mean 0.05) truncated to (0,1], N(0,1) forces and torques,
  FP64 path at relative RMS tolerance 1e-10 (plan set-up is not timed, Sec. 7).

Prints one JSON line.  ``value`` is whole-job Mtargets/s with inputs resident
on the device; ``e2e`` repeats the measurement with host inputs copied in and
velocities copied out inside the timed region.  ``--impl reference`` times the
FP64 CPU direct-sum oracle on a bounded target sample of the same workload.
Multi-GPU: independent replicas (one per rank), weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import KERNEL_S, KERNEL_W, problem  # noqa: E402

WORKLOAD = dict(
    name="hs_stokeslet_rotlet_n1m_nearwall",
    mask=KERNEL_S | KERNEL_W, n=1_000_000, dist="near_wall", index=2, tol=1e-10,
    # parameters checked against the FP64 oracle on a target sample (tests/test_gpu_parity.py):
    # xi r_c = 4.8, k_inf / xi = pi M / xi = 10.9, P = 18 give 3.0e-11 on 3000 targets (P = 16:
    # 3.2e-10; xi = 90 with the same grid: 7.3e-11); Mt = 320 = 2^6 x 5 is a fast cuFFT size
    xi=87.0, rc=0.0552, P=18, M=302,
)
# mixed-precision (FP32 arithmetic) configuration of the same workload at tolerance 1e-5;
# parameters checked against the FP64 oracle on a target sample (tests/test_gpu_parity.py):
# 2.9e-6 on 3000 targets (the plan's own rule at xi = 100 picks r_c 0.0367, P 14, M 306:
# 4.4e-7 at 1.5x the time); Mt = 256 is a power of two, markedly faster in FP32 cuFFT
MIXED = dict(tol=1e-5, xi=95.0, rc=0.035, P=12, M=244)
METRIC = "Mtargets/s, N=1M stokeslet @1e-10 FP64 vs 1e-5 mixed; serve p50/p99 ms"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 peak from unit counts and clock: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP32 peak likewise: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# Algorithmic FP64 work of the real-space stage (stokeslet + rotlet), counted
# from the written code (FMA = 2 flops): the radial part of a pair (distance,
# reciprocal square root charged 4, exp by reduction + degree-13 polynomial,
# erfcx by a degree-10 polynomial, the coefficients a1, g2) costs 82 flops and is
# evaluated once per unordered pair; each direction then adds its contribution,
# 37 flops for a free pair and 92 for an image pair with its wall corrections.
# Pairs in the outer shell [rc64, rc) run the same formulas in FP32; they are
# charged the same flops against the FP32 peak.
# DRAM bytes of one k_real_sym<double, 5> launch per point, measured with ncu
# (dram__bytes_read.sum + dram__bytes_write.sum = 16.1 MB + 0 at N = 100k of
# this workload); the kernel reads positions, strengths and cell lists about
# once, so the figure is scaled by the number of points.
REAL_TRAFFIC_BYTES_PER_POINT = 161.0
FLOPS_RADIAL = 82
FLOPS_FREE_DIR = 37
FLOPS_IMAGE_DIR = 92


def max_over_ranks(value: float, world: int, device) -> float:
    """Largest value over the ranks (the slowest replica sets the job time)."""
    if world <= 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_problem(rank: int, n: int):
    """The bench workload's inputs for one replica: same recipe, own seed."""
    return problem(WORKLOAD["mask"], n, 1.0, WORKLOAD["dist"], WORKLOAD["index"], sub=rank)


def whole_job_rate(points_per_rank: int, world: int, ms_max: float) -> float:
    """Mtargets/s of the whole job: every rank's points over the slowest rank's time."""
    return points_per_rank * world / (ms_max / 1e3) / 1e6


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

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
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "samples": len(sm),
                "power_w_max": float(max(power)) if power else None, "reasons": sorted(reasons)}


# ----------------------------------------------------------- CPU oracle
def time_oracle(pr, mask, budget_s: float, start_targets: int = 16):
    """Times the FP64 direct-sum oracle on a growing seeded sample of targets
    until about ``budget_s`` seconds of work; returns (targets/s, sample, cores)."""
    import oracle
    n = pr.src.shape[1]
    rng = np.random.default_rng(1802078440 + 99)
    k = start_targets
    t_used = 0.0
    while True:
        idx = np.sort(rng.choice(n, size=min(k, n), replace=False))
        t0 = time.perf_counter()
        oracle.direct(mask, pr.src, pr.strengths, pr.src[:, idx])
        dt = time.perf_counter() - t0
        t_used += dt
        if dt > 0.25 * budget_s or k >= n or t_used > budget_s:
            return len(idx) / dt, len(idx), dt
        k = int(min(n, max(2 * k, k * 0.5 * budget_s / max(dt, 1e-3))))


# ------------------------------------------------------------ main arm
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1802_07844_gb300 as pkg
    from paper_1802_07844_gb300 import build
    build.build_library()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    W = dict(WORKLOAD)
    if args.n:
        W["n"] = args.n
    mask = W["mask"]
    pr = replica_problem(rank, W["n"])
    if args.real_only:
        return run_real_only(args, pkg, torch, dev, W, pr)
    if args.fourier_small:
        return run_fourier_small(args, pkg, torch, dev, W)
    plan = pkg.Plan(mask, (1.0, 1.0, 1.0), xi=W["xi"], rc=W["rc"], P=W["P"], tol=0.0, M=W["M"])
    plan.set_timing(True)
    prm = plan.params
    src = torch.from_numpy(pr.src).to(dev)
    st = torch.from_numpy(pr.strengths).to(dev)
    vel = torch.empty((3, W["n"]), dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=dev)  # 512 MB > L2
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.eval(src, st, out=vel)
    torch.cuda.synchronize()
    # exact pair counts of the real-space stage (untimed); a target's own image
    # counts once, every other pair is shared by its two targets
    a, b = plan.neighbor_counts(src)
    n_free, n_img = int(a.sum().item()), int(b.sum().item())
    z = pr.src[2]
    n_own = int(np.sum((z + z) * (z + z) < W["rc"] * W["rc"]))
    # the same counts within rc64 (pairs evaluated in FP64), from a count-only plan
    rc64 = prm["rc64"]
    cplan = pkg.Plan(mask, (1.0, 1.0, 1.0), xi=W["xi"], rc=rc64, P=W["P"], tol=0.0)
    a64, b64 = cplan.neighbor_counts(src)
    n_free64, n_img64 = int(a64.sum().item()), int(b64.sum().item())
    n_own64 = int(np.sum((z + z) * (z + z) < rc64 * rc64))
    cplan.close()
    del a, b, a64, b64

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    stages = {k: [] for k in pkg.hse.STAGE_NAMES}
    launches = 0
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        plan.eval(src, st, out=vel)
        ev[i][1].record(stream)
        s = plan.stats()
        launches += s["n_kernel_launches"]
        overlapped = s["overlapped"]
        for k, v in s["stage_ms"].items():
            stages[k].append(v)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    total_ms = sum(e0.elapsed_time(e1) for e0, e1 in ev)
    ms_step = total_ms / args.steps
    ms_step_max = max_over_ranks(ms_step, world, dev)
    value = whole_job_rate(W["n"], world, ms_step_max)

    # end-to-end: pinned host inputs in, velocities out, inside the timed region
    h_src = torch.from_numpy(pr.src).pin_memory()
    h_st = torch.from_numpy(pr.strengths).pin_memory()
    h_vel = torch.empty((3, W["n"]), dtype=torch.float64).pin_memory()
    d_src = torch.empty_like(src)
    d_st = torch.empty_like(st)
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e_ms = 0.0
    for _ in range(e2e_steps):
        flush.zero_()
        e0.record(stream)
        d_src.copy_(h_src, non_blocking=True)
        d_st.copy_(h_st, non_blocking=True)
        plan.eval(d_src, d_st, out=vel)
        h_vel.copy_(vel, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e_ms += e0.elapsed_time(e1)
    e_ms /= e2e_steps
    e2e_value = whole_job_rate(W["n"], world, max_over_ranks(e_ms, world, dev))
    h2d = h_src.numel() * 8 + h_st.numel() * 8
    d2h = h_vel.numel() * 8

    # roofline of the dominant kernel of this library
    avg = {k: float(np.mean(v)) if v else 0.0 for k, v in stages.items()}
    own = {k: avg[k] for k in ("real", "spread", "scale", "gather")}
    dom = max(own, key=own.get)
    P, Mt, nc = prm["P"], prm["Mt"], prm["n_fft_in"]
    peaks = json.load(open(PEAKS_PATH)) if os.path.exists(PEAKS_PATH) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    if dom == "real":
        def flops(nf, ni, no):
            return ((nf // 2) * (FLOPS_RADIAL + 2 * FLOPS_FREE_DIR)
                    + ((ni - no) // 2) * (FLOPS_RADIAL + 2 * FLOPS_IMAGE_DIR) + no * (FLOPS_RADIAL + FLOPS_IMAGE_DIR))
        w64 = flops(n_free64, n_img64, n_own64)
        w32 = flops(n_free, n_img, n_own) - w64
        # FP64-equivalent rate: the FP32 shell flops weighted by the pipe ratio,
        # so achieved / peak = (ideal time on both pipes) / measured time
        work = w64 + w32 * FP64_PEAK_TFLOPS / FP32_PEAK_TFLOPS
        roof = {"kernel": "k_real_sym", "bound": "alu", "unit": "TFLOP/s", "peak": FP64_PEAK_TFLOPS,
                "peak_source": "FP64 units x clock (152 SMs x 2 FMA/clk x 2.07 GHz); FP32 shell flops "
                               "charged at FP64/FP32 = 1/64 (128 FP32 lanes/SM)",
                "achieved": work / (avg["real"] / 1e3) / 1e12,
                "work": {"free_pairs_ordered": n_free, "image_pairs_ordered": n_img, "own_images": n_own,
                         "fp64_free_pairs_ordered": n_free64, "fp64_image_pairs_ordered": n_img64,
                         "rc64": rc64, "flops_fp64": w64, "flops_fp32_shell": w32,
                         "flops_radial": FLOPS_RADIAL, "flops_free_direction": FLOPS_FREE_DIR,
                         "flops_image_direction": FLOPS_IMAGE_DIR}}
    elif dom in ("spread", "gather"):
        per = P ** 3 * (2 * nc + 2) if dom == "spread" else P ** 3 * 12
        work = W["n"] * per
        roof = {"kernel": "k_" + dom, "bound": "alu", "unit": "TFLOP/s", "peak": FP64_PEAK_TFLOPS,
                "peak_source": "FP64 units x clock", "achieved": work / (avg[dom] / 1e3) / 1e12}
    else:
        nh = (2 * Mt) * (2 * Mt) * (2 * Mt + 1)
        byts = (nc + 6) * nh * 16 + nh * 8 * 2
        roof = {"kernel": "k_scale", "bound": "hbm", "unit": "GB/s", "peak": hbm_peak,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs", "achieved": byts / (avg["scale"] / 1e3) / 1e9}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = REAL_TRAFFIC_BYTES_PER_POINT * W["n"] if dom == "real" else None
    if dom == "real":
        roof["traffic_source"] = "ncu dram bytes of one launch at N = 100k, scaled by points"
    roof["stage_ms"] = {k: round(v, 3) for k, v in avg.items()}
    if overlapped:
        roof["stage_ms_note"] = ("device time of each stage on its own stream: the real-space stage runs "
                                 "concurrently with spread..gather, so the stages overlap and their sum "
                                 "exceeds ms_per_step")

    out = {
        "metric": METRIC, "value": value, "unit": "Mtargets/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": W["name"], "n_sources": W["n"], "n_targets": W["n"], "kernels": "stokeslet+rotlet",
                   "distribution": "x,y ~ U[0,1), z ~ TruncExp(0.05) on (0,1]", "tol": W["tol"],
                   "precision": "fp64", "xi": prm["xi"], "rc": prm["rc"], "P": P, "M": prm["M"], "Mt": Mt,
                   "fft_in": nc, "fft_out": prm["n_fft_out"], "parallelism": f"replicas x{world}",
                   "l2": "512 MB buffer written between timed steps"},
        "e2e": {"value": e2e_value, "unit": "Mtargets/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "roofline": roof,
        "gpu_launches": launches,
        "clocks": clk,
    }
    if not args.no_mixed:
        out["mixed_1e-5"] = run_mixed(args, pkg, torch, dev, pr, src, st, vel, flush, stream, world)
    if args.serve_requests > 0:
        del flush
        plan.close()
        torch.cuda.empty_cache()
        out["serve"] = run_serve(args, pkg, torch, dev)
    if args.batch_instances > 0:
        torch.cuda.empty_cache()
        out["batch"] = run_batch(args, pkg, torch, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        tps, k, dt = time_oracle(pr, mask, args.cpu_budget)
        out["cpu_baseline"] = {"value": tps / 1e6, "unit": "Mtargets/s", "cores": os.cpu_count(), "kind": "oracle",
                               "sample": f"{k} seeded targets of the same workload against all {W['n']} sources "
                                         f"(FP64 direct half-space sum, OpenMP), {dt:.1f} s"}
    plan.close()
    return out


def run_mixed(args, pkg, torch, dev, pr, src, st, vel, flush, stream, world):
    """The same workload through the FP32-arithmetic path at tolerance 1e-5."""
    Mx = MIXED
    plan = pkg.Plan(WORKLOAD["mask"], (1.0, 1.0, 1.0), xi=Mx["xi"], rc=Mx["rc"], P=Mx["P"], tol=0.0, M=Mx["M"],
                    precision=pkg.HSE_MIXED)
    plan.set_timing(True)
    for _ in range(args.warmup):
        plan.eval(src, st, out=vel)
    torch.cuda.synchronize()
    stages = {k: [] for k in pkg.hse.STAGE_NAMES}
    ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.eval(src, st, out=vel)
        e1.record(stream)
        s = plan.stats()
        for k, v in s["stage_ms"].items():
            stages[k].append(v)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
    ms /= args.steps
    ms_max = max_over_ranks(ms, world, dev)
    prm = plan.params
    plan.close()
    n = src.shape[1]
    return {"value": whole_job_rate(n, world, ms_max), "unit": "Mtargets/s", "ms_per_step": ms_max,
            "dtype": "f32 arithmetic (FP64 sums, close image pairs, tables)", "tol": Mx["tol"], "xi": prm["xi"],
            "rc": prm["rc"], "P": prm["P"], "M": prm["M"], "Mt": prm["Mt"],
            "stage_ms": {k: round(float(np.mean(v)), 3) for k, v in stages.items()}}


def run_serve(args, pkg, torch, dev):
    """Poisson stream of requests through the continuous-batching server:
    kernel uniform over stokeslet/stresslet/rotlet, N log-uniform in [1e3, 2e5],
    half uniform and half near-wall (TruncExp 0.05), tol 1e-10 (FP64) or 1e-5
    (mixed) per request.  The offered load is 0.7 x the service capacity
    measured on a closed-loop warm-up of the same request mix."""
    from workloads import KERNEL_S, KERNEL_T, KERNEL_W, problem as mk
    rng = np.random.default_rng(1802078440 + 4)
    nreq = args.serve_requests
    kinds = [KERNEL_S, KERNEL_T, KERNEL_W]
    reqs = []
    for i in range(nreq):
        mask = kinds[int(rng.integers(3))]
        n = int(np.exp(rng.uniform(np.log(1e3), np.log(2e5))))
        dist = "uniform" if rng.uniform() < 0.5 else "near_wall"
        tol = 1e-10 if rng.uniform() < 0.5 else 1e-5
        pr = mk(mask, n, 1.0, dist, 4, sub=i)
        reqs.append((mask, tol, torch.from_numpy(pr.src).to(dev), torch.from_numpy(pr.strengths).to(dev)))
    srv = pkg.hse.Server(n_slots=args.serve_slots)
    try:
        return _serve_measure(srv, reqs, rng, pkg, args)
    finally:
        srv.close()


def _serve_measure(srv, reqs, rng, pkg, args):
    prec = lambda tol: pkg.HSE_MIXED if tol >= 1e-6 else pkg.HSE_FP64

    def closed_loop(batch):
        ts = [srv.submit(m, a, b, tol, prec(tol)) for m, tol, a, b in batch]
        for t in ts:
            srv.wait(t, 600.0)

    # warm the plan cache and measure the service capacity (requests/s)
    warm = reqs[: min(len(reqs), 3 * args.serve_slots * 8)]
    closed_loop(warm)
    srv.reset_stats()
    t0 = time.perf_counter()
    closed_loop(warm)
    cap = len(warm) / (time.perf_counter() - t0)
    srv.reset_stats()
    lam = 0.7 * cap
    gaps = rng.exponential(1.0 / lam, size=len(reqs))
    tickets = []
    t_start = time.perf_counter()
    t_next = t_start
    for (m, tol, a, b), g in zip(reqs, gaps):
        t_next += g
        now = time.perf_counter()
        if t_next > now:
            time.sleep(t_next - now)
        tickets.append(srv.submit(m, a, b, tol, prec(tol)))
    for t in tickets:
        srv.wait(t, 600.0)
    st = srv.stats()
    n_tgt = sum(int(a.shape[1]) for _, _, a, _ in reqs)
    return {"requests": len(reqs), "slots": args.serve_slots, "offered_load_req_per_s": lam,
            "capacity_req_per_s": cap, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
            "throughput_req_per_s": st["completed"] / st["busy_s"] if st["busy_s"] else None,
            "throughput_Mtargets_per_s": st["targets_per_s"] / 1e6, "targets": n_tgt, "failed": st["failed"],
            "plans_created": st["plans_created"], "plans_evicted": st["plans_evicted"]}


def run_batch(args, pkg, torch, dev):
    """Many small independent sums in one call: stokeslet / stresslet 50/50, N
    log-uniform in [200, 2e4], uniform positions in the unit box, N(0,1)
    strengths, FP32 arithmetic at tol 1e-5, xi autotuned per group.  A step is
    one hse_batch_eval over all instances (inputs resident on the device)."""
    from workloads import KERNEL_S, KERNEL_T, problem as mk
    import oracle
    n_inst = args.batch_instances
    rng = np.random.default_rng(1802078440 + 3)
    probs = []
    for i in range(n_inst):
        mask = KERNEL_S if i % 2 == 0 else KERNEL_T
        n = int(np.exp(rng.uniform(np.log(200), np.log(2e4))))
        probs.append(mk(mask, n, 1.0, "uniform", 3, sub=i))
    items = [(p.mask, torch.from_numpy(p.src).to(dev), torch.from_numpy(p.strengths).to(dev)) for p in probs]
    outs = [torch.empty((3, p.src.shape[1]), dtype=torch.float64, device=dev) for p in probs]
    n_tot = sum(p.src.shape[1] for p in probs)
    b = pkg.hse.Batch(1e-5, pkg.HSE_MIXED, autotune=True)
    try:
        t0 = time.perf_counter()
        b.eval(items, outs)  # first call: plans, autotuning, cuFFT plans
        torch.cuda.synchronize()
        t_first = time.perf_counter() - t0
        for _ in range(max(0, args.warmup - 1)):
            b.eval(items, outs)
        torch.cuda.synchronize()
        s0 = b.stats()
        stream = torch.cuda.current_stream()
        ms = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.eval(items, outs)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        s1 = b.stats()
    finally:
        b.close()
    ms_step = float(np.mean(ms))
    # error against the FP64 direct sum: all targets of 32 seeded instances,
    # and 64 seeded targets of every instance
    erng = np.random.default_rng(1802078440 + 97)
    errs, errs64 = [], []
    host = [u.cpu().numpy() for u in outs]
    for i in sorted(erng.choice(n_inst, size=min(32, n_inst), replace=False)):
        p = probs[i]
        ref = oracle.direct(p.mask, p.src, p.strengths)
        errs.append(oracle.rel_rms(host[i], ref))
    for i, p in enumerate(probs):
        n = p.src.shape[1]
        idx = np.sort(erng.choice(n, size=min(64, n), replace=False))
        ref = oracle.direct(p.mask, p.src, p.strengths, p.src[:, idx])
        errs64.append(oracle.rel_rms(host[i][:, idx], ref))
    steps = max(1, args.steps)
    return {"instances": n_inst, "targets": n_tot, "value": n_tot / (ms_step / 1e3) / 1e6, "unit": "Mtargets/s",
            "instances_per_s": n_inst / (ms_step / 1e3), "ms_per_step": ms_step,
            "first_call_s": t_first, "tol": 1e-5, "dtype": "f32 arithmetic (FP64 sums, close image pairs, tables)",
            "chunks_per_step": (s1["chunks"] - s0["chunks"]) / steps,
            "gpu_launches_per_step": (s1["kernel_launches"] - s0["kernel_launches"]) / steps,
            "fft_execs_per_step": (s1["fft_execs"] - s0["fft_execs"]) / steps,
            "plans": s1["plans"], "autotuned_groups": s1["autotuned_groups"],
            "err_vs_oracle_max": float(max(errs)),
            "err_sample": f"{len(errs)} seeded instances, all their targets, FP64 direct sum",
            "err_64_targets_median": float(np.median(errs64)), "err_64_targets_max": float(max(errs64)),
            "err_64_targets_sample": "64 seeded targets of every instance (norm of a 64-target sample of a "
                                     "heavy-tailed field: a noisy error estimate)",
            "graph_launches_per_step": (s1["graph_launches"] - s0["graph_launches"]) / steps}


def run_real_only(args, pkg, torch, dev, W, pr):
    if args.mixed:  # the mixed-precision leg's parameters, real-space half only
        plan = pkg.Plan(W["mask"], (1.0, 1.0, 1.0), xi=MIXED["xi"], rc=MIXED["rc"], P=MIXED["P"], tol=0.0,
                        precision=pkg.HSE_MIXED)
    else:
        plan = pkg.Plan(W["mask"], (1.0, 1.0, 1.0), xi=W["xi"], rc=W["rc"], P=W["P"], tol=0.0)
    src = torch.from_numpy(pr.src).to(dev)
    st = torch.from_numpy(pr.strengths).to(dev)
    for _ in range(args.warmup):
        plan.eval_parts(src, st, fourier=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        plan.eval_parts(src, st, fourier=False)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.steps
    plan.close()
    return {"profiling_run": "real-space half only" + (" (mixed precision)" if args.mixed else ""), "n": W["n"],
            "ms_per_step": dt * 1e3}


# Profiling aid: the Fourier half of the bench workload's kind at 1/8 of its
# grid (Mt = 160) and the same particle density and support (P = 18), small
# enough (3.7 GB of grids) for full ncu captures of the spread, transform,
# scale and gather kernels.
FOURIER_SMALL = dict(n=100000, xi=44.0, rc=0.11, P=18, M=142)


def run_fourier_small(args, pkg, torch, dev, W):
    F = dict(FOURIER_SMALL)
    if args.n:
        F["n"] = args.n
    pr = replica_problem(0, F["n"])
    plan = pkg.Plan(W["mask"], (1.0, 1.0, 1.0), xi=F["xi"], rc=F["rc"], P=F["P"], tol=0.0, M=F["M"])
    src = torch.from_numpy(pr.src).to(dev)
    st = torch.from_numpy(pr.strengths).to(dev)
    for _ in range(args.warmup):
        plan.eval_parts(src, st, real=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        plan.eval_parts(src, st, real=False)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.steps
    mt = plan.params["Mt"]
    plan.close()
    return {"profiling_run": "Fourier half only, small grid", "n": F["n"], "Mt": mt, "ms_per_step": dt * 1e3}


# ---------------------------------------------------------- reference arm
def run_reference(args):
    W = dict(WORKLOAD)
    if args.n:
        W["n"] = args.n
    mask = W["mask"]
    pr = problem(mask, W["n"], 1.0, W["dist"], W["index"])
    import oracle
    oracle.build()
    budget = max(2.0, 120.0 / max(1, args.steps + args.warmup))
    tps, k, _ = time_oracle(pr, mask, budget)  # sizes the per-step sample
    rng = np.random.default_rng(1802078440 + 98)
    for _ in range(args.warmup):
        idx = np.sort(rng.choice(W["n"], size=k, replace=False))
        oracle.direct(mask, pr.src, pr.strengths, pr.src[:, idx])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        idx = np.sort(rng.choice(W["n"], size=k, replace=False))
        oracle.direct(mask, pr.src, pr.strengths, pr.src[:, idx])
    dt = (time.perf_counter() - t0) / args.steps
    value = k / dt / 1e6
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mtargets/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": W["name"], "n_sources": W["n"], "targets_per_step": k, "kernels": "stokeslet+rotlet",
                   "tol": W["tol"], "precision": "fp64"},
        "cpu_baseline": {"value": value, "unit": "Mtargets/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"{k} seeded targets per step against all {W['n']} sources"},
        "e2e": {"value": value, "unit": "Mtargets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=0, help="override the number of sources (smaller test runs)")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the FP32-arithmetic measurement")
    ap.add_argument("--serve-requests", type=int, default=400, help="requests of the serving run (0: skip)")
    ap.add_argument("--serve-slots", type=int, default=3)
    ap.add_argument("--batch-instances", type=int, default=4096,
                    help="instances of the batched small-systems run (0: skip)")
    ap.add_argument("--real-only", action="store_true",
                    help="profiling aid: plan without a grid, time only the real-space half")
    ap.add_argument("--mixed", action="store_true", help="with --real-only: the mixed-precision leg's plan")
    ap.add_argument("--fourier-small", action="store_true",
                    help="profiling aid: Fourier half only on a grid of Mt = 160 (100k sources)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
