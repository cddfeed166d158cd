"""Throughput bench of the BSDE solver (path-steps/s at d = 10).

One step = one full solve of the American basket put d = 10 (n = 4000 points,
M = 4000 paths, N = 100 Euler steps, total degree 3 -> p = 364 basis
functions, K_it = 12 Picard iterations): every row of the hot path (points,
basis matrix, path simulation + evaluation + reduction, Gram + RHS, Cholesky
+ refinement, update, price/delta read-out) runs once per iteration.
Metric: path-steps/s = K_it n M N / time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank solves its own independent problem (its
own seed): weak scaling with no data-path collective.  With --shard the ranks
share one problem instead: each simulates a block of the points and the
corrections are all-gathered once per iteration (strong scaling).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "path-steps/s incl. u^k,∇u^k,Lu^k eval at d=10 (vs FP64 plain); p50/p99 solve ms"
UNIT = "path-steps/s"
CONFIG = "c4"

FP32_LANES = 128  # FP32 lanes per SM (sm_103a)
# DRAM bytes (read + write) of one path-kernel launch per point, from an ncu
# capture of the same kernel on the d = 10 workload with n = 800 points
# (146.2 KB read, 0 B written: the partial sums stay in L2), scaled to a
# launch over n points (the kernel reads the points and coefficients and
# writes one partial sum per (point, chunk), both proportional to n).
PATH_TRAFFIC_BYTES_PER_POINT = (134656.0 + 0.0) / 800.0
# instruction issue of the same capture: instructions per path-step and
# instructions issued per SM cycle (of 4), and the MUFU (XU) pipe's share
PATH_ISSUE = {"instructions_per_path_step": 251.2, "ipc": 2.44, "ipc_peak": 4.0, "xu_pipe_busy": 0.682,
              "fma_heavy_pipe_busy": 0.648}


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def rank_seed(base_seed, rank):
    """Seed of the independent problem that rank `rank` solves."""
    return base_seed + 1000 * rank


def weak_scaling_value(ms_local, steps, units_per_step, device=None):
    """Whole-job throughput under weak scaling: every rank solves its own
    problems, the job time is the slowest rank's.  Returns (value, ms_max)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    ms = float(ms_local)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * steps * units_per_step / (ms * 1e-3), ms


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_ready(self, samples=3, timeout_s=30.0):
        """Block until nvidia-smi delivers samples: its start-up (NVML
        initialisation, seconds on a fresh machine) must not overlap the
        timed region."""
        t0 = time.perf_counter()
        while self.proc is not None and len(self.lines) < samples:
            if time.perf_counter() - t0 > timeout_s or self.proc.poll() is not None:
                break
            time.sleep(0.05)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_rate(cfg, budget_s=12.0, gpu_c=None):
    """The oracle (FP64, C, threads over points) on this host's cores: one
    iteration's corrections at a bounded sample of points; path-steps/s.
    With gpu_c (the GPU's corrections of the same iteration from the same
    coefficients, at all points), also the largest difference between the
    two at the sampled points."""
    import numpy as np
    from oracle import bsde_oracle as O
    nth = os.cpu_count() or 1
    nu = O.multi_index_set(cfg["d"] + 1, cfg["eta"], cfg.get("q", 1.0))
    alpha = np.zeros(len(nu)); alpha[0] = 5.0
    t, x = O.points(cfg, 0)
    # calibrate on one point, then size the sample to the budget
    t0 = time.perf_counter()
    O.correction(cfg, nu, alpha, 0, np.arange(1), t[:1], x[:, :1], nthreads=1)
    per_point = max(1e-6, time.perf_counter() - t0)
    npts = max(nth, int(budget_s * nth / per_point) // nth * nth)
    npts = min(npts, cfg["n"])
    idx = np.arange(npts)
    t0 = time.perf_counter()
    c_or = O.correction(cfg, nu, alpha, 0, idx, t[idx], x[:, idx], nthreads=nth)
    el = time.perf_counter() - t0
    steps = npts * cfg["M"] * cfg["N"]
    out = {"value": steps / el, "unit": UNIT, "cores": nth, "kind": "oracle",
           "sample": "one Picard iteration, corrections c_i at %d of the %d points (M=%d paths, N=%d "
                     "steps each, p=%d), FP64 C oracle, %.1f s" % (npts, cfg["n"], cfg["M"], cfg["N"],
                                                                   len(nu), el)}
    if gpu_c is not None:
        err = float(np.max(np.abs(np.asarray(gpu_c)[idx] - c_or)))
        mag = float(np.max(np.abs(c_or)))
        out["parity_vs_gpu"] = {"points": int(npts), "gpu_precision": "mixed",
                                "max_abs_err_c": err, "max_abs_c": mag,
                                "max_err_relative_to_max_c": err / max(1.0, mag)}
    return out


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    cfg = workloads.config(CONFIG)
    # each step: a bounded sample of the same workload (one iteration at a
    # subset of points), sized so that warmup + steps take a few minutes
    for _ in range(max(0, min(args.warmup, 1))):
        cpu_oracle_rate(cfg, budget_s=2.0)
    vals = []
    last = None
    t_all = time.perf_counter()
    for _ in range(args.steps):
        last = cpu_oracle_rate(cfg, budget_s=max(2.0, min(20.0, 120.0 / max(1, args.steps))))
        vals.append(last["value"])
    el = time.perf_counter() - t_all
    v = sum(vals) / len(vals)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": cfg["name"], "d": 10, "n": cfg["n"], "M": cfg["M"], "N": cfg["N"],
                       "eta": 3, "p": 364, "K_it": cfg["K_it"], "sample": last["sample"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_profile_case(args):
    """A small launch of the same kernels for ncu: the d = 10 workload with
    n = 800 points and one iteration (every kernel of an iteration runs
    once per solve); `--case profile_tree`: the same model with a degree-4
    basis (p = 1365, prefix-tree evaluation), n = 2800, M = 2000, N = 50."""
    import torch
    import paper_1102_4666_gb300 as G
    if args.case == "profile_tree":
        cfg = workloads.config(CONFIG, n=2800, M=2000, N=50, eta=4, K_it=1)
        label = " eta=4 n=2800 M=2000 N=50 K_it=1"
    else:
        cfg = workloads.config(CONFIG, n=800, K_it=1)
        label = " n=800 K_it=1"
    s = G.Solver(cfg, precision=args.precision)
    for _ in range(2):
        r = s.solve(use_graph=0, timing=1)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "workload": cfg["name"] + label,
                      "precision": args.precision, "ms_paths": r.ms_paths, "ms_gram": r.ms_gram,
                      "ms_solve": r.ms_solve, "ms_total": r.ms_total, "price": r.price}))
    s.close()
    return 0


def serving_capacity(reqs, slots=16, precision="mixed"):
    """Path-steps/s of a warm server running the first requests of the mix
    back to back (after one untimed pass that warms the memory pool, the
    kernels' modules and the graph machinery)."""
    import paper_1102_4666_gb300 as G
    srv = G.Server(max_slots=slots, precision=precision)
    calib = reqs[:min(16, len(reqs))]
    for timed in (False, True):
        t0 = time.perf_counter()
        ids = [srv.submit(r) for r in calib]
        srv.drain()
        el = time.perf_counter() - t0
        for i in ids:
            srv.poll(i)
    srv.close()
    return sum(workloads.path_steps(r) for r in calib) / el


def arrival_times(n, rate_hz, seed):
    rng = __import__("random").Random(seed)
    t, out = 0.0, []
    for _ in range(n):
        t += rng.expovariate(rate_hz)
        out.append(t)
    return out


def run_serving(reqs, arrivals, precision="mixed", slots=16, policy="fifo", large_slots=2):
    """Continuous-batching serving: the requests of the mix submitted to
    bsde_server at their arrival times (seconds from the start).  Returns
    p50/p99 latency (submit to completion) and throughput."""
    import paper_1102_4666_gb300 as G
    srv = G.Server(max_slots=slots, precision=precision, policy=policy, large_slots=large_slots)
    t_start = time.perf_counter()
    ids = []
    for r, t_arr in zip(reqs, arrivals):
        now = time.perf_counter() - t_start
        if t_arr > now:
            time.sleep(t_arr - now)
        ids.append(srv.submit(r))
    srv.drain()
    wall = time.perf_counter() - t_start
    st = srv.stats()
    bad = 0
    for i in ids:
        rep = srv.poll(i)
        if rep is None or rep.status != 0:
            bad += 1
    srv.close()
    return {"requests": len(reqs), "precision": precision, "slots": slots, "policy": policy,
            "large_slots": large_slots if policy == "size_lanes" else None,
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "path_steps_per_s": st["path_steps"] / wall, "busy_path_steps_per_s": st["path_steps_per_s"],
            "wall_s": wall, "failed": bad}


def fp64_sequential_model(reqs, arrivals):
    """The plain comparator for serving: one request at a time in FP64 on
    the GPU, FIFO.  Its service rate is measured per number of assets d on
    one FP64 iteration of the first request with that d (M capped at 1000);
    each request's service time is its path-steps at that rate, and the
    latencies follow from the same arrival times through a single FIFO
    server.  Simulating the queue instead of running it keeps the bench
    short: the FP64 path needs minutes for this mix."""
    import numpy as np
    import paper_1102_4666_gb300 as G
    rates = {}
    for r in reqs:
        if r["d"] in rates:
            continue
        probe = dict(r)
        probe["K_it"] = 1
        probe["M"] = min(r["M"], 1000)
        s = G.Solver(probe, precision="fp64")
        s.solve(use_graph=0, K_it=1)
        rep = s.solve(use_graph=0, K_it=1, timing=1)
        s.close()
        rates[r["d"]] = rep.path_steps / (rep.ms_total * 1e-3)
    t_free, lat = 0.0, []
    for r, t_arr in zip(reqs, arrivals):
        start = max(t_arr, t_free)
        t_free = start + workloads.path_steps(r) / rates[r["d"]]
        lat.append((t_free - t_arr) * 1e3)
    lat = np.array(lat)
    total = sum(workloads.path_steps(r) for r in reqs)
    return {"precision": "fp64", "slots": 1, "policy": "fifo", "kind": "modeled from measured FP64 rates",
            "fp64_path_steps_per_s_by_d": {str(k): v for k, v in sorted(rates.items())},
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "path_steps_per_s": total / (t_free - 0.0)}


def run_serving_fp64_measured(n_requests=24, seed=17, load=0.7, m_div=8):
    """The plain comparator measured rather than modeled: a smaller mix (the
    serving mix with M divided by m_div) at an arrival rate the FP64
    one-request-at-a-time server sustains (`load` times its measured
    capacity), served by it and, on the same arrivals, by the mixed-precision
    continuous-batching server (4 slots, FIFO)."""
    reqs = workloads.serving_mix(n_requests, seed=seed)
    for r in reqs:
        r["M"] = max(200, r["M"] // m_div)
    mean_steps = sum(workloads.path_steps(r) for r in reqs) / len(reqs)
    cap64 = serving_capacity(reqs[:6], slots=1, precision="fp64")
    rate = load * cap64 / mean_steps
    arr = arrival_times(len(reqs), rate, seed)
    return {"requests": len(reqs), "M_divided_by": m_div, "arrival_rate_hz": rate,
            "fp64_capacity_path_steps_per_s": cap64, "load_of_fp64": load,
            "fp64_one_at_a_time": run_serving(reqs, arr, precision="fp64", slots=1, policy="fifo"),
            "mixed_4_slots": run_serving(reqs, arr, precision="mixed", slots=4, policy="fifo")}


def run_serving_suite(n_requests, seed=7, load=0.8, compare_requests=300):
    """One seeded request mix and one arrival stream (rate: `load` times the
    16-slot capacity).  The whole stream (n_requests; the configured mix has
    2000) is served by the size-lane continuous-batching server (16 slots)
    and one request at a time (mixed precision).  Its first compare_requests
    requests, with the same arrival times, are served by every policy and
    slot count for comparison: FIFO with 16 or 4 slots, shortest-first and
    response-ratio with 4, size lanes with 16 and one at a time.  Besides:
    the modeled one-at-a-time FP64 comparator on the whole stream and a
    measured one on a smaller mix."""
    reqs = workloads.serving_mix(n_requests, seed=seed)
    mean_steps = sum(workloads.path_steps(r) for r in reqs) / len(reqs)
    cap = serving_capacity(reqs)
    rate = load * cap / mean_steps
    arr = arrival_times(len(reqs), rate, seed)
    out = {"arrival_rate_hz": rate, "calibrated_capacity_path_steps_per_s": cap, "load": load,
           "requests": len(reqs)}
    out["size_lanes_16"] = run_serving(reqs, arr, slots=16, policy="size_lanes")
    out["one_at_a_time_mixed"] = run_serving(reqs, arr, slots=1, policy="fifo")
    out["one_at_a_time_fp64"] = fp64_sequential_model(reqs, arr)
    nc = min(compare_requests, len(reqs))
    if nc < len(reqs):
        cmp_ = {"requests": nc, "note": "the first %d requests of the same stream and arrival times" % nc}
        rq, ar = reqs[:nc], arr[:nc]
        cmp_["size_lanes_16"] = run_serving(rq, ar, slots=16, policy="size_lanes")
        cmp_["one_at_a_time_mixed"] = run_serving(rq, ar, slots=1, policy="fifo")
        cmp_["fifo_16"] = run_serving(rq, ar, slots=16, policy="fifo")
        cmp_["fifo_4"] = run_serving(rq, ar, slots=4, policy="fifo")
        cmp_["shortest_first_4"] = run_serving(rq, ar, slots=4, policy="shortest")
        cmp_["response_ratio_4"] = run_serving(rq, ar, slots=4, policy="response_ratio")
        out["policies_on_a_prefix"] = cmp_
    out["fp64_comparator_measured"] = run_serving_fp64_measured()
    return out


def precision_check(G, device, serving_sample=8, max_steps=1.5e9):
    """The error of the mixed-precision path against the plain FP64 path
    (the same kernels in FP64, the same random numbers), stated with the
    results: the d = 10 workload at the paper's penalty weight omega = 1
    (where the iteration converges) for 2 iterations, and a sample of the
    serving mix's requests (the first ones with at most max_steps
    path-steps, European and American alike; a request's served result
    equals its stand-alone solve bit for bit).  Relative errors of the price
    and of the largest delta."""
    import numpy as np

    def pair(cfg):
        out = []
        for prec in ("mixed", "fp64"):
            s = G.Solver(cfg, precision=prec, device=device)
            r = s.solve(use_graph=0)
            s.close()
            out.append((r.price, np.array(r.delta[:cfg["d"]]), r.status))
        (pm, dm, sm), (pf, df, sf) = out
        return {"price_rel_err": abs(pm - pf) / max(abs(pf), 1e-300),
                "delta_rel_err": float(np.max(np.abs(dm - df)) / max(np.max(np.abs(df)), 1e-300)),
                "status": [sm, sf]}

    res = {"tolerance": 1e-4}
    res["d10_omega1_K_it2"] = pair(workloads.config(CONFIG, K_it=2, **{"lambda": 1.0}))
    sample = [r for r in workloads.serving_mix(2000, seed=7) if workloads.path_steps(r) <= max_steps]
    sample = sample[:serving_sample]
    rows = [dict(pair(r), d=r["d"], eta=r["eta"], **{"lambda": r["lambda"]}) for r in sample]
    res["serving_sample"] = {"requests": len(rows),
                             "max_price_rel_err": max(x["price_rel_err"] for x in rows),
                             "max_delta_rel_err": max(x["delta_rel_err"] for x in rows),
                             "per_request": rows}
    return res


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1102_4666_gb300 as G

    cfg = workloads.config(CONFIG)
    shard = args.shard and world > 1
    if not shard:
        cfg["seed"] = rank_seed(cfg["seed"], rank)  # independent problem per rank
    from paper_1102_4666_gb300 import autotune
    shape = autotune.lookup(cfg, "mixed") or autotune.tune(cfg, "mixed", repeats=3)
    stream = torch.cuda.Stream(device=dev)
    s = G.Solver(cfg, precision="mixed", device=local, stream=stream.cuda_stream, launch_shape=shape,
                 gram_splits=autotune.lookup_gram_splits(cfg, "mixed"))
    if shard:
        # one problem, its points in blocks over the ranks, one all-gather of
        # the corrections per iteration (strong scaling)
        nb = (cfg["n"] + world - 1) // world
        xbuf = torch.zeros(world * nb, dtype=torch.float64, device=dev)
        s.set_shard(rank, world, xbuf, G.torch_distributed_exchange())
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def step(timing=1):
        return s.solve(use_graph=1, timing=timing)

    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.zero_()  # also loads the fill kernel's module before the timed region
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    clocks.wait_ready()  # nvidia-smi running before the timed region
    reps = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            flush.zero_()  # L2 flush between steps (on the solve's stream)
            reps.append(step())
        ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    steps_per_solve = workloads.path_steps(cfg)
    value, ms = weak_scaling_value(ms, args.steps, steps_per_solve, device=dev)
    if shard:  # every rank worked on the same problem
        value /= world
    launches = sum(r.kernel_launches for r in reps)
    path_ms = sum(r.ms_paths for r in reps) / max(1, sum(r.path_launches for r in reps))

    # end to end through the public API with host buffers: model, grid and
    # parameters copied from host, report (price, delta, residuals) to host
    # (every rank on its own problem; the job time is the slowest rank's)
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.set_model(cfg)
        s.set_grid(cfg)
        r = s.solve(use_graph=1, timing=0)
        _ = (r.price, list(r.delta))
    e2e_s = time.perf_counter() - t0
    e2e_val, e2e_ms = weak_scaling_value(e2e_s * 1e3, args.steps, steps_per_solve, device=dev)
    if shard:
        e2e_val /= world
    p = 364
    h2d = p * 8 + p + cfg["d"] * 8 + 8 + 4   # basis tables, log S0, key, status reset
    d2h = (1 + 16 + 3 * 64) * 8 + 4          # report block and status word

    # plain FP64 comparator: the same kernels in FP64, one request, no graph
    fp64 = None
    if rank == 0 and not args.no_fp64:
        cfg64 = dict(cfg)
        cfg64["K_it"] = 1
        s64 = G.Solver(cfg64, precision="fp64", device=local)
        s64.solve(use_graph=0, K_it=1)
        r64 = s64.solve(use_graph=0, K_it=1, timing=1)
        s64.close()
        fp64 = {"value": r64.path_steps_per_s, "unit": UNIT,
                "sample": "one iteration of the same workload in FP64, direct launches",
                "path_kernel_ms": r64.ms_paths}

    s.close()
    if rank != 0:
        return 0
    # the same d = 10 American basket put with the penalty weight of the
    # paper's American experiments (omega = 1), where the iteration converges
    chk = G.Solver(workloads.config(CONFIG, **{"lambda": 1.0}), precision="mixed", device=local)
    r1 = chk.solve(use_graph=1)
    chk.close()
    precision = None if args.no_fp64 else precision_check(G, local)
    omega1 = {"lambda": 1.0, "price": r1.price, "delta": list(r1.delta[:10]),
              "resid_l2": list(r1.resid_l2[:cfg["K_it"]]), "status": r1.status}
    # the other configured workloads (whole solves, graph replay, device time)
    others = {}
    for name, prec in (() if args.no_others else (("c1", "fp64"), ("c2", "mixed"), ("c3", "mixed"))):
        wc = workloads.config(name)
        ws = G.Solver(wc, precision=prec, device=local)
        ws.solve(use_graph=1)
        best = min((ws.solve(use_graph=1) for _ in range(3)), key=lambda r: r.ms_total)
        ws.close()
        others[name] = {"workload": wc["name"], "precision": prec, "p": best.p,
                        "path_steps": best.path_steps, "ms_per_solve": best.ms_total,
                        "path_steps_per_s": best.path_steps_per_s}
    # the paper's timing-table workloads (context: its CPU cluster wall times)
    paper = {}
    for name in (() if args.no_others else ("paper_d3", "paper_d6")):
        wc = workloads.config(name)
        t8, tbest, nbest = workloads.PAPER_TIMING_SECONDS[name]
        row = {"workload": wc["name"], "paper_seconds_8_procs": t8,
               "paper_seconds_best": tbest, "paper_best_procs": nbest}
        for prec in ("mixed", "fp64"):
            ws = G.Solver(wc, precision=prec, device=local)
            ws.solve(use_graph=1)
            best = min((ws.solve(use_graph=1) for _ in range(2)), key=lambda r: r.ms_total)
            ws.close()
            row[prec] = {"ms_per_solve": best.ms_total, "price": best.price,
                         "path_steps_per_s": best.path_steps_per_s}
        paper[name] = row
    sm_mhz = clk.get("sm_mhz") or 2070.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s at the sampled clock
    launch_steps = cfg["n"] * cfg["M"] * cfg["N"]
    from paper_1102_4666_gb300 import flops as FL
    fc = FL.per_path_step(cfg["d"], cfg["N"])
    tf = (lambda f: f * launch_steps / (path_ms * 1e-3) / 1e12 if path_ms > 0 else None)
    achieved = tf(fc["flops_with_eval"])
    achieved_steps = tf(fc["flops_steps_only"])
    cpu = None
    if not args.no_cpu:
        # the GPU's corrections of the iteration the oracle times (same
        # points, same coefficients), for the parity figure of the line
        pc = G.Solver(cfg, precision="mixed", device=local)
        a0 = np.zeros(pc.basis_size())
        a0[0] = 5.0
        _, _, c_gpu, _ = pc.iterate(0, a0)
        pc.close()
        cpu = cpu_oracle_rate(cfg, budget_s=args.cpu_budget, gpu_c=c_gpu)
    serving = run_serving_suite(args.serving_requests) if args.serving_requests > 0 else None
    rep0 = reps[-1]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if shard else "weak", "vs_baseline": None, "dtype": "f32",
        "dtype_detail": "f32 paths and evaluation, f64 per-point sums, 3xTF32 Gram, f64 Cholesky/refit",
        "data": "synthetic",
        "config": {"workload": cfg["name"], "d": 10, "n": cfg["n"], "M": cfg["M"], "N": cfg["N"],
                   "eta": 3, "p": rep0.p, "K_it": cfg["K_it"], "precision": "mixed",
                   "l2": "flushed between steps (256 MB write)", "graph": not shard,
                   "parallelism": ("points sharded over %d ranks, one all-gather of the corrections "
                                   "per iteration" % world) if shard else
                                  ("one independent problem per rank" if world > 1 else "one GPU"),
                   "paths_launch_shape": list(shape) if shape else None,
                   "gram_splits": autotune.lookup_gram_splits(cfg, "mixed") or "default (one wave)"},
        "roofline": {"bound": "alu", "kernel": "k_paths_lr<VK_TANH,EV_DENSE3,CC,float,10>",
                     "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
                     "traffic": (PATH_TRAFFIC_BYTES_PER_POINT * cfg["n"]
                                 if PATH_TRAFFIC_BYTES_PER_POINT else None),
                     "traffic_basis": "dram read+write per launch from the n=800 ncu capture, scaled by n",
                     "sm_count": sms,
                     "peak_basis": "%d SMs (device attribute) x 128 FP32 lanes x 2 flop x sampled SM clock "
                                   "%.0f MHz" % (sms, sm_mhz),
                     "flops_per_path_step": fc["flops_with_eval"],
                     "flops_breakdown": {
                         "euler_step": fc["step_flops"],
                         "per_path_eval_u_grad_Lu": fc["eval_flops_per_path"],
                         "per_path_bridge_payoff_driver": fc["other_flops_per_path"],
                         "N_steps": cfg["N"],
                         "basis": "FP32 operations of the kernel source (FMA = 2), "
                                  "paper_1102_4666_gb300/flops.py; MUFU operations apart",
                         "mufu_per_path_step": fc["mufu_per_step"]},
                     "achieved_steps_only": achieved_steps,
                     "frac_steps_only": (achieved_steps / peak) if achieved_steps else None,
                     "path_kernel_ms": path_ms,
                     "issue": dict(PATH_ISSUE, frac=PATH_ISSUE["ipc"] / PATH_ISSUE["ipc_peak"],
                                   basis="ncu capture of this kernel (d = 10, n = 800)")},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
                   "reasons": clk.get("reasons")},
        "fp64_plain": fp64,
        "solve": {"price": rep0.price, "delta0": rep0.delta[0], "ms_paths": rep0.ms_paths,
                  "ms_gram": rep0.ms_gram, "ms_solve": rep0.ms_solve, "ms_total": rep0.ms_total,
                  "ms_total_timed_steps": [r.ms_total for r in reps],
                  "resid_l2_first_last": [rep0.resid_l2[0], rep0.resid_l2[cfg["K_it"] - 1]],
                  "note": "penalty lambda T = 100 is far outside the range where the Picard "
                          "iteration contracts (error bound (lambda T)^k / k!): the iterates of this "
                          "throughput workload grow over its 12 iterations; see solve_omega1"},
        "solve_omega1": omega1,
        "precision_error": precision,
        "other_workloads": others,
        "paper_timing_context": paper,
        "cpu_baseline": cpu,
        "serving": serving,
    }
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--case", default="bench", choices=["bench", "profile", "profile_tree"])
    ap.add_argument("--no-others", action="store_true", help="skip the other configured workloads")
    ap.add_argument("--serving-requests", type=int, default=2000,
                    help="requests of the Poisson serving mix (0: skip; default: the configured 2000)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--shard", action="store_true",
                    help="under torchrun: shard the points of one problem over the ranks (strong "
                         "scaling) instead of one independent problem per rank (weak scaling)")
    args = ap.parse_args()
    if args.case in ("profile", "profile_tree"):
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
