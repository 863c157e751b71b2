"""Benchmark: solves/s to relative residual 1e-10 on the 1-D SPD peridynamic system.

Workload (one step = one whole solve, every row of the hot path): N = 2^22 intervals
(8,388,607 unknowns), horizon delta = 0.05 (r = 209,715), constant kernel, shifted-symmetric
system, V(1,1) damped Jacobi (omega = 2/3) down to 15 unknowns, seeded uniform[-1,1) right-hand
sides, tol 1e-10 on the FP64 residual. The headline solver runs its V-cycles in FP32 inside FP64
iterative refinement; the plain FP64 V-cycle solver is timed on the same right-hand sides and
reported beside it. Right-hand sides are resident in HBM before the timed region; the
per-solve working set (spectra, twiddles, level vectors: > 1 GB) is far larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--K 22]

With N > 1 (torchrun, one process per GPU) every rank solves its own independent problems
(replicas, no collective on the data path); the value is the total over ranks.
--impl reference times the oracle (dense FP64 CPU code) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synth import uniform_pm1  # noqa: E402

METRIC = ("solves/s to rel-res 1e-10 (1D SPD peridynamic system; mixed FP32 V-cycles in FP64 "
          "refinement, plain FP64 V-cycle reported beside it)")
UNIT = "solves/s"
FP64_FLOP_PER_CLK_PER_SM = 4      # 2 DFMA per clock per SM (FMA-loop probe: 1.19 TFLOP/s at 1995 MHz)
N_SMS = 152
# dram__bytes_read.sum + dram__bytes_write.sum of one k_mid_pair<double> launch at the finest
# level, from ncu (profiles/k_mid_pair_fp64_N2e22.md); unknown for other sizes
MID_TRAFFIC = {22: 356.8e6}
# Algorithmic bytes of the FP32 finest-level kernels per point of the FFT length m = 2N + 2
# (residual epilogue, no prologue; x, f, y hold about m floats; the Cross vectors q, zeta and
# p, xi hold m/2 entries each of which only the first r are nonzero and read, a fraction r/N):
#   forward pass:            reads x (4m), q and zeta (4m r/N); writes z (8m)   -> 12m + 4m r/N
#   contiguous-block kernel: reads z (8m), 16 B of spectra per pair (8m); writes z  -> 24m
#   inverse pass:            reads z (8m), p and xi (4m r/N), f (4m); writes y (4m) -> 16m + 4m r/N
def f32_bytes_per_point(r, N):
    frac = min(1.0, r / N)
    return (12.0 + 4.0 * frac, 24.0, 16.0 + 4.0 * frac)
# dram__bytes_read.sum + dram__bytes_write.sum per launch of the FP32 finest kernels, from ncu
# (profiles/fp32_transform_kernels_N2e22.md), keyed by (K, kernel index); unknown for other sizes
F32_TRAFFIC = {(22, 0): 54.3e6, (22, 1): 154.3e6, (22, 2): 115.9e6}


def measured_hbm_gbs():
    """The measured copy bandwidth of this GPU type, else the stated fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return {"gbs": float(json.load(fh)["hbm_gbs"]),
                    "source": "measured STREAM-style copy (MEASURED_PEAKS.json hbm_gbs)"}
    except (OSError, KeyError, ValueError):
        return {"gbs": 6800.0, "source": "fallback 6.8 TB/s (no measured peak file)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--K", type=int, default=22)
    ap.add_argument("--delta", type=float, default=0.05)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--inner", type=int, default=6, help="FP32 V-cycles per FP64 residual")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=512,
                    help="instances of the batched-uneven measurement (0 = skip it)")
    ap.add_argument("--serve-rates", default="50,100,200,500,1000,2000",
                    help="Poisson arrival rates (req/s) of the serving measurement ('' = skip)")
    ap.add_argument("--serve-seconds", type=float, default=2.0,
                    help="arrival window per rate of the serving measurement")
    ap.add_argument("--profile", action="store_true",
                    help="profiling case: set up, then 3 finest-level products, nothing timed")
    ap.add_argument("--profile-f32", action="store_true",
                    help="profiling case: mixed-precision setup, then 3 FP32 finest-level products")
    ap.add_argument("--profile-solve", choices=["fp64", "mixed"], default=None,
                    help="profiling case: set up, then one solve, nothing timed")
    return ap.parse_args()


def workload(K, delta):
    N = 1 << K
    r = int(np.floor(delta * N)) if delta > 1.0 / N else 1
    return {"workload": f"1D SPD peridynamic, N=2^{K}, delta={delta}, constant kernel, "
                        f"uniform[-1,1) RHS, V(1,1) omega=2/3, kc=3, tol 1e-10",
            "K": K, "N": N, "unknowns": 2 * N - 1, "delta": delta, "r": r, "variant": "spd",
            "precision": "mixed (FP32 inner V-cycles, FP64 residual/refinement); FP64 also timed",
            "l2": "working set > L2 (spectra + vectors > 1 GB); no flush"}


# --------------------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline object)
# --------------------------------------------------------------------------------------

def oracle_hierarchy(K_sample, delta):
    from oracle import amg, model
    N = 1 << K_sample
    return amg.Hierarchy(model.assemble(model.SPD, N, model.horizon_ratio(delta, 1.0 / N)), kc=3)


def oracle_sample(K_sample, delta, tol, reps, budget_s=20.0, H=None):
    """Time the dense oracle's solve at N = 2^K_sample; returns (solves/s measured, detail)."""
    from oracle import amg
    N = 1 << K_sample
    if H is None:
        H = oracle_hierarchy(K_sample, delta)
    times, its = [], []
    t_start = time.perf_counter()
    for i in range(reps):
        b = uniform_pm1(2 * N - 1, i)
        t0 = time.perf_counter()
        _, it, rel, _ = amg.solve(H, b, tol=tol)
        times.append(time.perf_counter() - t0)
        its.append(it)
        if time.perf_counter() - t_start > budget_s:
            break
    return len(times) / sum(times), {"solves": len(times), "seconds": sum(times), "iters": its}


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def extrapolate(value_sample, K_sample, K):
    """Dense oracle cost per solve grows as n^2 (dense matrix-vector products, same count)."""
    ratio = ((2 ** (K + 1) - 1) / (2 ** (K_sample + 1) - 1)) ** 2
    return value_sample / ratio


def cpu_baseline(args, K_sample=11):
    v, det = oracle_sample(K_sample, args.delta, args.tol, reps=8)
    return {"value": extrapolate(v, K_sample, args.K), "unit": UNIT, "cores": cpu_cores(),
            "kind": "oracle",
            "sample": f"dense FP64 oracle solve at N=2^{K_sample} ({2 ** (K_sample + 1) - 1} "
                      f"unknowns): {det['solves']} solves in {det['seconds']:.2f} s "
                      f"({v:.3f} solves/s, iters {det['iters'][0]}); value extrapolated to "
                      f"N=2^{args.K} by the n^2 cost of its dense products"}


def run_reference(args, rank):
    if rank != 0:
        return
    K_sample = 11
    H = oracle_hierarchy(K_sample, args.delta)
    per = []
    for s in range(args.warmup + args.steps):
        v, det = oracle_sample(K_sample, args.delta, args.tol, reps=1, H=H)
        if s >= args.warmup:
            per.append(1.0 / v)
    sec = float(np.mean(per))
    value = extrapolate(1.0 / sec, K_sample, args.K)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload(args.K, args.delta),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": f"each step one dense oracle solve at N=2^{K_sample} "
                                       f"({sec:.3f} s); extrapolated to N=2^{args.K} by n^2"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def time_solves(tpc, torch, S, stream, rhs, x, args, clocks=None):
    """Warm-up, then exactly args.steps solves between CUDA events on the solver's stream."""
    for s in range(args.warmup):
        rc, it, rel = S.solve(rhs[s % len(rhs)], x, tol=args.tol)
        assert rc == tpc.TPC_OK and rel < args.tol, (rc, rel)
    torch.cuda.synchronize()
    l0 = tpc.tpc_kernel_launches(S.handle)
    if clocks:
        clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters = []
    ev0.record(stream)
    for s in range(args.steps):
        rc, it, rel = S.solve(rhs[s % len(rhs)], x, tol=args.tol)
        assert rc == tpc.TPC_OK and rel < args.tol, (rc, rel)
        iters.append(it)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    return ev0.elapsed_time(ev1), iters, tpc.tpc_kernel_launches(S.handle) - l0, clk


def batch_workload(count, seed=0):
    """Uneven 1-D instances: N = 2^K with K uniform in 9..17 (1023 .. 262143 unknowns), delta
    uniform in [0.02, 0.25] (redrawn until r >= 1), SPD / nonsymmetric alternating, constant
    kernel (the V-cycle needs tens to hundreds of cycles with the fractional kernel), uniform[-1,1)
    right-hand sides. Entries: (K, delta, variant, kernel, a)."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        K = int(rng.integers(9, 18))
        while True:
            delta = float(rng.uniform(0.02, 0.25))
            if delta * (1 << K) >= 1.0:
                break
        specs.append((K, delta, i % 2, 0, 0.0))
    return specs


def time_batch(tpc, torch, args, rank):
    """One step = one tpc_solve_batch call over all instances (mixed precision)."""
    specs = batch_workload(args.batch)
    solvers = [tpc.Solver(d, 2.0 ** -K, variant=v, kernel=kk, kernel_a=a,
                          precision=tpc.TPC_MIXED) for K, d, v, kk, a in specs]
    bs = [torch.tensor(uniform_pm1(S.n, 5000 + i), device="cuda") for i, S in enumerate(solvers)]
    xs = [torch.zeros_like(b) for b in bs]
    handles = [S.handle for S in solvers]
    for _ in range(2):
        rc, its, rels, sts = tpc.tpc_solve_batch(handles, bs, xs, tol=args.tol)
        assert rc == tpc.TPC_OK, rc
    torch.cuda.synchronize()
    steps = min(5, max(1, args.steps))  # the batch is a secondary measurement: a few steps
    t0 = time.perf_counter()
    for _ in range(steps):
        rc, its, rels, sts = tpc.tpc_solve_batch(handles, bs, xs, tol=args.tol)
        assert rc == tpc.TPC_OK and max(rels) < args.tol
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / steps
    dof = sum(S.n for S in solvers)
    for S in solvers:
        S.close()
    return {"instances": len(specs), "solves_per_s": len(specs) / sec, "dof_per_s": dof / sec,
            "ms_per_batch": 1000.0 * sec, "unknowns_total": dof,
            "workload": "N=2^K, K uniform in 9..17, delta uniform in [0.02,0.25], SPD/nonsym, "
                        "constant kernel, mixed precision, tol 1e-10, one tpc_solve_batch per "
                        "step (host clock)"}


def time_fractional(tpc, torch, args, stream):
    """Secondary: the fractional kernel |s|^-(1+2a), a = 1/4, of the same size and horizon, with
    the geometric transfer (an option, not the paper's transfer, under which the V-cycle does
    not reach 1e-10 in 400 outer iterations at this size). Mixed and FP64, 3 timed solves each
    after one warm-up, CUDA events on the solver's stream."""
    out = {"workload": f"as the headline, fractional kernel a = 0.25 (reading of this build), "
                       f"transfer = geometric; 3 solves after 1 warm-up"}
    n = 2 ** (args.K + 1) - 1
    with torch.cuda.stream(stream):
        b = torch.tensor(uniform_pm1(n, 2024), device="cuda")
        x = torch.zeros_like(b)
    for name, prec in (("mixed", tpc.TPC_MIXED), ("fp64", tpc.TPC_FP64)):
        S = tpc.Solver(args.delta, 2.0 ** -args.K, stream=stream, precision=prec, kernel=1,
                       kernel_a=0.25, transfer=tpc.TPC_TRANSFER_GEOMETRIC)
        rc, it, rel = S.solve(b, x, tol=args.tol)
        assert rc == tpc.TPC_OK and rel < args.tol, (rc, rel)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(3):
            rc, it, rel = S.solve(b, x, tol=args.tol)
            assert rc == tpc.TPC_OK and rel < args.tol, (rc, rel)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / 3
        out[name] = {"value": 1000.0 / ms, "unit": UNIT, "ms_per_solve": ms,
                     ("outer_iters" if prec == tpc.TPC_MIXED else "vcycles"): it, "relres": rel}
        S.close()
    return out


def serve_keys():
    """Problems of the serving measurement: N = 2^K, K in 9..21 (1023 .. 4,194,303 unknowns,
    log-uniform when K is uniform), delta in {0.05, 0.1, 0.2}, SPD or nonsymmetric, constant
    kernel: (variant, delta, K, kernel, a)."""
    return [(v, d, K, 0, 0.0) for K in range(9, 22) for d in (0.05, 0.1, 0.2) for v in (0, 1)]


def time_serving(tpc, torch, args):
    """Poisson arrivals into the request server; p50 / p99 latency and throughput per rate."""
    rates = [float(r) for r in args.serve_rates.split(",") if r.strip()]
    keys = serve_keys()
    rng = np.random.default_rng(17)
    rhs = {K: torch.tensor(uniform_pm1((1 << (K + 1)) - 1, 900 + K)).pin_memory()
           for K in range(9, 22)}
    pool = {K: [] for K in rhs}

    def xbuf(K):
        return pool[K].pop() if pool[K] else torch.empty(rhs[K].numel(), dtype=torch.float64).pin_memory()

    srv = tpc.Server(hbm_budget_bytes=150 << 30, max_inflight=32, precision=tpc.TPC_MIXED)
    out = {"workload": "Poisson arrivals; N=2^K, K uniform in 9..21 (1023..4,194,303 unknowns), "
                       "delta in {0.05,0.1,0.2}, SPD/nonsym, constant kernel, mixed precision, "
                       "tol 1e-10, host buffers (pinned); hierarchies resident (HBM budget "
                       "150 GB, 32 slots)",
           "rates": []}
    try:
        owner = {}
        t0 = time.perf_counter()
        for v, d, K, kk, a in keys:                    # prewarm: build every hierarchy once
            x = xbuf(K)
            owner[srv.submit(v, d, 2.0 ** -K, rhs[K], x, args.tol, kk, a)] = (K, x)
        got = 0
        while got < len(keys):
            for r in srv.poll(256, wait_ms=20):
                K, x = owner.pop(r["ticket"])
                pool[K].append(x)
                got += 1
        out["prewarm_s"] = time.perf_counter() - t0
        for rate in rates:
            n_req = max(1, int(rate * args.serve_seconds))
            gaps = rng.exponential(1.0 / rate, n_req)
            picks = rng.integers(len(keys), size=n_req)
            lat, bad = [], 0
            start = time.perf_counter()
            t_next = start
            for i in range(n_req):
                t_next += gaps[i]
                while True:
                    for r in srv.poll(256, wait_ms=0):
                        K, x = owner.pop(r["ticket"])
                        pool[K].append(x)
                        lat.append(r["latency_s"])
                        bad += r["status"] != tpc.TPC_OK
                    dt = t_next - time.perf_counter()
                    if dt <= 0:
                        break
                    time.sleep(min(dt, 0.0005))
                v, d, K, kk, a = keys[picks[i]]
                x = xbuf(K)
                owner[srv.submit(v, d, 2.0 ** -K, rhs[K], x, args.tol, kk, a)] = (K, x)
            while owner:
                for r in srv.poll(256, wait_ms=20):
                    K, x = owner.pop(r["ticket"])
                    pool[K].append(x)
                    lat.append(r["latency_s"])
                    bad += r["status"] != tpc.TPC_OK
            wall = time.perf_counter() - start
            lat_ms = np.array(lat) * 1000.0
            out["rates"].append({"rate_req_s": rate, "requests": n_req,
                                 "throughput_req_s": n_req / wall,
                                 "p50_ms": float(np.percentile(lat_ms, 50)),
                                 "p99_ms": float(np.percentile(lat_ms, 99)),
                                 "failed": int(bad)})
    finally:
        srv.close()
    return out


def replica_throughput(local_ms, steps, world, dist=None, device=None):
    """Whole-job throughput of N replicas: every rank times `steps` of its own solves; the
    job's time is the maximum over ranks (all_reduce MAX), and the value counts the solves of
    all ranks: world * steps / max_ms. Returns (value per second, max ms)."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return world * steps / (ms_max / 1000.0), ms_max


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2202_11288_gb300 as tpc

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def max_over_ranks(v):
        return replica_throughput(v, 1, world, dist, "cuda")[1]

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    cfg = workload(args.K, args.delta)
    n = cfg["unknowns"]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        rhs = [torch.tensor(uniform_pm1(n, 1000 * rank + i), device="cuda") for i in range(4)]
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
    stream.synchronize()

    # plain FP64 V-cycle solver
    S64 = tpc.Solver(args.delta, 2.0 ** -args.K, stream=stream)
    barrier()
    ms64, it64, l64, _ = time_solves(tpc, torch, S64, stream, rhs, x, args)
    barrier()
    ms64 = max_over_ranks(ms64)
    # dominant FP64 kernel: the contiguous-block kernel of the finest level (forward transform
    # stages, spectral product, inverse transform stages), timed with CUDA events
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    ms3 = tpc.tpc_time_level_kernels(S64.handle, args.K, 5, x, rhs[0], y)
    S64.close()

    # mixed precision: FP32 V-cycles inside FP64 refinement (the headline)
    S = tpc.Solver(args.delta, 2.0 ** -args.K, stream=stream, precision=tpc.TPC_MIXED,
                   inner_cycles=args.inner)
    clocks = Clocks(local_rank)
    barrier()
    ms, iters, launches, clk = time_solves(tpc, torch, S, stream, rhs, x, args, clocks)
    barrier()
    ms_max = max_over_ranks(ms)
    value = world * args.steps / (ms_max / 1000.0)
    # check the last result against an FP64 residual computed by the FP64 product
    x_last = x.clone()

    # end to end through the host-buffer entry point (pinned host memory)
    b_host = torch.tensor(uniform_pm1(n, 77 + rank), dtype=torch.float64).pin_memory()
    x_host = torch.zeros(n, dtype=torch.float64).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for s in range(args.steps):
        rc, it, rel = tpc.tpc_solve_host(S.handle, b_host.numpy(), x_host.numpy(), args.tol)
        assert rc == tpc.TPC_OK
    torch.cuda.synchronize()
    e2e_value = world * args.steps / max_over_ranks(time.perf_counter() - t0)
    # the FP32 kernels of the finest level, which the FP32 V-cycles run most
    x32 = x.float()
    f32 = rhs[0].float()
    y32 = torch.empty_like(x32)
    ms3_32 = tpc.tpc_time_level_kernels_f32(S.handle, args.K, 5, x32, f32, y32)
    S.close()
    del x_last, x32, f32, y32

    m = 2 ** (args.K + 1)
    logL = min(12, (args.K + 2) // 2)
    flops_mid = m * (2 * 5 * logL + 14)       # DIF + DIT radix-2 stages, spectral product
    achieved = flops_mid / (ms3[1] * 1e-3) / 1e12
    sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
    peak = N_SMS * FP64_FLOP_PER_CLK_PER_SM * sm_max * 1e6 / 1e12
    roofline_fp64 = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": MID_TRAFFIC.get(args.K),
                     "kernel": "k_mid_pair<double> (finest level; the FP64 residual product)",
                     "peak_source": "FP64: 152 SMs x 4 flop/clk x max SM clock (unit counts "
                                    "and clocks; FMA-loop probe 1.19 TFLOP/s)",
                     "ms_per_launch": {"fwd_strided": ms3[0], "mid": ms3[1],
                                       "inv_strided": ms3[2]}}
    # headline path: the FP32 finest-level kernels, each launched once per FP32 product; the
    # dominant one is the slowest of the three
    names = ("k_fwd_strided<float>", "k_mid_pair<float>", "k_inv_strided<float>")
    dom = max(range(3), key=lambda i: ms3_32[i])
    nbytes = [b * m for b in f32_bytes_per_point(cfg["r"], 2 ** args.K)]
    hbm = measured_hbm_gbs()
    ach32 = nbytes[dom] / (ms3_32[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": ach32, "peak": hbm["gbs"], "unit": "GB/s",
                "frac": ach32 / hbm["gbs"], "traffic": F32_TRAFFIC.get((args.K, dom)),
                "kernel": names[dom] + " (finest level of the FP32 V-cycles)",
                "algorithmic_bytes_per_launch": nbytes[dom],
                "peak_source": hbm["source"],
                "ms_per_launch": dict(zip(("fwd_strided", "mid", "inv_strided"), ms3_32)),
                "achieved_all": {names[i]: nbytes[i] / (ms3_32[i] * 1e-3) / 1e9
                                 for i in range(3)}}
    # the fractional-kernel, batched and served measurements run on one GPU (a single-rank job)
    frac = time_fractional(tpc, torch, args, stream) if world == 1 else None
    batch = time_batch(tpc, torch, args, rank) if (args.batch > 0 and world == 1) else None
    serving = (time_serving(tpc, torch, args)
               if (args.serve_rates.strip() and world == 1) else None)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic", "config": cfg,
                "dof_per_s": value * n, "outer_iters_per_solve": iters,
                "inner_fp32_vcycles_per_outer_max": args.inner,
                "fp64": {"value": world * args.steps / (ms64 / 1000.0), "unit": UNIT,
                         "ms_per_step": ms64 / args.steps, "vcycles_per_solve": it64,
                         "gpu_launches": int(l64)},
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * n,
                        "d2h_bytes_per_step": 8 * n},
                "roofline": roofline, "roofline_fp64": roofline_fp64, "clocks": clk,
                "gpu_launches": int(launches)}
        line["speedup_mixed_vs_fp64"] = line["value"] / line["fp64"]["value"]
        if frac:
            line["fractional_a025"] = frac
        if batch:
            line["batch_uneven"] = batch
        if serving:
            line["serving"] = serving
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_profile_case(args):
    """A short, fixed launch sequence for profilers: setup, then three finest-level products."""
    import torch

    import paper_2202_11288_gb300 as tpc
    n = 2 ** (args.K + 1) - 1
    S = tpc.Solver(args.delta, 2.0 ** -args.K, autotune=0)  # no tuning launches in the list
    x = torch.tensor(uniform_pm1(n, 5), device="cuda")
    y = torch.empty_like(x)
    for _ in range(3):
        S.apply(args.K, x, y)
    torch.cuda.synchronize()
    assert torch.isfinite(y).all()
    S.close()
    print(json.dumps({"profile_case": f"N=2^{args.K}", "unknowns": n}))


def run_profile_f32(args):
    """A fixed launch sequence for profilers: mixed setup, then the FP32 finest-level kernels
    exactly as the bench's roofline times them (tpc_time_level_kernels_f32, residual epilogue):
    forward pass x2, contiguous-block kernel x2, inverse pass x2 (the first of each a warm-up)."""
    import torch

    import paper_2202_11288_gb300 as tpc
    n = 2 ** (args.K + 1) - 1
    S = tpc.Solver(args.delta, 2.0 ** -args.K, precision=tpc.TPC_MIXED, autotune=0)
    x = torch.tensor(uniform_pm1(n, 5), dtype=torch.float32, device="cuda")
    f = torch.tensor(uniform_pm1(n, 6), dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    ms = tpc.tpc_time_level_kernels_f32(S.handle, args.K, 1, x, f, y)
    torch.cuda.synchronize()
    assert torch.isfinite(y).all()
    S.close()
    print(json.dumps({"profile_f32": f"N=2^{args.K}", "unknowns": n, "ms": ms}))


def run_profile_solve(args):
    """A fixed launch sequence for profilers: setup, then one solve."""
    import torch

    import paper_2202_11288_gb300 as tpc
    n = 2 ** (args.K + 1) - 1
    prec = tpc.TPC_MIXED if args.profile_solve == "mixed" else tpc.TPC_FP64
    S = tpc.Solver(args.delta, 2.0 ** -args.K, precision=prec, inner_cycles=args.inner,
                   autotune=0)
    b = torch.tensor(uniform_pm1(n, 0), device="cuda")
    x = torch.zeros_like(b)
    rc, it, rel = S.solve(b, x, tol=args.tol)
    torch.cuda.synchronize()
    S.close()
    print(json.dumps({"profile_solve": args.profile_solve, "K": args.K, "rc": rc, "iters": it,
                      "relres": rel}))


def main():
    args = parse()
    if args.profile:
        run_profile_case(args)
        return
    if args.profile_solve:
        run_profile_solve(args)
        return
    if args.profile_f32:
        run_profile_f32(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
