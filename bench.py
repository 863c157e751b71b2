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


# Algorithmic bytes of one Toeplitz-plus-Cross product on a level with N_k nodes, ideal
# single-pass I/O (n = N_k): read the operand u (2n words), the spectra (SPD: real A^ and D^
# over n + 1 frequencies plus complex B^, i.e. 4 (n + 1) words; nonsymmetric: four complex
# spectra, 8 (n + 1) words), write y (2n words) and read the right-hand side of the fused
# epilogue (2n words). Words are 4 B (FP32) or 8 B (FP64): 40 n / 80 n B for the SPD system.
# Multi-pass transforms move more (the work array z between passes): that is measured
# traffic, not algorithmic bytes.
def product_bytes(n, word, nonsym=False):
    return word * (2 * n + (8 if nonsym else 4) * (n + 1) + 2 * n + 2 * n)


# The same bytes split over the three kernels of a strided-pipeline product: the forward pass
# reads u, the contiguous-block kernel reads the spectra, the inverse pass writes y and reads
# the right-hand side.
def product_bytes_split(n, word, nonsym=False):
    return (word * 2 * n, word * (8 if nonsym else 4) * (n + 1), word * 4 * n)


def solve_bytes(K, kc, vcycles, outer, mixed, nonsym=False):
    """Algorithmic bytes of one solve: V(1,1) cycles run two products per level above the
    coarsest (the residual after the first sweep, the post-smoothing sweep); a mixed solve
    adds one FP32 finest residual per inner cycle after the first of each outer iteration and
    one FP64 finest residual per outer iteration; an FP64 solve one FP64 finest residual per
    V-cycle."""
    word = 4 if mixed else 8
    per_cycle = sum(2 * product_bytes((1 << k) - 1, word, nonsym) for k in range(kc + 1, K + 1))
    nK = (1 << K) - 1
    total = vcycles * per_cycle + outer * product_bytes(nK, 8, nonsym)
    if mixed:
        total += (vcycles - outer) * product_bytes(nK, 4, nonsym)
    return total


# dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu capture, valid only for
# the kernel sources it was taken with (SHA-256 of the two device headers below, first 16 hex
# digits) and for the level it was taken at; any other build reports traffic as null.
KERNEL_SOURCES = ("paper_2202_11288_gb300/csrc/tpc_kernels.cuh",
                  "paper_2202_11288_gb300/csrc/tpc_fft.cuh",
                  "paper_2202_11288_gb300/csrc/tpc_f32.cuh")
# per launch, forward pass / contiguous-block kernel / inverse pass (k32_fwd<11, 0>,
# k32_mid<12, 0>, k32_inv<11, 1> at m = 2^23, cold cache), and the FP64 contiguous-block kernel
# k_mid_pair<double, 0, 0> of the same level
TRAFFIC = {"digest": "2483e8f3e9995ff5", "K": 22, "f32": (50.17e6, 152.96e6, 113.06e6), "f64_mid": 353.12e6}


def kernel_digest():
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(key, K):
    if TRAFFIC.get("digest") != kernel_digest() or TRAFFIC.get("K") != K:
        return None
    return TRAFFIC.get(key)


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
    ap.add_argument("--no-twod", action="store_true", help="skip the 2-D measurement")
    ap.add_argument("--batch", type=int, default=512,
                    help="instances of the batched-uneven measurement (0 = skip it)")
    ap.add_argument("--serve-rates", default="50,100,200,500,1000,2000",
                    help="Poisson arrival rates (req/s) of the serving measurement ('' = skip)")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="arrival window per rate of the serving measurement")
    ap.add_argument("--profile", action="store_true",
                    help="profiling case: set up, then 3 finest-level products, nothing timed")
    ap.add_argument("--profile-f32", action="store_true",
                    help="profiling case: mixed-precision setup, then 3 FP32 finest-level products")
    ap.add_argument("--profile-solve", choices=["fp64", "mixed", "fgmres"], default=None,
                    help="profiling case: set up, then one solve, nothing timed")
    ap.add_argument("--profile-batch", action="store_true",
                    help="profiling case: the 512-instance stage-batched solve, one solve "
                         "between cudaProfilerStart / Stop")
    ap.add_argument("--profile-twod", action="store_true",
                    help="profiling case: 2-D mixed set-up (n = 4095^2), then one solve")
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
    from oracle import amg, large, model
    N = 1 << K_sample
    r = model.horizon_ratio(delta, 1.0 / N)
    return amg.Hierarchy(large.rows(model.SPD, N, r, np.arange(2 * N - 1)), kc=3)


def oracle_sample(K_sample, delta, tol, reps, budget_s=20.0, H=None, seed0=0):
    """Time the dense oracle's solve at N = 2^K_sample (set-up not timed); returns
    (solves/s measured, detail, solution of the first right-hand side)."""
    from oracle import amg
    N = 1 << K_sample
    if H is None:
        H = oracle_hierarchy(K_sample, delta)
    times, its, first = [], [], None
    t_start = time.perf_counter()
    for i in range(reps):
        b = uniform_pm1(2 * N - 1, seed0 + i)
        t0 = time.perf_counter()
        u, it, rel, _ = amg.solve(H, b, tol=tol)
        times.append(time.perf_counter() - t0)
        its.append(it)
        if first is None:
            first = u
        if time.perf_counter() - t_start > budget_s:
            break
    return len(times) / sum(times), {"solves": len(times), "seconds": sum(times), "iters": its}, first


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def extrapolate(value_sample, K_sample, K):
    """Dense oracle cost per solve grows as n^2 (dense matrix-vector products, same count)."""
    ratio = ((2 ** (K + 1) - 1) / (2 ** (K_sample + 1) - 1)) ** 2
    return value_sample / ratio


ORACLE_K_SMALL, ORACLE_K_LARGE = 7, 12


def cpu_baseline(args, gpu_solutions=None):
    """The oracle timed on the host cores at two sizes: N = 128 (delta = 0.125, the small
    configuration) and N = 2^12 (the headline's delta), solves after set-up. The value is the
    N = 2^12 rate extrapolated to the headline size by the n^2 cost of dense products (an
    extrapolation: the dense oracle does not fit at N = 2^22). gpu_solutions(K, b), when given,
    returns {name: GPU solution} for the N = 2^12 right-hand side; their distance to the
    oracle's solution of it is reported."""
    v7, d7, _ = oracle_sample(ORACLE_K_SMALL, 0.125, args.tol, reps=8, budget_s=5.0)
    K = ORACLE_K_LARGE
    v12, d12, u12 = oracle_sample(K, args.delta, args.tol, reps=8, budget_s=15.0, seed0=4242)
    out = {"value": extrapolate(v12, K, args.K), "unit": UNIT, "cores": cpu_cores(),
           "kind": "oracle",
           "sample": f"dense FP64 oracle solves (set-up not timed): N=2^{ORACLE_K_SMALL}, "
                     f"delta=0.125: {d7['solves']} solves in {d7['seconds']:.3f} s "
                     f"({v7:.1f} solves/s); N=2^{K} ({2 ** (K + 1) - 1} unknowns), "
                     f"delta={args.delta}: {d12['solves']} solves in {d12['seconds']:.2f} s "
                     f"({v12:.3f} solves/s, {d12['iters'][0]} V-cycles); value = the N=2^{K} "
                     f"rate EXTRAPOLATED to N=2^{args.K} by the n^2 cost of dense products",
           "measured": {f"N=2^{ORACLE_K_SMALL}": v7, f"N=2^{K}": v12}}
    errs = {}
    if gpu_solutions is not None:
        b = uniform_pm1(2 ** (K + 1) - 1, 4242)
        for name, xg in gpu_solutions(K, b).items():
            errs[f"{name}_vs_oracle_N2e{K}"] = float(np.linalg.norm(xg - u12) / np.linalg.norm(u12))
    return out, errs


def run_reference(args, rank):
    if rank != 0:
        return
    K_sample = ORACLE_K_LARGE
    H = oracle_hierarchy(K_sample, args.delta)
    per = []
    for s in range(args.warmup + args.steps):
        v, det, _ = oracle_sample(K_sample, args.delta, args.tol, reps=1, H=H, seed0=s)
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
                                       f"({sec:.3f} s, set-up not timed); value EXTRAPOLATED "
                                       f"to N=2^{args.K} by the n^2 cost of dense products"},
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


def batch_mix_workload(count, seed=1):
    """Uneven 1-D and 2-D instances of 2^10 .. 2^18 unknowns: log2(unknowns) uniform in 10..18;
    an even exponent 2(K+1) is a 2-D instance with probability 1/2 (n = (2^(K+1) - 1)^2, K in
    4..8), else a 1-D one (n = 2^(K+1) - 1, K in 9..17). delta uniform in [0.02, 0.25] (redrawn
    until r >= 1); SPD / nonsymmetric alternating; a 1-D instance takes the fractional kernel
    with probability 1/2, a uniform in [0.1, 0.4], SPD, geometric transfer (the V-cycle does not
    converge beyond a ~ 0.43). Entries: (dim, K, delta, variant, kernel, a)."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        e = int(rng.integers(10, 19))
        dim = 2 if (e % 2 == 0 and rng.random() < 0.5) else 1
        K = e // 2 - 1 if dim == 2 else e - 1
        while True:
            delta = float(rng.uniform(0.02, 0.25))
            if delta * (1 << K) >= 1.0:
                break
        v, kk, a = i % 2, 0, 0.0
        if dim == 1 and rng.random() < 0.5:
            v, kk, a = 0, 1, float(rng.uniform(0.1, 0.4))
        specs.append((dim, K, delta, v, kk, a))
    return specs


def time_batch(tpc, torch, args, rank):
    """The batched configuration: one tpc_batch_solve over a mix of 1-D (constant and
    fractional) and 2-D instances; beside it, the earlier constant-kernel 1-D workload solved
    both stage-batched and as per-instance graphs on concurrent streams (tpc_solve_batch)."""
    steps = min(5, max(1, args.steps))  # the batch is a secondary measurement: a few steps

    def timed(f):
        for _ in range(2):
            f()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            f()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / steps

    # the mix
    specs = batch_mix_workload(args.batch)
    s1 = [s for s in specs if s[0] == 1]
    s2 = [s for s in specs if s[0] == 2]
    solvers = [tpc.Solver(d, 2.0 ** -K, variant=v, kernel=kk, kernel_a=a, precision=tpc.TPC_MIXED,
                          transfer=(tpc.TPC_TRANSFER_GEOMETRIC if kk else tpc.TPC_TRANSFER_PAPER))
               for _, K, d, v, kk, a in s1]
    # the 2-D instances take the FGMRES outer iteration (6 steps a cycle): those with r = 1 or 2
    # need 30 to 110 V-cycles of the stationary one
    twod = [tpc.Solver2D(d, 2.0 ** -K, variant=v, precision=tpc.TPC_MIXED,
                         outer=tpc.TPC_OUTER_FGMRES, inner_cycles=6) for _, K, d, v, _, _ in s2]
    sizes = [S.n for S in solvers] + [S.nn for S in twod]
    bs = [torch.tensor(uniform_pm1(n, 7000 + i), device="cuda") for i, n in enumerate(sizes)]
    xs = [torch.zeros_like(b) for b in bs]
    B = tpc.Batch([S.handle for S in solvers], [S.handle for S in twod])
    res = {}

    def mix():
        rc, its, rels, sts = B.solve(bs, xs, tol=args.tol)
        assert rc == tpc.TPC_OK and max(rels) < args.tol, (rc, max(rels))
        res["its"] = its

    sec = timed(mix)
    dof = sum(sizes)
    out = {"instances": len(specs), "instances_2d": len(s2),
           "instances_fractional": sum(1 for s in s1 if s[4]), "solves_per_s": len(specs) / sec,
           "dof_per_s": dof / sec, "ms_per_batch": 1000.0 * sec, "unknowns_total": dof,
           "groups": B.groups(), "grouped_instances": B.grouped_instances(),
           "max_outer_iters": max(res["its"]),
           "workload": "512 instances of 2^10..2^18 unknowns (log2 uniform in 10..18; even "
                       "exponents 2-D with probability 1/2), delta uniform in [0.02,0.25], "
                       "SPD/nonsym, 1-D: constant kernel or (probability 1/2) fractional a "
                       "uniform in [0.1,0.4] with the geometric transfer, 2-D: constant kernel "
                       "with the FGMRES(6) outer iteration; mixed precision, tol 1e-10; one "
                       "tpc_batch_solve per step (host clock)"}
    B.close()
    for S in solvers + twod:
        S.close()
    # the constant-kernel 1-D workload, stage-batched and on concurrent streams
    specs = batch_workload(args.batch)
    solvers = [tpc.Solver(d, 2.0 ** -K, variant=v, kernel=kk, kernel_a=a,
                          precision=tpc.TPC_MIXED) for K, d, v, kk, a in specs]
    bs = [torch.tensor(uniform_pm1(S.n, 5000 + i), device="cuda") for i, S in enumerate(solvers)]
    xs = [torch.zeros_like(b) for b in bs]
    handles = [S.handle for S in solvers]

    def streams():
        rc, its, rels, sts = tpc.tpc_solve_batch(handles, bs, xs, tol=args.tol)
        assert rc == tpc.TPC_OK and max(rels) < args.tol

    B = tpc.Batch(handles)

    def staged():
        rc, its, rels, sts = B.solve(bs, xs, tol=args.tol)
        assert rc == tpc.TPC_OK and max(rels) < args.tol

    sec_streams = timed(streams)
    sec_staged = timed(staged)
    dof = sum(S.n for S in solvers)
    out["constant_1d"] = {
        "instances": len(specs), "unknowns_total": dof, "groups": B.groups(),
        "stage_batched": {"solves_per_s": len(specs) / sec_staged, "dof_per_s": dof / sec_staged,
                          "ms_per_batch": 1000.0 * sec_staged},
        "streams": {"solves_per_s": len(specs) / sec_streams, "dof_per_s": dof / sec_streams,
                    "ms_per_batch": 1000.0 * sec_streams},
        "workload": "N=2^K, K uniform in 9..17, delta uniform in [0.02,0.25], SPD/nonsym, "
                    "constant kernel, mixed precision, tol 1e-10; stage_batched: tpc_batch_solve, "
                    "streams: tpc_solve_batch (instance graphs on concurrent streams)"}
    B.close()
    for S in solvers:
        S.close()
    return out


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


def time_fgmres(tpc, torch, args, stream, steps=4):
    """Secondary: the headline problem (and the fractional one of time_fractional) with the
    flexible GMRES outer iteration (an option, not the paper's: one restart cycle of at most
    `steps` V-cycle-preconditioned steps per FP64 residual). Mixed and FP64, 3 timed solves each
    after one warm-up, CUDA events on the solver's stream; cycles = V-cycles per solve."""
    out = {"workload": f"as the headline; outer iteration = FGMRES({steps}) with one V-cycle per "
                       f"step as preconditioner; 3 solves after 1 warm-up"}
    n = 2 ** (args.K + 1) - 1
    with torch.cuda.stream(stream):
        b = torch.tensor(uniform_pm1(n, 2024), device="cuda")
        x = torch.zeros_like(b)
    cases = (("mixed", tpc.TPC_MIXED, {}), ("fp64", tpc.TPC_FP64, {}),
             ("fractional_a025_mixed", tpc.TPC_MIXED,
              dict(kernel=1, kernel_a=0.25, transfer=tpc.TPC_TRANSFER_GEOMETRIC)))
    for name, prec, kw in cases:
        S = tpc.Solver(args.delta, 2.0 ** -args.K, stream=stream, precision=prec,
                       outer=tpc.TPC_OUTER_FGMRES, inner_cycles=steps, **kw)
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
        out[name] = {"value": 1000.0 / ms, "unit": UNIT, "ms_per_solve": ms, "outer_iters": it,
                     "vcycles": tpc.tpc_last_solve_cycles(S.handle), "relres": rel}
        S.close()
    return out


def time_twod(tpc, torch, args, stream, K=11, delta=0.1):
    """The 2-D configuration: the tensor-product reading of the constant kernel on the unit square
    with a square horizon, n x n unknowns with n = 2^(K+1) - 1 (K = 11: 4095^2 = 16.8 M), delta
    = 0.1, SPD and nonsymmetric, uniform[-1,1) right-hand sides, tol 1e-10; mixed (FP32 V-cycles,
    FP64 refinement) and FP64; 3 solves after 1 warm-up, CUDA events on the solver's stream."""
    out = {"workload": f"2-D constant kernel, square horizon, n = {2 ** (K + 1) - 1}^2 unknowns, "
                       f"delta = {delta}, uniform[-1,1) RHS, tol {args.tol}; 3 solves after 1 "
                       f"warm-up"}
    for vname, variant in (("spd", tpc.TPC_SPD), ("nonsym", tpc.TPC_NONSYM)):
        for pname, prec in (("mixed", tpc.TPC_MIXED), ("fp64", tpc.TPC_FP64)):
            S = tpc.Solver2D(delta, 2.0 ** -K, stream=stream, variant=variant, precision=prec)
            with torch.cuda.stream(stream):
                b = torch.tensor(uniform_pm1(S.nn, 3030), device="cuda")
                x = torch.zeros_like(b)
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
            out[f"{vname}_{pname}"] = {"value": 1000.0 / ms, "unit": UNIT, "ms_per_solve": ms,
                                       "dof_per_s": S.nn * 1000.0 / ms, "outer_iters": it,
                                       "vcycles": S.last_cycles(), "relres": rel}
            S.close()
    return out


def serve_keys():
    """Problems of the serving measurement, (dim, variant, delta, K, kernel, a, transfer), sizes
    2^10 .. 2^22 unknowns: 1-D N = 2^K, K in 9..21 (n = 2^(K+1) - 1), delta in {0.05, 0.1, 0.2},
    SPD or nonsymmetric with the constant kernel, or SPD with the fractional kernel a in {0.1,
    0.25, 0.4} (geometric transfer); 2-D K in 4..10 (n = (2^(K+1) - 1)^2, the even exponents),
    delta in {0.1, 0.2}, SPD or nonsymmetric, constant kernel. Requests pick the dimension with
    probability 1/2 each, then the size uniformly on the log scale, then the rest uniformly."""
    one = [(1, v, d, K, 0, 0.0, 0) for K in range(9, 22) for d in (0.05, 0.1, 0.2) for v in (0, 1)]
    one += [(1, 0, d, K, 1, a, 1) for K in range(9, 22) for d in (0.05, 0.2) for a in (0.1, 0.25, 0.4)]
    two = [(2, v, d, K, 0, 0.0, 0) for K in range(4, 11) for d in (0.1, 0.2) for v in (0, 1)]
    return one, two


def serve_outer(key):
    """Outer iteration of a served problem: FGMRES for the 2-D ones (their stationary iteration
    is slow at small r), the stationary one of section 5 otherwise."""
    return 1 if key[0] == 2 else 0


# Requests a client keeps outstanding at most (their host buffers are pinned); arrivals beyond
# it are turned away and counted as rejected.
MAX_OUTSTANDING = 2048


def serve_size(key):
    dim, K = key[0], key[3]
    n1 = (1 << (K + 1)) - 1
    return n1 * n1 if dim == 2 else n1


def time_serving(tpc, torch, args):
    """Poisson arrivals into the request server; p50 / p99 latency, throughput and the server's
    occupancy of the GPU (fraction of the window with a solve on it, mean solves on it at once)
    per rate."""
    rates = [float(r) for r in args.serve_rates.split(",") if r.strip()]
    one, two = serve_keys()
    keys = one + two
    rng = np.random.default_rng(17)
    sizes = sorted(set(serve_size(k) for k in keys))
    # three seeded right-hand sides per size, one drawn per request
    rhs = {n: [torch.tensor(uniform_pm1(n, 900 + 8 * i + j)).pin_memory() for j in range(3)]
           for i, n in enumerate(sizes)}
    pool = {n: [] for n in rhs}

    def xbuf(n):
        return pool[n].pop() if pool[n] else torch.empty(n, dtype=torch.float64).pin_memory()

    def pick():
        # dimension, then the size (log scale), then the rest
        group = one if rng.random() < 0.5 else two
        Ks = sorted(set(k[3] for k in group))
        K = Ks[int(rng.integers(len(Ks)))]
        cands = [k for k in group if k[3] == K]
        return cands[int(rng.integers(len(cands)))]

    srv = tpc.Server(hbm_budget_bytes=150 << 30, max_inflight=32, precision=tpc.TPC_MIXED)
    out = {"workload": "Poisson arrivals of 1-D and 2-D solves, 2^10..2^22 unknowns (dimension "
                       "1/2 each, size log-uniform): 1-D N=2^K, K in 9..21, constant kernel "
                       "(delta in {0.05,0.1,0.2}, SPD/nonsym) or fractional a in {0.1,0.25,0.4} "
                       "(SPD, geometric transfer, delta in {0.05,0.2}); 2-D K in 4..10, delta in "
                       "{0.1,0.2}, SPD/nonsym, constant kernel, FGMRES outer iteration; uniform[-1,1) "
                       "right-hand sides (one of "
                       "three seeded ones per size, drawn per request); "
                       "mixed precision, tol 1e-10, host buffers (pinned); hierarchies resident "
                       f"(HBM budget 150 GB, 32 slots); {args.serve_seconds:g} s of arrivals per rate; "
                       f"at most {MAX_OUTSTANDING} requests outstanding (later arrivals rejected)",
           "keys": len(keys), "rates": []}
    try:
        owner = {}
        t0 = time.perf_counter()
        failed_keys = []
        for key in keys:                    # prewarm: build every hierarchy once
            dim, v, d, K, kk, a, tr = key
            n = serve_size(key)
            x = xbuf(n)
            owner[srv.submit(v, d, 2.0 ** -K, rhs[n][0], x, args.tol, kk, a, dim=dim,
                             transfer=tr, outer=serve_outer(key))] = (n, x, key)
        got = 0
        while got < len(keys):
            for r in srv.poll(256, wait_ms=20):
                n, x, key = owner.pop(r["ticket"])
                pool[n].append(x)
                if r["status"] != tpc.TPC_OK:
                    failed_keys.append(list(key))
                got += 1
        out["prewarm_s"] = time.perf_counter() - t0
        out["prewarm_failed_keys"] = failed_keys
        out["resident_gb"] = srv.stats()["resident_bytes"] / 1e9
        for rate in rates:
            n_req = max(1, int(rate * args.serve_seconds))
            gaps = rng.exponential(1.0 / rate, n_req)
            lat, bad, rejected = [], 0, 0
            srv.stats(reset=True)
            start = time.perf_counter()
            t_next = start
            for i in range(n_req):
                t_next += gaps[i]
                while True:
                    for r in srv.poll(256, wait_ms=0):
                        n, x, _ = owner.pop(r["ticket"])
                        pool[n].append(x)
                        lat.append(r["latency_s"])
                        bad += r["status"] != tpc.TPC_OK
                    dt = t_next - time.perf_counter()
                    if dt <= 0:
                        break
                    time.sleep(min(dt, 0.0005))
                key = pick()
                if len(owner) >= MAX_OUTSTANDING:   # the client's queue is full: turned away
                    rejected += 1
                    continue
                dim, v, d, K, kk, a, tr = key
                n = serve_size(key)
                x = xbuf(n)
                owner[srv.submit(v, d, 2.0 ** -K, rhs[n][int(rng.integers(3))], x, args.tol, kk,
                                 a, dim=dim, transfer=tr, outer=serve_outer(key))] = (n, x, key)
            while owner:
                for r in srv.poll(256, wait_ms=20):
                    n, x, _ = owner.pop(r["ticket"])
                    pool[n].append(x)
                    lat.append(r["latency_s"])
                    bad += r["status"] != tpc.TPC_OK
            wall = time.perf_counter() - start
            st = srv.stats()
            lat_ms = np.array(lat) * 1000.0
            done = n_req - rejected
            out["rates"].append({"rate_req_s": rate, "requests": n_req, "rejected": rejected,
                                 "throughput_req_s": done / wall,
                                 "p50_ms": float(np.percentile(lat_ms, 50)),
                                 "p99_ms": float(np.percentile(lat_ms, 99)),
                                 "failed": int(bad),
                                 "gpu_busy_frac": st["busy_s"] / max(st["elapsed_s"], 1e-9),
                                 "mean_inflight_when_busy": st["inflight_s"] / max(st["busy_s"], 1e-9),
                                 "max_inflight": st["max_inflight_seen"]})
    finally:
        srv.close()
    return out


def gpu_solutions(tpc, torch, args, K, b):
    """GPU solutions (mixed and FP64, tol as the headline) of one right-hand side at N = 2^K."""
    out = {}
    for name, prec in (("mixed", tpc.TPC_MIXED), ("fp64", tpc.TPC_FP64)):
        S = tpc.Solver(args.delta, 2.0 ** -K, precision=prec)
        try:
            bd = torch.tensor(b, device="cuda")
            xd = torch.zeros_like(bd)
            rc, it, rel = S.solve(bd, xd, tol=args.tol)
            assert rc == tpc.TPC_OK and rel < args.tol
            torch.cuda.synchronize()
            out[name] = xd.cpu().numpy()
        finally:
            S.close()
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
    cyc64 = tpc.tpc_last_solve_cycles(S64.handle)
    # FP64 solution of rhs[0], the reference of the mixed solutions' error
    x64 = torch.zeros_like(x)
    rc, it, rel = S64.solve(rhs[0], x64, tol=args.tol)
    assert rc == tpc.TPC_OK and rel < args.tol
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
    cyc_mixed = tpc.tpc_last_solve_cycles(S.handle)
    # per-result error of the mixed solution against the FP64 solution of the same system
    xm = torch.zeros_like(x)
    rc, it_m, rel_m = S.solve(rhs[0], xm, tol=args.tol)
    assert rc == tpc.TPC_OK and rel_m < args.tol
    err_vs_fp64 = (torch.linalg.norm(xm - x64) / torch.linalg.norm(x64)).item()
    del xm, x64

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
    del x32, f32, y32

    NK = (1 << args.K) - 1
    hbm = measured_hbm_gbs()
    digest = kernel_digest()
    # headline path: one FP32 product of the finest level = forward strided pass +
    # contiguous-block kernel + inverse strided pass (residual epilogue), each timed alone
    reg = 20 <= args.K + 1 <= 23   # m = 2^(K+1): the register-resident FP32 kernels
    names = (("k32_fwd", "k32_mid", "k32_inv") if reg else
             ("k_fwd_strided<float>", "k_mid_pair<float>", "k_inv_strided<float>"))
    t_prod = sum(ms3_32) * 1e-3
    b_prod = product_bytes(NK, 4)
    split = product_bytes_split(NK, 4)
    ach32 = b_prod / t_prod / 1e9
    tr32 = traffic_for("f32", args.K)
    roofline = {"bound": "hbm", "achieved": ach32, "peak": hbm["gbs"], "unit": "GB/s",
                "frac": ach32 / hbm["gbs"],
                "traffic": (sum(tr32) if tr32 else None),
                "kernel": "FP32 finest-level product (%s, residual epilogue), N_K = 2^%d - 1"
                          % (" + ".join(names), args.K),
                "algorithmic_bytes_per_launch": b_prod,
                "algorithmic_bytes_rule": "40 n B per FP32 SPD product, n = N_K (read u 8n, "
                                          "spectra 16n, write y 8n, right-hand side 8n)",
                "peak_source": hbm["source"] + " (of measured)",
                "ms_per_launch": dict(zip(("fwd_strided", "mid", "inv_strided"), ms3_32)),
                "achieved_per_kernel": {names[i]: split[i] / (ms3_32[i] * 1e-3) / 1e9
                                        for i in range(3)},
                "traffic_per_kernel": (dict(zip(names, tr32)) if tr32 else None),
                "kernel_digest": digest}
    # FP64 residual product: bound by the FP64 pipe on GB300
    m = 2 ** (args.K + 1)
    logL = min(12, (args.K + 2) // 2)
    flops_mid = m * (2 * 5 * logL + 14)       # DIF + DIT radix-2 stages, spectral product
    achieved = flops_mid / (ms3[1] * 1e-3) / 1e12
    sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
    peak = N_SMS * FP64_FLOP_PER_CLK_PER_SM * sm_max * 1e6 / 1e12
    b64 = product_bytes(NK, 8)
    roofline_fp64 = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic_for("f64_mid", args.K),
                     "kernel": "k_mid_pair<double> (finest level; the FP64 residual product)",
                     "peak_source": "FP64: 152 SMs x 4 flop/clk x max SM clock (unit counts "
                                    "and clocks; FMA-loop probe 1.19 TFLOP/s)",
                     "ms_per_launch": {"fwd_strided": ms3[0], "mid": ms3[1],
                                       "inv_strided": ms3[2]},
                     "product_hbm": {"algorithmic_bytes": b64,
                                     "achieved_gbs": b64 / (sum(ms3) * 1e-3) / 1e9,
                                     "frac_of_hbm": b64 / (sum(ms3) * 1e-3) / 1e9 / hbm["gbs"]}}
    # whole solves: the algorithmic bytes of every product the solve runs over its time
    kc = 3
    sb_mixed = solve_bytes(args.K, kc, cyc_mixed, iters[-1], True)
    sb_fp64 = solve_bytes(args.K, kc, cyc64, it64[-1], False)
    solve_level = {
        "mixed": {"algorithmic_bytes": sb_mixed, "vcycles_fp32": cyc_mixed,
                  "outer_iters": iters[-1],
                  "achieved_gbs": sb_mixed / (ms_max / args.steps * 1e-3) / 1e9,
                  "frac_of_hbm": sb_mixed / (ms_max / args.steps * 1e-3) / 1e9 / hbm["gbs"]},
        "fp64": {"algorithmic_bytes": sb_fp64, "vcycles": cyc64,
                 "achieved_gbs": sb_fp64 / (ms64 / args.steps * 1e-3) / 1e9,
                 "frac_of_hbm": sb_fp64 / (ms64 / args.steps * 1e-3) / 1e9 / hbm["gbs"]},
        "rule": "sum over the solve's products of the per-product algorithmic bytes (40 n_k B "
                "FP32, 80 n_k B FP64, SPD): 2 per level above the coarsest per V-cycle, plus "
                "the finest residuals; element-wise kernels not counted"}
    errors = {"mixed_vs_fp64_gpu_N2e%d" % args.K: err_vs_fp64,
              "note": "||x_mixed - x_fp64|| / ||x_fp64|| for the same right-hand side, both "
                      "at relative residual < %g" % args.tol}
    # the fractional-kernel, batched and served measurements run on one GPU (a single-rank job)
    frac = time_fractional(tpc, torch, args, stream) if world == 1 else None
    fgmres = time_fgmres(tpc, torch, args, stream) if world == 1 else None
    twod = time_twod(tpc, torch, args, stream) if (world == 1 and not args.no_twod) else None
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
                "solve_level_hbm": solve_level, "result_errors": errors,
                "gpu_launches": int(launches)}
        line["speedup_mixed_vs_fp64"] = line["value"] / line["fp64"]["value"]
        if frac:
            line["fractional_a025"] = frac
        if fgmres:
            line["fgmres"] = fgmres
        if twod:
            line["twod"] = twod
        if batch:
            line["batch_uneven"] = batch
        if serving:
            line["serving"] = serving
        if not args.no_cpu_baseline:
            line["cpu_baseline"], oerr = cpu_baseline(args, lambda K, b: gpu_solutions(
                tpc, torch, args, K, b))
            errors.update(oerr)
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
    prec = tpc.TPC_FP64 if args.profile_solve == "fp64" else tpc.TPC_MIXED
    if args.profile_solve == "fgmres":   # mixed precision, FGMRES(4) outer iteration
        S = tpc.Solver(args.delta, 2.0 ** -args.K, precision=prec, inner_cycles=4, autotune=0,
                       outer=tpc.TPC_OUTER_FGMRES)
    else:
        S = tpc.Solver(args.delta, 2.0 ** -args.K, precision=prec, inner_cycles=args.inner,
                       autotune=0)
    b = torch.tensor(uniform_pm1(n, 0), device="cuda")
    x = torch.zeros_like(b)
    rc, it, rel = S.solve(b, x, tol=args.tol)
    torch.cuda.synchronize()
    S.close()
    print(json.dumps({"profile_solve": args.profile_solve, "K": args.K, "rc": rc, "iters": it,
                      "relres": rel}))


def run_profile_twod(args):
    """A fixed launch sequence for profilers: the 2-D mixed solver at n = 4095^2, one solve."""
    import torch

    import paper_2202_11288_gb300 as tpc
    S = tpc.Solver2D(0.1, 2.0 ** -11, precision=tpc.TPC_MIXED)
    b = torch.tensor(uniform_pm1(S.nn, 3030), device="cuda")
    x = torch.zeros_like(b)
    rc, it, rel = S.solve(b, x, tol=args.tol)
    torch.cuda.synchronize()
    S.close()
    print(json.dumps({"profile_twod": "n=4095^2", "rc": rc, "iters": it, "relres": rel}))


def run_profile_batch(args):
    """A fixed launch sequence for profilers: set up the constant-kernel batch of 512 uneven 1-D
    instances stage-batched (tpc_batch_*), solve it twice, then once more between
    cudaProfilerStart and cudaProfilerStop (capture with --profile-from-start off)."""
    import torch

    import paper_2202_11288_gb300 as tpc
    specs = batch_workload(512)
    solvers = [tpc.Solver(d, 2.0 ** -K, variant=v, kernel=kk, kernel_a=a, precision=tpc.TPC_MIXED,
                          autotune=0) for K, d, v, kk, a in specs]
    bs = [torch.tensor(uniform_pm1(S.n, 5000 + i), device="cuda") for i, S in enumerate(solvers)]
    xs = [torch.zeros_like(b) for b in bs]
    B = tpc.Batch([S.handle for S in solvers])
    for _ in range(2):
        rc, its, rels, sts = B.solve(bs, xs, tol=args.tol)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    rc, its, rels, sts = B.solve(bs, xs, tol=args.tol)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    B.close()
    for S in solvers:
        S.close()
    print(json.dumps({"profile_batch": 512, "groups": len(set((K, v) for K, _, v, _, _ in specs)),
                      "rc": rc, "max_iters": max(its), "max_relres": max(rels)}))


def main():
    args = parse()
    if args.profile_batch:
        run_profile_batch(args)
        return
    if args.profile_twod:
        run_profile_twod(args)
        return
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
