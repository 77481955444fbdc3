"""Benchmark: time-to-solution of the hybrid IPM / column-generation OT solver on GB300.

Workload: one 64x64 image pair (m = n = 4096, 16.8M variables), seeded log-normal Gaussian
random-field marginals, squared-Euclidean pixel cost, solved to relative gap 1e-6 with the mixed
precision path (FP32 pricing scan + FP64 recheck, FP32 dense factorisation preconditioning an
FP64 CG, which stops at relative residual 1e-6; at most one centrality corrector per iteration)
and the multiscale warm start (the 32x32 binned problem solved first, its duals seeding
the initial support).  A step = ot_ipm_create + ot_ipm_solve of that instance (the coarse solve
happens inside create), timed wall-clock with the device synchronised on both sides.  The cold
mixed solve, the plain FP64 path (cold and multiscale) and the learned network's warm start are
timed the same way beside it, and a batch of 64 uneven instances (24^2 .. 96^2, autotuned launch
shapes) is solved through the library's work queue.

JSON line (rank 0): metric/value/unit (seconds, lower is better), e2e through the public API
with host buffers, pricing throughput, the roofline of the dominant instrumented kernel, the
CPU oracle's time for one complete exact solve of the same instance (network simplex), clocks
sampled during the timed region.  --impl reference times one complete solve of the instance by
the oracle's rendition of the method (the paper ships no code).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--k 64]
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "OT time-to-solution at rel. gap 1e-6 (learned+mixed vs plain FP64); pricing Gcols/s"
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling (every 200 ms) while the timed region runs."""

    def __init__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self, gpu_index: int = 0) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.f.read().splitlines():
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9 or parts[0] != str(gpu_index):
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """The slowest rank's value (replicas: each rank times its own instance)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_instance_seed(rank: int) -> int:
    """Seed of the instance a rank solves: replicas of the same workload on different data."""
    return rank


# ------------------------------------------------------------------------------ oracle arm
def host_cpu() -> dict:
    """CPU model and core count of the host the oracle runs on."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                key = ln.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "processor name") and ":" in ln:
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for ln in out.splitlines():
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"model": model, "nproc": os.cpu_count()}


def oracle_ipm_solve(k: int, seed: int, tol: float = 1e-6):
    """One complete solve of the CPU oracle's rendition of the method (O2) to its stopping test;
    returns (seconds, iterations, status)."""
    from oracle import costs, ipm
    from paper_2206_11009_gb300 import synth
    inst = synth.image_pair(k, seed)
    t0 = time.perf_counter()
    r = ipm.solve(costs.square_grid(k), inst.a, inst.b, ipm.Options(tol=tol))
    return time.perf_counter() - t0, r.iters, r.status


def oracle_simplex_solve(k: int, seed: int):
    """One complete exact solve by the oracle's network simplex (O1); returns (seconds, pivots)."""
    from oracle import costs, netsimplex
    from paper_2206_11009_gb300 import synth
    inst = synth.image_pair(k, seed)
    t0 = time.perf_counter()
    r = netsimplex.solve(costs.square_grid(k), inst.a, inst.b)
    return time.perf_counter() - t0, r.pivots


def run_reference(args, world, rank):
    """The reference arm is the CPU oracle (the paper ships no code): one complete solve of the
    same instance by the oracle's rendition of the method, on one host core.  Its iterations are
    split evenly over the K timed steps, so the K steps together are exactly that one solve (the
    value is the solve's whole time); the W warm-up steps are complete oracle solves of a 16x16
    pair."""
    if rank != 0:
        return 0
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    for _ in range(args.warmup):
        oracle_ipm_solve(16, 0)
    v, iters, status = oracle_ipm_solve(args.k, 0)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3 / max(args.steps, 1),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args),
            "cpu_baseline": {"kind": "oracle", "value": v, "unit": "s", "cores": 1, "cpu": host_cpu(),
                             "sample": f"one complete solve of the {args.k}x{args.k} instance by the oracle's "
                                       f"float64 rendition of the method to its stopping test ({iters} iterations, "
                                       f"status {status}); its iterations split evenly over the {args.steps} steps"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_dict(args):
    return {"workload": f"{args.k}x{args.k} image pair (m=n={args.k * args.k}, {args.k ** 4} variables), "
                        "GRF marginals, squared-Euclidean cost, rel. gap 1e-6, multiscale warm start + mixed "
                        "precision, create + solve timed",
            "k": args.k, "m": args.k * args.k, "n": args.k * args.k, "tol": 1e-6,
            "l2": "flushed between steps (256 MiB write)", "seed": 0, "direct_cg_tol": 1e-6, "max_corr": 1}


# ------------------------------------------------------------------------------ GPU arm
def pcg_at(torch, synth, k: int, seed: int, steps: int):
    """The FP32 Jacobi PCG (one cooperative launch per refinement) and the FP64 one on the Newton
    system of a k x k pair's iterate `steps`: microseconds per CG iteration and algorithmic bytes
    per second (theta, index and gathered entry per pair in both passes, plus the vectors)."""
    from paper_2206_11009_gb300 import Solver, kernel_timing
    inst = synth.image_pair(k, seed)
    out = {"k": k, "seed": seed, "iterate": steps}
    with Solver(inst.a, inst.b, grid=(k, k), tol=1e-6, precision=1) as s:
        for _ in range(steps):
            s.step()
        out["psi"] = int(len(s.state()[0]))
        pk_d, _ = peaks()
        for name, solver in (("pcg32", "mixed"), ("pcg64", "pcg64")):
            s.newton_direction(solver, cg_tol=1e-8, max_cg=3000)
            torch.cuda.synchronize()
            kernel_timing(True)
            its = s.newton_direction(solver, cg_tol=1e-8, max_cg=3000)[4]
            torch.cuda.synchronize()
            ms, cnt, work = kernel_timing()[name]
            kernel_timing(False)
            gbs = work / (ms * 1e-3) / 1e9 if ms > 0 else None
            out[name] = {"cg_iters": its, "us_per_iter": ms * 1e3 / max(its, 1), "achieved_gbs": gbs,
                         "frac_hbm": gbs / pk_d.get("hbm_gbs", 6800.0) if gbs else None}
    return out


def pricing_at(torch, synth, k: int, seed: int, reps: int = 5):
    """Pricing + selection on a k x k pair with the duals and support of its 4th IPM iteration;
    full-call throughput and the scan pass against the FP32 ALU peak (4 lane-ops per pair)."""
    import numpy as np
    from paper_2206_11009_gb300 import Solver, kernel_timing, price_topk
    inst = synth.image_pair(k, seed)
    with Solver(inst.a, inst.b, grid=(k, k), tol=1e-6, precision=1, max_iter=4) as s:
        s.solve(raise_on_error=False)
        Is, Js, _, _, us, vs = s.state()
    x, y = synth.grid_coords(k)
    T = lambda arr, dt: torch.as_tensor(np.ascontiguousarray(arr), dtype=dt, device="cuda")
    tx, ty, tu, tv, ti, tj = (T(x, torch.int32), T(y, torch.int32), T(us, torch.float64), T(vs, torch.float64),
                              T(Is, torch.int32), T(Js, torch.int32))
    for _ in range(3):
        price_topk(tx, ty, tx, ty, tu, tv, ti, tj, kmax=k * k, precision=1)
    torch.cuda.synchronize()
    kernel_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        gi, _, _ = price_topk(tx, ty, tx, ty, tu, tv, ti, tj, kmax=k * k, precision=1)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    kt = kernel_timing()
    kernel_timing(False)
    pairs = float(k * k) ** 2
    pk_d, src = peaks()
    table = kernel_table(kt, pk_d, src)
    return {"k": k, "pairs": pairs, "support": int(len(Is)), "selected": int(gi.numel()), "ms_per_call": ms,
            "gcols_per_s": pairs / (ms * 1e-3) / 1e9, "scan_pass": table.get("scan_hist"),
            "gather_pass": table.get("scan_gather")}


def run_batch(torch, synth, count: int = 64, workers: int = 2):
    """64 uneven instances (sides 24..96, seeded), autotuned launch shapes, solved through the
    library's queue with `workers` host threads and with one; wall time around each whole batch
    (creation, solve, destruction: every host-device copy included)."""
    from paper_2206_11009_gb300 import autotune
    from paper_2206_11009_gb300.api import solve_batch
    t0 = time.perf_counter()
    autotune.tune([32, 64, 96], verbose=False)
    tune_s = time.perf_counter() - t0
    sides = synth.batch_sides(count, 24, 96, seed=1234)
    pairs = []
    for i, kk in enumerate(sides):
        inst = synth.image_pair(int(kk), i)
        pairs.append((inst.a, inst.b, int(kk)))
    out = {"instances": count, "sides": [int(x) for x in sides], "tuning_seconds": tune_s,
           "tuned": {key: v["options"] for key, v in autotune._load().items()}}
    for w in (workers, 1):
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = solve_batch(pairs, workers=w, tuning=autotune.lookup, create_threads=8)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t
        ok = sum(1 for r in res if r.status == 0)
        out[f"workers_{w}"] = {"wall_s": wall, "instances_per_s": count / wall, "solved": ok,
                               "mean_device_s": statistics.mean(r.seconds for r in res),
                               "mean_iters": statistics.mean(r.iters for r in res)}
    out["speedup_vs_one_worker"] = out["workers_1"]["wall_s"] / out[f"workers_{workers}"]["wall_s"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native")
    ap.add_argument("--k", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-big-pricing", action="store_true")
    ap.add_argument("--no-c3", action="store_true")
    ap.add_argument("--no-pcg256", action="store_true")
    args = ap.parse_args()
    world, rank, local = dist_init()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import numpy as np
    import torch
    import __graft_entry__
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        __graft_entry__.build()
    barrier(world)
    __graft_entry__.build()
    from paper_2206_11009_gb300 import Solver, kernel_launches, kernel_timing, price_topk, synth

    k = args.k
    inst = synth.image_pair(k, rank_instance_seed(rank))   # each rank: its own instance (replicas, weak scaling)
    a_pin = torch.from_numpy(inst.a).pin_memory()
    b_pin = torch.from_numpy(inst.b).pin_memory()
    a_np, b_np = a_pin.numpy(), b_pin.numpy()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    from paper_2206_11009_gb300 import learn
    net = learn.WarmNet.load() if os.path.exists(learn.WEIGHTS) else None
    a_dev, b_dev = a_pin.cuda(), b_pin.cuda()      # inputs resident in HBM for the device-timed value
    # the configuration measured: mixed precision and the multiscale warm start (one coarser level
    # solved first to relative tolerance 1e-3); ot_ipm_create is inside every timed region
    # the factor-preconditioned CG stops at relative residual 1e-6 (direct_cg_tol); at most one
    # centrality corrector per iteration (max_corr; the library's default is 3: at 64x64 one
    # corrector costs a few more iterations but less time, 3 seeds 5 % on average).  The
    # comparison arms below use the same IPM settings.
    IPM = dict(tol=1e-6, max_corr=1)
    MAIN = dict(IPM, precision=1, multiscale=1, ms_tol=1e-3, direct_cg_tol=1e-6)

    def timed_solve(a, b, want_solution=False, **opts):
        """Wall time of create + solve (+ solution read-back), synchronised on both sides."""
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with Solver(a, b, grid=(k, k), **opts) as s:
            r = s.solve(raise_on_error=False)
            sol = s.solution() if want_solution else None
        torch.cuda.synchronize()
        return time.perf_counter() - t0, r, sol

    # warm-up (untimed)
    for _ in range(args.warmup):
        timed_solve(a_dev, b_dev, **MAIN)
        timed_solve(a_np, b_np, want_solution=True, **MAIN)
    # timed: `value` = create + solve with the inputs on the device; `e2e` = the same through host
    # buffers (masses copied in by ot_ipm_create) plus the read-back of the coupling and duals
    clocks = Clocks()
    dev_times, e2e_times, results = [], [], []
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    launches0 = kernel_launches()
    kernel_timing(True)
    h2d = d2h = 0
    for _ in range(args.steps):
        flush.fill_(1)
        t, r, _ = timed_solve(a_dev, b_dev, **MAIN)
        dev_times.append(t)
        results.append(r)
        flush.fill_(1)
        t, r2, (I, J, P, u, v) = timed_solve(a_np, b_np, want_solution=True, **MAIN)
        e2e_times.append(t)
        h2d = a_np.nbytes + b_np.nbytes
        d2h = I.nbytes + J.nbytes + P.nbytes + u.nbytes + v.nbytes
    # every step runs two solves (device inputs for `value`, host buffers for `e2e`): the kernels of
    # the `value` solves are half of those counted over the region
    launches_per_solve = (kernel_launches() - launches0) / (2.0 * max(args.steps, 1))
    torch.cuda.synchronize()
    ktimes = kernel_timing()
    kernel_timing(False)
    launches = int(round(launches_per_solve * args.steps))
    clk = clocks.stop(local)
    barrier(world)
    t_dev = max_over_ranks(statistics.mean(dev_times), world)
    t_e2e = max_over_ranks(statistics.mean(e2e_times), world)

    # plain FP64 GPU path on the same instance (the comparison the metric names), and the mixed
    # path without the network
    def summary(t, r):
        return {"seconds": t, "solve_seconds": r.seconds, "create_seconds": r.create_seconds, "status": r.status,
                "iters": r.iters, "rel_gap": r.rel_gap, "warm_added": r.warm_added, "dropped": r.warm_restarts}
    plain = None
    if not args.no_plain:
        plain = summary(*timed_solve(a_dev, b_dev, precision=0, **IPM)[:2])
    mixed_cold = summary(*timed_solve(a_dev, b_dev, precision=1, direct_cg_tol=1e-6, **IPM)[:2])
    plain_ms = None if args.no_plain else summary(*timed_solve(a_dev, b_dev, precision=0, multiscale=1, **IPM,
                                                              ms_tol=1e-3)[:2])
    learned = None
    if net is not None:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        wd = net.predict(a_np, b_np, k)                 # network inference inside the timed region
        with Solver(a_dev, b_dev, grid=(k, k), precision=1, warm=wd, direct_cg_tol=1e-6, **IPM) as s:
            rl = s.solve(raise_on_error=False)
        torch.cuda.synchronize()
        learned = summary(time.perf_counter() - t0, rl)

    batch = None if args.no_batch else run_batch(torch, synth)

    # pricing throughput at this size with the final duals of a solve (realistic reduced costs)
    with Solver(a_np, b_np, grid=(k, k), tol=1e-6, precision=1) as s:
        s.solve(raise_on_error=False)
        Is, Js, Ps, Ss, us, vs = s.state()
    x, y = synth.grid_coords(k)
    T = lambda arr, dt: torch.as_tensor(np.ascontiguousarray(arr), dtype=dt, device="cuda")
    tx, ty = T(x, torch.int32), T(y, torch.int32)
    tu, tv = T(us, torch.float64), T(vs, torch.float64)
    ti, tj = T(Is, torch.int32), T(Js, torch.int32)
    for _ in range(3):
        price_topk(tx, ty, tx, ty, tu, tv, ti, tj, kmax=k * k, precision=1)
    torch.cuda.synchronize()
    kernel_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    e0.record()
    for _ in range(reps):
        price_topk(tx, ty, tx, ty, tu, tv, ti, tj, kmax=k * k, precision=1)
    e1.record()
    torch.cuda.synchronize()
    price_ms = e0.elapsed_time(e1) / reps
    pk = kernel_timing()
    kernel_timing(False)
    pairs = (k * k) ** 2
    gcols = pairs / (price_ms * 1e-3) / 1e9

    big = None if args.no_big_pricing else pricing_at(torch, synth, 256, 10000)
    pcg256 = None if args.no_pcg256 else pcg_at(torch, synth, 256, 10000, 25)

    # config 3: the 128x128 pair with 5 % spikes (mixed precision, one solve)
    c3 = None
    if not args.no_c3:
        inst3 = synth.image_pair(128, 0, spike_frac=0.05)
        with Solver(inst3.a, inst3.b, grid=(128, 128), tol=1e-6, precision=1) as s:
            r3 = s.solve(raise_on_error=False)
        c3 = {"k": 128, "spike_frac": 0.05, "seconds": r3.seconds, "status": r3.status, "iters": r3.iters,
              "direct_iters": r3.direct_iters, "rel_gap": r3.rel_gap, "r1_l1": r3.r1_l1, "psi": r3.psi}

    pk_d, src = peaks()
    # pricing against its roofline: the FP32 ALU issue rate over 4 lane-ops per pair (whole call:
    # both scan passes, recheck, sorts and the host synchronisations)
    roof_gcols = SM_COUNT * FP32_LANES_PER_SM * pk_d.get("sm_max_mhz", 2070.0) * 1e6 / 4 / 1e9
    if big:
        big["frac_full_call"] = big["gcols_per_s"] / roof_gcols
    table = kernel_table(ktimes, pk_d, src)
    roof = roofline(table)
    # the pricing scan beside it (ALU-bound hot loop of the pricing)
    ptable = kernel_table(pk, pk_d, src)

    r0 = results[-1]
    line = {
        "metric": METRIC, "value": t_dev, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_dev * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "config": config_dict(args),
        "e2e": {"value": t_e2e, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches), "gpu_launches_per_solve": int(round(launches_per_solve)),
        "e2e_steps_s": e2e_times, "value_steps_s": dev_times,
        "solve": {"status": r0.status, "iters": r0.iters, "direct_iters": r0.direct_iters, "cg_iters": r0.cg_iters,
                  "rel_gap": r0.rel_gap, "r1_l1": r0.r1_l1, "obj": r0.obj, "psi": r0.psi, "max_fill_pct": r0.max_fill},
        "plain_fp64": plain,
        "plain_fp64_multiscale": plain_ms,
        "mixed_cold": mixed_cold,
        "mixed_learned_network": learned,
        "warm_start": {"kind": "multiscale (one coarser level, tol 1e-3)", "levels": r0.ms_levels,
                       "added_pairs": r0.warm_added, "dropped": r0.warm_restarts,
                       "create_seconds": r0.create_seconds, "solve_seconds": r0.seconds},
        "batch": batch,
        "pricing": {"gcols_per_s": gcols, "ms_per_call": price_ms, "pairs": pairs, "kernels": ptable,
                    "roofline_gcols_per_s": roof_gcols, "frac_full_call": gcols / roof_gcols,
                    "at_256x256": big},
        "pcg_at_256x256": pcg256,
        "config3_128x128_spikes": c3,
        "kernels": table,
        "roofline": roof,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle's exact network simplex (plain C, one host core), one complete solve of the
        # same instance: the fastest CPU oracle for this workload
        sec, pivots = oracle_simplex_solve(k, 0)
        line["cpu_baseline"] = {"value": sec, "unit": "s", "cores": 1, "kind": "oracle", "cpu": host_cpu(),
                                "sample": f"one complete exact solve of the same {k}x{k} instance by the oracle's "
                                          f"network simplex ({pivots} pivots); the oracle's rendition of the "
                                          f"method itself is timed by --impl reference"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 rate (nominal; no measured FP64 peak is available)


def kernel_table(ktimes, pk_d, src):
    """Per instrumented kernel: total ms, launches and achieved rate against its bound."""
    mhz = pk_d.get("sm_max_mhz", 2070.0)
    alu_peak = SM_COUNT * FP32_LANES_PER_SM * mhz * 1e6            # FP32 lane-ops/s
    hbm_peak = pk_d.get("hbm_gbs", 6800.0)                          # GB/s
    out = {}
    for name, (ms, cnt, work) in ktimes.items():
        if not cnt:
            continue
        row = {"ms": ms, "launches": cnt, "ms_per_launch": ms / cnt}
        sec = ms * 1e-3
        if name in ("scan_hist", "scan_gather") and work:
            row.update(bound="alu", achieved=work / sec / 1e12, peak=alu_peak / 1e12, unit="TFLOP/s",
                       frac=work / sec / alu_peak,
                       peak_source=f"152 SMs x 128 FP32 lanes x {mhz:.0f} MHz (unit counts)")
        elif name == "d32_factor" and work:
            # FP32 flops (n^3 per factorisation: 2n^3/3 for L D L^T, n^3/3 for L^-1); an FMA is 2 flops
            row.update(bound="alu", achieved=work / sec / 1e12, peak=2 * alu_peak / 1e12, unit="TFLOP/s",
                       frac=work / sec / (2 * alu_peak),
                       peak_source=f"152 SMs x 128 FP32 FMA lanes x 2 flops x {mhz:.0f} MHz (unit counts)")
        elif name in ("pcg32", "pcg64", "ldl_solve", "d32_apply", "dcg") and work:
            row.update(bound="hbm", achieved=work / sec / 1e9, peak=hbm_peak, unit="GB/s",
                       frac=work / sec / 1e9 / hbm_peak, peak_source=f"MEASURED_PEAKS.json hbm_gbs ({src})")
        elif name == "ldl_numeric" and work:
            row.update(bound="alu", achieved=work / sec / 1e12, peak=FP64_NOMINAL_TFLOPS, unit="TFLOP/s",
                       frac=work / sec / 1e12 / FP64_NOMINAL_TFLOPS, peak_source="nominal GB300 FP64 rate")
        out[name] = row
    return out


# DRAM bytes (read + write) per launch from one ncu capture of the kernel as it stands, and the
# summary under profiles/ that gives the command; a kernel changed since then reports null.
NCU_TRAFFIC = {
    # one FP32 factorisation (n = 4096, all 190 kernel launches of its graph): 1,600.5 MB read +
    # 0.15 MB written; profiles/d32_factor_64x64.md
    "d32_factor": 1.6007e9,
}


def roofline(table):
    """Roofline object of the dominant instrumented kernel (largest total device time)."""
    name, row = max(table.items(), key=lambda kv: kv[1]["ms"])
    return {"kernel": name, "bound": row.get("bound"), "achieved": row.get("achieved"), "peak": row.get("peak"),
            "unit": row.get("unit"), "frac": row.get("frac"), "traffic": NCU_TRAFFIC.get(name),
            "ms_per_launch": row["ms_per_launch"], "launches": row["launches"],
            "peak_source": row.get("peak_source")}


if __name__ == "__main__":
    sys.exit(main())
