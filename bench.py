#!/usr/bin/env python
"""Benchmark of the KCM step on B300: one line of JSON on rank 0.

Workload (default): the 1,000-residue synthetic chain (10,506 atoms) from its stored compact
random-walk start, 10 A cutoff, N = 256 solvation samples, mixed precision (FP32 pair and
solvation arithmetic; kinematics, wrenches and torque scans in double-float, ~48 significant bits). A step is one KCM iteration (forward
kinematics, binning, pair forces, Algorithm 1, wrenches and torque suffix sums, energies, step),
launched as a CUDA graph. Metric: atom-iterations per second, whole job (all ranks).

Timing: W warm-up steps, then K steps timed on the device with CUDA events on the library's
stream (each step is bracketed by events recorded by the library; a 256 MiB buffer is written
between steps to flush L2), max over ranks. Every step starts from the stored compact start: theta
is restored by a device-to-device copy before the step's first event. (Consecutive steps with the
configured clamp, kappa = 1e-3 and |dtheta| <= 0.02 rad on all 2,000 joints, push the unrelaxed
chain into overlapping atoms within one or two iterations, after which the pair and solvation
work is no longer that of the workload.) With torchrun (N > 1) every rank runs an independent
replica of the workload on its own GPU (chains are independent; there is no data-path exchange).

--impl reference times the FP64 CPU oracle on the same workload (rank 0 only), one oracle
iteration per step.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
GOLDEN = os.path.join(ROOT, "tests", "golden")

# the benchmark's headline metric: throughput of the mixed-precision step, with the plain FP64 GPU path
# beside it at the stated torque tolerance, and the serving loop's latency percentiles
METRIC = "atom-iterations/s vs plain FP64 at torque err\u22641e-4; served p50/p99 latency"
UNIT = "atom-iterations/s"
# FP32 lanes per SM on B300 (4 SM sub-partitions x 32 FP32 lanes); FMA = 2 flops
FP32_LANES_PER_SM = 128
FLOPS_PER_SASA_TEST = 9  # w = v - o (3), |w|^2 (1 mul + 2 FMA = 5), compare with Roff^2 (1)
FLOPS_PER_PAIR = 31      # per unordered pair within the cutoff (distance, 1/d^2, Coulomb, LJ, weights, accumulate)
STATUS_BYTES = 88  # the library's status record, read back with every step call
BYTES_PER_ATOM = {"kinematics": 80, "binning": 50, "torques_step": 60}  # algorithmic HBM bytes per atom
# DRAM bytes (read + write) per launch of the stage's main kernel on the 1,000-residue workload, from one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the kernel as it is built now; a stage
# left out has no capture of its current kernel
DRAM_BYTES_PER_LAUNCH = {"solvation": 6.84e6}
BATCH_ORACLE_STRIDE = 32  # chains of the batch checked against the oracle: 16 of 512
MIXED_DTYPE = "f32 pair/solvation; double-float (~48-bit) kinematics, wrenches and torque scans"


def kernels_per_iteration(binning_kind):
    """Launches of one mixed-precision iteration of a single chain with solvation on: reset + kinematics 2
    + binning (1 with the cluster kernel, 2 with the count and placement kernels) + pairs 1 + solvation 2
    (the main kernel and the long-list kernel beside it) + wrenches, torques and step 1."""
    from paper_1712_05012_b300 import kcm

    return 1 + 2 + (1 if binning_kind == kcm.BIN_CLUSTER else 2) + 1 + 2 + 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=20)
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--chain8000-steps", type=int, default=20)
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-iters", type=int, default=200)
    ap.add_argument("--cell-edge", type=float, default=0.0, metavar="A",
                    help="cell edge (A) of the 1,000-residue and batch legs instead of the cell-edge autotuner's "
                         "choice (for profiling runs, where ncu's serialised launches distort the autotuner)")
    ap.add_argument("--profile-batch", type=int, default=0, metavar="K",
                    help="profiling workload only: the first K chains of the batch workload, mixed precision, "
                         "stepped from their stored starts four times (a few GB on the device for one-kernel ncu "
                         "captures); prints one line of sizes, no measurement")
    return ap.parse_args()


def workload():
    from paper_1712_05012_b300 import synth

    man = json.load(open(os.path.join(GOLDEN, "starts.json")))["chain1000"]
    seq = synth.sequence(man["residues"], man["sequence_seed"])
    theta = synth.theta_from_codes(np.load(os.path.join(GOLDEN, "start_chain1000.npy")))
    return seq, theta, man


def batch_workload():
    """The 512-chain batch (lengths 30-600 residues) and its stored compact starts, concatenated."""
    from paper_1712_05012_b300 import synth

    wl = synth.workload(4)
    seqs = [synth.sequence(m, synth.chain_seed(wl.seed, i)) for i, m in enumerate(wl.m)]
    theta = synth.theta_from_codes(np.load(os.path.join(GOLDEN, "start_batch512.npy")))
    return seqs, theta, wl


def serve_pool():
    """The pool of serving jobs (lengths log-uniform in 20-2000 residues) and their stored starts."""
    from paper_1712_05012_b300 import synth

    wl = synth.workload(5)
    lens = json.load(open(os.path.join(GOLDEN, "starts.json")))["serve256"]["residues"]
    codes = np.load(os.path.join(GOLDEN, "start_serve256.npy"))
    seqs, thetas, off = [], [], 0
    for i, m in enumerate(lens):
        seqs.append(synth.sequence(m, synth.chain_seed(wl.seed, i)))
        thetas.append(synth.theta_from_codes(codes[off:off + 2 * m]))
        off += 2 * m
    return seqs, thetas, wl


def run_serving(kcm, table, params, rate, seconds, max_iters, budget, chunk, seed=0, admission=(1, 0.0)):
    """Poisson arrivals at `rate` jobs/s for `seconds` (jobs drawn from the pool), each run until
    converged or `max_iters`; returns latencies and throughput from the server's own clock."""
    seqs, thetas, _ = serve_pool()
    rng = np.random.default_rng(seed)
    t_arr = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * seconds * 3) + 16))
    t_arr = t_arr[t_arr < seconds]
    pick = rng.integers(0, len(seqs), size=len(t_arr))
    ids = []
    with kcm.Server(params, budget, 512, chunk) as s:
        s.set_admission(*admission)
        t0 = time.perf_counter()
        k = 0
        while True:
            now = time.perf_counter() - t0
            while k < len(t_arr) and t_arr[k] <= now:
                ids.append(s.submit(seqs[pick[k]], table, thetas[pick[k]], max_iters))
                k += 1
            waiting, running = s.tick()
            if k == len(t_arr) and waiting == 0 and running == 0:
                break
            time.sleep(0.0005)
        wall = time.perf_counter() - t0
        info = [s.job(j, with_theta=False) for j in ids]
    lat = np.array([x["t_done"] - x["t_submit"] for x in info])
    queue = np.array([x["t_admit"] - x["t_submit"] for x in info])
    atom_its = sum(x["natoms"] * x["iters"] for x in info)
    return {"jobs": len(ids), "rate_per_s": rate, "arrival_seconds": seconds, "max_iters": max_iters,
            "wall_s": wall, "chains_per_s": len(ids) / wall, "atom_iterations_per_s": atom_its / wall,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "p50_queue_s": float(np.percentile(queue, 50)), "converged": int(sum(x["converged"] for x in info)),
            "errors": int(sum(x["error"] != 0 for x in info)),
            "error_codes": sorted({int(x["error"]) for x in info if x["error"] != 0}),
            "admission": {"min_jobs": admission[0], "max_wait_s": admission[1]}}


def run_serving_converging(kcm, table, rate=200.0, seconds=0.5, max_iters=3000, conv_tol=1e-3, seed=2):
    """A stream whose jobs reach the convergence test: short chains (10-40 residues, the same generator)
    from the extended start in vacuum (smooth forces; with Algorithm 1's piecewise-constant solvation
    forces the clamped step ends in a cycle at the clamp instead), max |dtheta| < conv_tol = 1e-3 rad or
    3,000 iterations, Poisson arrivals. Reports how many retired on convergence, and their latencies."""
    from paper_1712_05012_b300 import synth

    rng = np.random.default_rng(seed)
    t_arr = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * seconds * 3) + 16))
    t_arr = t_arr[t_arr < seconds]
    lens = rng.integers(10, 41, size=len(t_arr))
    params = synth.RunParams(precision=synth.PRECISION_MIXED, solvation=0, conv_tol=conv_tol)
    ids = []
    with kcm.Server(params, 8 << 30, 512, 50) as s:
        t0 = time.perf_counter()
        k = 0
        while True:
            now = time.perf_counter() - t0
            while k < len(t_arr) and t_arr[k] <= now:
                m = int(lens[k])
                ids.append(s.submit(synth.sequence(m, 7000 + k), table, synth.theta_extended(m), max_iters))
                k += 1
            waiting, running = s.tick()
            if k == len(t_arr) and waiting == 0 and running == 0:
                break
            time.sleep(0.0005)
        wall = time.perf_counter() - t0
        info = [s.job(j, with_theta=False) for j in ids]
    lat = np.array([x["t_done"] - x["t_submit"] for x in info])
    conv = [x for x in info if x["converged"]]
    return {"jobs": len(ids), "rate_per_s": rate, "arrival_seconds": seconds, "max_iters": max_iters,
            "conv_tol": conv_tol, "wall_s": wall, "chains_per_s": len(ids) / wall,
            "converged": len(conv), "mean_iters_converged": float(np.mean([x["iters"] for x in conv])) if conv else None,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "errors": int(sum(x["error"] != 0 for x in info)),
            "note": "10-40 residues, extended start, vacuum, mixed precision"}


def max_over_ranks(t_local: float, ws: int, device: str = "cuda") -> float:
    """The largest of every rank's timed seconds (all_reduce MAX over the default process group;
    the tensor lives on `device`: CUDA for NCCL, CPU for gloo)."""
    if ws <= 1:
        return t_local
    import torch
    import torch.distributed as dist

    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws: int, units_per_rank: int, steps: int, t_max: float) -> float:
    """Units processed by all ranks (every rank runs its own replica of the workload) per second of
    the slowest rank."""
    return ws * units_per_rank * steps / t_max


def rel_err(got, ref):
    """max |got - ref| / max |ref|"""
    return float(np.max(np.abs(np.asarray(got) - np.asarray(ref))) / np.max(np.abs(ref)))


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or parts[0] != str(self.index):
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_baseline(seq, theta, params, budget_s=12.0, budget_1core_s=8.0):
    """The oracle (FP64, all-pairs, OpenMP over atoms) on the machine's host cores: KCM iterations of
    the same workload for about `budget_s` seconds on all cores, then about `budget_1core_s` on one."""
    from oracle import oracle as O
    from paper_1712_05012_b300 import synth

    table = synth.type_table()
    ch = O.OracleChain(seq, table, synth.GEOMETRY)

    def timed(budget):
        t0 = time.perf_counter()
        ch.run(params, np.array(theta), 1)
        t1 = time.perf_counter() - t0
        iters = max(1, min(200, int(budget / max(t1, 1e-6))))
        t0 = time.perf_counter()
        for _ in range(iters):  # each iteration from the stored start, as the GPU steps are timed
            ch.run(params, np.array(theta), 1)
        return iters, time.perf_counter() - t0

    cores = O.num_threads()
    iters, wall = timed(budget_s)
    O.set_threads(1)
    iters1, wall1 = timed(budget_1core_s)
    O.set_threads(cores)
    return {"value": ch.n * iters / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "value_1core": ch.n * iters1 / wall1,
            "sample": f"{iters} FP64 oracle iterations of the 1,000-residue chain ({ch.n} atoms) on {cores} threads, "
                      f"{wall:.1f} s wall, and {iters1} on 1 thread, {wall1:.1f} s wall; each iteration from "
                      f"the compact start"}, ch


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_1712_05012_b300 import synth

    seq, theta, man = workload()
    table = synth.type_table()
    ch = O.OracleChain(seq, table, synth.GEOMETRY)
    p = synth.RunParams(precision=synth.PRECISION_FP64)
    for _ in range(args.warmup):
        ch.run(p, np.array(theta), 1)
    times = []
    for _ in range(args.steps):
        th = np.array(theta)  # each step from the stored start, as the GPU arm does
        t0 = time.perf_counter()
        ch.run(p, th, 1)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = ch.n * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "chain1000_compact_cut10", "residues": 1000, "atoms": ch.n, "cutoff": 10.0,
                       "n_sample": 256, "solvation": 1, "precision": "fp64 (oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"one full FP64 oracle iteration per step ({ch.n} atoms)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def time_steps(c, prep, stream, steps):
    """Device time (ms) of each of `steps` whole iterations: the loop-state reset and every kernel of one
    iteration, between two CUDA events on the library's stream. The restore of the start conformation
    and the L2 flush before each step are outside the events."""
    import torch

    evs = []
    for _ in range(steps):
        prep()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.step_async(1)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    c.step_status()  # raises if the device flagged an error
    return [a.elapsed_time(b) for a, b in evs]


def stage_breakdown(c, prep, steps):
    """Mean per-stage device time (ms) over `steps` instrumented iterations (a CUDA event between stages;
    each event node adds about 3 us to the iteration, so these stages sum to more than a plain step)."""
    from paper_1712_05012_b300 import kcm

    stg = {k: 0.0 for k in kcm.STAGES}
    for _ in range(steps):
        prep()
        _, st = c.step_timed()
        for k, v in st.items():
            stg[k] += v
    return {k: v / steps for k, v in stg.items()}


def stage_rooflines(ms_stage, stats, n, fp32_peak, peaks, sasa_tests=None):
    """Achieved rate of every stage against its bound: the FP32 pipes for the pair terms and Algorithm 1's
    tests, HBM for the rest (algorithmic bytes per atom). Algorithm 1's work is its overlap tests as the
    algorithm performs them (step 1 stopping at the second overlap, step 2's re-tests), counted by the
    oracle at the same conformation when `sasa_tests` is given; otherwise the kernel's own count (every
    valid point against every neighbour, no early exit: an upper bound on the algorithm's tests)."""
    rooflines = {}
    for stage, ms in ms_stage.items():
        sec = ms / 1e3
        if stage == "solvation":
            tests = sasa_tests if sasa_tests is not None else stats["sasa_tests"]
            work = tests * FLOPS_PER_SASA_TEST
            r = {"bound": "alu", "achieved": work / sec / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                 "peak_source": "FP32 FMA: SMs x 128 lanes x 2 x max SM clock",
                 "work_source": ("Algorithm 1 tests as performed (oracle count)" if sasa_tests is not None
                                 else "kernel count (every valid point x every neighbour)")}
        elif stage == "pairs":
            work = stats["pairs"] * FLOPS_PER_PAIR
            r = {"bound": "alu", "achieved": work / sec / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                 "peak_source": "FP32 FMA: SMs x 128 lanes x 2 x max SM clock"}
        else:
            work = BYTES_PER_ATOM[stage] * n
            r = {"bound": "hbm", "achieved": work / sec / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)"}
        r["frac"] = r["achieved"] / r["peak"]
        r["ms_per_launch"] = ms
        r["work_per_launch"] = work
        rooflines[stage] = r
    return rooflines


def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1712_05012_b300 import kcm, synth

    table = synth.type_table()
    seq, theta, man = workload()
    prec = synth.PRECISION_MIXED if args.precision == "mixed" else synth.PRECISION_FP64
    params = synth.RunParams(precision=prec)
    ch = kcm.Chain(seq, table, params)
    ch.set_theta(theta)
    n = ch.n
    lib_stream = torch.cuda.ExternalStream(ch.stream())
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")  # 256 MiB > 126 MB L2
    theta0 = torch.tensor(theta, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()

    def prepare(c, stream):
        # untimed: restore the start conformation and flush L2 on the library's stream
        c.set_theta_dev(theta0.data_ptr(), c.l)
        with torch.cuda.stream(stream):
            flush.add_(1)

    # pair kernel (warp per atom or cell-pair tiles) and tile shapes from the library's autotuner, at the
    # start conformation, before the warm-up
    prepare(ch, lib_stream)
    cell_cands = (args.cell_edge,) if args.cell_edge > 0 else (6.0, 7.0, 8.0, 9.0, 10.0, 12.0)
    cell_main, cell_main_ms = ch.autotune_cell(candidates=cell_cands, reps=20)
    prepare(ch, lib_stream)
    kind, kind_ms = ch.autotune_pair_kernel(reps=10)
    bin_kind, bin_ctas = ch.get_binning_kernel()
    tiles = {"used": list(ch.get_tiles()), "choices": list(kcm.TILE_CHOICES), "source": "autotuner",
             "pair_kernel": ("cell_tiles" if kind == kcm.PAIR_CELL_TILES else "warp_per_atom"),
             "pair_kernel_ms": {"warp_per_atom": float(kind_ms[0]), "cell_tiles": float(kind_ms[1])},
             "binning_kernel": {"kind": "cluster" if bin_kind == kcm.BIN_CLUSTER else "blocks", "ctas": bin_ctas},
             "cell_autotune_ms": dict(zip([f"{x:g}" for x in cell_cands], [float(x) for x in cell_main_ms]))}
    # the torques at the start conformation, compared with the oracle's in the oracle leg
    prepare(ch, lib_stream)
    tau_start = ch.torques()
    clocks = Clocks(local)
    prep_main = lambda: prepare(ch, lib_stream)  # noqa: E731
    for _ in range(args.warmup):
        prep_main()
        ch.step_timed()
        prep_main()
        ch.step(1)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    totals = time_steps(ch, prep_main, lib_stream, args.steps)
    ms_stage = stage_breakdown(ch, prep_main, args.steps)
    clk = clocks.stop()
    stats = ch.stats()
    # end to end through the C ABI with pinned host buffers: the start theta in, one step, theta out
    # (right after the device-timed steps, on the same handle, before the other legs' handles exist)
    pin_in = torch.empty(ch.l, dtype=torch.float64, pin_memory=True)
    pin_in.copy_(torch.from_numpy(theta))
    pin_out = torch.empty(ch.l, dtype=torch.float64, pin_memory=True)
    L = kcm.load()
    import ctypes
    din = ctypes.cast(pin_in.data_ptr(), ctypes.POINTER(ctypes.c_double))
    dout = ctypes.cast(pin_out.data_ptr(), ctypes.POINTER(ctypes.c_double))
    e2e_steps = max(args.steps, 20)
    it_out = (ctypes.c_int32 * 1)()
    dm_out = (ctypes.c_double * 1)()
    for _ in range(3):
        L.kcm_step_host(ch.handle, din, dout, ch.l, 1, it_out, dm_out)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        if L.kcm_step_host(ch.handle, din, dout, ch.l, 1, it_out, dm_out):
            raise RuntimeError("kcm call failed during the end-to-end run")
    e2e_wall = time.perf_counter() - t0
    # the same round trip as three calls (kcm_set_theta, kcm_step, kcm_get_theta), each with its own wait
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        rc = L.kcm_set_theta(ch.handle, din, ch.l)
        rc |= L.kcm_step(ch.handle, 1, it_out, dm_out)
        rc |= L.kcm_get_theta(ch.handle, dout, ch.l)
        if rc:
            raise RuntimeError("kcm call failed during the end-to-end run")
    e2e_wall3 = time.perf_counter() - t0
    e2e = {"value": ws * n * e2e_steps / e2e_wall, "unit": UNIT, "h2d_bytes_per_step": 8 * ch.l,
           "d2h_bytes_per_step": 8 * ch.l + STATUS_BYTES, "steps": e2e_steps,
           "value_three_calls": ws * n * e2e_steps / e2e_wall3,
           "note": "per step: kcm_step_host from pinned host buffers (the start theta read by the first "
                   "kernel from the handle's page-locked mapped buffer, one iteration, theta and the status "
                   "record written back to host memory by the kernels: one graph launch, one wait); host "
                   "wall clock. value_three_calls: kcm_set_theta, kcm_step, kcm_get_theta"}
    t_sum = max_over_ranks(sum(totals) / 1e3, ws)
    value = whole_job_rate(ws, n, args.steps, t_sum)

    # roofline denominators (the rooflines themselves are formed after the oracle leg, which counts
    # Algorithm 1's tests at the start conformation)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sm_max = (clk or {}).get("sm_max_mhz") or 2032.0
    fp32_peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6400.0}

    # the same step with solvation off (the paper's vacuum runs), measured the same way
    vacuum_value = None
    if args.fp64_steps > 0:
        with kcm.Chain(seq, table, synth.RunParams(precision=prec, solvation=0)) as cv:
            sv = torch.cuda.ExternalStream(cv.stream())
            prepare(cv, sv)
            cv.autotune_pair_kernel(reps=3)  # kernel and tile shapes chosen as on the headline leg
            for _ in range(3):
                prepare(cv, sv)
                cv.step(1)
            tt = time_steps(cv, lambda: prepare(cv, sv), sv, args.fp64_steps)
            vacuum_value = n * args.fp64_steps / (sum(tt) / 1e3)

    # the same step with the pairwise solvation surrogate instead of the enumeration, measured the same way
    surrogate_value = None
    if args.fp64_steps > 0:
        with kcm.Chain(seq, table, synth.RunParams(precision=prec, solvation=2)) as cs:
            ss = torch.cuda.ExternalStream(cs.stream())
            prepare(cs, ss)
            cs.autotune_pair_kernel(reps=3)
            for _ in range(3):
                prepare(cs, ss)
                cs.step(1)
            tt = time_steps(cs, lambda: prepare(cs, ss), ss, args.fp64_steps)
            surrogate_value = n * args.fp64_steps / (sum(tt) / 1e3)

    # the same step with the side-chain joints on (chi_1..chi_4 per residue, stepped with the main chain),
    # each step from the same start (chi = 0), measured the same way
    side_value = None
    if args.fp64_steps > 0:
        with kcm.Chain(seq, table, synth.RunParams(precision=prec, side_joints=1)) as cx:
            sx = torch.cuda.ExternalStream(cx.stream())
            chi0 = torch.zeros(cx.ls, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()

            def prep_x():
                cx.set_side_theta_dev(chi0.data_ptr())
                prepare(cx, sx)

            prep_x()
            cx.autotune_pair_kernel(reps=3)
            for _ in range(3):
                prep_x()
                cx.step(1)
            tt = time_steps(cx, prep_x, sx, args.fp64_steps)
            side_value = n * args.fp64_steps / (sum(tt) / 1e3)

    # the 8,000-residue chain (83,746 atoms, 12 A cutoff), the cell edge chosen by the autotuner among
    # 6-12 A, measured the same way, with its FP64 path beside it
    chain8000 = None
    if args.chain8000_steps > 0:
        man8 = json.load(open(os.path.join(GOLDEN, "starts.json")))["chain8000"]
        seq8 = synth.sequence(man8["residues"], man8["sequence_seed"])
        th8 = torch.tensor(synth.theta_from_codes(np.load(os.path.join(GOLDEN, "start_chain8000.npy"))),
                           dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        leg = {"workload": "chain8000_compact_cut12", "residues": man8["residues"]}
        for name, pr in (("mixed", synth.PRECISION_MIXED), ("fp64", synth.PRECISION_FP64)):
            with kcm.Chain(seq8, table, synth.RunParams(precision=pr, cutoff=12.0)) as c8:
                s8 = torch.cuda.ExternalStream(c8.stream())

                def prep8():
                    c8.set_theta_dev(th8.data_ptr(), c8.l)
                    with torch.cuda.stream(s8):
                        flush.add_(1)

                prep8()
                cell, cand_ms = c8.autotune_cell(candidates=(6.0, 7.0, 8.0, 9.0, 10.0, 12.0), reps=3)
                kind8, _ = c8.autotune_pair_kernel(reps=3)
                tiles8 = c8.get_tiles()
                if name == "mixed":
                    prep8()
                    tau8_start = c8.torques()
                steps8 = args.chain8000_steps if name == "mixed" else max(2, args.chain8000_steps // 10)
                for _ in range(3):
                    prep8()
                    c8.step(1)
                tt = time_steps(c8, prep8, s8, steps8)
                st8 = c8.stats()
                r = {"value": ws * c8.n * steps8 / (sum(tt) / 1e3), "ms_per_step": sum(tt) / steps8,
                     "steps": steps8, "cell_size": cell, "autotune_ms": dict(zip(("6", "7", "8", "9", "10", "12"),
                                                                             [float(x) for x in cand_ms])),
                     "pairs": st8["pairs"], "sasa_tests": st8["sasa_tests"], "tiles": list(tiles8),
                     "pair_kernel": "cell_tiles" if kind8 == kcm.PAIR_CELL_TILES else "warp_per_atom"}
                if name == "mixed":
                    stg8 = stage_breakdown(c8, prep8, steps8)
                    r["stage_ms"] = stg8
                    r["rooflines"] = stage_rooflines(stg8, st8, c8.n, fp32_peak, peaks)
                leg["atoms"] = c8.n
                leg[name] = r
        leg["speedup_vs_fp64"] = leg["mixed"]["value"] / leg["fp64"]["value"]
        chain8000 = leg

    # the batch workload: 512 chains stepped together, one launch per stage, measured the same way
    batch = None
    if args.batch_steps > 0:
        bseqs, btheta, bwl = batch_workload()
        with kcm.Batch(bseqs, table, synth.RunParams(precision=prec)) as bb:
            sb = torch.cuda.ExternalStream(bb.stream())
            bth0 = torch.tensor(btheta, dtype=torch.float64, device="cuda")

            def prep_b():
                bb.set_theta_dev(bth0.data_ptr(), bb.l)
                with torch.cuda.stream(sb):
                    flush.add_(1)

            prep_b()
            bcell, bcand_ms = bb.autotune_cell(candidates=cell_cands, reps=2)
            prep_b()
            bkind, bkind_ms = bb.autotune_pair_kernel(reps=2)
            btiles = bb.get_tiles()
            prep_b()
            btau_start = bb.split(bb.torques(), per="joint")  # compared with the oracle's in the oracle leg
            bthetas = bb.split(np.asarray(btheta), per="joint")
            for _ in range(3):
                prep_b()
                bb.step_timed()
                prep_b()
                bb.step(1)
            tt = time_steps(bb, prep_b, sb, args.batch_steps)
            stg = stage_breakdown(bb, prep_b, args.batch_steps)
            bst = bb.stats()
            batch = {"workload": bwl.name, "chains": bb.nchains, "atoms": bb.n, "residues": int(sum(bwl.m)),
                     "value": ws * bb.n * args.batch_steps / (sum(tt) / 1e3), "unit": UNIT,
                     "ms_per_step": sum(tt) / args.batch_steps,
                     "stage_ms": stg,
                     "steps": args.batch_steps, "pairs": bst["pairs"], "sasa_tests": bst["sasa_tests"],
                     "cell_size": bcell, "autotune_ms": dict(zip([f"{x:g}" for x in cell_cands],
                                                                  [float(x) for x in bcand_ms])),
                     "rooflines": stage_rooflines(stg, bst, bb.n, fp32_peak, peaks),
                     "tiles": {"chosen": list(btiles), "order": "[pair warps or tile split][solvation warps][persistent pair grid]",
                               "pair_kernel": "cell_tiles" if bkind == kcm.PAIR_CELL_TILES else "warp_per_atom",
                               "pair_kernel_ms": {"warp_per_atom": float(bkind_ms[0]), "cell_tiles": float(bkind_ms[1])}},
                     "start": "every step from the stored compact starts (theta restored untimed)"}

    # serving: Poisson arrivals into the continuous-batching server, next to the same jobs one at a time
    serving = None
    if args.serve_seconds > 0:
        sp = synth.RunParams(precision=prec)
        serving = run_serving(kcm, table, sp, 200.0, args.serve_seconds, args.serve_iters, 120 << 30, 25)
        seqs_p, thetas_p, _ = serve_pool()
        rng = np.random.default_rng(1)
        one = []  # one job at a time, plain FP64 single-chain path, a sample of the pool
        for i in rng.integers(0, len(seqs_p), size=6):
            t0 = time.perf_counter()
            with kcm.Chain(seqs_p[i], table, synth.RunParams(precision=synth.PRECISION_FP64)) as c1:
                c1.set_theta(thetas_p[i])
                try:
                    it1, _ = c1.step(args.serve_iters)
                except kcm.KcmError:  # the job failed (e.g. its chain collapsed): count what it ran
                    it1 = int(c1.chain_state()[0][0])
                one.append((time.perf_counter() - t0, c1.n * it1))
        serving["one_at_a_time_fp64"] = {
            "jobs": len(one), "mean_latency_s": float(np.mean([x[0] for x in one])),
            "atom_iterations_per_s": float(sum(x[1] for x in one) / sum(x[0] for x in one))}
        serving["note"] = (f"jobs drawn from 256 stored compact starts, lengths log-uniform 20-2000 residues; "
                           f"capped at {args.serve_iters} iterations (5,000 in the full stream); 120 GB budget; "
                           f"server clock")
        serving["converging_stream"] = run_serving_converging(kcm, table)

    # the plain FP64 single-chain GPU path, measured the same way
    fp64_value = None
    if args.fp64_steps > 0 and prec == synth.PRECISION_MIXED:
        with kcm.Chain(seq, table, synth.RunParams(precision=synth.PRECISION_FP64)) as c64:
            s64 = torch.cuda.ExternalStream(c64.stream())
            for _ in range(3):
                prepare(c64, s64)
                c64.step(1)
            tt = time_steps(c64, lambda: prepare(c64, s64), s64, args.fp64_steps)
            fp64_value = n * args.fp64_steps / (sum(tt) / 1e3)

    ch.close()

    # the oracle leg (rank 0, one GPU, host cores): the CPU baseline, and one FP64 oracle evaluation at
    # the start conformation of the timed workloads, for the torque error of the GPU path's result and
    # Algorithm 1's test count
    cpu, accuracy, sasa_oracle = None, None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, och = oracle_baseline(seq, theta, synth.RunParams(precision=synth.PRECISION_FP64))
        t0 = time.perf_counter()
        ref = och.evaluate(synth.RunParams(precision=synth.PRECISION_FP64), theta)
        accuracy = {"reference": "FP64 oracle at the start conformation (max-norm relative torque error)",
                    "chain1000": {"torque_rel_err": rel_err(tau_start, ref["tau"]),
                                  "oracle_s": time.perf_counter() - t0}}
        sasa_oracle = ref["stats"]["sasa_tests1"] + ref["stats"]["sasa_tests2"]
        if chain8000 is not None:
            from oracle import oracle as O
            t0 = time.perf_counter()
            o8 = O.OracleChain(seq8, table, synth.GEOMETRY)
            ref8 = o8.evaluate(synth.RunParams(precision=synth.PRECISION_FP64, cutoff=12.0), th8.cpu().numpy())
            accuracy["chain8000"] = {"torque_rel_err": rel_err(tau8_start, ref8["tau"]),
                                     "oracle_s": time.perf_counter() - t0}
            chain8000["mixed"]["rooflines"] = stage_rooflines(
                chain8000["mixed"]["stage_ms"], {"pairs": chain8000["mixed"]["pairs"]}, chain8000["atoms"],
                fp32_peak, peaks, ref8["stats"]["sasa_tests1"] + ref8["stats"]["sasa_tests2"])
        if batch is not None:  # a sample of the batch's chains, each against the oracle alone
            from oracle import oracle as O
            t0 = time.perf_counter()
            sample = list(range(0, len(bseqs), BATCH_ORACLE_STRIDE))
            errs = [rel_err(btau_start[c], O.OracleChain(bseqs[c], table, synth.GEOMETRY).evaluate(
                synth.RunParams(precision=synth.PRECISION_FP64), bthetas[c])["tau"]) for c in sample]
            accuracy["batch"] = {"torque_rel_err": max(errs), "chains": len(sample),
                                 "sample": f"chains 0, {BATCH_ORACLE_STRIDE}, {2 * BATCH_ORACLE_STRIDE}, ... of the batch, each against the "
                                           f"FP64 oracle alone; the largest error",
                                 "oracle_s": time.perf_counter() - t0}

    # rooflines of every stage; the dominant one is the headline "roofline"
    rooflines = stage_rooflines(ms_stage, stats, n, fp32_peak, peaks, sasa_oracle)
    dom = max(ms_stage, key=ms_stage.get)
    roof = {k: v for k, v in rooflines[dom].items()}
    roof["kernel"] = dom
    roof["traffic"] = DRAM_BYTES_PER_LAUNCH.get(dom)

    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_sum / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": MIXED_DTYPE if prec == synth.PRECISION_MIXED else "f64",
                "data": "synthetic",
                "config": {"workload": "chain1000_compact_cut10", "residues": 1000, "atoms": n, "cutoff": 10.0,
                           "n_sample": 256, "solvation": 1, "precision": args.precision,
                           "replicas": ws, "l2": "flushed between timed steps (256 MiB write)",
                           "start": "every step from the stored compact start (theta restored untimed)"},
                "roofline": roof, "rooflines": rooflines, "stage_ms": ms_stage,
                "stage_note": "stage_ms from a second pass of the same steps with a CUDA event between stages "
                              "(each event node adds ~3 us); value and ms_per_step time whole steps only",
                "fp64_value": fp64_value, "surrogate_value": surrogate_value, "side_joints_value": side_value,
                "vacuum_value": vacuum_value, "tiles": tiles, "chain8000": chain8000, "batch": batch, "serving": serving,
                "speedup_vs_fp64": (value / ws / fp64_value) if fp64_value else None,
                "cpu_baseline": cpu, "accuracy": accuracy, "e2e": e2e, "gpu_launches": kernels_per_iteration(bin_kind) * args.steps,
                "clocks": clk, "stats": {k: stats[k] for k in ("pairs", "sasa_tests", "sasa_neighbors",
                                                                 "max_neighbors", "guard_rechecks", "cells")},
                "cell_size": stats["cell_size"]}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_profile_batch(k):
    """The first k chains of the batch workload, stepped four times from their stored starts: a small
    case of the batch's kernels for ncu captures that collect more than launch times."""
    import torch

    from paper_1712_05012_b300 import kcm, synth

    torch.cuda.set_device(0)
    seqs, theta, _ = batch_workload()
    with kcm.Batch(seqs[:k], synth.type_table(), synth.RunParams(precision=synth.PRECISION_MIXED)) as bb:
        for _ in range(4):
            bb.set_theta(theta[:bb.l])  # the chains' joints come first in the concatenated starts
            bb.step(1)
        torch.cuda.synchronize()
        print(json.dumps({"profile_batch": {"chains": bb.nchains, "atoms": bb.n, "joints": bb.l, "steps": 4}}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_batch > 0:
        return run_profile_batch(args.profile_batch)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
