"""Benchmark: RJMCMC proposals/s of the path-integral chain kernel on GB300.

One bench step is one pass of the whole hot path over one batch: chain
initialisation, n_steps RJMCMC steps of every chain (random numbers, move
choice, perturb / birth / death, delta log-density, accept, estimator
accumulation) and the per-pair estimator reduction.  The default workload is
the detector-scale pair: source-sensor distance 50 m, sensor radius 0.165 m,
scattering length 5 m, absorption length 100 m, g = 0.94, 65,536 chains x
100,000 steps, vertex cap 256.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the host cores on the same workload and metric (bounded sample per step).
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

METRIC = "RJMCMC proposals/s"
UNIT = "proposals/s"

# Algorithmic work of one proposal, per move type, counted from the method's
# formulas: FP32 operations of the proposal and of the changed factors
# (O(n) scans for births and deaths, n the vertex count), the integer work of
# the two Philox4x32-10 blocks every step draws (2 blocks x 10 rounds x 6
# multiply / xor operations), and special-function (MUFU) operations.  The
# lane-op roofline bounds a proposal by max((FP32 + INT) / (128 N_SM f),
# MUFU / (16 N_SM f)) at SM clock f.
LANE_OPS = {"perturb": (90.0, 8.0), "birth": (150.0, 16.0), "death": (130.0, 14.0)}  # FP32 (+ n), MUFU
INT_PER_PROPOSAL = 120.0
# The same FP32 count from the delta evaluator's own formulas (interior / end
# vertex moves, births, deaths), without the integer work.
FP32_PER_PROPOSAL = {"interior": 145.0, "end": 95.0, "birth": 206.0, "death": 122.0}
FP32_LANES_PER_SM = 128
MUFU_LANES_PER_SM = 16
ISSUE_PER_CLK_PER_SM = 4

WORKLOAD_TEXT = {
    "detector": "detector: 1 pair, D=50 m, R=0.165 m, lambda_s=5 m, lambda_a=100 m, g=0.94, 65,536 chains x "
                "100,000 steps, cap 256",
    "plain": "plain: 1 pair, D=1 m, R=0.1 m, lambda_s=0.5 m, lambda_a=5 m, g=0.9, cap 64",
    "gradients": "gradients: plain geometry, MALA eps=0.02 m, 65,536 chains, score accumulation",
    "batched": "batched: 4,096 pairs, D~U(5,150) m, chains~U{16..512}, caps 64..1024, lambda_s=0.5 m, "
               "lambda_a=5 m, g=0.9",
    "layered": "layered: 100 x 10 m layers, 60 sensors x 8,192 chains, cap 1,024, g=0.94",
}

# Counters of the lane kernel on the detector workload from an ncu capture,
# valid only for the kernel source they were taken from (sha256 of
# csrc/pmc_lane.cu, csrc/pmc_device.cuh, csrc/pmc_tree.cuh and
# csrc/pmc_internal.h, in that order): warp instructions per proposal and DRAM
# bytes (read + write) of one 65,536-chain x 100,000-step launch (window 20).
# With another source the bench reports them as null.
LANE_CAPTURE = {"source_sha256": "3364a28ea771d3f3e2ca9e7e8bde99009a16bde4c14f1235f194a05bdfa0842b",
                "inst_per_proposal": 49.53, "dram_bytes_per_launch": 79878400.0,
                "capture": "ncu dram__bytes_read.sum + dram__bytes_write.sum (57.2 MB + 22.7 MB) of one "
                           "65,536-chain x 100,000-step launch, window 20, 2 warps per CTA"}


def lane_kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in ("pmc_lane.cu", "pmc_device.cuh", "pmc_tree.cuh", "pmc_internal.h"):
        with open(os.path.join(ROOT, "paper_1811_04156_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def parse(argv=None):
    return parse_args(argv)


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="detector")
    p.add_argument("--chains", type=int, default=65_536)
    p.add_argument("--run-steps", type=int, default=100_000)
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU-baseline sample budget")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the other workloads' rates and the time-to-1%% comparison after the timed steps")
    p.add_argument("--ttt-limit", type=float, default=25.0, help="seconds per method of the time-to-target runs")
    p.add_argument("--warps-per-block", type=int, default=0)
    p.add_argument("--within", choices=["default", "perturb", "mala", "tree"], default="default",
                   help="within-dimension moves of the timed workload (default: the workload's own)")
    p.add_argument("--layout", choices=["auto", "warp", "lane"], default="auto",
                   help="chain layout of the kernel: the autotuner's choice, one warp or one lane per chain")
    p.add_argument("--smem-window", type=int, default=0,
                   help="vertices per chain in shared memory (0: whole cap, or the autotuner's choice)")
    p.add_argument("--time-to-target", type=float, default=0.0,
                   help="instead of the throughput line: wall time to this relative intensity error for plain "
                        "RJMCMC, batched MALA chains and the GPU forward tracer on the plain / detector geometry")
    p.add_argument("--geometry", default="plain", help="geometry of --time-to-target: plain or detector")
    p.add_argument("--ttt-methods", default="",
                   help="comma list of --time-to-target methods to run (default all): plain_rjmcmc, batched_mala, "
                        "batched_mala_tracer_seeded, batched_perturb_tracer_seeded, batched_tree_moves, "
                        "tree_moves_optimal_bridge, gpu_tracer")
    p.add_argument("--ttt-ref", default="",
                   help="I,se,photons of a reference tracer run to use instead of running it again")
    p.add_argument("--two-sensor", action="store_true",
                   help="instead of the throughput line: the paper's two-sensor scene (relative light yield B "
                        "through the map T and path-length distributions for each b1, beside the GPU tracer)")
    p.add_argument("--ts-b1", default="0.1,0.2,0.3,0.4,0.5")
    p.add_argument("--ts-chains", type=int, default=2048, help="chains per sensor")
    p.add_argument("--ts-steps", type=int, default=1_000_000, help="steps per chain (10%% burn-in)")
    p.add_argument("--ts-thin", type=int, default=200, help="steps between observations of B and lengths")
    p.add_argument("--ts-photons", type=int, default=0, help="tracer photons per sensor and b1 (0: no tracer)")
    p.add_argument("--ts-out", default="", help="file for the full result (histograms included)")
    p.add_argument("--ts-within", default="perturb", choices=["perturb", "tree", "mala", "hmc"],
                   help="within-dimension moves: Gaussian vertex steps, the paper's tree-coordinate moves, MALA or "
                        "full-path HMC")
    p.add_argument("--ts-hmc-steps", type=int, default=10, help="leapfrog steps of an HMC move")
    p.add_argument("--ts-sigma", type=float, default=0.0,
                   help="step scale (m for perturb; dimensionless for tree; MALA epsilon); 0 = the scene default")
    p.add_argument("--ts-ttt", type=float, default=0.0,
                   help="two-sensor scene: wall time until B reaches this relative error for tree-move chains, "
                        "Cartesian chains (straight starts and tracer seeds) and the GPU tracer")
    p.add_argument("--ts-grad", action="store_true",
                   help="also observe the per-layer scores: d log B / d theta and d log B / d b1")
    p.add_argument("--ts-cpu-seconds", type=float, default=0.0,
                   help="also time the FP64 oracle's chains (same moves) on the host cores for about this long")
    p.add_argument("--ts-seed", action="store_true",
                   help="start the chains from weight-thinned tracer paths (exact draws, as the paper seeds its "
                        "chains) instead of straight jittered paths")
    return p.parse_args(argv)


def measure_pipes(device: int, stream) -> dict:
    """Measured FP32 FMA and MUFU lane-operations per second of the device,
    from the harness's pipe-rate microbenchmark (libpmcprobe.so, built beside
    the product library; not part of its C ABI)."""
    import ctypes as C
    from paper_1811_04156_gb300 import build as B
    B.build()
    lib = C.CDLL(B.PROBE_LIB)
    fn = lib.pmcprobe_measure_pipes
    fn.argtypes = [C.c_int, C.POINTER(C.c_double), C.c_void_p]
    fn.restype = C.c_int
    out = (C.c_double * 2)()
    rc = fn(int(device), out, C.c_void_p(stream.cuda_stream if stream is not None else 0))
    if rc != 0:
        raise RuntimeError(f"pipe-rate microbenchmark failed (cudaError {rc})")
    return {"fp32_per_s": float(out[0]), "mufu_per_s": float(out[1])}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                pass
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), r[2:]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def scene_for(args, world: int = 1):
    """The workload.  Single-pair workloads grow with the ranks (weak scaling:
    `--chains` chains per GPU, one pair of world x chains chains); multi-pair
    workloads are split as they are (strong scaling)."""
    from paper_1811_04156_gb300 import scenes as S
    if args.workload == "detector":
        return S.detector(n_chains=args.chains * world, n_steps=args.run_steps)
    if args.workload == "plain":
        return S.plain(n_chains=args.chains * world, n_steps=args.run_steps)
    if args.workload == "gradients":
        return S.gradients(n_chains=args.chains * world, n_steps=args.run_steps)
    if args.workload == "batched":
        return S.batched(n_steps=args.run_steps)
    if args.workload == "layered":
        return S.layered(n_steps=args.run_steps)
    raise SystemExit(f"unknown workload {args.workload}")


def host_initial_paths(sc, lo: int, hi: int):
    """The run's initial paths (straight, init_k interior vertices jittered by
    N(0, init_jitter^2); the direct path when init_k = 0) of the geometry's
    chains [lo, hi), built on the host (seeded), as a user passes them
    through the C ABI: absolute positions [chain][3][stride], counts [chain]."""
    import numpy as np
    from paper_1811_04156_gb300 import scenes as S
    k = sc.run.init_k if sc.run.init == S.INIT_STRAIGHT else 0
    stride = k + 2
    rng = np.random.default_rng(S.BASE_SEED + 17)
    xyz = np.zeros((hi - lo, 3, stride), dtype=np.float32)
    c0 = 0
    fr = np.arange(1, k + 1) / (k + 1)
    for pr in sc.pairs:
        a, b = max(c0, lo), min(c0 + pr.n_chains, hi)
        c0 += pr.n_chains
        if b <= a:
            continue
        src = np.asarray(sc.sources[pr.source].pos, float)
        c = np.asarray(sc.sensors[pr.sensor].centre, float)
        u = (src - c) / np.linalg.norm(src - c)
        e = c + sc.sensors[pr.sensor].radius * u
        m = b - a
        inner = src[None, None, :] + fr[None, :, None] * (e - src)[None, None, :] + \
            sc.run.init_jitter * rng.normal(size=(m, k, 3))
        xyz[a - lo:b - lo, :, 0] = src
        xyz[a - lo:b - lo, :, 1:k + 1] = inner.transpose(0, 2, 1)
        xyz[a - lo:b - lo, :, k + 1] = e
    n = np.full(hi - lo, k + 2, dtype=np.int32)
    return xyz, n


def _oracle_sample(sc, seconds, threads, steps_cap=10_000):
    """Size a bounded sample of the workload for the FP64 oracle: every chain
    runs min(workload steps, steps_cap) steps from the workload's initial
    paths; the chain count is chosen to take about `seconds` on `threads`."""
    import oracle as O
    p = sc.pairs[0]
    steps = int(min(sc.run.n_steps, steps_cap))
    probe_chains = max(threads, 8)
    probe_steps = min(steps, 1000)
    ch = O.Chains(sc.medium, sc.sources[0], sc.sensors[p.sensor], sc.run, probe_chains, p.cap)
    t = time.perf_counter()
    ch.run(probe_steps, threads=threads)
    rate = probe_chains * probe_steps / max(time.perf_counter() - t, 1e-6)
    chains = int(max(threads, min(p.n_chains, round(rate * seconds / steps))))
    return chains, steps


def _oracle_run(sc, chains, steps, threads):
    import oracle as O
    p = sc.pairs[0]
    ch = O.Chains(sc.medium, sc.sources[0], sc.sensors[p.sensor], sc.run, chains, p.cap)
    t = time.perf_counter()
    ch.run(steps, threads=threads)
    return time.perf_counter() - t


def cpu_baseline(sc, seconds, threads):
    """The oracle as it stands on the host cores, on a bounded sample of the
    workload; also its single-core rate on a smaller sample."""
    chains, steps = _oracle_sample(sc, seconds, threads)
    dt = _oracle_run(sc, chains, steps, threads)
    c1, s1 = _oracle_sample(sc, max(2.0, seconds / 5), 1)
    dt1 = _oracle_run(sc, c1, s1, 1)
    return {"value": chains * steps / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "value_1core": c1 * s1 / dt1,
            "sample": f"{chains} of the {sc.pairs[0].n_chains} chains x the first {steps} of "
                      f"{sc.run.n_steps} steps of the {sc.name} workload, FP64, {dt:.1f} s; 1 core: "
                      f"{c1} chains x {s1} steps, {dt1:.1f} s"}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    sc = scene_for(args)
    threads = os.cpu_count() or 1
    import oracle as O
    O.build()
    per_step = max(3.0, 150.0 / max(args.steps + args.warmup, 1))
    chains, steps = _oracle_sample(sc, per_step, threads)
    times = []
    for i in range(args.warmup + args.steps):
        dt = _oracle_run(sc, chains, steps, threads)
        if i >= args.warmup:
            times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = chains * steps / (ms / 1e3)
    sample = (f"{chains} of the {sc.pairs[0].n_chains} chains x the first {steps} of {sc.run.n_steps} "
              f"steps per bench step, FP64")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{sc.name} (bounded sample: {sample})", "global_batch": chains,
                       "vertex_cap": sc.pairs[0].cap},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def max_over_ranks(ms: float, dist, device="cpu") -> float:
    """The bench's step time is the slowest rank's."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def lane_op_roofline(est, rate, n_sm, clk_mhz, pipes):
    """Lane-op roofline of a proposal (FP32 + INT against 128 lanes/clk/SM,
    MUFU against 16 lanes/clk/SM, each pipe's peak the larger of that unit
    count and the microbenchmark's measured rate) at the measured move mix and
    mean vertex count: achieved and peak lane-operations per second of the
    binding pipe, and the FP32-only fraction of the delta evaluator's own
    per-move counts beside it."""
    prop = est["proposals"]
    tot = sum(prop)
    mix = {k: prop[i] / tot for i, k in enumerate(("interior", "end", "birth", "death"))}
    nbar = est["mean_n"]
    p_pert, p_b, p_d = mix["interior"] + mix["end"], mix["birth"], mix["death"]
    fp32 = p_pert * LANE_OPS["perturb"][0] + p_b * (LANE_OPS["birth"][0] + nbar) + \
        p_d * (LANE_OPS["death"][0] + nbar)
    alu = fp32 + INT_PER_PROPOSAL
    mufu = p_pert * LANE_OPS["perturb"][1] + p_b * LANE_OPS["birth"][1] + p_d * LANE_OPS["death"][1]
    f = clk_mhz * 1e6
    alu_peak = max(FP32_LANES_PER_SM * n_sm * f, pipes["fp32_per_s"])
    mufu_peak = max(MUFU_LANES_PER_SM * n_sm * f, pipes["mufu_per_s"])
    if mufu / mufu_peak >= alu / alu_peak:
        pipe, work, peak = "MUFU", mufu, mufu_peak
    else:
        pipe, work, peak = "FP32+INT", alu, alu_peak
    fp32_own = sum(mix[k] * FP32_PER_PROPOSAL[k] for k in mix)
    fp32_peak = max(FP32_LANES_PER_SM * n_sm * f, pipes["fp32_per_s"])
    return {"bound": "alu", "achieved": rate * work / 1e12, "peak": peak / 1e12, "unit": "T lane-ops/s",
            "frac": rate * work / peak, "pipe": pipe,
            "lane_ops_per_proposal": {"fp32": fp32, "int": INT_PER_PROPOSAL, "mufu": mufu, "mean_n": nbar},
            "peak_source": f"{pipe}: lanes/clk/SM x {n_sm} SMs x {clk_mhz:.0f} MHz (median SM clock sampled during "
                           f"the timed region), or the pipe microbenchmark's rate where higher",
            "frac_fp32_only": rate * fp32_own / fp32_peak, "fp32_own_per_proposal": fp32_own,
            "pipes_measured": pipes}


def ours(args):
    import numpy as np
    import torch
    from paper_1811_04156_gb300 import build as B
    B.build()
    from paper_1811_04156_gb300 import api

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    sc = scene_for(args, world)
    # the sharded form: each rank holds a contiguous window of the chain set,
    # balanced by vertex cap; a chain keeps its global index, so its Philox
    # stream is the one it has on a single GPU
    lo, hi = api.shard_range(sc.pairs, rank, world)
    ctx = api.Context(local)
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    sc.run.layout = {"auto": 0, "warp": 1, "lane": 2}[args.layout]  # scenes.LAYOUT_*
    if args.within != "default":
        from paper_1811_04156_gb300 import scenes as S
        sc.run.within = {"perturb": S.WITHIN_PERTURB, "mala": S.WITHIN_MALA, "tree": S.WITHIN_TREE}[args.within]
        if args.within == "tree":
            sc.run.sigma = 0.3
    chains = api.Chains(ctx, medium, geom, sc.run, warps_per_block=args.warps_per_block,
                        smem_window=args.smem_window, chain_window=(lo, hi))
    stream = torch.cuda.current_stream()
    n_local = hi - lo
    props_local = n_local * sc.run.n_steps
    props_all = sc.total_chains * sc.run.n_steps
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def estimate():
        # one sum all-reduce of the per-pair moments (NCCL) when sharded
        return chains.read_estimator_sharded()[0][0] if dist else chains.read_estimator()[0]

    def one_step(ev=None):
        chains.reset()
        if ev is not None:
            ev[0].record(stream)
        chains.run_steps(sc.run.n_steps)
        if ev is not None:
            ev[1].record(stream)
        return estimate()

    for _ in range(args.warmup):
        one_step()
    pipes = measure_pipes(local, stream) if rank == 0 else None
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clock = ClockSampler(local) if rank == 0 else None
    if clock:
        clock.start()
    step_ms, kern_ms = [], []
    est = None
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        est = one_step((k0, k1))
        s1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(s0.elapsed_time(s1))
        kern_ms.append(k0.elapsed_time(k1))
    clocks = clock.stop() if clock else None
    total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    ms_per_step = total_ms / args.steps
    value = props_all / (ms_per_step / 1e3)

    # end to end through the public API with host buffers: each step uploads
    # this rank's initial paths from pinned memory, steps, and reads the estimate
    e2e = None
    if not args.no_e2e:
        hx, hn = host_initial_paths(sc, lo, hi)
        px = torch.from_numpy(hx).pin_memory()
        pn = torch.from_numpy(hn).pin_memory()
        hx, hn = px.numpy(), pn.numpy()

        def e2e_step():
            chains.set_states(hx, hn)
            chains.run_steps(sc.run.n_steps)
            return estimate()

        e2e_step()
        torch.cuda.synchronize()
        ts = []
        for _ in range(max(1, min(args.steps, 2))):
            flush.zero_()
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            t0 = time.perf_counter()
            e2e_step()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(sum(ts) / len(ts), dist, "cuda")
        from paper_1811_04156_gb300._lib import PMC_MOMENT_WORDS
        e2e = {"value": props_all / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(hx.nbytes + hn.nbytes),
               "d2h_bytes_per_step": int(8 * PMC_MOMENT_WORDS * len(sc.pairs))}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    peaks, peak_kind = load_peaks()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    clk = (clocks or {}).get("sm_mhz") or float(peaks.get("sm_max_mhz", 2070.0))
    kern_s = statistics.mean(kern_ms) / 1e3
    rate = props_local / kern_s
    li = chains.launch_info()
    kind = li[0]["general"] if len(li) == 1 else None
    roof = lane_op_roofline(est, rate, n_sm, clk, pipes)
    roof["kernel"] = "lane_chain_kernel" if kind in (4, 5) else "chain_kernel"
    if args.within != "default":
        roof["within"] = args.within
    roof["kernel_ms"] = statistics.mean(kern_ms)
    roof["clock_max_mhz"] = float(peaks.get("sm_max_mhz", 2070.0))
    roof["peak_kind"] = peak_kind
    # counters of the committed capture, only while the kernel source matches it
    fresh = (kind == 4 and sc.name == "detector" and li[0]["smem_cap"] == 20 and
             LANE_CAPTURE["source_sha256"] == lane_kernel_source_hash())
    have_traffic = fresh and LANE_CAPTURE["dram_bytes_per_launch"] is not None and sc.run.n_steps == 100_000
    roof["traffic"] = LANE_CAPTURE["dram_bytes_per_launch"] * n_local / 65536.0 if have_traffic else None
    roof["traffic_source"] = LANE_CAPTURE["capture"] if have_traffic else \
        "null: no ncu capture of this kernel source and launch"
    issue = None
    if fresh:
        inst = LANE_CAPTURE["inst_per_proposal"]
        issue_peak = ISSUE_PER_CLK_PER_SM * n_sm * clk * 1e6
        issue = {"achieved": rate * inst, "peak": issue_peak, "unit": "warp instructions/s",
                 "frac": rate * inst / issue_peak, "inst_per_proposal": inst,
                 "source": "warp instructions per proposal from the ncu capture of this kernel source; peak = 4 "
                           "warp instructions/clk/SM x SMs x median SM clock under load"}
    converged = bool(est.get("rhat") is not None and math.isfinite(est["rhat"]) and est["rhat"] < 1.2)
    estimate_block = {k: est[k] for k in ("intensity", "std_err", "pi_direct", "rhat", "mean_n", "accept", "ess")}
    estimate_block["converged"] = converged
    estimate_block["note"] = ("R-hat on the path length below 1.2 (the paper's stopping rule)" if converged else
                              "not converged: R-hat on the path length >= 1.2, so the chains have not forgotten "
                              "their initial paths; intensity and std_err describe the run, not the target")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak" if len(sc.pairs) == 1 else "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT.get(sc.name, sc.name) +
                       ("" if args.within == "default" else f", {args.within} moves"),
                       "chains": sc.total_chains, "steps_per_chain": sc.run.n_steps,
                       "vertex_cap": max(p.cap for p in sc.pairs), "global_batch": sc.total_chains,
                       "parallelism": f"sharded chain windows x{world}" if world > 1 else "1 GPU",
                       "l2": "flushed between steps (256 MB write)", "accumulators": "f64",
                       "launch": li},
            "roofline": roof, "issue_roofline": issue,
            "gpu_launches": (len(li) + 2) * args.steps,
            "effective_samples_per_s": (est["ess"] / (ms_per_step / 1e3)) if (converged and est.get("ess"))
            else None,
            "estimate": estimate_block, "clocks": clocks, "e2e": e2e}
    if world == 1 and not args.no_extras:
        # reports beside the timed line: a failure here must not lose the line
        for key, fn in (("other_configs", lambda: other_configs(api, ctx)),
                        ("time_to_1pct", lambda: time_to_1pct(api, ctx, args))):
            try:
                line[key] = fn()
            except Exception as exc:
                line[key] = {"error": f"{type(exc).__name__}: {exc}"}
    if not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline(sc, args.cpu_seconds, os.cpu_count() or 1)
        except Exception as exc:  # the baseline is a report, not the product
            line["cpu_baseline"] = {"error": str(exc)}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def other_configs(api, ctx):
    """Proposals/s of the other workloads, each a timed launch after a warm-up
    launch of the same chain set (autotuned launch shapes): the batched uneven
    pairs under one CUDA graph (one launch per cap class, and one persistent
    launch for every cap), the gradients workload (MALA moves and score
    accumulation) and the layered string of sensors."""
    import torch
    from paper_1811_04156_gb300 import scenes as S
    from paper_1811_04156_gb300._lib import PMC_FLAG_ONE_LAUNCH
    out = {}
    for name, sc, flags in (("batched", S.batched(n_steps=5000), 0),
                            ("batched_one_launch", S.batched(n_steps=5000), PMC_FLAG_ONE_LAUNCH),
                            ("gradients", S.gradients(n_steps=10_000), 0),
                            ("layered", S.layered(n_steps=5000), 0)):
        medium = api.Medium(ctx, sc.medium)
        geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
        ch = api.Chains(ctx, medium, geom, sc.run, flags=flags)
        ch.run_steps(sc.run.n_steps)
        ch.read_estimator()
        ch.reset()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ch.run_steps(sc.run.n_steps)
        e1.record()
        est = ch.read_estimator()
        ms = e0.elapsed_time(e1)
        props = sc.total_chains * sc.run.n_steps
        out[name] = {"workload": WORKLOAD_TEXT[sc.name] + (", one persistent launch for every cap" if flags else ""),
                     "chains": sc.total_chains, "steps_per_chain": sc.run.n_steps,
                     "proposals_per_s": props / (ms / 1e3), "ms": ms, "launch": ch.launch_info(),
                     "mean_n": sum(e["mean_n"] * e["n_samples"] for e in est) / max(sum(e["n_samples"] for e in est),
                                                                                     1.0)}
        if name == "gradients":
            g, gse = ch.grad_estimator()
            out[name]["d_intensity_d_theta"] = {"theta": "lambda_s, lambda_a, g", "value": g[0].tolist(),
                                                "se": gse[0].tolist()}
        ch.close()
    return out


def ttt_geometry(api, ctx, geom_name, tgt, methods=None, limit=120.0, ref=None, ref_photons=None):
    """Wall time until the intensity estimate reaches relative standard error
    `tgt` and lies within max(tgt, 3 combined SE) of a reference value from a
    long forward-tracer run (the criterion of the method's time-to-error
    comparison), for each method on the plain (D = 1 m) or detector (D = 50 m)
    geometry: plain RJMCMC (64 chains, Gaussian steps); batched MALA chains
    (65,536; from the direct path, or from tracer seeds as the paper seeds
    its chains, seeding inside the timed region); batched Gaussian chains with
    seeds; batched tree-move chains; tree-move chains whose intensity comes
    from the optimal bridge against the reference density; the GPU forward
    tracer.  Budgets double until the criterion holds or `limit` seconds
    have passed."""
    import torch
    from paper_1811_04156_gb300 import scenes as S
    sc_plain = S.plain() if geom_name == "plain" else S.detector(n_chains=64)
    med = api.Medium(ctx, sc_plain.medium)
    cap = sc_plain.pairs[0].cap
    g1 = api.Geometry(ctx, sc_plain.sources, sc_plain.sensors, [S.Pair(0, 0, 1, cap)])
    if ref_photons is None:
        ref_photons = 4_000_000_000 if geom_name == "plain" else 16_000_000_000
    t0 = time.perf_counter()
    if ref is not None:
        I_ref, se_ref, N = ref
    else:
        parts = []
        left = ref_photons
        while left > 0:
            k = min(left, 4_000_000_000)
            parts.append(api.trace(ctx, med, g1, 0, 123457, k, photon0=ref_photons - left, max_scatter=cap - 2))
            left -= k
        N = sum(p["photons"] for p in parts)
        I_ref = sum(p["sum_w"] for p in parts) / N
        se_ref = math.sqrt(sum((p["se"] * p["photons"]) ** 2 for p in parts)) / N
    out = {"target_rel_err": tgt, "geometry": geom_name, "limit_s": limit,
           "reference": {"intensity": I_ref, "std_err": se_ref, "photons": N, "seconds": time.perf_counter() - t0,
                         "how": "GPU forward tracer (Algorithm 1), cap-truncated"}}

    def ok(I, se):
        return I > 0 and se / I <= tgt and abs(I - I_ref) <= max(tgt * I_ref, 3 * math.hypot(se, se_ref))

    def run_chains(n_chains, within, increment, seeded=False, seed_rounds=64, seed_photons=1 << 26):
        sc = S.plain(n_chains=n_chains) if geom_name == "plain" else S.detector(n_chains=n_chains)
        sc.run.within = within
        sc.run.burn_in = 0 if seeded else (1000 if geom_name == "plain" else 10_000)
        if within == S.WITHIN_MALA:
            sc.run.mala_step = 0.02 if geom_name == "plain" else 0.5
        if within == S.WITHIN_TREE:
            sc.run.sigma = 0.3
        geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
        ch = api.Chains(ctx, med, geom, sc.run)
        torch.cuda.synchronize()
        t = time.perf_counter()
        seed_s = 0.0
        if seeded:
            # equilibrium seeds from the forward tracer (inside the timed region)
            api.seed_from_tracer(ch, seed=4321, photons_per_round=seed_photons, max_rounds=seed_rounds)
            seed_s = time.perf_counter() - t
        steps = 0
        while True:
            ch.run_steps(increment)
            steps += increment
            e = ch.read_estimator()[0]
            if steps > sc.run.burn_in and e["n_samples"] > 0 and ok(e["intensity"], e["std_err"]):
                break
            if time.perf_counter() - t > limit:
                break
            increment = min(increment * 2, 1_000_000)
        dt = time.perf_counter() - t
        ch.close()
        return {"seconds": dt, "seed_seconds": seed_s, "steps_per_chain": steps, "chains": n_chains,
                "intensity": e["intensity"], "std_err": e["std_err"], "rhat": e["rhat"],
                "reached": bool(ok(e["intensity"], e["std_err"]))}

    def run_tree_bridge(n_chains, burn, thin, n_draws, rows0):
        """Tree-move chains and the optimal bridge against the normalised
        reference density: after `burn` steps, one row of log ratios (n_draws
        reference draws, every chain's state) every `thin` steps; the row
        count doubles until the criterion holds."""
        sc = S.plain(n_chains=n_chains) if geom_name == "plain" else S.detector(n_chains=n_chains)
        sc.run.within, sc.run.sigma, sc.run.burn_in = S.WITHIN_TREE, 0.3, 0
        geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
        torch.cuda.synchronize()
        t = time.perf_counter()
        ch = api.Chains(ctx, med, geom, sc.run)
        ch.run_steps(burn)
        rows, target, ob = [], rows0, None
        while True:
            while len(rows) < target:
                ch.run_steps(thin)
                row = torch.empty(n_draws + n_chains, dtype=torch.float32, device="cuda")
                ch.bridge_observe_log(0, n_draws, len(rows) * n_draws, 4242, row)
                rows.append(row)
            ob = api.bridge_ratio(ctx, torch.stack(rows), n_draws, n_chains, groups=32)
            if ok(ob["r"], ob["se"]) or time.perf_counter() - t > limit:
                break
            target *= 2
        dt = time.perf_counter() - t
        ch.close()
        return {"seconds": dt, "steps_per_chain": burn + thin * len(rows), "chains": n_chains, "rows": len(rows),
                "draws_per_row": n_draws, "intensity": ob["r"], "std_err": ob["se"],
                "geometric": ob["geometric"], "reached": bool(ok(ob["r"], ob["se"]))}

    def want(name):
        return methods is None or name in methods

    if want("plain_rjmcmc"):
        out["plain_rjmcmc"] = run_chains(64, S.WITHIN_PERTURB, 20_000)
    if want("batched_mala"):
        out["batched_mala"] = run_chains(65_536, S.WITHIN_MALA, 2_000)
    # seeds cost tracer photons: 1 / I of them per seed (I ~ 2e-3 at 1 m, ~2e-6 at 50 m), so the
    # detector geometry seeds 8,192 chains (about 4e9 photons) and lets each run longer
    n_seeded = 65_536 if geom_name == "plain" else 8_192
    seed_kw = {} if geom_name == "plain" else {"seed_rounds": 32, "seed_photons": 1 << 28}
    if want("batched_mala_tracer_seeded"):
        out["batched_mala_tracer_seeded"] = run_chains(n_seeded, S.WITHIN_MALA, 500, seeded=True, **seed_kw)
    if want("batched_perturb_tracer_seeded"):
        out["batched_perturb_tracer_seeded"] = run_chains(n_seeded, S.WITHIN_PERTURB, 500, seeded=True, **seed_kw)
    if want("batched_tree_moves"):
        out["batched_tree_moves"] = run_chains(65_536, S.WITHIN_TREE, 2_000)
    if want("tree_moves_optimal_bridge"):
        out["tree_moves_optimal_bridge"] = run_tree_bridge(65_536, 10_000 if geom_name == "plain" else 40_000,
                                                           500, 65_536, 8)
    if want("gpu_tracer"):
        t = time.perf_counter()
        photons, acc = 1_000_000, []
        while True:
            acc.append(api.trace(ctx, med, g1, 0, 99, photons, photon0=sum(a["photons"] for a in acc),
                                 max_scatter=cap - 2))
            Nn = sum(a["photons"] for a in acc)
            I = sum(a["sum_w"] for a in acc) / Nn
            se = math.sqrt(sum((a["se"] * a["photons"]) ** 2 for a in acc)) / Nn
            if ok(I, se) or time.perf_counter() - t > limit:
                break
            photons *= 2
        out["gpu_tracer"] = {"seconds": time.perf_counter() - t, "photons": Nn, "intensity": I, "std_err": se,
                             "reached": bool(ok(I, se))}
    reached = {k: v["seconds"] for k, v in out.items() if isinstance(v, dict) and v.get("reached")}
    out["fastest"] = min(reached, key=reached.get) if reached else None
    if "plain_rjmcmc" in out and "batched_mala_tracer_seeded" in out:
        pl, bm = out["plain_rjmcmc"], out["batched_mala_tracer_seeded"]
        out["batched_gradient_beats_plain"] = bool(bm["reached"] and (not pl["reached"] or
                                                                      bm["seconds"] < pl["seconds"]))
    return out


def time_to_1pct(api, ctx, args):
    """The metric's second half on both geometries, in the bench process."""
    plain = ttt_geometry(api, ctx, "plain", 0.01, ["plain_rjmcmc", "batched_mala_tracer_seeded", "gpu_tracer"],
                         limit=args.ttt_limit)
    det = ttt_geometry(api, ctx, "detector", 0.01, ["plain_rjmcmc", "batched_mala_tracer_seeded",
                                                     "tree_moves_optimal_bridge", "gpu_tracer"],
                       limit=args.ttt_limit)
    return {"plain_geometry": plain, "detector_geometry": det}


def time_to_target(args):
    """--time-to-target: every method on one geometry (--geometry), printed."""
    from paper_1811_04156_gb300 import build as B
    B.build()
    from paper_1811_04156_gb300 import api
    ctx = api.Context(0)
    ref = tuple(float(x) for x in args.ttt_ref.split(",")) if args.ttt_ref else None
    methods = set(args.ttt_methods.split(",")) if args.ttt_methods else None
    out = ttt_geometry(api, ctx, args.geometry, args.time_to_target, methods, limit=args.ttt_limit, ref=ref,
                       ref_photons=4_000_000_000 if args.geometry == "plain" else 100_000_000_000)
    print(json.dumps(out), flush=True)
    return 0


# The paper's table of its two-sensor scene (section "Comparison of relative
# light yield", Table tbl:results): B with its uncertainty for each b1, the
# ray tracer's and the path sampler's, and the CPU seconds of each.
TWO_SENSOR_PAPER = {0.1: {"tracer": (0.67, 0.03), "sampler": (0.64, 0.07), "sampler_cpu_s": 23.0, "tracer_cpu_s": 45.9e3},
            0.2: {"tracer": (0.79, 0.02), "sampler": (0.77, 0.01), "sampler_cpu_s": 74.4, "tracer_cpu_s": 78.1e3},
            0.3: {"tracer": (0.73, 0.02), "sampler": (0.76, 0.07), "sampler_cpu_s": 232.0, "tracer_cpu_s": 99.6e3},
            0.4: {"tracer": (0.68, 0.02), "sampler": (0.64, 0.04), "sampler_cpu_s": 373.0, "tracer_cpu_s": 122e3},
            0.5: {"tracer": (0.59, 0.02), "sampler": (0.50, 0.06), "sampler_cpu_s": 416.0, "tracer_cpu_s": 156e3}}


def two_sensor_experiment(args):
    """Relative light yield B of the paper's two sensors and their path-length
    distributions, for each b1: chains of both sensors from straight jittered
    paths, 10% burn-in, then B (geometric estimator through the map T) and the
    length histograms observed every --ts-thin steps; optionally I_1/I_0 and
    the length histograms of the GPU forward tracer (rejection radius 400 m,
    scatterings capped at the chains' vertex cap)."""
    import numpy as np
    import torch
    from paper_1811_04156_gb300 import build as B
    B.build()
    from paper_1811_04156_gb300 import api, scenes as S
    ctx = api.Context(0)
    stream = torch.cuda.current_stream()
    lo, hi, nb = 115.0, 215.0, 50
    results = []
    for b1 in [float(x) for x in args.ts_b1.split(",")]:
        sc = S.two_sensor(b1, n_chains=args.ts_chains, n_steps=args.ts_steps)
        sc.run.within = {"perturb": S.WITHIN_PERTURB, "tree": S.WITHIN_TREE, "mala": S.WITHIN_MALA,
                         "hmc": S.WITHIN_HMC}[args.ts_within]
        if args.ts_within == "tree":
            sc.run.sigma = args.ts_sigma or 0.3
        elif args.ts_within in ("mala", "hmc"):
            sc.run.mala_step = args.ts_sigma or 0.5
            sc.run.hmc_steps = args.ts_hmc_steps
        elif args.ts_sigma:
            sc.run.sigma = args.ts_sigma
        medium = api.Medium(ctx, sc.medium)
        geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
        ch = api.Chains(ctx, medium, geom, sc.run)
        seed_s, seed_photons = 0.0, None
        if args.ts_seed:
            ts = time.perf_counter()
            seed_photons = api.seed_from_tracer(ch, seed=2468, photons_per_round=1 << 28, r_reject=400.0)
            seed_s = time.perf_counter() - ts
        burn = sc.run.burn_in
        thin = args.ts_thin
        n_obs = (sc.run.n_steps - burn + thin - 1) // thin
        Y = api.YieldRatio(ch, 0, 1, max_obs=n_obs)
        hist = torch.zeros((2, nb), dtype=torch.float64, device="cuda")
        nth = medium.n_theta
        ssum = torch.zeros((2, 2 * nth), dtype=torch.float64, device="cuda") if args.ts_grad else None
        sobs = []
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        ev0.record(stream)
        ch.run_steps(burn)
        done = burn
        while done < sc.run.n_steps:
            k = min(thin, sc.run.n_steps - done)
            ch.run_steps(k)
            done += k
            Y.observe()
            ch.length_hist(lo, hi, hist)
            if ssum is not None:
                ch.score_observe(ssum)
                sobs.append(ssum[:, :nth].clone())
        ev1.record(stream)
        est = Y.estimate()
        ob = Y.estimate_bridge(groups=32)
        e = ch.read_estimator()
        wall = time.perf_counter() - t0
        gpu_s = ev0.elapsed_time(ev1) / 1e3
        h = hist.cpu().numpy()
        row = {"b1": b1, "B": est["B"], "B_se": est["se"], "B_bridge": ob["r"], "B_bridge_se": ob["se"],
               "bridge_iterations": ob["iterations"], "rhat": [e[0]["rhat"], e[1]["rhat"]],
               "accept": [e[0]["accept"], e[1]["accept"]], "mean_n": [e[0]["mean_n"], e[1]["mean_n"]],
               "mean_length_m": [e[0]["mean_length"], e[1]["mean_length"]], "observations": Y.n_obs,
               "proposals": 2 * args.ts_chains * sc.run.n_steps, "gpu_seconds": gpu_s, "wall_seconds": wall,
               "proposals_per_s": 2 * args.ts_chains * sc.run.n_steps / gpu_s,
               "length_hist": {"lo": lo, "hi": hi, "bins": nb, "sensor0": (h[0] / max(h[0].sum(), 1)).tolist(),
                               "sensor1": (h[1] / max(h[1].sum(), 1)).tolist()},
               "init": "tracer seeds" if args.ts_seed else "straight, 30 interior vertices, N(0, 0.5 m) jitter",
               "within": args.ts_within, "sigma": sc.run.sigma, "mala_step": sc.run.mala_step,
               "seed_seconds": seed_s, "seed_photons": seed_photons, "paper": TWO_SENSOR_PAPER.get(b1)}
        if ssum is not None:
            # per-observation mean scores of each sensor's chains, then batch means over 20 batches
            cum = torch.stack(sobs).cpu().numpy()                        # (obs, 2, nth) running sums
            per = np.diff(np.concatenate([np.zeros_like(cum[:1]), cum]), axis=0) / args.ts_chains
            d = per[:, 1, :] - per[:, 0, :]                               # d log B / d theta per observation
            nbat = 20
            bm = np.array([b.mean(axis=0) for b in np.array_split(d, nbat)])
            g, gse = d.mean(axis=0), bm.std(axis=0, ddof=1) / math.sqrt(nbat)
            lam1 = 1.0 / b1                                               # layer 1 = the x >= 0 half-space
            row["dlogB_dtheta"] = {"theta": "lambda_s[0], lambda_s[1], lambda_a[0], lambda_a[1] (m)",
                                   "value": g.tolist(), "se": gse.tolist()}
            row["dlogB_db1"] = {"value": float(-lam1 * lam1 * g[1]), "se": float(lam1 * lam1 * gse[1])}
        if args.ts_photons > 0:
            cap = sc.pairs[0].cap
            tr, th = [], []
            t1 = time.perf_counter()
            for p, sd in ((0, 701), (1, 702)):
                r, hh = api.trace_lengths(ctx, medium, geom, p, sd, args.ts_photons, lo, hi, nb, r_reject=400.0,
                                          max_scatter=cap - 2)
                tr.append(r)
                th.append(hh)
            Bt = tr[1]["I"] / tr[0]["I"]
            row["tracer"] = {"B": Bt, "B_se": Bt * math.hypot(tr[0]["se"] / tr[0]["I"], tr[1]["se"] / tr[1]["I"]),
                             "I0": tr[0]["I"], "I0_se": tr[0]["se"], "I1": tr[1]["I"], "I1_se": tr[1]["se"],
                             "hits": [tr[0]["hits"], tr[1]["hits"]], "photons_per_sensor": args.ts_photons,
                             "seconds": time.perf_counter() - t1,
                             "length_hist": {"sensor0": (th[0] / max(th[0].sum(), 1e-300)).tolist(),
                                             "sensor1": (th[1] / max(th[1].sum(), 1e-300)).tolist()}}
        if args.ts_cpu_seconds > 0:
            import oracle as O
            ts = time.perf_counter()
            oc = [O.Chains(sc.medium, sc.sources[0], sc.sensors[k], sc.run, 256, sc.pairs[k].cap, chain_offset=k * 256)
                  for k in (0, 1)]
            steps = 0
            while time.perf_counter() - ts < args.ts_cpu_seconds:
                for k in (0, 1):
                    oc[k].run(200)
                steps += 200
            cs = time.perf_counter() - ts
            row["cpu_baseline"] = {"kind": "oracle", "value": 2 * 256 * steps / cs, "unit": "proposals/s",
                                   "cores": os.cpu_count() or 1,
                                   "sample": f"2 x 256 chains x the first {steps} steps from the same starts"}
        results.append(row)
        brief = {k: row[k] for k in ("b1", "within", "B", "B_se", "B_bridge", "B_bridge_se", "rhat", "accept",
                                     "mean_n", "gpu_seconds", "proposals_per_s", "seed_seconds")}
        if "cpu_baseline" in row:
            brief["cpu_proposals_per_s"] = row["cpu_baseline"]["value"]
        if "dlogB_db1" in row:
            brief["dlogB_db1"] = row["dlogB_db1"]
        if "tracer" in row:
            brief["tracer_B"] = (row["tracer"]["B"], row["tracer"]["B_se"], row["tracer"]["hits"],
                                 row["tracer"]["seconds"])
        print(json.dumps(brief), flush=True)
        ch.close()
    out = {"experiment": "two-sensor scene (relative light yield, path lengths)", "chains_per_sensor": args.ts_chains,
           "steps_per_chain": args.ts_steps, "thin": args.ts_thin, "results": results}
    if args.ts_out:
        with open(args.ts_out, "w") as f:
            json.dump(out, f)
    print(json.dumps({"experiment": out["experiment"],
                      "B": [(r["b1"], r["B"], r["B_se"], r["B_bridge"], r["B_bridge_se"], r.get("tracer", {}).get("B"))
                            for r in results]}),
          flush=True)
    return 0


def two_sensor_time_to_target(args):
    """Wall time until the relative light yield B of the two-sensor scene
    (b1 = first --ts-b1 value) reaches relative standard error --ts-ttt and
    lies within max(target, 3 combined SE) of a reference from a long
    tree-move run.  Chains keep running with doubling step budgets (the first
    10 % of the steps run so far as burn-in is never observed); the tracer
    doubles its photons.  Each method stops after 120 s."""
    import torch
    from paper_1811_04156_gb300 import build as B
    B.build()
    from paper_1811_04156_gb300 import api, scenes as S
    ctx = api.Context(0)
    b1 = float(args.ts_b1.split(",")[0])
    tgt = args.ts_ttt
    limit = 120.0

    def chains_run(within, sigma, n_chains, steps_total, seeded=False, budget0=20_000, thin=200, ref=None):
        sc = S.two_sensor(b1, n_chains=n_chains, n_steps=steps_total)
        sc.run.within = within
        sc.run.sigma = sigma
        medium = api.Medium(ctx, sc.medium)
        geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ch = api.Chains(ctx, medium, geom, sc.run)
        if seeded:
            api.seed_from_tracer(ch, seed=2468, photons_per_round=1 << 28, r_reject=400.0)
        done, budget, hist = 0, budget0, []
        est = None
        while True:
            # burn-in: the first 10 % of the final budget, then observe every `thin` steps
            burn = budget // 10
            Y = api.YieldRatio(ch, 0, 1)
            # continue the same chains for `budget` more steps: burn-in, then observations
            ch.run_steps(burn)
            k = burn
            while k < budget:
                ch.run_steps(thin)
                k += thin
                Y.observe()
            est = Y.estimate()
            done += budget
            el = time.perf_counter() - t0
            hist.append({"steps": done, "seconds": el, "B": est["B"], "se": est["se"]})
            ok = ref is None or (est["se"] / est["B"] <= tgt and
                                 abs(est["B"] - ref[0]) <= max(tgt * ref[0], 3 * math.hypot(est["se"], ref[1])))
            if ref is None and done >= steps_total:
                break
            round_s = el - (hist[-2]["seconds"] if len(hist) > 1 else 0.0)
            if ref is not None and (ok or el + 2.0 * round_s > 1.5 * limit):
                break
            budget *= 2
        ch.close()
        return {"seconds": time.perf_counter() - t0, "steps_per_chain": done, "chains_per_sensor": n_chains,
                "B": est["B"], "se": est["se"], "reached": bool(ref is not None and ok), "trace": hist}

    out = {"experiment": "two-sensor scene: time to B within target", "b1": b1, "target_rel_err": tgt}
    r = chains_run(S.WITHIN_TREE, 0.3, 2048, 400_000, budget0=400_000)
    ref = (r["B"], r["se"])
    out["reference"] = {"B": ref[0], "se": ref[1], "seconds": r["seconds"], "how": "tree moves, 2 x 2048 chains x 4e5"}
    out["tree_moves"] = chains_run(S.WITHIN_TREE, 0.3, 2048, 0, budget0=5_000, ref=ref)
    out["cartesian_straight_starts"] = chains_run(S.WITHIN_PERTURB, 0.5, 2048, 0, budget0=50_000, ref=ref)
    out["cartesian_tracer_seeds"] = chains_run(S.WITHIN_PERTURB, 0.5, 1024, 0, seeded=True, budget0=50_000, ref=ref)
    # GPU tracer: I1/I0 with doubling photon budgets
    sc = S.two_sensor(b1, n_chains=1)
    medium = api.Medium(ctx, sc.medium)
    geom = api.Geometry(ctx, sc.sources, sc.sensors, sc.pairs)
    cap = sc.pairs[0].cap
    t0 = time.perf_counter()
    photons, acc = 1 << 28, [[], []]
    while True:
        for p in (0, 1):
            done = sum(a["photons"] for a in acc[p])
            acc[p].append(api.trace(ctx, medium, geom, p, 901 + p, photons, photon0=done, r_reject=400.0,
                                    max_scatter=cap - 2))
        I, se = [], []
        for p in (0, 1):
            Nn = sum(a["photons"] for a in acc[p])
            I.append(sum(a["I"] * a["photons"] for a in acc[p]) / Nn)
            se.append(math.sqrt(sum((a["se"] * a["photons"]) ** 2 for a in acc[p])) / Nn)
        Bt = I[1] / I[0]
        st = Bt * math.hypot(se[0] / I[0], se[1] / I[1])
        el = time.perf_counter() - t0
        ok = st / Bt <= tgt and abs(Bt - ref[0]) <= max(tgt * ref[0], 3 * math.hypot(st, ref[1]))
        if ok or el > limit:
            break
        photons *= 2
    out["gpu_tracer"] = {"seconds": time.perf_counter() - t0, "photons_per_sensor": sum(a["photons"] for a in acc[0]),
                         "B": Bt, "se": st, "reached": bool(ok)}
    out["paper_cpu_seconds"] = {"sampler": TWO_SENSOR_PAPER.get(b1, {}).get("sampler_cpu_s"),
                                "tracer": TWO_SENSOR_PAPER.get(b1, {}).get("tracer_cpu_s")}
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.time_to_target > 0:
        return time_to_target(args)
    if args.ts_ttt > 0:
        return two_sensor_time_to_target(args)
    if args.two_sensor:
        return two_sensor_experiment(args)
    if args.impl == "reference":
        return reference_arm(args)
    return ours(args)


if __name__ == "__main__":
    sys.exit(main())
