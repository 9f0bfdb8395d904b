"""Benchmark of the KAFMM evaluator on one GB300 (or N replicas under torchrun).

Workload: Stokeslet KAFMM, N = 262144 uniform points in the unit cube (FP32), forces
N(0,1)^3, order p = 10, <= 128 points per leaf, four-channel Laplace ML-tree table, mixed
precision.  A step is the whole hot path on one batch: kafmm_set_points (Morton keys, radix
sort, octree, U/V/W/X lists) + kafmm_eval (upward, M->L, downward, near field) -- the paper
rebuilds the tree whenever points move (t_tree + t_run, Sec. III).

value  = targets / (device time of set_points + eval), inputs resident in HBM, L2 flushed
         (256 MiB write) between timed steps, timed per step with CUDA events.
e2e    = the same through the C ABI with pinned HOST buffers (copies inside the timed region).
--impl reference: the CPU oracle (direct FP64 sum, oracle/direct.c) on the host cores,
         on a bounded sample of targets per step.
--workload batched: 512 independent Stokeslet problems, N_k log-uniform in [1024, 65536]
         (about 8 million points), p = 8, q = 64, mixed precision, set and evaluated as one
         batch (kafmm_set_points_batched + kafmm_eval) and, for comparison, as 512 sequential
         single-problem calls.
--workload periodic: triply periodic Stokeslet, 2^22 uniform points, p = 12, q = 128, G table.
--workload rpy: RPY sphere velocities, 2^20 clustered points, p = 8, q = 128 (set_points +
         eval + rpy_velocity per step).
--workload convergence: the paper's convergence benchmark (10^6 log-normal points, L = 32,
         q = 2000, m = 6..16 relative to m = 16, FP64), Laplace and Stokeslet.
--workload leafsweep: the leaf-size trade-off on the paper's log-normal cloud (10^6 points,
         p = 10, mixed form, q = 32 .. 2000): step time and error against the direct sum.
--workload errors: error of every form (FP64, FP32, mixed) against the direct FP64 sum per
         kernel and order (65536 uniform points, 512 sampled targets).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

N_POINTS, P_ORDER, Q_LEAF = 262144, 10, 128
METRIC = "Stokeslet KAFMM Mpoints/s at rel L2 err <=1e-5 vs plain FP64 GPU form; S->T GFLOP/s"
WORKLOAD = "stokeslet_uniform_256k_p10_q128_l4"
# FLOP counts of one pair evaluation (add/mul = 1, FMA = 2, rsqrt = 1): the Stokeslet S->T
# pair in the leaf kernel (stk_st): 3 sub, r^2 (5), rsqrt, ir^3 (2), r.f (5), scale (1),
# 3 x (mul + FMA + FMA = 5) -> 29.
FLOP_ST_PAIR = 29
# DRAM bytes (read + written) of one M->L launch of this workload in the default mixed form
# (compressed coordinates, rank rounded to 64, automatic split, tiles per parent neighbour),
# from an ncu capture of the current kernel: 80.07 MB read + 224.42 MB written.  Reported only
# for that configuration; None when the kernel changes until it is captured again.
M2L_DRAM_BYTES = 304.49e6


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def _dist_init(world, backend="nccl"):
    """One process per GPU (torchrun): joins the process group when world > 1."""
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend)


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(value, world, device=None):
    """The slowest rank's time: the whole job's step time."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _rank_seed(base, rank):
    """Every rank works on its own seeded inputs (replicas, or its own batch of problems): the
    units are partitioned across ranks and no data crosses them."""
    return base + rank


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 20 ms during the timed region."""

    def __init__(self, index=0):
        self.path = os.path.join(tempfile.gettempdir(), f"kafmm_clocks_{os.getpid()}.csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            v = [x.strip() for x in line.split(",")]
            if len(v) < 9:
                continue
            try:
                sm.append(float(v[1]))
                mx.append(float(v[2]))
            except ValueError:
                continue
            for nm, val in zip(names, v[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    """Rates measured on this GPU by the library's micro-benchmarks (kafmm_measure_peak)."""
    from paper_2010_15155_gb300 import kafmm as K
    out = {}
    for what, name in ((K.PEAK_FFMA, "fp32_fma_tflops"), (K.PEAK_RSQRT, "mufu_rsqrt_tops"),
                       (K.PEAK_DFMA, "fp64_fma_tflops"), (K.PEAK_MMA_TF32, "tf32_mma_tflops"),
                       (K.PEAK_MMA_BF16, "bf16_mma_tflops")):
        out[name] = K.kafmm_measure_peak(what)[0] / 1e12
    return out


def cpu_baseline_o2(n=32768):
    """The oracle's plain CPU KAFMM (numpy, FP64) on a bounded problem of the same kind:
    n uniform points, the same order, leaf size and table; the operator precompute runs first
    and is not timed."""
    from oracle.kafmm import KAFMM
    pts, f = workloads.stokes_uniform(n, seed=1, dtype=np.float32)
    p64, f64 = pts.astype(np.float64), f.astype(np.float64)
    F = KAFMM("stokeslet_l4", P_ORDER, Q_LEAF)
    t0 = time.perf_counter()
    F.evaluate(p64[:2048], f64[:2048])   # builds and caches the operators
    t_ops = time.perf_counter() - t0
    t0 = time.perf_counter()
    F.evaluate(p64, f64)
    dt = time.perf_counter() - t0
    return {"value": n / dt / 1e6, "unit": "Mpoints/s", "kind": "oracle O2 (plain CPU KAFMM, numpy)",
            "sample": f"{n} uniform points, p = {P_ORDER}, q = {Q_LEAF}, four-channel table: "
                      f"{dt:.1f} s per evaluation (operators cached; their build took {t_ops:.1f} s)"}


def cpu_baseline(max_seconds=15.0):
    """The oracle's direct FP64 sum on the host cores over a bounded sample of targets of the
    same workload (all sources); scaled to Mpoints/s (targets per second)."""
    from oracle import direct
    pts, f = workloads.stokes_uniform(N_POINTS, seed=1, dtype=np.float32)
    pts64, f64 = pts.astype(np.float64), f.astype(np.float64)
    cores = os.cpu_count() or 1
    nt = 64
    direct.direct("stokeslet", pts64[:8], pts64, f64)  # load + warm
    while True:
        t0 = time.perf_counter()
        direct.direct("stokeslet", pts64[:nt], pts64, f64)
        dt = time.perf_counter() - t0
        if dt > max_seconds / 4 or nt >= N_POINTS:
            break
        nt = min(N_POINTS, int(nt * max(2.0, (max_seconds / 4) / max(dt, 1e-3))))
    # the same sums on one thread, a sample sized for about min(3 s, max_seconds / 4)
    t1 = min(3.0, max_seconds / 4)
    nt1 = int(min(N_POINTS, max(4, nt / dt / max(cores, 1) * t1)))
    prev = direct.set_threads(1)
    try:
        t0 = time.perf_counter()
        direct.direct("stokeslet", pts64[:nt1], pts64, f64)
        dt1 = time.perf_counter() - t0
    finally:
        direct.set_threads(prev)
    return {"value": nt / dt / 1e6, "unit": "Mpoints/s", "cores": cores, "kind": "oracle",
            "value_1thread": nt1 / dt1 / 1e6,
            "sample": f"O1 direct FP64 sum, {nt} of {N_POINTS} targets x all sources, "
                      f"{dt:.2f} s on {cores} threads; {nt1} targets in {dt1:.2f} s on 1 thread"}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    res = []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(max_seconds=max(2.0, 40.0 / max(1, args.steps + args.warmup)))
        if i >= args.warmup:
            res.append(r)
    v = float(np.median([r["value"] for r in res]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mpoints/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": N_POINTS / (v * 1e6) * 1e3,
            "ms_per_step_note": "extrapolated: N divided by the rate measured on the sampled "
                                "targets of each step (see cpu_baseline.sample)",
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_points": N_POINTS, "p": P_ORDER, "q": Q_LEAF,
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "Mpoints/s", "cores": res[-1]["cores"],
                             "value_1thread": float(np.median([r["value_1thread"] for r in res])),
                             "kind": "oracle", "sample": res[-1]["sample"]},
            "e2e": {"value": v, "unit": "Mpoints/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch

    from paper_2010_15155_gb300 import kafmm as K

    rank, world, local = _env_rank()
    _dist_init(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    pts, f = workloads.stokes_uniform(N_POINTS, seed=_rank_seed(1, rank), dtype=np.float32)
    y = torch.from_numpy(pts).to(dev)
    s = torch.from_numpy(f).to(dev)
    g = torch.empty((N_POINTS, 3), dtype=torch.float32, device=dev)
    prec = {"mixed": K.PREC_MIXED, "fp32": K.PREC_FP32, "fp64": K.PREC_FP64}[args.precision]
    split = {"tf32x3": K.TC_TF32X3, "bf16x3": K.TC_BF16X3, "auto": K.TC_AUTO}[args.tc_split]
    mpk = measured_peaks()
    # plan: operator precompute (SVD pseudo-inverses, translation operators), not in a step
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    plan = K.Plan(K.STOKESLET, p=P_ORDER, q=Q_LEAF, precision=prec, variant=K.ML_L4,
                  stream=stream.cuda_stream, tc_split=split, compress=args.compress)
    R = 6 * (P_ORDER - 1) ** 2 + 2
    K.kafmm_get_operator(plan.h, 0, R)   # builds the operators
    torch.cuda.synchronize(dev)
    plan_ms = (time.perf_counter() - t0) * 1e3
    K.kafmm_set_option(plan.h, K.OPT_TC_TILING, args.tc_tiling)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # accuracy against the plain FP64 GPU form and against the oracle's direct FP64 sum on
    # 4096 sampled targets (outside the timed region)
    err, err_o1 = None, None
    if rank == 0 and not args.skip_check:
        from oracle import direct as D
        ref_plan = K.Plan(K.STOKESLET, p=P_ORDER, q=Q_LEAF, precision=K.PREC_FP64,
                          variant=K.ML_L4, stream=stream.cuda_stream)
        ref_plan.set_points(y.double())
        gref = ref_plan.eval(s.double())
        plan.set_points(y)
        plan.eval(s, g)
        torch.cuda.synchronize(dev)
        err = float(torch.linalg.norm(g.double() - gref) / torch.linalg.norm(gref))
        idx = workloads.sample_targets(N_POINTS, 4096)
        p64, f64 = pts.astype(np.float64), f.astype(np.float64)
        o1 = D.direct("stokeslet", p64[idx], p64, f64)
        err_o1 = {"form": D.rel_l2(g.double().cpu().numpy()[idx], o1),
                  "fp64_form": D.rel_l2(gref.cpu().numpy()[idx], o1),
                  "targets": "4096 sampled (oracle O1, direct FP64 sum over all sources)"}
        ref_plan.close()
        del gref

    # tensor-core kernel configuration picked by the autotuner on these points (untimed setup)
    tuned = None
    if args.precision == "mixed" and args.tc_tiling == 0:
        plan.set_points(y)
        tuned = K.kafmm_autotune(plan.h, s, g, K.F32)

    def step():
        plan.set_points(y)
        plan.eval(s, g)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize(dev)
    _barrier(world)
    clocks = ClockSampler(local)
    times, phases = [], []
    torch.cuda.synchronize(dev)
    for _ in range(args.steps):
        flush.fill_(float(_))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        phases.append(plan.phase_times())
    torch.cuda.synchronize(dev)
    _barrier(world)
    clk = clocks.stop()
    ms = float(np.mean(times))
    ms = _max_over_ranks(ms, world, dev)
    value = world * N_POINTS / (ms * 1e-3) / 1e6

    # end to end through the C ABI with pinned host buffers
    yh = torch.from_numpy(pts).pin_memory()
    sh = torch.from_numpy(f).pin_memory()
    gh = torch.empty((N_POINTS, 3), dtype=torch.float32).pin_memory()
    for _ in range(2):
        plan.set_points(yh)
        plan.eval(sh, gh)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ne = max(3, args.steps // 2)
    for _ in range(ne):
        plan.set_points(yh)
        plan.eval(sh, gh)
    torch.cuda.synchronize(dev)
    e2e_ms = (time.perf_counter() - t0) / ne * 1e3

    info = plan.info()
    ph = {k: float(np.median([p[k] for p in phases])) for k in phases[0]}
    eval_only = eval_graph_timing(plan, s, g, stream, flush, args.steps)
    st_ms = near_only_timing(plan, s, g, flush)
    peaks, src = _peaks()
    cnt = K.kafmm_get_counters(plan.h)
    # dominant kernel: M->L.  Algorithmic flops per launch = V translations x 2 n^2 x 4
    # channels: the method's dense translation of an n-point check potential (the per-unit
    # figure of the path); in compressed coordinates the kernel executes r_dn x r_up per
    # translation instead (reported beside it, with the three split products and padding).
    n = 6 * (P_ORDER - 1) ** 2 + 2
    m2l_flops = info["n_v"] * 2.0 * n * n * 4
    if cnt["compressed_rows"]:
        m2l_cmp = info["n_v"] * 2.0 * cnt["rank_dn"] * cnt["rank_up"] * 4
        m2l_exec = info["n_v"] * 2.0 * cnt["compressed_rows"] ** 2 * 4 * 3
        coords = (f"executed in compressed coordinates: {cnt['rank_dn']} x {cnt['rank_up']} per "
                  f"translation (padded {cnt['compressed_rows']})")
    else:
        m2l_cmp = m2l_flops
        m2l_exec = info["n_v"] * 2.0 * n * ((n + 63) // 64 * 64) * 4 * 3
        coords = f"check potentials: {n} x {n} per translation"
    m2l_s = ph["m2l"] * 1e-3
    split_used = cnt["tc_split"]
    default_m2l = (M2L_DRAM_BYTES is not None and args.precision == "mixed" and args.compress == 2 and
                   args.tc_split == "auto" and cnt["m2l_tiling"] == "per parent neighbour")
    if args.precision == "mixed" and plan_uses_tc(plan):
        # achieved counts useful flops only (the three split products and the padding are not
        # counted); tf32x3 is measured against the TF32 MMA rate of kafmm_measure_peak
        bound, unit = "tensor", "TFLOP/s"
        if split_used == "tf32x3":
            peak = mpk["tf32_mma_tflops"]
            pk = "tf32 tcgen05 MMA rate measured by kafmm_measure_peak"
        else:
            peak = peaks["bf16_tflops"]
            pk = f"bf16 dense burst (cuBLAS), {src}"
        achieved = m2l_flops / m2l_s / 1e12
        peak_note = (f"{split_used}: {pk}; achieved = algorithmic flops (V translations x 2 x {n}^2 x 4, "
                     f"the dense translation on check potentials) / M->L time; {coords}: "
                     f"{m2l_cmp / m2l_s / 1e12:.0f} TFLOP/s useful, "
                     f"{m2l_exec / m2l_s / 1e12:.0f} TFLOP/s executed with the three split products "
                     f"and padding")
    elif args.precision == "fp64":
        bound, unit = "alu", "TFLOP/s"
        peak = mpk["fp64_fma_tflops"]
        achieved = m2l_flops / m2l_s / 1e12
        peak_note = "FP64 FMA rate measured by kafmm_measure_peak"
    else:
        bound, unit = "alu", "TFLOP/s"
        peak = mpk["fp32_fma_tflops"]
        achieved = m2l_flops / m2l_s / 1e12
        peak_note = "FP32 FMA rate measured by kafmm_measure_peak"
    # near field alone (the leaf kernel in near-only mode: U-list S->T, no L->T)
    st_gflops = info["near_pairs"] * FLOP_ST_PAIR / (st_ms * 1e-3) / 1e9
    fp32_peak = mpk["fp32_fma_tflops"]
    rsqrt_frac = info["near_pairs"] / (st_ms * 1e-3) / (mpk["mufu_rsqrt_tops"] * 1e12)
    # tree build + lists: ~48 algorithmic bytes per point (coordinates read 12, keys 8 + 8,
    # permutation 4 + 4, sorted coordinates 12) against the measured HBM copy bandwidth
    tree_gbs = N_POINTS * 48 / ((ph["tree"] + ph["lists"]) * 1e-3) / 1e9
    launches = plan_launches(plan)
    line = {
        "metric": METRIC, "value": value, "unit": "Mpoints/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": f"f32+{split_used}" if args.precision == "mixed"
        else ("f32" if args.precision == "fp32" else "f64"),
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_points": N_POINTS, "p": P_ORDER, "q": Q_LEAF,
                   "ml_table": "four-channel Laplace", "precision": args.precision,
                   "compress": args.compress,
                   "tc_split": split_used if args.precision == "mixed" else None,
                   "autotuned": tuned,
                   "m2l_tiling": K.kafmm_get_counters(plan.h)["m2l_tiling"],
                   "l2": "flushed (256 MiB write) between timed steps",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "rel_l2_vs_fp64": err,
        "rel_l2_vs_o1": err_o1,
        "plan_ms": plan_ms,
        "st_gflops": st_gflops,
        "st_roofline": {"bound": "alu", "achieved": st_gflops / 1e3, "peak": fp32_peak,
                        "unit": "TFLOP/s", "frac": st_gflops / 1e3 / fp32_peak,
                        "ms": st_ms, "rsqrt_frac": rsqrt_frac,
                        "note": "U-list pairs x 29 flop over the near-field-only leaf kernel "
                                "(CUDA events); peak = FP32 FMA rate measured by "
                                "kafmm_measure_peak; rsqrt_frac = pairs/s over the measured "
                                "MUFU rsqrt rate (one per pair)"},
        "measured_peaks": mpk,
        "tree_roofline": {"bound": "hbm", "achieved": tree_gbs, "peak": peaks["hbm_gbs"],
                          "unit": "GB/s", "frac": tree_gbs / peaks["hbm_gbs"],
                          "note": "48 B/point over tree + lists time; launch-latency bound"},
        "eval_only": eval_only,
        "phases_ms": ph,
        "tree": info,
        "roofline": {"bound": bound, "kernel": "m2l", "achieved": achieved, "peak": peak,
                     "unit": unit, "frac": achieved / peak,
                     "traffic": M2L_DRAM_BYTES if default_m2l else None,
                     "traffic_source": "DRAM bytes of one M->L launch from an ncu capture of the "
                                       "current kernel in this configuration" if default_m2l else
                                       "not captured for this configuration",
                     "peak_source": peak_note},
        "e2e": {"value": world * N_POINTS / (e2e_ms * 1e-3) / 1e6, "unit": "Mpoints/s",
                "h2d_bytes_per_step": int(pts.nbytes + f.nbytes),
                "d2h_bytes_per_step": int(gh.numel() * 4)},
        "clocks": clk,
        "gpu_launches": launches * args.steps if launches is not None else None,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
        line["cpu_baseline"]["o2"] = cpu_baseline_o2()
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_gpu_batched(args):
    """The batched workload: one forest for 512 problems vs 512 sequential calls."""
    import torch

    from paper_2010_15155_gb300 import kafmm as K

    rank, world, local = _env_rank()
    _dist_init(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    p_ord, q_leaf, n_prob = 8, 64, 512
    sizes = workloads.batched_sizes(n_prob, seed=_rank_seed(3, rank))
    pts, f, off = workloads.batched_stokes(sizes, seed=_rank_seed(3, rank))
    ntot = int(off[-1])
    y = torch.from_numpy(pts).to(dev)
    s = torch.from_numpy(f).to(dev)
    g = torch.empty((ntot, 3), dtype=torch.float32, device=dev)
    plan = K.Plan(K.STOKESLET, p=p_ord, q=q_leaf, precision=K.PREC_MIXED, variant=K.ML_L4,
                  stream=stream.cuda_stream, tc_split={"tf32x3": K.TC_TF32X3, "bf16x3": K.TC_BF16X3, "auto": K.TC_AUTO}[args.tc_split])
    K.kafmm_set_option(plan.h, K.OPT_TC_TILING, args.tc_tiling)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    err = None
    if rank == 0 and not args.skip_check:
        ref_plan = K.Plan(K.STOKESLET, p=p_ord, q=q_leaf, precision=K.PREC_FP64,
                          variant=K.ML_L4, stream=stream.cuda_stream)
        ref_plan.set_points_batched(y.double(), off)
        gref = ref_plan.eval(s.double())
        plan.set_points_batched(y, off)
        plan.eval(s, g)
        torch.cuda.synchronize(dev)
        d = (g.double() - gref).square().sum(dim=1)
        r = gref.square().sum(dim=1)
        idx = torch.from_numpy(np.repeat(np.arange(n_prob), np.diff(off))).to(dev)
        num = torch.zeros(n_prob, dtype=torch.float64, device=dev).index_add_(0, idx, d)
        den = torch.zeros(n_prob, dtype=torch.float64, device=dev).index_add_(0, idx, r)
        err = float(torch.sqrt(num / den).max())
        ref_plan.close()
        del gref

    plan.set_points_batched(y, off)
    tuned = K.kafmm_autotune(plan.h, s, g, K.F32) if args.tc_tiling == 0 else None

    def step():
        plan.set_points_batched(y, off)
        plan.eval(s, g)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize(dev)
    _barrier(world)
    clocks = ClockSampler(local)
    times, phases = [], []
    for i in range(args.steps):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        phases.append(plan.phase_times())
    torch.cuda.synchronize(dev)
    _barrier(world)
    clk = clocks.stop()
    ms = float(np.mean(times))
    ms = _max_over_ranks(ms, world, dev)
    value = world * ntot / (ms * 1e-3) / 1e6
    info = plan.info()
    ph = {k: float(np.median([p[k] for p in phases])) for k in phases[0]}
    launches = plan_launches(plan)
    # kafmm_eval of the whole batch alone: eager (host launches) and replayed from one CUDA
    # graph; their difference bounds what host launch overhead costs the batch
    eager = []
    for i in range(max(3, min(5, args.steps))):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.eval(s, g)
        e1.record(stream)
        e1.synchronize()
        eager.append(e0.elapsed_time(e1))
    eval_graph = eval_graph_timing(plan, s, g, stream, flush, args.steps)
    eval_graph["eager_ms"] = float(np.mean(eager))
    eval_graph["launches_per_eval"] = K.kafmm_get_counters(plan.h)["launches_eval"]
    split_used = K.kafmm_get_counters(plan.h)["tc_split"]
    tiling = K.kafmm_get_counters(plan.h)["m2l_tiling"]
    _, roof = _m2l_roofline(K, plan, info["n_v"], 6 * (p_ord - 1) ** 2 + 2, 4, ph["m2l"])
    plan.close()

    # the same 512 problems as sequential single-problem calls (one plan, one stream)
    seq = K.Plan(K.STOKESLET, p=p_ord, q=q_leaf, precision=K.PREC_MIXED, variant=K.ML_L4,
                 stream=stream.cuda_stream)

    def seq_step():
        for k in range(n_prob):
            a, b = int(off[k]), int(off[k + 1])
            seq.set_points(y[a:b])
            seq.eval(s[a:b], g[a:b])

    seq_step()
    torch.cuda.synchronize(dev)
    seq_ms = []
    for i in range(max(1, min(3, args.steps))):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        seq_step()
        e1.record(stream)
        e1.synchronize()
        seq_ms.append(e0.elapsed_time(e1))
    seq_launches = plan_launches(seq) * n_prob
    seq.close()
    seq_v = ntot / (float(np.mean(seq_ms)) * 1e-3) / 1e6

    line = {
        "metric": METRIC, "value": value, "unit": "Mpoints/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": f"f32+{split_used}", "data": "synthetic",
        "config": {"workload": f"stokeslet_batched_{n_prob}x_loguniform_1k_64k_p8_q64_l4",
                   "n_problems": n_prob, "n_points": ntot, "p": p_ord, "q": q_leaf,
                   "autotuned": tuned, "m2l_tiling": tiling,
                   "l2": "flushed (256 MiB write) between timed steps",
                   "parallelism": f"one batch per GPU x{world}" if world > 1 else "1 GPU"},
        "max_problem_rel_l2_vs_fp64": err,
        "st_gflops": info["near_pairs"] * FLOP_ST_PAIR / (ph["leaves"] * 1e-3) / 1e9,
        "phases_ms": ph,
        "tree": info,
        "roofline": roof,
        "eval_only": eval_graph,
        "sequential": {"value": seq_v, "unit": "Mpoints/s", "ms_per_step": float(np.mean(seq_ms)),
                       "gpu_launches_per_step": seq_launches,
                       "what": "the same problems, one kafmm_set_points + kafmm_eval each"},
        "clocks": clk,
        "gpu_launches": launches * args.steps if launches is not None else None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _timed_steps(step, plan, args, world, dev, stream, flush, local):
    """W untimed warm-up steps, then K steps timed one by one with CUDA events (L2 flushed in
    between), clocks sampled meanwhile; returns (mean ms max over ranks, median phases, clocks)."""
    import torch
    for i in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize(dev)
    _barrier(world)
    clocks = ClockSampler(local)
    times, phases = [], []
    for i in range(args.steps):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        phases.append(plan.phase_times())
    torch.cuda.synchronize(dev)
    _barrier(world)
    clk = clocks.stop()
    ms = _max_over_ranks(float(np.mean(times)), world, dev)
    ph = {k: float(np.median([p[k] for p in phases])) for k in phases[0]}
    return ms, ph, clk


def _m2l_roofline(K, plan, n_v, dense_rows, cols, m2l_ms):
    """M->L roofline of a tensor-core plan: achieved = algorithmic flops (V translations x 2 x
    dense_rows^2 x columns: the dense translation on check potentials) / M->L time; the flops
    executed in compressed coordinates (r_dn x r_up per translation) reported beside it; peak:
    the measured BF16 burst, or the TF32 MMA rate kafmm_measure_peak measured."""
    peaks, src = _peaks()
    cnt = K.kafmm_get_counters(plan.h)
    split_used, tiling = cnt["tc_split"], cnt["m2l_tiling"]
    flops = n_v * 2.0 * dense_rows * dense_rows * cols
    s = m2l_ms * 1e-3
    if cnt["compressed_rows"]:
        cmp = n_v * 2.0 * cnt["rank_dn"] * cnt["rank_up"] * cols
        note = (f"executed in compressed coordinates {cnt['rank_dn']} x {cnt['rank_up']} (padded "
                f"{cnt['compressed_rows']}): {cmp / s / 1e12:.0f} TFLOP/s useful")
    else:
        note = f"check potentials {dense_rows} x {dense_rows}"
    if split_used == "tf32x3":
        peak, pk = measured_peaks()["tf32_mma_tflops"], "tf32 tcgen05 MMA rate measured by kafmm_measure_peak"
    else:
        peak, pk = peaks["bf16_tflops"], f"bf16 dense burst (cuBLAS), {src}"
    achieved = flops / s / 1e12
    return split_used, {"bound": "tensor", "kernel": "m2l", "achieved": achieved, "peak": peak,
                        "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                        "peak_source": f"{split_used}: {pk}; achieved = algorithmic flops (the dense "
                                       f"translation, 2 x {dense_rows}^2 x {cols} per V entry) / M->L time; "
                                       f"{note}",
                        "m2l_tiling": tiling}


def run_gpu_periodic(args):
    """Triply periodic Stokeslet: 2^22 uniform points, forces minus their mean, p = 12,
    q = 128, G table (the periodic far field acts on the root's G multipole), mixed form."""
    import torch

    from paper_2010_15155_gb300 import kafmm as K

    rank, world, local = _env_rank()
    _dist_init(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    n_pts, p_ord, q_leaf = 1 << 22, 12, 128
    pts, f = workloads.stokes_uniform(n_pts, seed=_rank_seed(4, rank), zero_mean=True)
    y = torch.from_numpy(pts).to(dev)
    s = torch.from_numpy(f).to(dev)
    g = torch.empty((n_pts, 3), dtype=torch.float32, device=dev)
    plan = K.Plan(K.STOKESLET, p=p_ord, q=q_leaf, bc=K.BC_PXYZ, precision=K.PREC_MIXED,
                  variant=K.ML_G, stream=stream.cuda_stream, tc_split={"tf32x3": K.TC_TF32X3, "bf16x3": K.TC_BF16X3, "auto": K.TC_AUTO}[args.tc_split])
    K.kafmm_set_option(plan.h, K.OPT_TC_TILING, args.tc_tiling)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    plan.set_points(y)
    plan.eval(s, g)
    acc = None
    if rank == 0 and not args.skip_check:
        # a rigid shift modulo the cell (Sec. III.B) and the FP32 CUDA-core form
        sh = ((pts.astype(np.float64) + np.array([0.4173, 0.2281, 0.9011])) % 1.0).astype(np.float32)
        sh = np.minimum(sh, np.float32(1) - np.float32(2 ** -24))
        g0 = g.clone()
        plan.set_points(torch.from_numpy(sh).to(dev))
        g1 = plan.eval(s)
        p32 = K.Plan(K.STOKESLET, p=p_ord, q=q_leaf, bc=K.BC_PXYZ, precision=K.PREC_FP32,
                     variant=K.ML_G, stream=stream.cuda_stream)
        p32.set_points(y)
        g32 = p32.eval(s)
        torch.cuda.synchronize(dev)
        p32.close()

        def rel(a, b):
            return float(torch.linalg.norm(a.double() - b.double()) / torch.linalg.norm(b.double()))
        acc = {"translation_rel_l2": rel(g1, g0), "rel_l2_vs_fp32_form": rel(g0, g32)}
        del g0, g1, g32

    def step():
        plan.set_points(y)
        plan.eval(s, g)

    ms, ph, clk = _timed_steps(step, plan, args, world, dev, stream, flush, local)
    info = plan.info()
    n = 6 * (p_ord - 1) ** 2 + 2
    split_used, roof = _m2l_roofline(K, plan, info["n_v"], 3 * n, 1, ph["m2l"])
    launches = plan_launches(plan)
    line = {
        "metric": METRIC, "value": world * n_pts / (ms * 1e-3) / 1e6, "unit": "Mpoints/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": f"f32+{split_used}", "data": "synthetic",
        "config": {"workload": "stokeslet_periodic_4m_p12_q128_g", "n_points": n_pts, "p": p_ord,
                   "q": q_leaf, "bc": "pxyz", "ml_table": "G",
                   "l2": "inputs larger than L2; flushed (256 MiB write) between timed steps",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "accuracy": acc, "phases_ms": ph, "tree": info, "roofline": roof, "clocks": clk,
        "gpu_launches": launches * args.steps if launches is not None else None,
    }
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_gpu_rpy(args):
    """RPY sphere velocities: 2^20 points in 64 Gaussian clusters, radii U(0.002, 0.006),
    p = 8, q = 128, four-channel table, mixed form with the contact split; a step is
    kafmm_set_points + kafmm_eval + kafmm_rpy_velocity (overlap pass and assembly)."""
    import torch

    from oracle import direct as D
    from paper_2010_15155_gb300 import kafmm as K

    rank, world, local = _env_rank()
    _dist_init(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    n_pts, p_ord, q_leaf = 1 << 20, 8, 128
    pts, f, a = workloads.rpy_clusters(n_pts, seed=_rank_seed(2, rank))
    fb = np.concatenate([f, a[:, None]], axis=1).astype(np.float32)
    y = torch.from_numpy(pts).to(dev)
    s = torch.from_numpy(fb).to(dev)
    rad = torch.from_numpy(a).to(dev)
    g = torch.empty((n_pts, 6), dtype=torch.float32, device=dev)
    ua = torch.empty((n_pts, 3), dtype=torch.float32, device=dev)
    plan = K.Plan(K.RPY, p=p_ord, q=q_leaf, precision=K.PREC_MIXED, variant=K.ML_L4,
                  stream=stream.cuda_stream, tc_split={"tf32x3": K.TC_TF32X3, "bf16x3": K.TC_BF16X3, "auto": K.TC_AUTO}[args.tc_split])
    K.kafmm_set_option(plan.h, K.OPT_RPY_CONTACT, 1)
    K.kafmm_set_option(plan.h, K.OPT_TC_TILING, args.tc_tiling)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        plan.set_points(y)
        plan.eval(s, g)
        K.kafmm_rpy_velocity(plan.h, s, rad, g, ua, K.F32)

    step()
    torch.cuda.synchronize(dev)
    err = None
    if rank == 0 and not args.skip_check:
        # brute-force pair mobilities (FP64 oracle) at 1024 sampled spheres
        idx = workloads.sample_targets(n_pts, 1024)
        p64, fb64, a64 = pts.astype(np.float64), fb.astype(np.float64), a.astype(np.float64)
        ref = D.rpy_velocity(p64[idx], a64[idx], p64, fb64, same_set=False)
        ref -= fb64[idx, :3] / (6 * np.pi * a64[idx, None])
        err = D.rel_l2(ua.double().cpu().numpy()[idx], ref)
    ms, ph, clk = _timed_steps(step, plan, args, world, dev, stream, flush, local)
    info = plan.info()
    n = 6 * (p_ord - 1) ** 2 + 2
    split_used, roof = _m2l_roofline(K, plan, info["n_v"], n, 4, ph["m2l"])
    launches = plan_launches(plan)
    line = {
        "metric": METRIC, "value": world * n_pts / (ms * 1e-3) / 1e6, "unit": "Mpoints/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": f"f32+{split_used}", "data": "synthetic",
        "config": {"workload": "rpy_clusters_1m_64c_p8_q128_l4", "n_points": n_pts, "p": p_ord,
                   "q": q_leaf, "ml_table": "four-channel Laplace", "contact_split": True,
                   "l2": "flushed (256 MiB write) between timed steps",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "velocity_rel_l2_vs_brute_force_1024_sampled": err,
        "phases_ms": ph, "tree": info, "roofline": roof, "clocks": clk,
        "gpu_launches": launches * args.steps if launches is not None else None,
        "gpu_launches_note": "set_points + eval launches; the velocity pass adds its own",
    }
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_convergence(args):
    """The paper's convergence benchmark (Sec. III.A): 10^6 points with log-normal coordinates
    (Eq. ptdist, m = -1, s = 0.5) in [0, 32)^3, source values U(-1, 1), leaves of at most 2000
    points, orders m = 6..16, eps_L2 of every target value relative to m = 16; plain FP64
    form.  Laplace and Stokeslet (four-channel table).  The m = 16 result is also checked
    against the oracle's direct FP64 sum on 256 sampled targets."""
    import torch

    from oracle import direct as D
    from paper_2010_15155_gb300 import kafmm as K

    rank, world, local = _env_rank()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    n, L, q = 1000000, 32.0, 2000
    orders = (6, 8, 10, 12, 14, 16)
    pts = workloads.lognormal_points(n, seed=5) * L
    rng = np.random.default_rng(6)
    y = torch.from_numpy(pts).cuda()
    idx = workloads.sample_targets(n, 256)
    out = {"metric": "eps_L2 relative to m = 16 (Sec. III.A)", "impl": "gb300",
           "data": "synthetic", "dtype": "f64",
           "config": {"workload": "lognormal_1m_L32_q2000", "n_points": n, "L": L, "q": q,
                      "orders": list(orders), "precision": "fp64"}, "kernels": {}}
    for name, kern, ks in (("laplace", K.LAPLACE, 1), ("stokeslet", K.STOKESLET, 3)):
        sv = rng.uniform(-1.0, 1.0, (n, ks))
        s = torch.from_numpy(sv).cuda()
        g, ms, info = {}, {}, None
        for m in orders:
            plan = K.Plan(kern, p=m, q=q, precision=K.PREC_FP64, variant=K.ML_L4,
                          origin=(0.0, 0.0, 0.0), L=L)
            plan.set_points(y)
            g[m] = plan.eval(s).cpu().numpy()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.set_points(y)
            plan.eval(s)
            e1.record()
            e1.synchronize()
            ms[m] = e0.elapsed_time(e1)
            info = plan.info()
            plan.close()
        ref = D.direct(name, pts[idx], pts, sv)
        out["kernels"][name] = {
            "eps_l2_vs_m16": {m: D.rel_l2(g[m], g[16]) for m in orders[:-1]},
            "m16_vs_direct_256_sampled": D.rel_l2(g[16][idx], ref),
            "ms_per_step": ms, "tree": {k: info[k] for k in ("nbox", "nleaf", "nlevels", "n_v")}}
    print(json.dumps(out), flush=True)
    return 0


def run_errors(args):
    """FMM error of every form against the oracle's direct FP64 sum (O1), per kernel and order:
    N = 65536 uniform points, q = 64, 512 sampled targets (Sec. III.A's eps_L2 on a sample).
    Forms: plain FP64, FP32 on CUDA cores, mixed (tensor cores, compressed coordinates)."""
    import torch

    from oracle import direct as D
    from paper_2010_15155_gb300 import kafmm as K

    rank, world, local = _env_rank()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    n, q = 65536, 64
    rng = np.random.default_rng(7)
    pts = np.minimum(rng.random((n, 3)), 1.0 - 2.0 ** -24)
    p32 = pts.astype(np.float32).astype(np.float64)
    idx = workloads.sample_targets(n, 512)
    cases = [  # name, kernel, ML variant, oracle kernel, orders
        ("laplace", K.LAPLACE, K.ML_L4, "laplace", (6, 8, 10, 12)),
        ("stokeslet_four_channel", K.STOKESLET, K.ML_L4, "stokeslet", (6, 8, 10, 12)),
        ("stokeslet_g_table", K.STOKESLET, K.ML_G, "stokeslet", (6, 8, 10)),
        ("rpy_four_channel", K.RPY, K.ML_L4, "rpy", (6, 8, 10, 12)),
        ("regularized_stokeslet", K.STOKES_REG, K.ML_G, "stokeslet_reg", (6, 8, 10)),
        ("laplace_charge_dipole", K.LAPLACE_QD, K.ML_L4, "laplace_qd", (6, 8, 10, 12)),
        ("stokes_double_layer", K.STOKES_DL, K.ML_L4, "stokes_dl", (6, 8, 10)),
    ]
    forms = (("fp64", K.PREC_FP64), ("fp32", K.PREC_FP32), ("mixed", K.PREC_MIXED))
    out = {"metric": "relative L2 error against the direct FP64 sum (O1), 512 sampled targets",
           "impl": "gb300", "data": "synthetic",
           "config": {"workload": "errors_uniform_64k_q64", "n_points": n, "q": q,
                      "targets": "512 sampled"}, "table": {}}
    for name, kern, var, okern, orders in cases:
        ks = K.KDIM[kern][0]
        s = rng.standard_normal((n, ks))
        if kern == K.RPY:
            s[:, 3] = rng.uniform(0.0, 2e-3, n)
        if kern == K.STOKES_REG:
            s[:, 3] = rng.uniform(0.0, 1e-4, n)
        s32 = s.astype(np.float32).astype(np.float64)
        ref = {"fp64": D.direct(okern, pts[idx], pts, s),
               "f32in": D.direct(okern, p32[idx], p32, s32)}
        row = {}
        for p in orders:
            cell = {}
            for fname, prec in forms:
                dt = torch.float64 if prec == K.PREC_FP64 else torch.float32
                plan = K.Plan(kern, p=p, q=q, precision=prec, variant=var)
                src = pts if prec == K.PREC_FP64 else p32
                plan.set_points(torch.from_numpy(src).to(dt).cuda())
                sv = s if prec == K.PREC_FP64 else s32
                g = plan.eval(torch.from_numpy(sv).to(dt).cuda()).double().cpu().numpy()
                plan.close()
                cell[fname] = D.rel_l2(g[idx], ref["fp64" if prec == K.PREC_FP64 else "f32in"])
            row[p] = cell
        out["table"][name] = row
    print(json.dumps(out), flush=True)
    return 0


def run_leafsweep(args):
    """The leaf-size trade-off (Sec. III.A uses at most 2000 points per leaf): the paper's
    log-normal cloud (10^6 points, Eq. ptdist, m = -1, s = 0.5, L = 32), Stokeslet, p = 10,
    mixed form, q = 32 .. 2000: step time (set_points + eval, CUDA events, L2 flushed between
    steps) and the error against the direct FP64 sum on 512 sampled targets."""
    import torch

    from oracle import direct as D
    from paper_2010_15155_gb300 import kafmm as K

    rank, world, local = _env_rank()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    n, L = 1000000, 32.0
    pts = (workloads.lognormal_points(n, seed=5) * L).astype(np.float32)
    f = np.random.default_rng(6).uniform(-1.0, 1.0, (n, 3)).astype(np.float32)
    idx = workloads.sample_targets(n, 512)
    ref = D.direct("stokeslet", pts[idx].astype(np.float64), pts.astype(np.float64), f.astype(np.float64))
    y = torch.from_numpy(pts).to(dev)
    s = torch.from_numpy(f).to(dev)
    g = torch.empty((n, 3), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    rows = {}
    for q in (32, 64, 128, 256, 512, 1000, 2000):
        plan = K.Plan(K.STOKESLET, p=10, q=q, precision=K.PREC_MIXED, variant=K.ML_L4,
                      origin=(0.0, 0.0, 0.0), L=L, stream=stream.cuda_stream)

        def step():
            plan.set_points(y)
            plan.eval(s, g)
        ms, ph, _ = _timed_steps(step, plan, argparse.Namespace(warmup=2, steps=5), 1, dev, stream, flush, local)
        err = D.rel_l2(g.double().cpu().numpy()[idx], ref)
        info = plan.info()
        rows[q] = {"ms_per_step": ms, "mpoints_s": n / (ms * 1e-3) / 1e6, "rel_l2_vs_o1": err,
                   "phases_ms": ph, "nleaf": info["nleaf"], "nlevels": info["nlevels"],
                   "near_pairs": info["near_pairs"], "n_v": info["n_v"]}
        plan.close()
    out = {"metric": "Stokeslet KAFMM step time and error vs leaf size q (Sec. III.A cloud)",
           "impl": "gb300", "data": "synthetic", "dtype": "f32+bf16x3",
           "config": {"workload": "lognormal_1m_L32_p10_leafsweep", "n_points": n, "L": L, "p": 10,
                      "precision": "mixed", "l2": "flushed (256 MiB write) between timed steps"},
           "by_q": rows}
    print(json.dumps(out), flush=True)
    return 0


def eval_graph_timing(plan, s, g, stream, flush, steps):
    """kafmm_eval alone for the current points, captured once in a CUDA graph (the plan in
    asynchronous mode) and replayed; per replay CUDA-event time with L2 flushed in between."""
    import torch

    from paper_2010_15155_gb300 import kafmm as K
    K.kafmm_set_option(plan.h, K.OPT_SYNC, 0)
    K.kafmm_eval(plan.h, s, g, K.F32)   # every buffer exists before the capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        K.kafmm_set_option(plan.h, K.OPT_STREAM, torch.cuda.current_stream().cuda_stream)
        K.kafmm_eval(plan.h, s, g, K.F32)
    K.kafmm_set_option(plan.h, K.OPT_STREAM, stream.cuda_stream)
    times = []
    for i in range(max(3, steps)):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    K.kafmm_status(plan.h)
    K.kafmm_set_option(plan.h, K.OPT_SYNC, 1)
    del graph
    ms = float(np.mean(times))
    n = g.shape[0]
    return {"value": n / (ms * 1e-3) / 1e6, "unit": "Mpoints/s", "ms": ms,
            "how": "kafmm_eval captured once in a CUDA graph and replayed (tree kept)"}


def near_only_timing(plan, s, g, flush, reps=5):
    """The leaf kernel alone in near-only mode (U-list S->T, no far field): median of its
    CUDA-event phase time over reps evaluations, L2 flushed before each."""
    import torch

    from paper_2010_15155_gb300 import kafmm as K
    K.kafmm_set_option(plan.h, K.OPT_NEAR_ONLY, 1)
    t = []
    for i in range(reps):
        flush.fill_(float(i))
        K.kafmm_eval(plan.h, s, g, K.F32)
        t.append(K.kafmm_phase_times(plan.h)["leaves"])
    torch.cuda.synchronize()
    K.kafmm_set_option(plan.h, K.OPT_NEAR_ONLY, 0)
    return float(np.median(t))


def plan_uses_tc(plan):
    from paper_2010_15155_gb300 import kafmm as K
    return bool(K.kafmm_get_counters(plan.h)["tensor_core_m2l"])


def plan_launches(plan):
    from paper_2010_15155_gb300 import kafmm as K
    return K.kafmm_get_counters(plan.h)["launches_per_step"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp32", "fp64"])
    ap.add_argument("--tc-split", default="auto", choices=["auto", "tf32x3", "bf16x3"])
    ap.add_argument("--workload", default="stokeslet",
                    choices=["stokeslet", "batched", "periodic", "rpy", "convergence", "errors",
                             "leafsweep"])
    ap.add_argument("--tc-tiling", type=int, default=0, choices=[0, 1, 2],
                    help="M->L tiling: 0 automatic, 1 whole V lists, 2 per parent neighbour")
    ap.add_argument("--compress", type=int, default=2, choices=[0, 1, 2],
                    help="mixed form: 0 check potentials, 1 compressed coordinates, 2 compressed "
                         "with the rank rounded down to a multiple of 64")
    ap.add_argument("--skip-check", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_gpu_batched(args)
    if args.workload == "periodic":
        return run_gpu_periodic(args)
    if args.workload == "rpy":
        return run_gpu_rpy(args)
    if args.workload == "convergence":
        return run_convergence(args)
    if args.workload == "errors":
        return run_errors(args)
    if args.workload == "leafsweep":
        return run_leafsweep(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
