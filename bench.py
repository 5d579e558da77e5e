#!/usr/bin/env python3
"""Benchmark of the FP64 H12 least-squares path on GB300.

One step = one pass of the whole hot path over the two FP64 matrices of the
plain-method workload, with inputs resident in HBM:
  tall 16384 x 2048 and square 8192 x 8192, iid N(0,1) (seeds 2 and 3):
  restore A from its pristine copy, in-place H12 factorization (slqr_factor,
  keeping the compact-WY store), Q^T applied to 1 and to 64 N(0,1) right-hand
  sides (slqr_apply_qt), back-substitution of all 65 (slqr_solve_r).
Throughput is counted with the algorithmic Householder flop counts
(2mn^2 - 2n^3/3 per factorization, 4mn - 2n^2 per right-hand side for Q^T,
n^2 per right-hand side for the solve), whatever the blocking does.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one process per GPU: the path does not shard, so
every rank runs its own replica of the workload ("replicas only"; weak
scaling).  --impl reference times the CPU oracle (plain sequential C, FP64) on
a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "QR GFLOP/s & batched QR+solves/s vs plain FP64 at <=1e-10 err; p50/p99 latency"
UNIT = "GFLOP/s"
SHAPES = [(16384, 2048, 2), (8192, 8192, 3)]   # (m, n, seed)
NRHS = (1, 64)
WORKLOAD = ("plain FP64 H12 least squares: tall 16384x2048 + square 8192x8192 iid N(0,1); "
            "factor + Q^T (1 and 64 RHS) + back-substitution (65 RHS)")
# FP64 FMA pipe: 2 DFMA (4 flops) per clock per SM x 152 SMs x 2070 MHz
FP64_PEAK_TFLOPS = 4 * 152 * 2.070e9 / 1e12
CPU_SAMPLE_COLS = 512   # oracle sample: leading m x 512 block of each matrix
# factorization-only timings reported beside the step (N(0,1), seeds 2, 3, 4)
FACTOR_ONLY_SHAPES = [(16384, 2048, 2), (8192, 8192, 3), (8192, 4096, 4)]
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the two
# trailing-update kernels, scaled to this program's launches from a one-pass
# capture of those two kernels alone on a small case larger than L2:
#   python bench.py --ncu-case 8192 2048 && ncu --metrics dram__bytes_read.sum,\
#     dram__bytes_write.sum,gpu__time_duration.sum --clock-control none \
#     -k regex:"gemm_(vtx|upd)_kernel" -c 400 --csv python bench.py --ncu-case 8192 2048
# There vtx moved 1.119 and upd 0.638 times their algorithmic bytes (vtx: 8 M (N + 64)
# read; upd: X read and written, V and W' read); times this program's average algorithmic
# bytes per launch (vtx 52.23 MB, upd 101.72 MB).  Re-measure the same way (never the
# full-size program with DRAM counters) and reset to None whenever either kernel changes.
TRAFFIC_PER_LAUNCH = {"vtx": {"dram": 1.119 * 52.23e6, "algorithmic": 52.23e6},
                      "upd": {"dram": 0.638 * 101.72e6, "algorithmic": 101.72e6}}


def max_over_ranks(ms, dist=None, device="cpu"):
    """The slowest rank's time (the job's time): an all-reduce MAX over the
    ranks (NCCL on the GPU, gloo on the CPU), or `ms` itself on one rank."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(flops_per_step, steps, world, t_max_ms):
    """Whole-job GFLOP/s of `world` replicas, each doing `steps` steps, timed
    by the slowest rank (weak scaling: the work per rank is fixed)."""
    return world * flops_per_step * steps / (t_max_ms / 1e3) / 1e9


def step_flops(shapes=SHAPES, nrhs=NRHS):
    total = 0.0
    for m, n, _ in shapes:
        total += 2.0 * m * n * n - 2.0 * n ** 3 / 3.0
        r = sum(nrhs)
        total += r * (4.0 * m * n - 2.0 * n * n)
        total += r * float(n) * n
    return total


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"slqr_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            out = parse_clock_samples(f)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return out


def parse_clock_samples(lines):
    """Median and maximum SM clock and the throttle reasons seen in the lines
    of `nvidia-smi --query-gpu=<ClockSampler.FIELDS> --format=csv,noheader,nounits`."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
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
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# CPU oracle on a bounded sample (the cpu_baseline leg and the reference arm)
# ----------------------------------------------------------------------------
def oracle_sample(mats):
    """Run the oracle's full LS solve on the leading m x CPU_SAMPLE_COLS block of
    each matrix; returns (flops, seconds)."""
    import oracle
    oracle.build()
    flops, secs = 0.0, 0.0
    for (m, n, _), (A, b) in zip(SHAPES, mats):
        p = min(n, CPU_SAMPLE_COLS)
        As = np.asfortranarray(A[:, :p])
        t0 = time.perf_counter()
        oracle.lstsq(As, b)
        secs += time.perf_counter() - t0
        flops += 2.0 * m * p * p - 2.0 * p ** 3 / 3.0 + (4.0 * m * p - 2.0 * p * p) + p * p
    return flops, secs


def cpu_sample_desc():
    return (f"oracle (gcc -O2, 1 thread) factor + Q^T b + solve of the leading m x "
            f"{CPU_SAMPLE_COLS} column block of each matrix (16384x{CPU_SAMPLE_COLS}, "
            f"8192x{CPU_SAMPLE_COLS})")


SERVE_ORACLE_SAMPLE = 24       # requests of the serving stream timed on the oracle
BATCH_ORACLE_PER_CORE = 200    # batch problems per host core in the all-cores oracle run


def start_oracle_legs(mixed_in):
    """The CPU legs beyond the headline sample, started before the GPU work so
    that they run on the host cores meanwhile (spawned worker processes,
    oracle/jobs.py): the oracle's solves of the 8192 x 4096 conditioned
    matrices (their timing, and the reference solutions every mixed-precision
    cell is compared with) and a sample of the request stream, one request at
    a time on one core."""
    from oracle import jobs
    import workloads
    r = jobs.Runner(workers=4)
    for kappa, (A, bc, xt, br) in (mixed_in or {}).items():
        r.submit(f"cond_{kappa:.0e}", A.cpu().numpy(), [bc.cpu().numpy(), br.cpu().numpy()])
    t, n, meq, seeds = workloads.serving_stream(SERVE_ORACLE_SAMPLE, 100.0)
    r.submit_call("requests", jobs.requests_job,
                  list(zip(n.tolist(), meq.tolist(), seeds.tolist())))
    return r


def _warm(_):
    return os.getpid()


def oracle_batch_all_cores():
    """The oracle on a bounded sample of the 20,000-problem batch (its first
    BATCH_ORACLE_PER_CORE x cores problems: the same shape distribution), one
    chunk of problems per host core in spawned processes, and the same
    per-core rate.  Returns problems/s over all cores and per core."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import oracle
    import workloads
    from oracle import jobs
    oracle.build()
    cores = os.cpu_count() or 1
    ms, ns = workloads.batch_shapes(BATCH_COUNT)
    count = min(BATCH_COUNT, BATCH_ORACLE_PER_CORE * cores)
    chunks = [(ms[i:count:cores].tolist(), ns[i:count:cores].tolist(), workloads.SEED_BATCH + 17 + i)
              for i in range(cores)]
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as pool:
        list(pool.map(_warm, range(cores)))                  # workers started and imported
        t0 = time.perf_counter()
        secs = list(pool.map(jobs.batch_chunk_job, *zip(*chunks)))
        wall = time.perf_counter() - t0
    flops = sum(2.0 * m * n * n - 2.0 * n ** 3 / 3.0 + 4.0 * m * n - n * n
                for m, n in zip(ms[:count].tolist(), ns[:count].tolist()))
    return {"problems": count, "cores": cores, "wall_s": wall,
            "problems_per_s_all_cores": count / wall, "gflops_all_cores": flops / wall / 1e9,
            "problems_per_s_per_core": count / sum(secs),
            "sample": f"the first {count} problems of the seeded batch (m ~ U{{16..512}}, "
                      f"n ~ U{{ceil(m/4)..m}}), one chunk per core"}


def finish_oracle_legs(r, mixed, sols, inputs):
    """Collect the background legs, state every mixed cell's error against the
    oracle, then time the all-cores batch sample and the 256 x 128 problem."""
    import oracle
    import workloads
    res, oracle_x = {}, {}
    m3, n3 = MIXED_SHAPE
    fl3 = 2.0 * m3 * n3 * n3 - 2.0 * n3 ** 3 / 3.0
    for kappa in (MIXED_KAPPAS if inputs else ()):
        out = r.result(f"cond_{kappa:.0e}", timeout=1200)
        oracle_x[kappa] = out["x"]
        res[f"config3_8192x4096_kappa_{kappa:.0e}"] = {
            "factor_s": out["factor_seconds"], "solve_s_2rhs": out["solve_seconds"],
            "factor_gflops": fl3 / out["factor_seconds"] / 1e9, "cores": 1}
    if mixed is not None and inputs:
        mixed_errors(mixed, sols, inputs, oracle_x)
    req = np.array(r.value("requests", timeout=900)) * 1e3
    res["config5_requests"] = {"count": int(req.size), "p50_ms": float(np.percentile(req, 50)),
                               "p99_ms": float(np.percentile(req, 99)),
                               "mean_ms": float(req.mean()), "cores": 1,
                               "sample": f"the first {req.size} requests of the seeded stream "
                                         "(dense oracle LS solve of [L^T; C], one at a time)"}
    r.shutdown()
    res["config4_batch"] = oracle_batch_all_cores()
    A1, b1 = workloads.gaussian(256, 128, workloads.SEED_SMALL)
    ts = []
    for _ in range(25):
        t0 = time.perf_counter()
        oracle.lstsq(A1, b1)
        ts.append(time.perf_counter() - t0)
    res["config1_256x128_us"] = float(np.median(ts) * 1e6)
    return res


def gen_inputs():
    import workloads
    mats = []
    for m, n, seed in SHAPES:
        A, b = workloads.gaussian(m, n, seed)
        mats.append((A, b))
    return mats


# ----------------------------------------------------------------------------
# reference arm: the oracle as it stands, on the host cores
# ----------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    mats = gen_inputs()
    for _ in range(args.warmup):
        oracle_sample(mats)
    tot_f, tot_s = 0.0, 0.0
    for _ in range(args.steps):
        f, s = oracle_sample(mats)
        tot_f += f
        tot_s += s
    value = tot_f / tot_s / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_s / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": cpu_sample_desc()},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": cpu_sample_desc()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def colmajor_cuda(a, device):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a.T)).to(device).t()


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2506_09463_gb300 import abi, api

    device = torch.device("cuda", local_rank)
    torch.cuda.set_device(device)
    dist = None
    if world > 1:
        import torch.distributed as dist
    ctx = api.Context(local_rank)
    stream = torch.cuda.current_stream(device)
    mats_h = gen_inputs()
    # the 8192 x 4096 conditioned matrices, and the CPU legs that run on the
    # host cores while the GPU works (rank 0 of a single-GPU run only)
    cpu_legs = (rank == 0 and world == 1 and not args.no_cpu_baseline)
    mixed_in = mixed_inputs(device) if not args.no_mixed else None
    legs = start_oracle_legs(mixed_in if cpu_legs else None) if cpu_legs else None

    # device-resident inputs and working buffers
    bufs = []
    import workloads
    for (m, n, seed), (A, b) in zip(SHAPES, mats_h):
        A0 = colmajor_cuda(A, device)
        Aw = A0.t().clone().t()
        B0 = torch.empty(m, sum(NRHS), dtype=torch.float64, device=device)
        B0[:, 0] = torch.from_numpy(b).to(device)
        B0[:, 1:] = torch.from_numpy(workloads.gaussian_rhs(m, NRHS[1], seed)).to(device)
        B0 = B0.t().contiguous().t()
        Bw = B0.t().clone().t()
        up = torch.empty(n, dtype=torch.float64, device=device)
        wy = ctx.wy_buffer(m, n, device=device)
        bufs.append(dict(m=m, n=n, A0=A0, A=Aw, B0=B0, B=Bw, up=up, wy=wy))

    def step(timed_copy=True):
        for d in bufs:
            d["A"].copy_(d["A0"])
            d["B"].copy_(d["B0"])
            ctx.factor(d["A"], d["up"], d["wy"])
            ctx.apply_qt(d["A"], d["up"], d["B"][:, :1], wy=d["wy"])
            ctx.apply_qt(d["A"], d["up"], d["B"][:, 1:], wy=d["wy"])
            ctx.solve_r(d["A"], d["B"])

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(device)

    for _ in range(args.warmup):
        step()
    st = ctx.sync()
    if st != 0:
        raise RuntimeError(f"device status {st} after warm-up: {abi.slqr_last_error(ctx.ctx)}")

    # ---- timed region (device-resident inputs) ----
    clocks = ClockSampler(local_rank)
    abi.slqr_profile(ctx.ctx, True)
    launches0 = abi.slqr_launch_count(ctx.ctx)
    barrier()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    launches = abi.slqr_launch_count(ctx.ctx) - launches0
    ms = e0.elapsed_time(e1)
    prof = {name: abi.slqr_profile_read(ctx.ctx, k) for k, name in enumerate(abi.KERNEL_NAMES)}
    abi.slqr_profile(ctx.ctx, False)
    st = ctx.sync()
    if st != 0:
        raise RuntimeError(f"device status {st}: {abi.slqr_last_error(ctx.ctx)}")
    t_max = max_over_ranks(ms, dist, device)
    ms_per_step = t_max / args.steps
    flops = step_flops()
    value = job_throughput(flops, args.steps, world, t_max)

    # ---- end-to-end through the public API with host buffers ----
    pinned = []
    for d, (A, b) in zip(bufs, mats_h):
        Ah = torch.from_numpy(np.ascontiguousarray(A.T)).pin_memory()       # n x m = A^T rows
        Bh = d["B0"].t().contiguous().cpu().pin_memory()                     # nrhs x m
        Xh = torch.empty(sum(NRHS), d["n"], dtype=torch.float64).pin_memory()
        pinned.append((Ah, Bh, Xh))
    h2d = sum(Ah.numel() * 8 + Bh.numel() * 8 for Ah, Bh, _ in pinned)
    d2h = sum(Xh.numel() * 8 for _, _, Xh in pinned)

    # The host-to-device copies run on a second stream, each as soon as its
    # device buffer is free: the copy of the second matrix overlaps the solve
    # of the first, and the next step's copy of the first matrix overlaps the
    # solve of the second.  Every copy is inside the timed region.
    copy_stream = torch.cuda.Stream(device)
    free_ev = [torch.cuda.Event() for _ in bufs]      # buffer i may be overwritten
    ready_ev = [torch.cuda.Event() for _ in bufs]     # buffer i holds this step's input

    def e2e_step():
        for i, (d, (Ah, Bh, Xh)) in enumerate(zip(bufs, pinned)):
            copy_stream.wait_event(free_ev[i])
            with torch.cuda.stream(copy_stream):
                d["A"].t().copy_(Ah, non_blocking=True)
                d["B"].t().copy_(Bh, non_blocking=True)
            ready_ev[i].record(copy_stream)
        for i, (d, (Ah, Bh, Xh)) in enumerate(zip(bufs, pinned)):
            stream.wait_event(ready_ev[i])
            ctx.factor(d["A"], d["up"], d["wy"])
            ctx.apply_qt(d["A"], d["up"], d["B"][:, :1], wy=d["wy"])
            ctx.apply_qt(d["A"], d["up"], d["B"][:, 1:], wy=d["wy"])
            ctx.solve_r(d["A"], d["B"])
            Xh.copy_(d["B"][: d["n"]].t(), non_blocking=True)
            free_ev[i].record(stream)

    e2e_step()
    barrier()
    e0.record(stream)
    for ev in free_ev:                                 # the timed copies start after e0
        ev.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), dist, device)
    e2e_value = job_throughput(flops, args.steps, world, e2e_ms)
    if ctx.sync() != 0:
        raise RuntimeError(abi.slqr_last_error(ctx.ctx))

    # ---- factorization alone, per shape (context for the paper's QR-only times) ----
    factor_only = {}
    for (m, n, seed) in FACTOR_ONLY_SHAPES:
        A0 = colmajor_cuda(workloads.gaussian(m, n, seed)[0], device)
        Aw = A0.t().clone().t()
        up = torch.empty(n, dtype=torch.float64, device=device)
        times = []
        for rep in range(3):
            Aw.copy_(A0)
            barrier()
            e0.record(stream)
            ctx.factor(Aw, up)
            e1.record(stream)
            barrier()
            times.append(e0.elapsed_time(e1))
        t = min(times)
        fl = 2.0 * m * n * n - 2.0 * n ** 3 / 3.0
        factor_only[f"{m}x{n}"] = {"ms": t, "gflops": fl / (t / 1e3) / 1e9,
                                   "frac_of_fp64_peak": fl / (t / 1e3) / 1e12 / FP64_PEAK_TFLOPS}
        del A0, Aw
    if ctx.sync() != 0:
        raise RuntimeError(abi.slqr_last_error(ctx.ctx))

    # ---- the 256 x 128 single problem: latency of one LS solve ----
    single = single_problem_latency(ctx, device, stream, barrier)

    # ---- batched workload: 20,000 uneven problems in one persistent launch ----
    batch = run_batch_workload(ctx, device, stream, barrier) if not args.no_batch else None
    mixed, sols = (run_mixed_workload(ctx, device, stream, barrier, mixed_in)
                   if not args.no_mixed else (None, None))
    serving = run_serving_workload(local_rank) if not args.no_serving else None

    # ---- measured arithmetic peaks (diagnostic probes of the library) ----
    peaks = {}
    for name, kind in (("fp64_fma_tflops", abi.SLQR_PEAK_FP64_FMA),
                       ("tf32_tensor_tflops", abi.SLQR_PEAK_TF32_TC)):
        stp, v = abi.slqr_measure_peak(ctx.ctx, kind)
        peaks[name] = v if stp == abi.SLQR_OK else None

    # ---- roofline of the dominant kernel (most device time in the timed region) ----
    # the dominant kernel is the family carrying most of the algorithmic flops
    # (the two trailing-update GEMMs carry equal shares; take the slower one);
    # panel launches overlap those GEMMs on a second stream, so their event
    # times are not exclusive
    dom = max(("vtx", "upd"), key=lambda k: prof[k][0])
    dms, dn, dfl = prof[dom]
    achieved = (dfl / dn) / (dms / dn / 1e3) / 1e12 if dn else 0.0
    tr = TRAFFIC_PER_LAUNCH.get(dom)
    roofline = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": tr["dram"] if tr else None,
                "traffic_algorithmic": tr["algorithmic"] if tr else None,
                "traffic_unit": "bytes per launch (ncu on 8192x2048, scaled to this program's launches)",
                "peak_source": "derived: FP64 FMA pipe 4 flop/clk/SM x 152 SMs x 2070 MHz",
                "peak_measured": peaks.get("fp64_fma_tflops"),
                "frac_of_measured": (achieved / peaks["fp64_fma_tflops"]
                                     if peaks.get("fp64_fma_tflops") else None)}
    kernels = {k: {"ms": v[0], "launches": v[1], "share_of_step_time": v[0] / max(1e-9, ms),
                   "tflops": (v[2] / (v[0] / 1e3) / 1e12) if v[0] > 0 else 0.0}
               for k, v in prof.items()}

    if rank != 0:
        return 0
    cpu, oracle_legs = None, None
    if cpu_legs:
        oracle_legs = finish_oracle_legs(legs, mixed, sols, mixed_in)
        single["oracle_us"] = oracle_legs["config1_256x128_us"]
        f, s = oracle_sample(mats_h)
        cpu = {"value": f / s / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": cpu_sample_desc(), "seconds": s}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded N(0,1))",
        "config": {"workload": WORKLOAD, "shapes": [[m, n] for m, n, _ in SHAPES],
                   "nrhs": list(NRHS), "panel_width": [abi.slqr_panel_width(m, n) for m, n, _ in SHAPES],
                   "l2": "inputs larger than L2 (268 MB and 537 MB matrices, no flush)",
                   "parallelism": "replicas only" if world > 1 else "single GPU"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "clocks": clk,
        "peaks_measured": peaks,
        "gpu_launches": launches,
        "kernels": kernels,
        "factor_only": factor_only,
        "single_256x128": single,
        "batch": batch,
        "mixed_8192x4096": mixed,
        "serving": serving,
        "oracle": oracle_legs,
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


MIXED_KAPPAS = (1e2, 1e6, 1e10)
MIXED_SHAPE = (8192, 4096)
U64 = 2.0 ** -53


def mixed_inputs(device):
    """The 8192 x 4096 conditioned matrices (kappa 1e2 / 1e6 / 1e10, seeds 4 / 5 /
    6), drawn on the device: {kappa: (A, b_consistent, x_true, b_random)}."""
    import workloads
    m, n = MIXED_SHAPE
    return {k: workloads.conditioned_device(m, n, k, device=device) for k in MIXED_KAPPAS}


def run_mixed_workload(ctx, device, stream, barrier, inputs):
    """Every (kappa, b, precision) cell of the 8192 x 4096 conditioned workload:
    the FP64 path (factor + Q^T b + solve) and slqr_lstsq_mixed_ex in its
    automatic mode (Bjorck sweeps, then GMRES-IR, then the flagged FP64
    fallback) for SLQR_FP32 / SLQR_TF32 / SLQR_BF16X3.  Returns the timings and
    statuses, and the solutions (host) whose errors against the oracle
    mixed_errors() states once the oracle's solves are done."""
    import torch
    from paper_2506_09463_gb300 import abi
    m, n = MIXED_SHAPE
    out, sols = {}, {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flops = 2.0 * m * n * n - 2.0 * n ** 3 / 3.0 + (4.0 * m * n - 2.0 * n * n) + n * n
    precs = (("fp32", abi.SLQR_FP32), ("tf32", abi.SLQR_TF32), ("bf16x3", abi.SLQR_BF16X3))
    # one untimed solve per precision first: the first call of a precision
    # loads its kernels and builds its tensor maps and workspaces (1-2 ms)
    A0, _, _, b0 = inputs[MIXED_KAPPAS[0]]
    for _, prec in precs:
        x = torch.zeros(n, dtype=torch.float64, device=device)
        abi.slqr_lstsq_mixed_ex(ctx.ctx, m, n, A0.data_ptr(), m, b0.data_ptr(), x.data_ptr(), prec,
                                stream.cuda_stream, fp64_fallback=1)
    stream.synchronize()
    for kappa in MIXED_KAPPAS:
        A, b_cons, x_true, b_rand = inputs[kappa]
        rec = {}
        for name, b in (("consistent", b_cons), ("random", b_rand)):
            Aw, bw = A.t().clone().t(), b.clone()
            barrier()
            e0.record(stream)
            x64, _ = ctx.lstsq(Aw, bw)
            e1.record(stream)
            barrier()
            t64 = e0.elapsed_time(e1)
            r = {"fp64_ms": t64, "fp64_gflops": flops / (t64 / 1e3) / 1e9}
            sols[(kappa, name, "fp64")] = x64.cpu().numpy().copy()
            del Aw, bw
            for pname, prec in precs:
                x = torch.zeros(n, dtype=torch.float64, device=device)
                barrier()
                e0.record(stream)
                st, info = abi.slqr_lstsq_mixed_ex(ctx.ctx, m, n, A.data_ptr(), m, b.data_ptr(),
                                                   x.data_ptr(), prec, stream.cuda_stream,
                                                   fp64_fallback=1)
                e1.record(stream)
                barrier()
                tm = e0.elapsed_time(e1)
                method = {abi.SLQR_REFINE_BJORCK: "bjorck", abi.SLQR_REFINE_GMRES: "gmres-ir",
                          abi.SLQR_REFINE_FP64: "fp64-fallback"}.get(info["method"], info["method"])
                r[pname] = {"ms": tm, "speedup_vs_fp64": t64 / tm,
                            "status": abi.STATUS_NAMES.get(st, st), "method": method,
                            "sweeps": info["sweeps"], "gmres_steps": info["gmres_steps"],
                            "gmres_iters": info["gmres_iters"], "last_step": info["err"],
                            "kappa_est": info["kappa_est"]}
                sols[(kappa, name, pname)] = x.cpu().numpy().copy()
            if name == "consistent":
                xt = x_true.cpu().numpy()
                r["fp64_err_vs_x_true"] = float(np.linalg.norm(sols[(kappa, name, "fp64")] - xt)
                                                / np.linalg.norm(xt))
            rec[name] = r
        out[f"kappa_{kappa:.0e}"] = rec
    if ctx.sync() != 0:
        raise RuntimeError("device status after the mixed workload")
    return out, sols


def mixed_errors(mixed, sols, inputs, oracle_x):
    """Per cell: ||x - x_o|| / ||x_o|| and max |x_i - x_o,i| / ||x_o||_inf against
    the oracle's solution x_o, and the tolerance max(1e-10, 64 (kappa + kappa^2
    ||r|| / (||A|| ||x_o||)) u) (||A|| = 1 by construction)."""
    for kappa in MIXED_KAPPAS:
        if kappa not in oracle_x:
            continue
        A, b_cons, x_true, b_rand = inputs[kappa]
        rec = mixed[f"kappa_{kappa:.0e}"]
        for j, (name, b) in enumerate((("consistent", b_cons), ("random", b_rand))):
            x_o = oracle_x[kappa][:, j]
            r_o = b.cpu().numpy() - A.cpu().numpy() @ x_o
            tol = max(1e-10, 64.0 * (kappa + kappa ** 2 * np.linalg.norm(r_o) /
                                     np.linalg.norm(x_o)) * U64)
            rec[name]["tol_vs_oracle"] = tol
            for pname in ("fp64", "fp32", "tf32", "bf16x3"):
                x = sols[(kappa, name, pname)]
                rel = float(np.linalg.norm(x - x_o) / np.linalg.norm(x_o))
                mx = float(np.max(np.abs(x - x_o)) / np.max(np.abs(x_o)))
                if pname == "fp64":
                    rec[name]["fp64_err_vs_oracle"] = rel
                    rec[name]["fp64_maxerr_vs_oracle"] = mx
                else:
                    rec[name][pname]["err_vs_oracle"] = rel
                    rec[name][pname]["maxerr_vs_oracle"] = mx
                    rec[name][pname]["within_tol"] = bool(rel <= tol and mx <= tol)


def single_problem_latency(ctx, device, stream, barrier, reps=50):
    """The 256 x 128 problem (seed 1): one factor + Q^T b + back-substitution,
    device time (CUDA events) and host time through the API (from the first
    call to the end of the solve, with a stream synchronisation), medians."""
    import torch
    import workloads
    A, b = workloads.gaussian(256, 128, workloads.SEED_SMALL)
    A0 = colmajor_cuda(A, device)
    b0 = torch.from_numpy(b.copy()).to(device)
    Aw = A0.t().clone().t()
    bw = b0.clone()
    up = torch.empty(128, dtype=torch.float64, device=device)
    wy = ctx.wy_buffer(256, 128, device=device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dev_us, host_us = [], []
    for _ in range(reps + 5):
        Aw.copy_(A0)
        bw.copy_(b0)
        barrier()
        t0 = time.perf_counter()
        e0.record(stream)
        ctx.factor(Aw, up, wy)
        ctx.apply_qt(Aw, up, bw, wy=wy)
        ctx.solve_r(Aw, bw)
        e1.record(stream)
        stream.synchronize()
        host_us.append((time.perf_counter() - t0) * 1e6)
        dev_us.append(e0.elapsed_time(e1) * 1e3)
    if ctx.sync() != 0:
        raise RuntimeError("device status after the 256 x 128 problem")
    return {"device_us": float(np.median(dev_us[5:])), "host_us": float(np.median(host_us[5:])),
            "reps": reps}


def run_serving_workload(ctx_device, rates=(100.0, 400.0, 1600.0), count=1000):
    """Poisson request streams of SLSQP-shaped LS subproblems [L^T; C]
    (n ~ log-U[50, 2000], m_eq ~ U{0..n/2}), FACTOR_SOLVE each, through
    slqr_submit / slqr_poll; reports solves/s and p50/p99 latency per rate
    (`count` requests, so that p99 is a percentile of 1000 samples), in FP64
    and in mixed precision (every request SLQR_FP32: the batched FP32 launch
    for m <= 512, a mixed lane above, the FP64 fallback flagged), each as a
    dense request and as a stacked one (SLQR_STACKED).  Every mixed-precision
    solution is compared with the FP64 request's solution of the same problem
    at the same rate."""
    import time
    import workloads
    from paper_2506_09463_gb300 import abi, api
    t_arr, ns, meqs, seeds = workloads.serving_stream(count, rate=1.0)
    problems = [workloads.slsqp_stack(int(ns[i]), int(meqs[i]), int(seeds[i])) for i in range(count)]
    gflop = sum(2.0 * (n + me) * n * n - 2.0 * n ** 3 / 3.0 for n, me in zip(ns, meqs)) / 1e9
    out = {"requests_per_rate": count, "mean_gflop_per_request": gflop / count,
           "shapes": "[L^T; C], n ~ log-U[50,2000], m_eq ~ U{0..n/2}, Poisson arrivals"}
    modes = (("fp64", abi.SLQR_DENSE), ("mixed", abi.SLQR_DENSE),
             ("fp64_stacked", abi.SLQR_STACKED), ("mixed_stacked", abi.SLQR_STACKED))
    x_fp64 = {}
    for mode, structure in modes:
        res_mode = {}
        mixed = mode.startswith("mixed")
        for rate in rates:
            with api.Context(ctx_device) as sctx:
                srv = api.Server(sctx)
                # warm the loop (streams, pools, lanes, kernels) with two requests
                for A, b in (problems[0], workloads.slsqp_stack(700, 200, 1)):
                    srv.wait(srv.submit(abi.SLQR_REQ_FACTOR_SOLVE, A=A, b=b,
                                        prec=abi.SLQR_FP32 if mixed else abi.SLQR_FP64))
                gaps = np.random.default_rng(int(rate)).exponential(1.0 / rate, size=count)
                arrivals = np.cumsum(gaps) - gaps[0]
                tickets = []
                t0 = time.perf_counter()
                for i in range(count):
                    while time.perf_counter() - t0 < arrivals[i]:
                        pass
                    A, b = problems[i]
                    prec = abi.SLQR_FP32 if mixed else abi.SLQR_FP64
                    tickets.append(srv.submit(abi.SLQR_REQ_FACTOR_SOLVE, A=A, b=b, prec=prec,
                                              structure=structure))
                lat, bad, fallback, xs = [], 0, 0, []
                for t in tickets:
                    r, x = srv.wait(t, timeout_s=600)
                    lat.append(r.latency_ms)
                    bad += int(r.status not in (abi.SLQR_OK, abi.SLQR_FALLBACK))
                    fallback += int(r.status == abi.SLQR_FALLBACK)
                    xs.append(x)
                wall = time.perf_counter() - t0
                lat = np.array(lat)
                rec = {"offered_req_per_s": rate, "solves_per_s": count / wall,
                       "p50_ms": float(np.percentile(lat, 50)),
                       "p99_ms": float(np.percentile(lat, 99)),
                       "failed": bad, "fp64_fallbacks": fallback, "gflops": gflop / wall}
                key = (structure, rate)
                if not mixed:
                    x_fp64[key] = xs
                elif key in x_fp64:
                    rel = [float(np.max(np.abs(a - c)) / np.max(np.abs(c)))
                           for a, c in zip(xs, x_fp64[key])]
                    rec["max_rel_diff_vs_fp64"] = max(rel)
                    rec["over_1e-10_vs_fp64"] = int(sum(r_ > 1e-10 for r_ in rel))
                res_mode[f"rate_{rate:g}"] = rec
        out[mode] = res_mode
    return out


BATCH_COUNT = 20000


def run_batch_workload(ctx, device, stream, barrier, count=BATCH_COUNT, reps=2, serial=300):
    """Factor + Q^T b + solve of `count` problems (m ~ U{16..512}, n ~ U{m/4..m},
    N(0,1), seed 7) in one persistent launch, FP64 and mixed FP32 (FP32
    factorization + FP64-residual refinement); beside it the plain
    one-at-a-time FP64 path (slqr_factor + slqr_apply_qt + slqr_solve_r per
    problem, serially on one stream) timed on the first `serial` problems."""
    import torch
    import workloads
    from paper_2506_09463_gb300 import abi
    ms, ns = workloads.batch_shapes(count)
    A_flat, b_flat, a_off, b_off = workloads.batch_problems_device(ms, ns, workloads.SEED_BATCH,
                                                                   device=device)
    A0, b0 = A_flat.clone(), b_flat.clone()
    up_flat = torch.zeros(int(ns.sum()) + 1, dtype=torch.float64, device=device)
    up_off = np.concatenate([[0], np.cumsum(ns)[:-1]])
    A_ptrs = [A_flat.data_ptr() + int(o) * 8 for o in a_off]
    b_ptrs = [b_flat.data_ptr() + int(o) * 8 for o in b_off]
    up_ptrs = [up_flat.data_ptr() + int(o) * 8 for o in up_off]
    lda = [int(m) for m in ms]
    status = torch.zeros(count, dtype=torch.int32, device=device)
    err = torch.zeros(count, dtype=torch.float64, device=device)
    flops = float(np.sum(2.0 * ms * ns * ns - 2.0 * ns ** 3 / 3.0 + 6.0 * ms * ns))
    out = {"problems": count, "shapes": "m ~ U{16..512}, n ~ U{ceil(m/4)..m}, N(0,1), seed 7",
           "algorithmic_gflop": flops / 1e9}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def time_batch(prec):
        times = []
        for rep in range(reps + 1):
            A_flat.copy_(A0)
            b_flat.copy_(b0)
            barrier()
            e0.record(stream)
            st = abi.slqr_batch_factor(ctx.ctx, list(ms), list(ns), A_ptrs, lda,
                                       up_ptrs if prec == abi.SLQR_FP64 else None, b_ptrs, prec,
                                       status.data_ptr(), err.data_ptr(), stream.cuda_stream)
            abi.check(ctx.ctx, st, "slqr_batch_factor")
            e1.record(stream)
            barrier()
            if rep:
                times.append(e0.elapsed_time(e1))
        return min(times)

    import time as _t
    for name, prec in (("fp64", abi.SLQR_FP64), ("mixed_fp32", abi.SLQR_FP32)):
        # the default setting (panels of 16, tiles of 32 for every size class),
        # then the autotuner's choice per size class, which the batch uses
        abi.slqr_batch_set_tuning(prec, -1, 0, 0)
        t_default = time_batch(prec)
        t0 = _t.perf_counter()
        stt, choice, tms = abi.slqr_batch_autotune(ctx.ctx, prec, list(ms), list(ns))
        abi.check(ctx.ctx, stt, "slqr_batch_autotune")
        tune_s = _t.perf_counter() - t0
        t = time_batch(prec)
        stv = status.cpu().numpy()
        rec = {"ms": t, "problems_per_s": count / (t / 1e3), "gflops": flops / (t / 1e3) / 1e9,
               "ok": int(np.sum(stv == 0)), "erank": int(np.sum(stv == abi.SLQR_ERANK)),
               "no_conv": int(np.sum(stv == abi.SLQR_ENOCONV)),
               "default_setting_ms": t_default,
               "default_setting_problems_per_s": count / (t_default / 1e3),
               "autotune_s": tune_s,
               "autotune_sample_ms_before_after": list(tms),
               "tuned_settings": [{"m_max": abi.slqr_batch_class_rows(c), "panel_width": nb,
                                   "tile_cols": tc, "resident": bool(rs)}
                                  for c, (nb, tc, rs) in enumerate(choice)]}
        if prec == abi.SLQR_FP32:
            ev = err.cpu().numpy()
            rec["refine_err_max"] = float(ev[stv == 0].max()) if np.any(stv == 0) else None
            # refined solutions against the FP64 batch solutions of the same problems
            x32 = b_flat.clone()
            rec["max_rel_diff_vs_fp64_batch"] = None
            if x64 is not None:
                worst = 0.0
                for i in range(0, count, max(1, count // 400)):
                    o, n_ = int(b_off[i]), int(ns[i])
                    a, c = x32[o:o + n_], x64[o:o + n_]
                    worst = max(worst, float(torch.linalg.norm(a - c) / torch.linalg.norm(c)))
                rec["max_rel_diff_vs_fp64_batch"] = worst
        else:
            x64 = b_flat.clone()
        out[name] = rec
    # the same FP64 batch as a plan (problem table uploaded once, CUDA-graph
    # launch), with the tuned settings
    stp, plan = abi.slqr_batch_plan_create(ctx.ctx, list(ms), list(ns), None, A_ptrs, lda,
                                           up_ptrs, b_ptrs, abi.SLQR_FP64, status.data_ptr(),
                                           None)
    abi.check(ctx.ctx, stp, "slqr_batch_plan_create")
    times = []
    for rep in range(reps + 1):
        A_flat.copy_(A0)
        b_flat.copy_(b0)
        barrier()
        e0.record(stream)
        abi.check(ctx.ctx, abi.slqr_batch_plan_launch(plan, stream.cuda_stream), "plan launch")
        e1.record(stream)
        barrier()
        if rep:
            times.append(e0.elapsed_time(e1))
    abi.slqr_batch_plan_destroy(plan)
    out["fp64_plan"] = {"ms": min(times), "problems_per_s": count / (min(times) / 1e3),
                        "ok": int(np.sum(status.cpu().numpy() == 0))}
    # per-call latency of a small batch (256 problems, m ~ U{16..64}) from the
    # host: slqr_batch_factor (table built and uploaded per call) against a plan
    import time as _time
    sms, sns = workloads.batch_shapes(256, seed=71, m_lo=16, m_hi=64)
    SA, Sb, sa_off, sb_off = workloads.batch_problems_device(sms, sns, 71, device=device)
    SA0, Sb0 = SA.clone(), Sb.clone()
    sup = torch.zeros(int(sns.sum()) + 1, dtype=torch.float64, device=device)
    sup_off = np.concatenate([[0], np.cumsum(sns)[:-1]])
    sargs = ([int(m) for m in sms], [int(n) for n in sns],
             [SA.data_ptr() + int(o) * 8 for o in sa_off], [int(m) for m in sms],
             [sup.data_ptr() + int(o) * 8 for o in sup_off],
             [Sb.data_ptr() + int(o) * 8 for o in sb_off])
    sstat = torch.zeros(256, dtype=torch.int32, device=device)
    small = {}
    for mode in ("batch_factor", "plan"):
        if mode == "plan":
            stp, splan = abi.slqr_batch_plan_create(ctx.ctx, sargs[0], sargs[1], None, sargs[2],
                                                    sargs[3], sargs[4], sargs[5], abi.SLQR_FP64,
                                                    sstat.data_ptr(), None)
            abi.check(ctx.ctx, stp, "slqr_batch_plan_create")
        lat = []
        for rep in range(21):
            SA.copy_(SA0)
            Sb.copy_(Sb0)
            torch.cuda.synchronize()
            t0 = _time.perf_counter()
            if mode == "plan":
                st = abi.slqr_batch_plan_launch(splan, stream.cuda_stream)
            else:
                st = abi.slqr_batch_factor(ctx.ctx, *sargs, abi.SLQR_FP64, sstat.data_ptr(), None,
                                           stream.cuda_stream)
            abi.check(ctx.ctx, st, mode)
            torch.cuda.synchronize()
            if rep:
                lat.append((_time.perf_counter() - t0) * 1e3)
        if mode == "plan":
            abi.slqr_batch_plan_destroy(splan)
        small[mode] = {"median_ms": float(np.median(lat)), "min_ms": float(np.min(lat))}
    out["small_batch_256_call_latency"] = small
    # the same small batch after the autotuner has seen its shapes (all in the
    # class m <= 64, where the shared-memory-resident kernel is a candidate)
    stt, choice, tms = abi.slqr_batch_autotune(ctx.ctx, abi.SLQR_FP64, sargs[0], sargs[1])
    abi.check(ctx.ctx, stt, "slqr_batch_autotune (small batch)")
    lat = []
    for rep in range(21):
        SA.copy_(SA0)
        Sb.copy_(Sb0)
        torch.cuda.synchronize()
        t0 = _time.perf_counter()
        abi.check(ctx.ctx, abi.slqr_batch_factor(ctx.ctx, *sargs, abi.SLQR_FP64, sstat.data_ptr(),
                                                 None, stream.cuda_stream), "small batch")
        torch.cuda.synchronize()
        if rep:
            lat.append((_time.perf_counter() - t0) * 1e3)
    nb, tc, rs = choice[0]
    out["small_batch_256_tuned"] = {"panel_width": nb, "tile_cols": tc, "resident": bool(rs),
                                    "median_ms": float(np.median(lat)),
                                    "tuner_sample_ms_before_after": list(tms),
                                    "ok": int(np.sum(sstat.cpu().numpy() == 0))}
    abi.slqr_batch_set_tuning(abi.SLQR_FP64, -1, 0, 0)
    del SA, Sb, SA0, Sb0
    # plain one-at-a-time FP64 GPU path on the first `serial` problems
    A_flat.copy_(A0)
    b_flat.copy_(b0)
    barrier()
    e0.record(stream)
    sflops = 0.0
    for i in range(serial):
        m, n = int(ms[i]), int(ns[i])
        Ai = A_flat[int(a_off[i]):int(a_off[i]) + m * n].view(n, m).t()
        bi = b_flat[int(b_off[i]):int(b_off[i]) + m]
        upi = up_flat[int(up_off[i]):int(up_off[i]) + n]
        ctx.factor(Ai, upi)
        ctx.apply_qt(Ai, upi, bi)
        ctx.solve_r(Ai, bi)
        sflops += 2.0 * m * n * n - 2.0 * n ** 3 / 3.0 + 6.0 * m * n
    e1.record(stream)
    barrier()
    t = e0.elapsed_time(e1)
    out["one_at_a_time_fp64"] = {"problems": serial, "ms": t,
                                 "problems_per_s": serial / (t / 1e3),
                                 "gflops": sflops / (t / 1e3) / 1e9}
    out["speedup_fp64_batch_vs_one_at_a_time"] = (out["fp64"]["problems_per_s"] /
                                                  out["one_at_a_time_fp64"]["problems_per_s"])
    out["speedup_mixed_batch_vs_one_at_a_time"] = (out["mixed_fp32"]["problems_per_s"] /
                                                   out["one_at_a_time_fp64"]["problems_per_s"])
    if ctx.sync() != 0:
        raise RuntimeError("device status after the batch workload")
    del A_flat, b_flat, A0, b0
    torch.cuda.empty_cache()
    return out


def run_tune():
    """Factorization times under the panel tuning knobs (panel width, smallest
    row slice per panel CTA) for the plain-workload shapes and 8192 x 4096;
    prints one JSON line with the table and the best setting per shape."""
    import torch
    import workloads
    from paper_2506_09463_gb300 import abi, api
    dev = torch.device("cuda", 0)
    shapes = [(8192, 4096, 4), (16384, 2048, 2), (8192, 8192, 3)]
    settings = [(64, 32), (64, 128), (64, 160), (64, 192), (64, 224), (64, 256), (64, 320),
                (32, 192), (32, 256)]
    mats = {(m, n): colmajor_cuda(workloads.gaussian(m, n, seed)[0], dev) for m, n, seed in shapes}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    table = {}
    with api.Context(0) as ctx:
        for nb, rmin in settings:
            abi.slqr_set_tuning(nb, rmin)
            for (m, n), A0 in mats.items():
                Aw = A0.t().clone().t()
                up = torch.empty(n, dtype=torch.float64, device=dev)
                ts = []
                try:
                    for rep in range(3):
                        Aw.copy_(A0)
                        torch.cuda.synchronize()
                        e0.record()
                        ctx.factor(Aw, up)
                        e1.record()
                        torch.cuda.synchronize()
                        ts.append(e0.elapsed_time(e1))
                except abi.SlqrError:
                    continue                  # setting outside the kernel's limits
                if ctx.sync() != 0:
                    raise RuntimeError("device status")
                fl = 2.0 * m * n * n - 2.0 * n ** 3 / 3.0
                table.setdefault(f"{m}x{n}", {})[f"nb{nb}_rmin{rmin}"] = {
                    "ms": min(ts), "gflops": fl / (min(ts) / 1e3) / 1e9}
        abi.slqr_set_tuning(0, 0)
    best = {k: min(v.items(), key=lambda kv: kv[1]["ms"]) for k, v in table.items()}
    print(json.dumps({"tune": table, "best": {k: {"setting": b[0], **b[1]} for k, b in best.items()}}))
    return 0


def run_ncu_mixed(m, n, prec_name="tf32"):
    """Two mixed-precision LS solves (TF32, BF16 hi + lo or FP32 factorization)
    of an iid N(0,1) m x n matrix: a small program for ncu captures of the
    mixed path's kernels (no torch.linalg call, which does not load under the
    profiler)."""
    import torch
    import workloads
    from paper_2506_09463_gb300 import abi, api
    dev = torch.device("cuda", 0)
    A_h, b_h = workloads.gaussian(m, n, workloads.SEED_TALL)
    A = colmajor_cuda(A_h, dev)
    b = torch.from_numpy(b_h).to(dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    with api.Context(0) as ctx:
        for _ in range(2):
            prec = {"bf16x3": abi.SLQR_BF16X3, "fp32": abi.SLQR_FP32}.get(prec_name, abi.SLQR_TF32)
            st, its, err = abi.slqr_lstsq_mixed(ctx.ctx, m, n, A.data_ptr(), m, b.data_ptr(),
                                                x.data_ptr(), prec, 0, 0.0,
                                                torch.cuda.current_stream().cuda_stream)
            if st != 0:
                raise RuntimeError(f"mixed status {st}")
    print(f"ncu mixed case {m}x{n} done ({its} sweeps)")
    return 0


def run_ncu_batch(count):
    """A batch of `count` problems of the batched workload, FP64 then FP32."""
    import torch
    import workloads
    from paper_2506_09463_gb300 import abi, api
    ms, ns = workloads.batch_shapes(count)
    A_flat, b_flat, a_off, b_off = workloads.batch_problems_device(ms, ns, workloads.SEED_BATCH)
    up = torch.zeros(int(ns.sum()) + 1, dtype=torch.float64, device=A_flat.device)
    up_off = np.concatenate([[0], np.cumsum(ns)[:-1]])
    A0, b0 = A_flat.clone(), b_flat.clone()
    with api.Context(0) as ctx:
        for prec in (abi.SLQR_FP64, abi.SLQR_FP32):
            A_flat.copy_(A0)
            b_flat.copy_(b0)
            st = abi.slqr_batch_factor(ctx.ctx, list(ms), list(ns),
                                       [A_flat.data_ptr() + int(o) * 8 for o in a_off],
                                       [int(m) for m in ms],
                                       [up.data_ptr() + int(o) * 8 for o in up_off],
                                       [b_flat.data_ptr() + int(o) * 8 for o in b_off], prec,
                                       None, None, torch.cuda.current_stream().cuda_stream)
            abi.check(ctx.ctx, st, "batch")
            if ctx.sync() != 0:
                raise RuntimeError("device status")
    print(f"ncu batch case {count} done")
    return 0


def run_ncu_gmres(m, n):
    """GMRES-IR alone (a budget of 8 Krylov iterations) on an m x n matrix of
    condition 1e6 (the conditioned recipe drawn on the host with numpy: no
    torch.linalg call, which does not load under ncu), FP32 and split-BF16
    factorizations: a short program for ncu captures of the preconditioner."""
    import torch
    import workloads
    from paper_2506_09463_gb300 import abi, api
    A, b_cons, x_true, b_rand = workloads.conditioned(m, n, 1e6, seed=5)
    dev = torch.device("cuda", 0)
    Ad = colmajor_cuda(A, dev)
    bd = torch.from_numpy(b_rand.copy()).to(dev)
    with api.Context(0) as ctx:
        for prec in (abi.SLQR_FP32, abi.SLQR_BF16X3):
            x = torch.zeros(n, dtype=torch.float64, device=dev)
            st, info = abi.slqr_lstsq_mixed_ex(ctx.ctx, m, n, Ad.data_ptr(), m, bd.data_ptr(),
                                               x.data_ptr(), prec, 0,
                                               refine=abi.SLQR_REFINE_GMRES, gmres_max_iters=8)
            if st not in (abi.SLQR_OK, abi.SLQR_ENOCONV):
                raise RuntimeError(f"status {st}")
            print(prec, abi.STATUS_NAMES.get(st, st), info)
    return 0


def run_ncu_case(m, n):
    """One factorization + Q^T (64 RHS) + back-substitution of an m x n N(0,1)
    matrix after one warm-up pass: a small, short program for ncu captures."""
    import torch
    import workloads
    from paper_2506_09463_gb300 import api
    A, _ = workloads.gaussian(m, n, 4)
    dev = torch.device("cuda", 0)
    A0 = colmajor_cuda(A, dev)
    B0 = colmajor_cuda(workloads.gaussian_rhs(m, 64, 4), dev)
    with api.Context(0) as ctx:
        for _ in range(2):
            Aw, Bw = A0.t().clone().t(), B0.t().clone().t()
            up = torch.empty(n, dtype=torch.float64, device=dev)
            wy = ctx.wy_buffer(m, n)
            ctx.factor(Aw, up, wy)
            ctx.apply_qt(Aw, up, Bw, wy=wy)
            ctx.solve_r(Aw, Bw)
            st = ctx.sync()
            if st != 0:
                raise RuntimeError(f"device status {st}")
    print(f"ncu case {m}x{n} done")
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched workload")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision workload")
    ap.add_argument("--no-serving", action="store_true", help="skip the request-stream workload")
    ap.add_argument("--ncu-mixed", type=int, nargs=2, metavar=("M", "N"),
                    help="run one TF32 mixed-precision solve for profiling and exit")
    ap.add_argument("--ncu-prec", default="tf32", choices=["tf32", "bf16x3", "fp32"],
                    help="factorization precision of --ncu-mixed")
    ap.add_argument("--ncu-batch", type=int, metavar="COUNT",
                    help="run one FP64 and one FP32 batch for profiling and exit")
    ap.add_argument("--tune", action="store_true",
                    help="time the factorization under the panel tuning knobs and exit")
    ap.add_argument("--ncu-gmres", type=int, nargs=2, metavar=("M", "N"),
                    help="GMRES-IR alone on an M x N matrix of condition 1e6 (ncu captures)")
    ap.add_argument("--ncu-case", type=int, nargs=2, metavar=("M", "N"),
                    help="run one small factor/apply/solve pass for profiling and exit")
    args = ap.parse_args()
    if args.ncu_case:
        return run_ncu_case(*args.ncu_case)
    if args.ncu_gmres:
        return run_ncu_gmres(*args.ncu_gmres)
    if args.tune:
        return run_tune()
    if args.ncu_mixed:
        return run_ncu_mixed(*args.ncu_mixed, prec_name=args.ncu_prec)
    if args.ncu_batch:
        return run_ncu_batch(args.ncu_batch)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    rc = run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
