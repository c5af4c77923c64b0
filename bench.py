"""Benchmark of the matrix-free GP hot path on one or more GB300 GPUs.

One step = one log-marginal-likelihood + gradient evaluation (the path of the
C ABI entry point lgp_lml_and_grad) on the mBCG workload: N=100,000 points in
D=8 (X ~ U[-1,1]^8), Matern-5/2 with ARD lengthscales log-spaced over [0.3, 2],
t=32 right-hand sides (y plus 31 Rademacher probes), 50 Lanczos steps, batched
CG (tolerance 1e-3) with the split tensor-core product, then the adjoint gradient pass.
The line also records how far that step's LML and gradient are from a tighter solve,
the plain FP32 single-column path timed in full at N=20,000 beside the batched path,
and the device memory the library holds.

value = pair-RHS evaluations per second over the step: every product of the
step contributes N^2 * t (the CG products and the adjoint pass). ms_per_step is
the LML+grad time. Multi-GPU: the path of one GP does not shard without an
exchange, so N GPUs run N independent replicas (weak scaling, no collective on
the data path; the barrier and the max-over-ranks timing use torch.distributed).

--impl reference times the FP64 CPU oracle as it stands on the host cores, on a
bounded row sample of the same product.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "matvec pair·RHS evals/s and LML+grad time, N=100k t=32, vs plain FP32 path"
# DRAM bytes (read + write) of one full-size product launch (N=100000, D=8, M52, t=32), from one
# `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum` capture (profiles/), valid only for the
# kernel source it was taken on: the bench reports null once a header of that kernel changes.
TRAFFIC = {"mv_tc_kernel": {"bytes": None, "source_sha256_16": None},
           "mv_tcs_kernel": {"bytes": 38.476032e6, "source_sha256_16": "ff3939601c16953a"}}
KERNEL_SOURCES = {"mv_tc_kernel": ["mv_tc.cuh"], "mv_tcs_kernel": ["mv_tcs.cuh", "mv_tc.cuh", "tile_walk.cuh"]}
UNIT = "pair*RHS/s"
SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128
MUFU_EX2_PER_SM = 32
MAX_SM_MHZ_NOMINAL = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["lgp", "reference"], default="lgp")
    ap.add_argument("--N", type=int, default=100000)
    ap.add_argument("--t", type=int, default=32)
    ap.add_argument("--lanczos", type=int, default=50)
    # CG tolerance of the step: at 1e-3 the step's LML and gradient stay within 1e-3 (measured: 3e-4 and 1.2e-4)
    # of a tol-1e-6 solve on the same draw and probes, which the line's accuracy record re-measures each run
    ap.add_argument("--tol", type=float, default=1e-3)
    ap.add_argument("--max-iter", type=int, default=3000)
    ap.add_argument("--prec", choices=["auto", "fp32", "split_bf16", "split_f16"], default="auto")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--plain", action="store_true", help="also time the plain FP32 single-RHS path")
    ap.add_argument("--mode", choices=["lml", "matvec", "predict", "batch", "memory"], default="lml",
                    help="lml: the LML+grad step (default); matvec: only the product, for kernel profiling; "
                         "predict: posterior mean and variance at --M test points; "
                         "batch: the 64 uneven GPs of the batch workload in one call vs one call each; "
                         "memory: device memory of the LML+grad call for N in 1e3..5e5")
    ap.add_argument("--precond-rank", type=int, default=0,
                    help="pivoted-Cholesky preconditioner rank of the CG solves (0: the paper's plain CG)")
    ap.add_argument("--workload", choices=["cfg3", "cfg4", "cfg5-large"], default="cfg3",
                    help="--mode lml problem: cfg3 (N=100000, D=8, Matern-5/2, t=32; the default) or cfg4 "
                         "(N=50000, D=8, RBF, t=16, 10 hyperparameters; the line adds the adjoint pass's own time); "
                         "cfg5-large (--mode matvec only): one RBF product at N=500000, D=2, t=32 on a N(0,1) block")
    ap.add_argument("--ref-tol", type=float, default=1e-6,
                    help="tolerance of the tight solve the timed step's LML and gradient are compared with")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the accuracy record of the timed step")
    ap.add_argument("--plain-N", type=int, default=20000,
                    help="N at which the plain FP32 single-column path is timed in full beside the batched path")
    ap.add_argument("--M", type=int, default=10000, help="test points of --mode predict")
    ap.add_argument("--var-probes", type=int, default=31,
                    help="--mode predict: probes of the variance estimate (0: exact per-point variance)")
    return ap.parse_args()


def dist_init(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("LGP_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def job_rate(local_units, local_seconds, world, device):
    """Whole-job throughput: the units every rank processed over the slowest rank's time.
    Returns (rate, max seconds)."""
    if world == 1:
        return local_units / local_seconds, local_seconds
    import torch
    import torch.distributed as dist
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    s = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()) / float(s.item()), float(s.item())


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.proc = None
        # raw samples go to LGP_CLOCKS_DIR when set (kept for inspection), else to a temporary file
        out_dir = os.environ.get("LGP_CLOCKS_DIR") or tempfile.gettempdir()
        os.makedirs(out_dir, exist_ok=True)
        self.path = os.path.join(out_dir, f"lgp_clocks_{os.getpid()}.csv")
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if uuid:
            cmd[1:1] = ["-i", uuid]
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), float(parts[2]), parts[3:]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [r[0] for r in rows]
        loaded = [r for r in rows if r[2] > 200.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in loaded:
            for nm, v in zip(names, r[3][1:]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median([r[0] for r in loaded]), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "power_w_max": max(r[2] for r in rows), "reasons": sorted(reasons),
                "sm_mhz_min": min(sm)}


def gpu_uuid(dev_index):
    try:
        import torch
        u = torch.cuda.get_device_properties(dev_index).uuid
        s = str(u)
        return s if s.startswith("GPU-") else f"GPU-{s}"
    except Exception:
        return None


def measured_peaks():
    """The machine's measured copy bandwidth and bf16 GEMM rates (MEASURED_PEAKS.json), else the
    earlier single measurement used as fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"bf16_tflops": float(d["bf16_tflops"]), "hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"bf16_tflops": 1900.0, "hbm_gbs": 6800.0, "source": "fallback"}


def kernel_source_hash(name):
    """First 16 hex digits of the sha256 of the headers that define kernel `name`."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[name]:
        h.update(open(os.path.join(ROOT, "paper_2605_17898_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def kernel_traffic(name):
    """Recorded DRAM bytes per launch of `name`, or None if its source changed since the capture."""
    rec = TRAFFIC.get(name)
    if not rec or rec["bytes"] is None:
        return None
    return rec["bytes"] if kernel_source_hash(name) == rec["source_sha256_16"] else None


def flush_l2(buf):
    buf.add_(1.0)


def per_pair_ops(kind: int, D: int, split: bool, t: int, dot: bool = False) -> tuple[float, dict]:
    """Algorithmic FP32-pipe operations and MUFU operations per generated entry k(x_i, x_j).

    Difference form: D subtractions + D multiply-adds for r^2 (RBF starts the
    accumulation at -log2 s^2, so its exponent costs nothing more); Matern-5/2:
    exponent multiply-add, polynomial multiply-add, final multiply-add. Split
    (tensor-core) path: 2 per entry (the lo subtraction and two half-width roundings
    counted as half an op each); the contraction runs on the tensor pipe. Dot form:
    r^2 = a_i - d from the tensor-core Gram value (1 add), the kernel value as above,
    and the float32 hi/lo split (3 for the rounding, 1 for lo). FP32 SIMT path: t
    multiply-adds. MUFU: RBF one ex2; the Matern forms one sqrt and one ex2.
    """
    # kernel value beyond the squared distance: RBF 0, M52 3, M12 1 (the exponent), M32 2
    kval = {0: 0, 1: 3, 2: 1, 3: 2}[kind]
    mufu = {"ex2": 1.0, "sqrt": 0.0 if kind == 0 else 1.0}
    if not split:
        return 2 * D + kval + t, mufu
    if dot:
        return 1.0 + kval + 4.0, mufu
    return 2 * D + kval + 2.0, mufu


def binding_pipe(entries: float, pairs: float, ops_pair: float, mufu_pair: dict, t: int, D: int, split: bool,
                 dot: bool, seconds: float, n_sm: int, bf16_tflops: float) -> dict:
    """The product's pipe bounds and the one that binds (the largest time bound).

    FP32 pipe: entries x FP32 ops over n_sm x 128 lanes x 2070 MHz. MUFU: entries x (ex2 + 2 sqrt)
    ex2 slots over n_sm x 32 ex2/cycle x 2070 MHz (sqrt runs at half the ex2 rate). Tensor: N^2 6t
    contraction flops (+ 2 kg per entry for the dot form's Gram tile, kg = 32) over the bf16
    burst peak. Returns achieved and peak in the binding pipe's unit, frac = achieved / peak, and the
    three time fractions.
    """
    fp32_peak = n_sm * FP32_LANES_PER_SM * MAX_SM_MHZ_NOMINAL * 1e6
    ex2_peak = n_sm * MUFU_EX2_PER_SM * MAX_SM_MHZ_NOMINAL * 1e6
    mufu_work = entries * (mufu_pair["ex2"] + 2.0 * mufu_pair["sqrt"])
    kg = 32  # the Gram operand rows: 3 Dp split coordinates + 6 norm and unit columns, padded to 32
    tensor_flops = (pairs * 6 * t + (entries * 2 * kg if dot else 0.0)) if split else 0.0
    bf16_peak = bf16_tflops * 1e12
    times = {"fp32": entries * ops_pair / fp32_peak, "mufu": mufu_work / ex2_peak, "tensor": tensor_flops / bf16_peak}
    binding = max(times, key=times.get)
    work, peak, unit = {"fp32": (entries * ops_pair, fp32_peak, "Tops/s (FP32 pipe)"),
                        "mufu": (mufu_work, ex2_peak, "T ex2-slots/s (MUFU; sqrt = 2 slots)"),
                        "tensor": (tensor_flops, bf16_peak, "TFLOP/s (tensor, f16/bf16)")}[binding]
    achieved = work / seconds / 1e12
    return {"binding": binding, "achieved": achieved, "peak": peak / 1e12, "unit": unit, "frac": achieved / (peak / 1e12),
            "pipe_fracs": {k: v / seconds for k, v in times.items()}, "tensor_flops": tensor_flops}


def run_cpu_baseline(p, t, seconds, seed=0):
    """The oracle's FP64 streaming product on a bounded row sample of the workload."""
    import numpy as np
    import oracle
    from oracle import gp_oracle as go
    import workloads as wl
    hyp = go.hyper_of(p)
    V = wl.rhs_block(p.N, t, seed=seed, kind="sign")
    rng = np.random.default_rng(seed)
    rows = rng.choice(p.N, 64, replace=False)
    t0 = time.perf_counter()
    _, used = oracle.kyv_rows_c(p.X, V, hyp, rows=rows)
    dt = time.perf_counter() - t0
    n_rows = int(max(64, min(p.N, 64 * seconds / max(dt, 1e-3))))
    rows = rng.choice(p.N, n_rows, replace=False)
    t0 = time.perf_counter()
    _, used = oracle.kyv_rows_c(p.X, V, hyp, rows=rows)
    dt = time.perf_counter() - t0
    value = n_rows * p.N * t / dt
    return {"value": value, "unit": UNIT, "cores": int(used), "kind": "oracle",
            "sample": f"{n_rows} sampled rows of K_y V (all {p.N} columns, t={t}), FP64 C/OpenMP row-streamed "
                      f"oracle; {dt:.1f} s", "seconds": dt}


def bench_reference(args, rank, world):
    """The oracle as it stands, timed on the host cores (rank 0 only)."""
    import workloads as wl
    if rank != 0:
        return
    p = wl.cfg3(N=args.N, t=args.t)
    for _ in range(max(args.warmup, 0)):
        run_cpu_baseline(p, args.t, min(1.0, args.cpu_seconds / 10))
    vals = []
    times = []
    per_step = max(1.0, min(args.cpu_seconds, 60.0 / max(args.steps, 1)))
    base = None
    for _ in range(args.steps):
        base = run_cpu_baseline(p, args.t, per_step)
        vals.append(base["value"])
        times.append(base["seconds"])
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": p.name, "N": p.N, "D": p.D, "t": args.t, "kernel": "matern52",
                                            "sample": "row sample of the product per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        # the oracle runs on rank 0's host cores only; no process group is needed
        bench_reference(args, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")))
        return
    rank, world, local = dist_init(args.gpus)
    import numpy as np
    import torch
    import paper_2605_17898_gb300 as lgp
    import workloads as wl

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lgp.load()
    ctx = lgp.Context(local)
    prec = {"auto": lgp.LGP_PREC_AUTO, "fp32": lgp.LGP_PREC_FP32, "split_bf16": lgp.LGP_PREC_SPLIT_BF16,
            "split_f16": lgp.LGP_PREC_SPLIT_F16}[args.prec]

    V_large = None
    if args.workload == "cfg4":
        if args.N == 100000:
            args.N = 50000
        if args.t == 32:
            args.t = 16
        p = wl.cfg4(N=args.N, t=args.t)
    elif args.workload == "cfg5-large":
        if args.mode != "matvec":
            raise SystemExit("--workload cfg5-large is a single product: use it with --mode matvec")
        if args.N == 100000:
            args.N = 500000
        p, V_large = wl.cfg5_large(N=args.N, t=args.t)
    else:
        p = wl.cfg3(N=args.N, t=args.t)
    kernel_name = {wl.RBF: "rbf", wl.MATERN52: "matern52"}.get(p.kind, str(p.kind))
    m = args.t - 1
    if args.mode == "memory":
        bench_memory(lgp, args, dev, prec, rank)
        return
    if args.mode == "matvec":
        bench_matvec_only(lgp, ctx, p, args, dev, prec, rank, V_large)
        return
    if args.mode == "predict":
        bench_predict(lgp, ctx, p, args, dev, prec, rank)
        return
    if args.mode == "batch":
        bench_batch(lgp, ctx, args, dev, rank)
        return
    X = torch.as_tensor(p.X, device=dev)
    y = torch.as_tensor(p.y, device=dev)
    flush_buf = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def step(Xd, yd):
        return lgp.lgp_lml_and_grad(Xd, yd, p, n_probes=m, lanczos_steps=args.lanczos, seed=1234 + rank,
                                    tol=args.tol, max_iter=args.max_iter, prec=prec, ctx=ctx,
                                    precond_rank=args.precond_rank)

    for _ in range(args.warmup):
        step(X, y)
    torch.cuda.synchronize()

    # ---------------- timed region: K steps, per-step CUDA events, L2 flushed between steps
    sampler = ClockSampler(gpu_uuid(local)) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    infos = []
    for k in range(args.steps):
        flush_l2(flush_buf)
        starts[k].record()
        lml, grad, info = step(X, y)
        ends[k].record()
        infos.append(info)
    torch.cuda.synchronize()
    barrier(world)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    local_total_s = sum(step_ms) / 1e3
    clocks = sampler.stop() if sampler else None

    iters = [i["iters_max"] for i in infos]
    chunks = [i["cg_chunks"] for i in infos]
    # products per step: one per CG iteration replayed (graph chunks of 8 iterations) + the adjoint pass
    n_products = [8 * c for c in chunks]
    pairs_rhs = [(n + 1) * float(p.N) ** 2 * args.t for n in n_products]
    # useful work only: products of iterations that ran (later iterations of a chunk exit early)
    useful = [(it + 1) * float(p.N) ** 2 * args.t for it in iters]
    # whole job: every rank's useful products over the slowest rank's time
    value, total_s = job_rate(sum(useful), local_total_s, world, dev)
    ms_per_step = 1e3 * total_s / args.steps
    launches = int(sum(i["launches"] for i in infos))

    # ---------------- dominant kernel timing on the launching stream (torch's current stream)
    V = torch.as_tensor(wl.rhs_block(p.N, args.t, seed=3, kind="sign"), device=dev)
    out = torch.empty_like(V)
    kprec = ctx.matvec_precision(args.t, prec)
    for _ in range(2):
        lgp.lgp_kernel_matvec(X, p, V, prec=kprec, out=out, ctx=ctx)
    torch.cuda.synchronize()
    kev = []
    for _ in range(5):
        flush_l2(flush_buf)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        lgp.lgp_kernel_matvec(X, p, V, prec=kprec, out=out, ctx=ctx)
        b.record()
        kev.append((a, b))
    torch.cuda.synchronize()
    call_ms = statistics.mean(a.elapsed_time(b) for a, b in kev)
    # the product kernel alone (the roofline's duration): CUDA events the library records on its launching
    # stream immediately around the kernel, after the per-call V split
    ctx.set_kernel_timing(True)
    kms = []
    for _ in range(5):
        flush_l2(flush_buf)
        lgp.lgp_kernel_matvec(X, p, V, prec=kprec, out=out, ctx=ctx)
        kms.append(ctx.last_kernel_ms())
    ctx.set_kernel_timing(False)
    mv_ms = statistics.mean(kms)
    split = kprec in (lgp.LGP_PREC_SPLIT_BF16, lgp.LGP_PREC_SPLIT_F16)
    symmetric = split and ctx.tc_kernel_choice(p.N, p.D, p.kind, args.t, kprec) == lgp.LGP_TC_SYMMETRIC
    form, norm_max = ctx.tc_distance_form() if symmetric else (lgp.LGP_DIST_NONE, -1.0)
    dot = form == lgp.LGP_DIST_DOT
    kname = "mv_tcs_kernel" if symmetric else ("mv_tc_kernel" if split else "mv_simt_kernel")
    ops_pair, mufu_pair = per_pair_ops(p.kind, p.D, split, args.t, dot)
    pairs = float(p.N) ** 2
    # entries the kernel must generate: the symmetric kernel needs each unordered pair once
    entries = float(p.N) * (p.N + 1) / 2 if symmetric else pairs
    mv_s = mv_ms / 1e3
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    peaks = measured_peaks()
    meas = {name: lgp.lgp_measure_pipe_peak(i) for i, name in
            enumerate(["ffma", "ffma2_fmas", "mufu_ex2", "mufu_sqrt"])}
    # peaks from unit counts and the maximum SM clock: 128 FP32 lanes, 32 ex2 per SM per cycle (sqrt
    # at half that rate; both confirmed by the pipe microbenchmarks in measured_pipe_peaks_per_s)
    bp = binding_pipe(entries, pairs, ops_pair, mufu_pair, args.t, p.D, split, dot, mv_s, n_sm, peaks["bf16_tflops"])
    binding, achieved, peak, unit = bp["binding"], bp["achieved"], bp["peak"], bp["unit"]
    tensor_flops = bp["tensor_flops"]
    psrc = {"fp32": f"{n_sm} SMs x 128 FP32 lanes x 2070 MHz (unit counts and max clock)",
            "mufu": f"{n_sm} SMs x 32 ex2/cycle x 2070 MHz (unit counts and max clock)",
            "tensor": peaks["source"] + " bf16 burst (f16 dense rate = bf16)"}[binding]
    roofline = {"bound": "tensor" if binding == "tensor" else "alu", "achieved": achieved, "peak": peak,
                "unit": unit, "frac": achieved / peak,
                "traffic": kernel_traffic(kname) if split and p.N == 100000 and args.t == 32 else None,
                "kernel": kname, "binding_pipe": binding, "peak_source": psrc,
                "distance_form": {lgp.LGP_DIST_DOT: "dot", lgp.LGP_DIST_DIFF: "difference"}.get(form, None),
                "centred_norm_max": norm_max if dot else None,
                "per_entry_fp32_ops": ops_pair, "mufu_per_entry": mufu_pair, "matvec_ms": mv_ms,
                "product_call_ms": call_ms,
                "timing": "matvec_ms: the product kernel's launch alone (library-recorded CUDA events on its stream, "
                          "mean of 5, L2 flushed); product_call_ms: the whole lgp_kernel_matvec call, which also "
                          "splits V",
                "entries_per_launch": entries, "pairs_per_launch": pairs, "sm_count": n_sm,
                "tensor_flops_per_launch": tensor_flops,
                "pipe_fracs": bp["pipe_fracs"],
                "measured_pipe_peaks_per_s": meas,
                "tensor_peak_source": peaks["source"] + " bf16 burst (f16 dense rate = bf16)"}

    # ---------------- device memory of the step (the library allocates only its O(N) workspace)
    free_b, total_b = torch.cuda.mem_get_info(dev)
    memory = {"lgp_workspace_bytes": int(ctx.workspace_bytes),
              "torch_max_allocated_bytes": int(torch.cuda.max_memory_allocated(dev)),
              "device_used_bytes": int(total_b - free_b),
              "note": "workspace: the library's own device buffers (O(N)); torch: the caller's inputs, the "
                      "kernel-timing blocks and the 256 MB L2-flush buffer; device_used includes the CUDA context"}

    # ---------------- end to end through the public API with host buffers
    Xh = torch.as_tensor(p.X).pin_memory()
    yh = torch.as_tensor(p.y).pin_memory()
    Xd = torch.empty_like(X)
    yd = torch.empty_like(y)
    e2e_ms = []
    e2e_iters = []
    for k in range(2):
        flush_l2(flush_buf)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        Xd.copy_(Xh, non_blocking=True)
        yd.copy_(yh, non_blocking=True)
        lml_e, grad_e, info_e = step(Xd, yd)  # returns host scalars (device->host read inside)
        b.record()
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))
        e2e_iters.append(info_e["iters_max"])
    e2e_value, _ = job_rate(sum((it + 1) * float(p.N) ** 2 * args.t for it in e2e_iters), sum(e2e_ms) / 1e3,
                            world, dev)
    # the CG state read back per step: 8 int32 + 1 float64, 2 x 64 int32, 6 x 64 float64
    cg_state_bytes = 8 * 4 + 8 + 2 * 64 * 4 + 6 * 64 * 8
    d2h = cg_state_bytes + (2 * 64 + 4 + 10) * 8 + 16 + 4 * statistics.mean(chunks)
    e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(Xh.numel() * 4 + yh.numel() * 4),
           "d2h_bytes_per_step": int(d2h), "ms_per_step": statistics.mean(e2e_ms)}

    adjoint = None
    if args.workload == "cfg4":
        adjoint = time_adjoint(lgp, ctx, p, X, y, args, dev, prec, rank, flush_buf)
    accuracy = None
    if not args.no_accuracy:
        accuracy = bench_accuracy(lgp, ctx, p, X, y, args, prec, 1234 + rank, lml, grad)
    plain = estimate_plain(lgp, ctx, p, X, y, args, dev, iters, ms_per_step)
    plain["measured_equal_accuracy"] = bench_plain_equal(lgp, args, dev, prec, 1234 + rank)
    if args.plain:
        plain["measured_full_size"] = bench_plain(lgp, ctx, p, X, y, args, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(p, args.t, args.cpu_seconds)
        cpu.pop("seconds", None)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": ("f32+f16x3" if kprec == lgp.LGP_PREC_SPLIT_F16 else "f32+bf16x3") if split else "f32",
            "data": "synthetic",
            "config": {"workload": p.name, "N": p.N, "D": p.D, "t": args.t, "kernel": kernel_name,
                       "tc_kernel": kname,
                       "lanczos_steps": args.lanczos, "tol": args.tol, "max_iter": args.max_iter,
                       "precond_rank": args.precond_rank,
                       "cg_iterations": iters,
                       "precision": {1: "fp32", 2: "split_bf16", 3: "split_f16"}.get(kprec, str(kprec)),
                       "l2": "flushed between steps (256 MB write outside the step events)",
                       "parallelism": f"replicas{world}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "lml": lml, "grad": [float(g) for g in grad], "memory": memory, "accuracy": accuracy,
        }
        if adjoint is not None:
            line["adjoint"] = adjoint
        if plain is not None:
            line["plain_fp32"] = plain
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def bench_batch(lgp, ctx, args, dev, rank):
    """Batched solves (t = 8, CG tol 1e-6): the batch workload (64 GPs, N_g log-uniform in [500, 30000],
    D_g in 1..6) and 256 small GPs (N_g in [200, 2000]), each as one lgp_batch_cg_solve call against the
    same solves as one lgp_cg_solve call per problem."""
    import torch
    import workloads as wl
    lines = []
    for label, probs in [("cfg5: 64 GPs, N in [500, 30000]", wl.cfg5_batch(t=8)),
                         ("256 small GPs, N in [200, 2000]", wl.cfg5_batch(n_gp=256, t=8, seed=15, n_lo=200, n_hi=2000))]:
        lines.append(_bench_batch_set(lgp, ctx, args, dev, label, probs))
    if rank == 0:
        for line in lines:
            print(json.dumps(line), flush=True)


def _bench_batch_set(lgp, ctx, args, dev, label, probs):
    import torch
    import workloads as wl
    Xs = [torch.as_tensor(q.X, device=dev) for q in probs]
    Bs = []
    for g, q in enumerate(probs):
        B = wl.rhs_block(q.N, 8, seed=g, kind="sign")
        B[:, 0] = q.y
        Bs.append(torch.as_tensor(B, device=dev))

    def batched():
        return lgp.lgp_batch_cg_solve(Xs, probs, Bs, tol=1e-6, max_iter=3000, ctx=ctx)

    def one_by_one():
        its = []
        for X, q, B in zip(Xs, probs, Bs):
            _, it, _, _ = lgp.lgp_cg_solve(X, q, B, tol=1e-6, max_iter=3000, ctx=ctx)
            its.append(int(it.max()))
        return its

    res = {}
    for name, fn in [("batched", batched), ("one_call_per_gp", one_by_one)]:
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            out = fn()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        res[name] = {"ms": statistics.mean(ms), "ms_all": ms}
        if name == "batched":
            res[name]["iters_max"] = int(out[1].max())
        else:
            res[name]["iters_max"] = max(out)
    pairs = sum(float(q.N) ** 2 for q in probs)
    _, it_b, _, _ = batched()
    # useful work of the batched call: each problem's products (one per iteration of its slowest column,
    # plus the initial one) over the call's time; and the FP32-pipe operations the same products cost on
    # the float32 route (2D + kernel value + t per entry), against the FP32 peak, as the persistent
    # product's pipe fraction (tensor-route problems counted at that float32 cost, so an upper bound)
    kval = {wl.RBF: 0, wl.MATERN52: 3, wl.MATERN12: 1, wl.MATERN32: 2}
    it_g = [int(it_b[g].max()) + 1 for g in range(len(probs))]
    pr = sum(i * float(q.N) ** 2 * 8 for i, q in zip(it_g, probs)) / (res["batched"]["ms"] / 1e3)
    ops = sum(i * float(q.N) ** 2 * (2 * q.D + kval[q.kind] + 8) for i, q in zip(it_g, probs))
    n_sm = torch.cuda.get_device_properties(dev.index or 0).multi_processor_count
    fp32_peak = n_sm * FP32_LANES_PER_SM * MAX_SM_MHZ_NOMINAL * 1e6
    routes = [ctx.batch_route_choice(q.N, q.D, q.kind, 8) for q in probs]
    # column splits of the persistent-route problems: the timed choice against the fixed rule
    splits = [(q.N, ctx.batch_split_choice(q.N, q.D, q.kind, 8), ctx.batch_split_rule(q.N))
              for q, r in zip(probs, routes) if r == lgp.LGP_BATCH_PERSISTENT]
    return {"mode": "batch", "workload": label, "n_gp": len(probs), "t": 8, "pairs_per_product": pairs,
            "N_min": min(q.N for q in probs), "N_max": max(q.N for q in probs), **res,
            "speedup": res["one_call_per_gp"]["ms"] / res["batched"]["ms"],
            "batched_pair_rhs_per_s": pr,
            "batched_fp32_equiv_frac": ops / (res["batched"]["ms"] / 1e3) / fp32_peak,
            "tensor_route_problems": sum(1 for r in routes if r == lgp.LGP_BATCH_TENSOR),
            "tensor_route_N": sorted(q.N for q, r in zip(probs, routes) if r == lgp.LGP_BATCH_TENSOR),
            "persistent_splits": {"tuned_equal_to_rule": sum(1 for _, a, b in splits if a == b),
                                  "tuned_differs": [[n, a, b] for n, a, b in sorted(splits) if a != b],
                                  "note": "[N, timed split count, fixed rule's count] of persistent-route problems"}}


def bench_predict(lgp, ctx, p, args, dev, prec, rank):
    """Posterior mean and variance at M test points drawn like the training inputs (one call of
    lgp_predict per step: CG solve(s), the cross products and the variance finalisation)."""
    import numpy as np
    import torch
    X = torch.as_tensor(p.X, device=dev)
    y = torch.as_tensor(p.y, device=dev)
    Xs = torch.as_tensor(np.random.default_rng(7).uniform(-1.0, 1.0, (args.M, p.D)).astype(np.float32), device=dev)

    def step():
        return lgp.lgp_predict(X, y, p, Xs, n_probes=args.var_probes, seed=99, tol=args.tol,
                               max_iter=args.max_iter, prec=prec, ctx=ctx, precond_rank=args.precond_rank)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ms, infos = [], []
    for _ in range(args.steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        _, _, info, _ = step()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        infos.append(info)
    if rank == 0:
        print(json.dumps({"mode": "predict", "workload": p.name, "M": args.M, "var_probes": args.var_probes,
                          "tol": args.tol, "ms": statistics.mean(ms), "ms_all": ms,
                          "solves": infos[-1]["solves"], "iters_max": infos[-1]["iters_max"],
                          "prec_used": infos[-1]["prec_used"]}), flush=True)


def bench_matvec_only(lgp, ctx, p, args, dev, prec, rank, V_host=None):
    """Only the product K_y V on the workload (a small, fast command for kernel profiling). Reports the
    whole call and, from the library's kernel-timing events, the product kernel alone with its binding
    pipe (the same bounds as the LML line's roofline)."""
    import torch
    import workloads as wl
    X = torch.as_tensor(p.X, device=dev)
    if V_host is None:
        V_host = wl.rhs_block(p.N, args.t, seed=3, kind="sign")
    V = torch.as_tensor(V_host, device=dev)
    out = torch.empty_like(V)
    kprec = ctx.matvec_precision(args.t, prec)
    for _ in range(args.warmup):
        lgp.lgp_kernel_matvec(X, p, V, prec=kprec, out=out, ctx=ctx)
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        lgp.lgp_kernel_matvec(X, p, V, prec=kprec, out=out, ctx=ctx)
        b.record()
        evs.append((a, b))
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
    ctx.set_kernel_timing(True)
    kms = []
    for _ in range(args.steps):
        lgp.lgp_kernel_matvec(X, p, V, prec=kprec, out=out, ctx=ctx)
        kms.append(ctx.last_kernel_ms())
    ctx.set_kernel_timing(False)
    kernel_ms = statistics.mean(kms)
    split = kprec in (lgp.LGP_PREC_SPLIT_BF16, lgp.LGP_PREC_SPLIT_F16)
    symmetric = split and ctx.tc_kernel_choice(p.N, p.D, p.kind, args.t, kprec) == lgp.LGP_TC_SYMMETRIC
    form = ctx.tc_distance_form()[0] if symmetric else lgp.LGP_DIST_NONE
    dot = form == lgp.LGP_DIST_DOT
    ops_pair, mufu_pair = per_pair_ops(p.kind, p.D, split, args.t, dot)
    entries = float(p.N) * (p.N + 1) / 2 if symmetric else float(p.N) ** 2
    bp = binding_pipe(entries, float(p.N) ** 2, ops_pair, mufu_pair, args.t, p.D, split, dot, kernel_ms / 1e3,
                      torch.cuda.get_device_properties(dev).multi_processor_count, measured_peaks()["bf16_tflops"])
    if rank == 0:
        print(json.dumps({"mode": "matvec", "workload": p.name, "precision": kprec, "ms": ms,
                          "pair_rhs_per_s": float(p.N) ** 2 * args.t / (ms / 1e3), "kernel_ms": kernel_ms,
                          "kernel": "mv_tcs_kernel" if symmetric else ("mv_tc_kernel" if split else "mv_simt_kernel"),
                          "distance_form": {lgp.LGP_DIST_DOT: "dot", lgp.LGP_DIST_DIFF: "difference"}.get(form),
                          "binding_pipe": bp["binding"], "frac": bp["frac"], "pipe_fracs": bp["pipe_fracs"]}),
              flush=True)


def estimate_plain(lgp, ctx, p, X, y, args, dev, iters, ms_per_step):
    """The plain FP32 path's cost for the same step: t single-RHS CG solves with the t=1 FP32
    SIMT product at the same tolerance, plus one single-column product per column for the
    gradient. Measured: the solve of y and of the first probe column; the other t-2 probe columns
    are counted at the first probe's time (probe columns converge alike).
    """
    import torch
    Z = lgp.lgp_rademacher_probes(1234, p.N, 1, device=dev.index, ctx=ctx)
    cols = [y.reshape(-1, 1).contiguous(), Z[:, :1].contiguous()]
    ms = []
    its = []
    for c in cols:
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        _, it, _, _ = lgp.lgp_cg_solve(X, p, c, tol=args.tol, max_iter=args.max_iter, prec=lgp.LGP_PREC_FP32,
                                       ctx=ctx)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        its.append(int(it[0]))
    out = torch.empty_like(cols[0])
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    lgp.lgp_kernel_matvec(X, p, cols[0], prec=lgp.LGP_PREC_FP32, out=out, ctx=ctx)
    b.record()
    torch.cuda.synchronize()
    mv1 = a.elapsed_time(b)
    est = ms[0] + ms[1] * (args.t - 1) + args.t * mv1
    return {"ms_solve_y": ms[0], "ms_solve_probe": ms[1], "iters_y": its[0], "iters_probe": its[1],
            "ms_single_column_product": mv1, "est_ms_per_step": est, "batched_ms_per_step": ms_per_step,
            "speedup_batched_over_plain_est": est / ms_per_step,
            "note": "plain = t single-RHS FP32 CG solves (t=1 SIMT product) at the same tol + t single-column "
                    "products for the gradient; y and one probe solve timed, the other probes counted at the "
                    "probe's time"}


def bench_plain(lgp, ctx, p, X, y, args, dev):
    """The plain FP32 path at the bench's own size: the whole LML+grad step with every column solved on its
    own (lgp_lml_and_grad with LGP_OPT_SINGLE_RHS), one timed step."""
    import torch
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    lml, grad, info = lgp.lgp_lml_and_grad(X, y, p, n_probes=args.t - 1, lanczos_steps=args.lanczos, seed=1234,
                                           tol=args.tol, max_iter=args.max_iter, ctx=ctx, single_rhs=True)
    b.record()
    torch.cuda.synchronize()
    return {"ms_per_step": a.elapsed_time(b), "iters_max": info["iters_max"], "lml": lml,
            "note": "t single-column FP32 CG solves and t single-column adjoint passes, measured"}


def bench_plain_equal(lgp, args, dev, prec, seed):
    """Both paths on the same problem, probes, tolerance and Lanczos length, each timed in full: the batched
    split-F16 mBCG step and the plain FP32 single-column step (LGP_OPT_SINGLE_RHS), at --plain-N points of
    the bench workload's distribution (the plain path at N=100000 takes minutes), with the two paths' LML
    and gradient differences."""
    import numpy as np
    import torch
    import workloads as wl
    q = wl.cfg4(N=args.plain_N, t=args.t) if args.workload == "cfg4" else wl.cfg3(N=args.plain_N, t=args.t)
    X = torch.as_tensor(q.X, device=dev)
    y = torch.as_tensor(q.y, device=dev)
    ctx = lgp.Context(dev.index or 0)
    out = {"N": q.N, "workload": q.name, "tol": args.tol, "lanczos_steps": args.lanczos}
    res = {}
    for name, single in (("batched", False), ("plain_fp32", True)):
        def step():
            return lgp.lgp_lml_and_grad(X, y, q, n_probes=args.t - 1, lanczos_steps=args.lanczos, seed=seed,
                                        tol=args.tol, max_iter=args.max_iter, prec=prec, ctx=ctx, single_rhs=single)
        step()
        torch.cuda.synchronize()
        ms = []
        for _ in range(2):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            lml, grad, info = step()
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        res[name] = (lml, np.asarray(grad), info)
        out[name] = {"ms_per_step": statistics.mean(ms), "iters_max": info["iters_max"], "lml": lml,
                     "precision": {1: "fp32", 2: "split_bf16", 3: "split_f16"}.get(info["prec_used"])}
    ctx.close()
    (l0, g0, _), (l1, g1, _) = res["batched"], res["plain_fp32"]
    gs = np.maximum(np.abs(g1), 1e-2 * np.abs(g1).max())
    out["lml_rel_diff"] = abs(l0 - l1) / abs(l1)
    out["grad_rel_diff_max"] = float((np.abs(g0 - g1) / gs).max())
    out["speedup_batched_over_plain"] = out["plain_fp32"]["ms_per_step"] / out["batched"]["ms_per_step"]
    return out


def bench_accuracy(lgp, ctx, p, X, y, args, prec, seed, lml, grad):
    """How accurate the timed step is, on the same draw and probes: the true residual of the block solve
    at the step's tolerance (recomputed with the float32 product, whose own error is ~1e-7), its
    componentwise backward error, and the LML and gradient shift against a solve at --ref-tol."""
    import numpy as np
    import torch
    m = args.t - 1
    Z = lgp.lgp_rademacher_probes(seed, p.N, m, device=X.device.index or 0, ctx=ctx)
    B = torch.cat([y.reshape(-1, 1), Z], dim=1).contiguous()
    x, iters, rel, _ = lgp.lgp_cg_solve(X, p, B, tol=args.tol, max_iter=args.max_iter, prec=prec, ctx=ctx)
    Kx = lgp.lgp_kernel_matvec(X, p, x, prec=lgp.LGP_PREC_FP32, ctx=ctx)
    Kabs = lgp.lgp_kernel_matvec(X, p, x.abs().contiguous(), prec=lgp.LGP_PREC_FP32, ctx=ctx)
    R = B.double() - Kx.double()
    res = (torch.linalg.norm(R, dim=0) / torch.linalg.norm(B.double(), dim=0)).cpu().numpy()
    berr = float((R.abs() / (Kabs.double() + B.double().abs())).max().item())
    t0 = time.perf_counter()
    lml_ref, grad_ref, info_ref = lgp.lgp_lml_and_grad(X, y, p, n_probes=m, lanczos_steps=args.lanczos, seed=seed,
                                                       tol=args.ref_tol, max_iter=20000, prec=prec, ctx=ctx,
                                                       precond_rank=args.precond_rank)
    ref_s = time.perf_counter() - t0
    # the Lanczos truncation of the log-determinant: the step's tolerance and probes with the longest
    # tridiagonal the library keeps
    lml_lmax, _, info_lmax = lgp.lgp_lml_and_grad(X, y, p, n_probes=m, lanczos_steps=lgp.LGP_MAX_LANCZOS_STEPS,
                                                  seed=seed, tol=args.tol, max_iter=args.max_iter, prec=prec, ctx=ctx,
                                                  precond_rank=args.precond_rank, want_grad=False)
    g = np.asarray(grad)
    gr = np.asarray(grad_ref)
    gs = np.maximum(np.abs(gr), 1e-2 * np.abs(gr).max())
    return {"tol": args.tol, "true_rel_residual_y": float(res[0]), "true_rel_residual_max": float(res.max()),
            "recursive_rel_residual_max": float(np.max(rel)), "backward_error_max": berr,
            "ref_tol": args.ref_tol, "ref_iters_max": info_ref["iters_max"], "ref_seconds": ref_s,
            "lml_ref": lml_ref, "lml_rel_shift": abs(lml - lml_ref) / abs(lml_ref),
            "grad_rel_shift_max": float((np.abs(g - gr) / gs).max()),
            "lanczos_steps": args.lanczos, "lanczos_max": lgp.LGP_MAX_LANCZOS_STEPS, "lml_lanczos_max": lml_lmax,
            "logdet_lanczos_max": info_lmax["logdet"], "lml_rel_shift_lanczos": abs(lml - lml_lmax) / abs(lml_lmax),
            "note": "residuals of [y | probes] solved at tol with the step's product, recomputed with the FP32 "
                    "product over all rows; shifts = |step - tight solve| on the same probes (gradient relative "
                    "to max(|g_p|, 1e-2 max|g|)); lml_rel_shift_lanczos = |step - the same step with "
                    "lanczos_max Lanczos steps|, the truncation of the log-determinant quadrature"}


def time_adjoint(lgp, ctx, p, X, y, args, dev, prec, rank, flush_buf):
    """The LML call with and without the gradient (the adjoint pass is the difference), 3 timed calls each."""
    import torch
    out = {}
    for name, want in (("lml_only", False), ("lml_and_grad", True)):
        ms = []
        for _ in range(3):
            flush_l2(flush_buf)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            lgp.lgp_lml_and_grad(X, y, p, n_probes=args.t - 1, lanczos_steps=args.lanczos, seed=1234 + rank,
                                 tol=args.tol, max_iter=args.max_iter, prec=prec, ctx=ctx, want_grad=want)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        out[name + "_ms"] = statistics.median(ms)
    out["adjoint_ms"] = out["lml_and_grad_ms"] - out["lml_only_ms"]
    out["hyperparameters"] = p.D + 2
    return out


def bench_memory(lgp, args, dev, prec, rank):
    """Device memory of one LML+grad call (16 CG iterations; the workspace does not depend on the iteration
    count) on the bench workload's distribution at N = 1e3, 1e4, 1e5, 5e5: the library's workspace grows as
    O(N) (Sec. 4.4 reports the matrix-free CG path's peak memory flat in N for its single column)."""
    import torch
    import workloads as wl
    rows = []
    for N in (1000, 10000, 100000, 500000):
        q = wl.cfg3(N=N, t=args.t)
        X = torch.as_tensor(q.X, device=dev)
        y = torch.as_tensor(q.y, device=dev)
        ctx = lgp.Context(dev.index or 0)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info(dev)
        lgp.lgp_lml_and_grad(X, y, q, n_probes=args.t - 1, lanczos_steps=args.lanczos, seed=1, tol=1e-30,
                             max_iter=16, prec=prec, ctx=ctx)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info(dev)
        ws = ctx.workspace_bytes
        rows.append({"N": N, "lgp_workspace_bytes": int(ws), "workspace_bytes_per_point": ws / N,
                     "device_bytes_taken_by_call": int(free0 - free1),
                     "input_bytes": int(X.numel() * 4 + y.numel() * 4)})
        ctx.close()
        del X, y
    if rank == 0:
        print(json.dumps({"mode": "memory", "workload": f"cfg3 distribution, D=8, t={args.t}", "rows": rows}),
              flush=True)


if __name__ == "__main__":
    main()
