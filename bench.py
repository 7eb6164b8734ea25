#!/usr/bin/env python3
"""HPL benchmark: FP64 LU with partial pivoting + solve on the GPU.

Default workload (N=1 GPU): the random FP64 system of Sec. II with N=32768,
NB=384, seed 42, one right-hand side -- factor with depth-1 look-ahead, solve,
and report HPL TFLOP/s = ((2/3) N^3 + (3/2) N^2) / time.  --config 2 selects
N=131072, NB=512: about 20 minutes per step on one GB300 at FP64 peak, so a
run of 20 timed and 5 warm-up steps (8 hours) does not fit a default run;
that size is run on its own with --config 2 --steps 1 --warmup-n.

The default line also carries an "mxp" block: the mixed-precision variant at
N=65536, NB=1536 (BF16 and FP8-E4M3 LU on tcgen05 + FP64 GMRES-IR), with the
same --steps/--warmup, its effective TFLOP/s, the roofline of its tcgen05
trailing update, and each result's FP64-relative error against one FP64 LU
solve of the same system (--no-mxp leaves it out; --config 3 prints it as a
line of its own).

One step = hpl_getrf + hpl_getrs on a freshly generated system already
resident in HBM (8.6 GB at N=32768, far larger than the 129 MB L2; generation
is outside the timed region, one fresh system per step).  Each timed step is
bracketed by a barrier and a device synchronize; the reported time is the sum
over the K timed steps, max over ranks.  Under torchrun (N > 1 GPUs) every rank
solves its own replica (the factorization has no data-parallel split on one
node that the method defines without collectives): "replicas only".

--impl reference times the CPU oracle (plain C, OpenMP on the host cores) on a
bounded sample of the same workload: the first S elimination steps of the same
N x N system, rated by their algorithmic flops.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CONFIGS = {
    0: dict(n=2048, nb=256),
    1: dict(n=32768, nb=384),
    2: dict(n=131072, nb=512),
    3: dict(n=65536, nb=1536),   # mixed precision (BF16 / FP8-E4M3 LU + FP64 GMRES-IR)
}
L2_BYTES = 129e6  # GB300 L2
METRIC = "HPL FP64 TFLOP/s"
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def hpl_flops(n: int) -> float:
    return (2.0 / 3.0) * n ** 3 + 1.5 * n ** 2


# ------------------------------------------------------------ distributed

def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(value: float, world: int, device=None) -> float:
    """Max over ranks (identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while timing."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix="hpl_clocks_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + CLOCK_FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                                     active=int(parts[4], 16), hw=parts[5], hwt=parts[6], swt=parts[7],
                                     swp=parts[8]))
                except ValueError:
                    continue
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [r for r in rows if r["power"] > 300] or rows
        reasons = set()
        for r in load:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load), "sm_max_mhz": max(r["smax"] for r in rows),
                "power_w_max": max(r["power"] for r in rows), "samples": len(load), "reasons": sorted(reasons)}


# --------------------------------------------------------- CPU oracle sample

def oracle_sample(n: int, seed: int, target_s: float = 12.0, reps: int = 1):
    """Time the oracle on the first S elimination steps of the n x n system.

    S is chosen from a short calibration so one sample takes about target_s.
    Returns (TFLOP/s, seconds, flops, steps, threads)."""
    import numpy as np
    import oracle as O
    A0, _ = O.generate(n, seed)
    A0 = np.asfortranarray(A0)
    # calibration: 2 steps
    A = A0.copy(order="F")
    t0 = time.perf_counter()
    O.getrf_steps_inplace(A, 2)
    per_step = max(1e-4, (time.perf_counter() - t0) / 2)
    steps = int(max(2, min(n, target_s / per_step)))
    best = None
    for _ in range(reps):
        A = A0.copy(order="F")
        t0 = time.perf_counter()
        O.getrf_steps_inplace(A, steps)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    fl = O.getrf_steps_flops(n, steps)
    return fl / best / 1e12, best, fl, steps, O.num_threads()


# ------------------------------------------------------------------- arms

def run_reference(args, cfg):
    """The CPU oracle as the reference arm (rank 0 only)."""
    world, rank, _ = dist_info()
    if rank != 0:
        return 0
    n = cfg["n"]
    import numpy as np
    import oracle as O
    O.build()
    A0, _ = O.generate(n, args.seed)
    A0 = np.asfortranarray(A0)
    A = A0.copy(order="F")
    t0 = time.perf_counter()
    O.getrf_steps_inplace(A, 2)
    per_step = max(1e-4, (time.perf_counter() - t0) / 2)
    budget = 150.0 / max(1, args.steps + args.warmup)  # whole run within a few minutes
    steps = int(max(2, min(n, budget / per_step)))
    times = []
    for it in range(args.warmup + args.steps):
        A[...] = A0
        t0 = time.perf_counter()
        O.getrf_steps_inplace(A, steps)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    fl = O.getrf_steps_flops(n, steps)
    total = sum(times)
    value = fl * len(times) / total / 1e12
    sample = ("first %d of %d elimination steps of the N=%d system (seed %d) per step; oracle = "
              "unblocked right-looking LU, plain C, OpenMP" % (steps, n, n, args.seed))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args, cfg),
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": O.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(args, cfg):
    n, nb = cfg["n"], cfg["nb"]
    return {"workload": "HPL FP64 LU+solve N=%d NB=%d seed=%d 1 RHS, depth-1 look-ahead" % (n, nb, args.seed)
            + (" (warm-up steps at N=%d)" % args.warmup_n if getattr(args, "warmup_n", 0) else ""),
            "N": n, "NB": nb, "seed": args.seed, "lookahead": 0 if args.no_lookahead else 1,
            "l2": (("inputs larger than L2 (%.1f GB matrix per step, fresh each step)" % (8.0 * n * n / 1e9))
                   if 8.0 * n * n > L2_BYTES else
                   ("inputs smaller than L2 (%.1f MB matrix, regenerated each step, no flush): a parity-size "
                    "case, not a bench workload" % (8.0 * n * n / 1e6))),
            "parallelism": "replicas"}


def mxp_block(args, n, nb, seed, with_fp64, H):
    """The mixed-precision variant at (n, nb): LU of the diagonally dominant
    system in BF16 and in FP8-E4M3 (tcgen05) + FP64 GMRES-IR to the HPL
    residual bound.  One step = hpl_mxp_getrf + hpl_gmres_ir on the resident
    FP64 system (32 GB at n = 65536, larger than L2); effective TFLOP/s =
    ((2/3) n^3 + (3/2) n^2) / time.  With with_fp64 the plain FP64 LU solve of
    the same system runs once (untimed against the steps) for the speedup and
    the FP64-relative error ||x - x64||_inf / ||x64||_inf of each result."""
    import torch
    A64, b = H.generate(n, seed, dd=True)
    results = {}
    x64 = None
    if with_fp64:
        A = H.colmajor(n, n)
        A.copy_(A64)
        xf = b.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ipiv, inf64 = H.getrf(A, 512, lookahead=True)
        H.getrs("N", A, ipiv, xf)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        res64 = H.residual(n, seed, xf, dd=True)
        x64 = xf
        del A
        results["fp64"] = {"seconds": t64, "tflops": hpl_flops(n) / t64 / 1e12, "residual": float(res64[0]),
                           "NB": 512, "info": int(inf64.item())}
    LU = H.colmajor(n, n, dtype=torch.float32)
    x = torch.empty(n, device="cuda", dtype=torch.float64)
    info = torch.zeros(1, device="cuda", dtype=torch.int32)
    stream = torch.cuda.current_stream()
    launches0 = H.kernel_launches()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    extra_launches = 0  # those of the untimed update-kernel passes
    precs = [(0, "bf16"), (1, "e4m3")]
    if args.mxp_precs:
        precs = [p for p in precs if p[1] in args.mxp_precs.split(",")]
    for prec, name in precs:
        times = []
        for it in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e2 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            H.mxp_getrf(A64, nb, prec, LU32=LU, info=info)
            e1.record(stream)
            _, st = H.gmres_ir(A64, LU, b, x=x, restart=50, max_outer=50, inner_tol=1e-10, target=16.0)
            e2.record(stream)
            torch.cuda.synchronize()
            if it >= args.warmup:
                times.append((e0.elapsed_time(e1), e1.elapsed_time(e2), st))
        # the trailing-update kernel on its own: one more LU (untimed against
        # the steps) without the look-ahead, whose overlap would put the next
        # diagonal kernel inside the events around each update
        prev = os.environ.get("HPLGB_MXP_LOOKAHEAD")
        os.environ["HPLGB_MXP_LOOKAHEAD"] = "0"
        H.set_gemm_timing(True)
        lc0 = H.kernel_launches()
        H.mxp_getrf(A64, nb, prec, LU32=LU, info=info)
        torch.cuda.synchronize()
        extra_launches += H.kernel_launches() - lc0
        gt = H.gemm_timing()
        H.set_gemm_timing(False)
        if prev is None:
            del os.environ["HPLGB_MXP_LOOKAHEAD"]
        else:
            os.environ["HPLGB_MXP_LOOKAHEAD"] = prev
        res = H.residual(n, seed, x, dd=True)
        lu_ms = sum(t[0] for t in times) / len(times)
        ir_ms = sum(t[1] for t in times) / len(times)
        st = times[-1][2]
        entry = {"lu_ms": lu_ms, "ir_ms": ir_ms, "total_ms": lu_ms + ir_ms,
                 "effective_tflops": hpl_flops(n) / ((lu_ms + ir_ms) * 1e-3) / 1e12,
                 "lu_tflops": (2.0 / 3.0) * n ** 3 / (lu_ms * 1e-3) / 1e12,
                 "outer": st["outer"], "inner": st["inner"], "residual": float(res[0]), "info": int(info.item())}
        if gt["launches"]:
            entry["trailing_update"] = {"launches": gt["launches"], "ms": gt["ms"], "bytes": gt["bytes"],
                                        "flops": gt["flops"], "achieved_gbs": gt["bytes"] / gt["ms"] / 1e6,
                                        "achieved_tflops": gt["flops"] / gt["ms"] / 1e9}
        if x64 is not None:
            entry["fp64_relative_error"] = float((x - x64).abs().max() / x64.abs().max())
            entry["speedup_vs_fp64"] = results["fp64"]["seconds"] / ((lu_ms + ir_ms) * 1e-3)
        results[name] = entry
    clk = clocks.stop()
    names = [nm for _, nm in precs]
    head = "e4m3" if "e4m3" in names else names[0]
    block = {
        "metric": "MxP+IR effective TFLOP/s", "value": results[head]["effective_tflops"], "unit": "TFLOP/s",
        "head": head, "ms_per_step": results[head]["total_ms"], "steps": args.steps, "warmup": args.warmup,
        "dtype": head + "+f32+f64",
        "config": {"workload": "diagonally dominant N=%d seed=%d, unpivoted LU NB=%d in BF16 and FP8-E4M3 "
                               "(tcgen05, per-tile 2^e scales, FP32 accumulate) + FP64 GMRES(50)-IR to "
                               "scaled residual < 16" % (n, seed, nb), "N": n, "NB": nb,
                   "l2": "inputs larger than L2 (%.1f GB FP64 + %.1f GB FP32)" % (8.0 * n * n / 1e9,
                                                                                    4.0 * n * n / 1e9)},
        "results": results, "best_effective_tflops": max(results[nm]["effective_tflops"] for nm in names),
        "gpu_launches": H.kernel_launches() - launches0 - extra_launches, "clocks": clk,
    }
    tu = results[head].get("trailing_update")
    if tu:
        hbm = measured_hbm_gbs()
        alg = tu["bytes"] / tu["launches"]
        traffic = None
        if mxp_gemm_source_sha() == MXP_TRAFFIC_CAPTURE["mxp_gemm_cu_sha256"]:
            traffic = MXP_TRAFFIC_CAPTURE["dram_bytes"] / MXP_TRAFFIC_CAPTURE["alg_bytes"] * alg
        block["roofline"] = {
            "bound": "hbm", "kernel": "mxp_gemm_kernel (tcgen05 trailing update, %s)" % head,
            "achieved": tu["achieved_gbs"], "peak": hbm[0], "unit": "GB/s",
            "frac": tu["achieved_gbs"] / hbm[0] if hbm[0] else None, "traffic": traffic,
            "traffic_source": "ncu dram bytes of the m=n=16384 K=1536 E4M3 launch, as a ratio to its algorithmic "
                              "bytes, times the algorithmic bytes of the average timed launch",
            "algorithmic_bytes_per_launch": alg, "launches": tu["launches"],
            "avg_launch_ms": tu["ms"] / tu["launches"], "peak_source": hbm[1]}
    del A64, b, LU, x
    return block


def emulated_block(args, H, n, nb, seed, la, A, b, x, ipiv, info, stream):
    """HPL with the trailing-update DGEMMs replaced by the emulated FP64
    update (hpl_getrf_emulated: error-free BF16 slice products on tcgen05,
    after Ozaki et al. 2012), same system, --steps/--warmup, with the FP64
    path's pivots (ipiv of its last timed step) as the accuracy check."""
    import torch
    gp64 = ipiv.clone()
    times = []
    clocks = ClockSampler(torch.cuda.current_device())
    launches0 = H.kernel_launches()
    for it in range(args.warmup + args.steps):
        H.generate(n, seed, A=A, b=b)
        x.copy_(b)
        torch.cuda.synchronize()
        if it == args.warmup:
            clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        H.getrf_emulated(A, nb, slices=args.slices, ipiv=ipiv, info=info, lookahead=la)
        H.getrs("N", A, ipiv, x)
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            times.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    launches = H.kernel_launches() - launches0
    H.sync_check()
    res = H.residual(n, seed, x)
    pivots_equal = bool(torch.equal(ipiv, gp64))
    inf = int(info.item())
    # the update kernels on their own: one more factorization (untimed against
    # the steps) without the look-ahead, whose partition and joining launches
    # would put FACT inside the events around each update
    H.generate(n, seed, A=A, b=b)
    H.set_gemm_timing(True)
    H.getrf_emulated(A, nb, slices=args.slices, ipiv=ipiv, info=info, lookahead=False)
    torch.cuda.synchronize()
    gt = H.gemm_timing()
    H.set_gemm_timing(False)
    ms = sum(times) / len(times)
    out = {"metric": "HPL TFLOP/s with the emulated FP64 trailing update", "value": hpl_flops(n) / (ms * 1e-3) / 1e12,
           "unit": "TFLOP/s", "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
           "dtype": "f64 (update: bf16 slice products, exact, summed in f64)",
           "method": "not the paper's: every A22 -= L21 U12 from error-free BF16 slices (Ozaki, Ogita, Oishi, Rump "
                     "2012) on tcgen05; FACT, RS and the U12 solve in FP64",
           "residual": float(res[0]), "info": inf,
           "pivots_equal_fp64_path": pivots_equal, "gpu_launches": launches, "clocks": clk}
    if gt["launches"]:
        # the trailing updates as a whole (split, level products, level sum):
        # FP64-equivalent rate, and the BF16 rate of the level products they
        # contain (s(s+1)/2 products of 2 m n kp each), taken over the whole
        # update time, so a lower bound of the tensor kernels' own rate
        # one pass for k = nb <= 1024: 8 slices for k <= 409, else 9 (unless
        # --slices says otherwise): s (s + 1) / 2 level products
        sl = args.slices or (8 if nb <= 409 else 9)
        levels = sl * (sl + 1) / 2.0
        kp = (nb + 63) // 64 * 64
        bf16_flops = gt["flops"] / nb * kp * levels
        peak = measured_bf16_tflops()
        out["update"] = {"timed": "one more factorization without look-ahead",
                         "launches": gt["launches"], "ms": gt["ms"],
                         "fp64_equivalent_tflops": gt["flops"] / gt["ms"] / 1e9}
        out["roofline"] = {"bound": "tensor", "kernel": "emulated update (level products on tcgen05 kind::f16)",
                           "achieved": bf16_flops / gt["ms"] / 1e9, "peak": peak[0], "unit": "TFLOP/s",
                           "frac": bf16_flops / gt["ms"] / 1e9 / peak[0], "traffic": None,
                           "peak_source": peak[1],
                           "note": "BF16 flops of the level products over the whole update time (split and level "
                                   "sum included): a lower bound of the product kernel's rate"}
    return out


def measured_bf16_tflops():
    """(sustained dense BF16 TFLOP/s, source) from the measured peaks file."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            v = float(json.load(fh)["bf16_tflops_sustained"])
        return v, "measured: MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS, seconds-long loop)"
    except Exception:
        return 1700.0, "fallback: 1.7 PFLOP/s sustained BF16"


def run_mxp(args, cfg):
    """--config 3: the mixed-precision block as a line of its own."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2304_10397_gb300 as H
    block = mxp_block(args, cfg["n"], cfg["nb"], args.seed, args.with_fp64, H)
    line = {"metric": block["metric"], "value": block["value"], "unit": block["unit"], "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": block["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": block["dtype"],
            "data": "synthetic"}
    line.update({k: v for k, v in block.items() if k not in line and k not in ("head",)})
    print(json.dumps(line), flush=True)
    return 0


# DRAM traffic of the tcgen05 trailing update from one ncu capture (bench.py
# --case mxp_gemm --m 16384 --k 1536 --mxp-precs e4m3, ncu --metrics
# dram__bytes_read.sum,dram__bytes_write.sum -k regex:mxp_gemm -s 3 -c 1):
# dram__bytes_read.sum + dram__bytes_write.sum of C(16384 x 16384) -= qL qU^T
# with K = 1536 E4M3,
# against its algorithmic bytes 8 m n + (m + n) K.  Valid for the kernel
# source with this SHA-256 prefix (mxp_gemm_source_sha); reported as null once
# that source changes.
MXP_TRAFFIC_CAPTURE = {"dram_bytes": 1.149409e9 + 1.013075e9,
                       "alg_bytes": 8.0 * 16384 * 16384 + 2.0 * 16384 * 1536,
                       "mxp_gemm_cu_sha256": "e6f9c0cd40ed36a7"}


def mxp_gemm_source_sha() -> str:
    """SHA-256 prefix of mxp_gemm.cu without the sections of the two kernels
    that the trailing update does not run (the SM-pair variant and the fused
    emulated FP64 update): what the captured launch executed, its helpers,
    tensor maps and launcher included."""
    import hashlib
    with open(os.path.join(ROOT, "paper_2304_10397_gb300", "csrc", "mxp_gemm.cu"), "rb") as fh:
        src = fh.read()
    a = src.find(b"// ----------------------------------------- trailing update on SM pairs")
    c = src.find(b"// ------------------------------------------------------------ tensor maps")
    if 0 <= a < c:
        src = src[:a] + src[c:]
    return hashlib.sha256(src).hexdigest()[:16]


def measured_hbm_gbs():
    """(HBM copy GB/s, source) from the measured peaks file, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            v = float(json.load(fh)["hbm_gbs"])
        return v, "measured: MEASURED_PEAKS.json hbm_gbs (STREAM-style copy)"
    except Exception:
        return 6800.0, "fallback: 6.8 TB/s (no measured peaks file)"


def run_ours(args, cfg):
    import numpy as np
    import torch

    world, rank, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    device = torch.device("cuda", torch.cuda.current_device())
    import __graft_entry__
    __graft_entry__.build()
    import paper_2304_10397_gb300 as H

    n, nb = cfg["n"], cfg["nb"]
    la = not args.no_lookahead
    seed = args.seed + rank  # each replica its own system
    stream = torch.cuda.current_stream()

    props = torch.cuda.get_device_properties(device)
    n_sms = props.multi_processor_count

    A = H.colmajor(n, n, device=device)
    b = torch.empty(n, device=device, dtype=torch.float64)
    x = torch.empty(n, device=device, dtype=torch.float64)
    ipiv = torch.empty(n, device=device, dtype=torch.int32)
    info = torch.zeros(1, device=device, dtype=torch.int32)

    def one_step(timed: bool):
        H.generate(n, seed, A=A, b=b)
        x.copy_(b)
        torch.cuda.synchronize()
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        H.getrf(A, nb, ipiv=ipiv, info=info, lookahead=la)
        H.getrs("N", A, ipiv, x)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        return e0.elapsed_time(e1)

    if args.warmup_n:
        # warm-up on a smaller system of the same kind (for sizes whose single
        # step takes tens of minutes); the timed steps use the full size
        Aw = H.colmajor(args.warmup_n, args.warmup_n, device=device)
        bw = torch.empty(args.warmup_n, device=device, dtype=torch.float64)
        ipw = torch.empty(args.warmup_n, device=device, dtype=torch.int32)
        for _ in range(args.warmup):
            H.generate(args.warmup_n, seed, A=Aw, b=bw)
            H.getrf(Aw, nb, ipiv=ipw, info=info, lookahead=la)
            H.getrs("N", Aw, ipw, bw)
        torch.cuda.synchronize()
        del Aw, bw, ipw
    else:
        for _ in range(args.warmup):
            one_step(False)
    H.sync_check()

    clocks = ClockSampler(local)
    launches0 = H.kernel_launches()
    H.set_gemm_timing(True)
    clocks.start()
    times = [one_step(True) for _ in range(args.steps)]
    clk = clocks.stop()
    gt = H.gemm_timing()
    H.set_gemm_timing(False)
    launches = H.kernel_launches() - launches0
    H.sync_check()
    res = H.residual(n, seed, x)
    res_oracle = None
    if args.oracle_residual and rank == 0:
        import oracle as O
        O.build()
        res_oracle = O.residual_seeded(n, seed, x.cpu().numpy())
    total_ms = sum(times)
    total_ms_max = reduce_max(total_ms, world, device)
    flops_all = reduce_sum(hpl_flops(n) * args.steps, world, device)
    value = flops_all / (total_ms_max * 1e-3) / 1e12

    # the same workload with every trailing update emulated in FP64 accuracy
    # from BF16 slice products (not the paper's method: a separate block)
    emulated = None
    if world == 1 and not args.no_emulated:
        emulated = emulated_block(args, H, n, nb, seed, la, A, b, x, ipiv, info, stream)

    # end to end through the public API with host buffers (pinned), per step:
    # H2D of A and b, getrf, getrs, D2H of x
    e2e = None
    if not args.no_e2e:
        H.generate(n, seed, A=A, b=b)  # A holds factors now: regenerate once for the host copy
        hA = torch.empty((n, n), dtype=torch.float64, pin_memory=True)  # column j = row j of hA
        hb = torch.empty(n, dtype=torch.float64, pin_memory=True)
        hx = torch.empty(n, dtype=torch.float64, pin_memory=True)
        hA.copy_(A.t())
        hb.copy_(b)
        torch.cuda.synchronize()
        et = []
        e2e_steps = max(1, min(args.steps, args.e2e_steps))
        for it in range(e2e_steps):
            barrier(world)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            A.t().copy_(hA, non_blocking=True)
            x.copy_(hb, non_blocking=True)
            H.getrf(A, nb, ipiv=ipiv, info=info, lookahead=la)
            H.getrs("N", A, ipiv, x)
            hx.copy_(x, non_blocking=True)
            torch.cuda.synchronize()
            et.append(time.perf_counter() - t0)
            barrier(world)
        res_e2e = H.residual(n, seed, hx.cuda())
        et_max = reduce_max(sum(et), world, device)
        e2e = {"value": flops_all / args.steps * e2e_steps / et_max / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": 8 * n * n + 8 * n, "d2h_bytes_per_step": 8 * n,
               "steps": e2e_steps, "residual": float(res_e2e[0])}
        del hA, hb, hx

    # the mixed-precision variant (second half of the headline metric), one GPU
    mxp = None
    if world == 1 and not args.no_mxp:
        del A, b, x, ipiv
        torch.cuda.empty_cache()
        c3 = CONFIGS[3]
        mxp = mxp_block(args, c3["n"], c3["nb"], args.seed, True, H)
        torch.cuda.empty_cache()

    line = None
    if rank == 0:
        gemm_avg_ms = gt["ms"] / max(1, gt["launches"])
        gemm_avg_flops = gt["flops"] / max(1, gt["launches"])
        achieved = gemm_avg_flops / (gemm_avg_ms * 1e-3) / 1e12 if gt["launches"] else None
        # FP64 ALU roofline: 2 DFMA per clock per SM (unit count measured by the
        # DFMA probe) x 2 flop x SMs x the maximum SM clock
        smax = clk.get("sm_max_mhz") or 2070.0
        peak_tf = n_sms * 2 * 2 * smax * 1e6 / 1e12
        traffic = None
        if gt["launches"] and gemm_source_sha() == DGEMM_TRAFFIC_CAPTURE["gemm_cu_sha256"] \
                and cfg["nb"] == DGEMM_TRAFFIC_CAPTURE["k"]:
            mn_avg = gemm_avg_flops / (2.0 * cfg["nb"])
            traffic = DGEMM_TRAFFIC_CAPTURE["bytes"] * mn_avg / DGEMM_TRAFFIC_CAPTURE["mn"]
        roofline = {"bound": "alu", "kernel": "dgemm_kernel (trailing update, DFMA)",
                    "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                    "frac": (achieved / peak_tf) if achieved else None, "traffic": traffic,
                    "traffic_source": "ncu dram bytes of the m=n=8192 k=384 launch scaled by m*n to the "
                                      "average timed launch",
                    "algorithmic_bytes_per_launch": (16.0 * gemm_avg_flops / (2.0 * cfg["nb"])
                                                     if gt["launches"] else None),
                    "peak_source": "derived: %d SMs x 2 DFMA/clk x 2 flop x %.0f MHz max SM clock" % (n_sms, smax),
                    "launches": gt["launches"], "avg_launch_ms": gemm_avg_ms,
                    "avg_launch_gflop": gemm_avg_flops / 1e9}
        cpu = None
        if not args.no_cpu_baseline:
            tf, secs, fl, steps, cores = oracle_sample(n, args.seed)
            cpu = {"value": tf, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                   "sample": "first %d of %d elimination steps of the N=%d system (%.3g flops, %.1f s)"
                             % (steps, n, n, fl, secs)}
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, cfg),
            "frac_of_fp64_peak": value / peak_tf,
            "fp64_peak_tflops": peak_tf,
            "residual": float(res[0]), "info": int(info.item()),
            "residual_oracle": (float(res_oracle[0]) if res_oracle is not None else None),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk, "mxp": mxp, "emulated": emulated,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# DRAM traffic of the trailing-update DGEMM from one ncu capture (bench.py
# --case dgemm --m 8192 --k 384, ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum
# -k regex:dgemm_kernel -s 3 -c 1): dram__bytes_read.sum + dram__bytes_write.sum
# of the launch C(8192 x 8192) -= A(8192 x 384) B(384 x 8192).  Scaled to a
# launch of the timed region by m*n (k = NB is fixed).  Valid for the kernel
# source with this SHA-256 prefix; reported as null once gemm.cu changes.
DGEMM_TRAFFIC_CAPTURE = {"bytes": 590.515200e6 + 491.534336e6, "mn": 8192 * 8192, "k": 384,
                         "gemm_cu_sha256": "d4a919771786ba28"}


def gemm_source_sha() -> str:
    import hashlib
    with open(os.path.join(ROOT, "paper_2304_10397_gb300", "csrc", "gemm.cu"), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def run_case(args):
    """Single-kernel cases for profiling (ncu -k ...) and phase breakdowns."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2304_10397_gb300 as H
    if args.case == "dgemm":
        m, n, k = args.m, args.n_cols or args.m, args.k
        A = H.colmajor(m, k)
        B = H.colmajor(k, n)
        Cm = H.colmajor(m, n)
        for T in (A, B, Cm):
            T.uniform_(-0.5, 0.5)
        for _ in range(3):
            H.dgemm("N", "N", -1.0, A, B, 1.0, Cm)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        H.dgemm("N", "N", -1.0, A, B, 1.0, Cm)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        print(json.dumps({"case": "dgemm", "m": m, "n": n, "k": k, "ms": ms, "tflops": 2.0 * m * n * k / ms / 1e9}))
        return 0
    if args.case == "ozaki":
        # the emulated FP64 update alone against the FP64 DGEMM: C -= A B,
        # m x n x k (k = NB), slices = --slices (0 = chosen per k)
        m, n, k = args.m, args.n_cols or args.m, args.k
        A = H.colmajor(m, k)
        B = H.colmajor(k, n)
        Cm = H.colmajor(m, n)
        for T in (A, B, Cm):
            T.uniform_(-0.5, 0.5)
        out = {"case": "ozaki", "m": m, "n": n, "k": k, "slices": args.slices}
        def unfused():
            os.environ["HPLGB_OZAKI_UNFUSED"] = "1"
            try:
                H.dgemm_emulated(A, B, Cm, slices=args.slices)
            finally:
                del os.environ["HPLGB_OZAKI_UNFUSED"]
        for name, fn in (("emulated", lambda: H.dgemm_emulated(A, B, Cm, slices=args.slices)),
                         ("emulated_unfused", unfused),
                         ("dfma", lambda: H.dgemm("N", "N", -1.0, A, B, 1.0, Cm))):
            for _ in range(2):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            out[name + "_ms"] = ms
            out[name + "_fp64_tflops"] = 2.0 * m * n * k / ms / 1e9
        out["speedup"] = out["dfma_ms"] / out["emulated_ms"]
        print(json.dumps(out))
        return 0
    if args.case == "hpl_emulated":
        # HPL with the emulated FP64 update alone (look-ahead on): --steps timed
        # after --warmup, N and NB from --config / --n / --nb
        cfg = dict(CONFIGS[args.config])
        n, nb = args.n or cfg["n"], args.nb or cfg["nb"]
        A = H.colmajor(n, n)
        b = torch.empty(n, device="cuda", dtype=torch.float64)
        x = torch.empty(n, device="cuda", dtype=torch.float64)
        ipiv = torch.empty(n, device="cuda", dtype=torch.int32)
        info = torch.zeros(1, device="cuda", dtype=torch.int32)
        ts = []
        for it in range(args.warmup + args.steps):
            H.generate(n, args.seed, A=A, b=b)
            x.copy_(b)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            H.getrf_emulated(A, nb, slices=args.slices, ipiv=ipiv, info=info, lookahead=not args.no_lookahead)
            H.getrs("N", A, ipiv, x)
            e1.record()
            torch.cuda.synchronize()
            if it >= args.warmup:
                ts.append(e0.elapsed_time(e1))
        res = H.residual(n, args.seed, x)
        ms = sum(ts) / len(ts)
        out = {"case": "hpl_emulated", "n": n, "nb": nb, "ms": ms, "tflops": hpl_flops(n) / ms / 1e9,
               "residual": float(res[0]), "info": int(info.item())}
        if args.oracle_residual:
            # the same residual from the oracle's streamed regeneration of A and b
            import oracle as O
            O.build()
            out["residual_oracle"] = float(O.residual_seeded(n, args.seed, x.cpu().numpy())[0])
        print(json.dumps(out))
        return 0
    if args.case == "adjoint":
        # differentiable solve: N=8192, 64 right-hand sides, seeds 42 (A), 43 (B), 44 (W)
        from paper_2304_10397_gb300.autograd import HplSolve
        n, k, nb = args.n or 8192, 64, args.nb or 256
        A0, _ = H.generate(n, 42, with_b=False)
        gB = torch.Generator(device="cuda").manual_seed(43)
        gW = torch.Generator(device="cuda").manual_seed(44)
        B = (torch.rand((n, k), device="cuda", dtype=torch.float64, generator=gB) - 0.5)
        W = (torch.rand((n, k), device="cuda", dtype=torch.float64, generator=gW) - 0.5)
        fw, bw = [], []
        for it in range(args.warmup + args.steps):
            A = A0.detach().clone().requires_grad_(True)
            Bt = B.clone().requires_grad_(True)
            torch.cuda.synchronize()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            X = HplSolve.apply(A, Bt, nb, True)
            e1.record()
            X.backward(W)
            e2.record()
            torch.cuda.synchronize()
            if it >= args.warmup:
                fw.append(e0.elapsed_time(e1))
                bw.append(e1.elapsed_time(e2))
        fl_fw = (2.0 / 3.0) * n ** 3 + 2.0 * n * n * k
        fl_bw = 2.0 * n * n * k + 2.0 * n * n * k
        f, b_ = sum(fw) / len(fw), sum(bw) / len(bw)
        print(json.dumps({"case": "adjoint", "n": n, "nrhs": k, "nb": nb, "forward_ms": f, "backward_ms": b_,
                          "backward_over_forward": b_ / f, "forward_tflops": fl_fw / f / 1e9,
                          "backward_tflops": fl_bw / b_ / 1e9, "steps": args.steps, "warmup": args.warmup}))
        return 0
    if args.case == "laswp":
        # RS alone: the NB interchanges of one panel (random valid pivots) applied
        # to all N columns of an N x N matrix
        n, nb = args.n or 32768, args.nb or 384
        A = H.colmajor(n, n)
        A.uniform_(-0.5, 0.5)
        g = torch.Generator(device="cpu").manual_seed(7)
        ipiv = torch.tensor([int(torch.randint(j, n, (1,), generator=g)) + 1 for j in range(nb)], dtype=torch.int32)
        ipiv_full = torch.arange(1, n + 1, dtype=torch.int32)
        ipiv_full[:nb] = ipiv
        ipd = ipiv_full.cuda()
        for _ in range(3):
            H.laswp(A, 0, nb, ipd)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        H.laswp(A, 0, nb, ipd)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        # algorithmic bytes: each moved element read once and written once
        moved = nb + len(set(int(v) - 1 for v in ipiv.tolist()) - set(range(nb)))
        byts = 16.0 * moved * n
        print(json.dumps({"case": "laswp", "n": n, "nb": nb, "rows_moved_per_column": moved, "ms": ms,
                          "algorithmic_gbs": byts / ms / 1e6}))
        return 0
    if args.case == "panel":
        m, w = args.m, args.nb or 384
        A = H.colmajor(m, w)
        A.uniform_(-0.5, 0.5)
        A0 = A.clone()
        ts = []
        for it in range(4):
            A.copy_(A0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            H.panel_getrf(A)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        H.sync_check()
        ms = min(ts[1:])
        print(json.dumps({"case": "panel", "m": m, "w": w, "ms": ms,
                          "gflops": (m * w * w - w ** 3 / 3.0) / ms / 1e6,
                          "panel_bytes_gbs": 16.0 * m * w / ms / 1e6}))
        return 0
    if args.case == "mxp_gemm":
        # the tcgen05 trailing update alone: C (m x m FP32) -= 2^-(eL+eU) qL qU^T, K = args.k
        prec = 1 if (args.mxp_precs or "e4m3").startswith("e4m3") else 0
        m, kp = args.m, args.k
        dt = torch.int16 if prec == 0 else torch.uint8
        qL = torch.randint(0, 0x3000 if prec == 0 else 0x70, (m, kp), device="cuda", dtype=torch.int32).to(dt)
        qU = torch.randint(0, 0x3000 if prec == 0 else 0x70, (m, kp), device="cuda", dtype=torch.int32).to(dt)
        nt = (m + 127) // 128
        eL = torch.zeros(nt, device="cuda", dtype=torch.int32)
        eU = torch.zeros(nt, device="cuda", dtype=torch.int32)
        C32 = H.colmajor(m, m, dtype=torch.float32)
        C32.zero_()
        for _ in range(3):
            H.mxp_gemm(prec, qL, qU, eL, eU, C32)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        H.mxp_gemm(prec, qL, qU, eL, eU, C32)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        print(json.dumps({"case": "mxp_gemm", "prec": "bf16" if prec == 0 else "e4m3", "m": m, "n": m, "k": kp,
                          "ms": ms, "tflops": 2.0 * m * m * kp / ms / 1e9,
                          "c_bytes_gbs": 8.0 * m * m / ms / 1e6}))
        return 0
    if args.case == "mxp_once":
        # one mixed-precision LU + GMRES-IR of the diagonally dominant system
        # (for launch lists and profiles): --n, --nb, --mxp-precs
        n, nb = args.n or 16384, args.nb or CONFIGS[3]["nb"]
        prec = 1 if (args.mxp_precs or "e4m3").startswith("e4m3") else 0
        A64, b = H.generate(n, args.seed, dd=True)
        LU, info = H.mxp_getrf(A64, nb, prec)
        x, st = H.gmres_ir(A64, LU, b)
        torch.cuda.synchronize()
        print(json.dumps({"case": "mxp_once", "n": n, "nb": nb, "prec": "bf16" if prec == 0 else "e4m3",
                          "info": int(info.item()), "ir": st}))
        return 0
    if args.case == "peaks":
        # the FP64 pipe: DFMA 4x4 register tiles (the DGEMM's inner step), DMMA
        # m8n8k4 chains, and both at once (in every warp, or split by warp)
        out = {"case": "peaks", "unit": "GFLOP/s"}
        for it in (4096, 20000):
            out["dfma_tile_iters%d" % it] = H.fp64_peak(it)
        out["dmma_m8n8k4"] = H.fp64_dmma_peak(10000)
        for r in (1, 2, 4):
            out["mixed_in_warp_dfma_tiles%d" % r] = H.fp64_mixed_peak(4096, r, False)
            out["mixed_split_warps_dfma_tiles%d" % r] = H.fp64_mixed_peak(4096, r, True)
        print(json.dumps(out))
        return 0
    if args.case == "phases" and args.config == 3:
        cfg = dict(CONFIGS[3])
        n, nb = args.n or cfg["n"], args.nb or cfg["nb"]
        os.environ["HPLGB_TIMERS"] = "1"
        A64, b = H.generate(n, args.seed, dd=True)
        out = {"case": "phases", "config": 3, "n": n, "nb": nb}
        for prec, name in ((0, "bf16"), (1, "e4m3")):
            for rep in range(2):  # the second repetition is reported
                LU, info = H.mxp_getrf(A64, nb, prec)
                lu = H.phase_times()
                x, st = H.gmres_ir(A64, LU, b)
                ir = H.phase_times()
            out[name] = {"lu_phases_ms": lu, "ir_phases_ms": ir, "ir_stats": st}
            del LU
        print(json.dumps(out))
        return 0
    if args.case == "phases":
        cfg = dict(CONFIGS[args.config])
        n, nb = args.n or cfg["n"], args.nb or cfg["nb"]
        os.environ["HPLGB_TIMERS"] = "1"
        A = H.colmajor(n, n)
        b = torch.empty(n, device="cuda", dtype=torch.float64)
        H.generate(n, args.seed, A=A, b=b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if args.emulated:
            H.getrf_emulated(A, nb, slices=args.slices, lookahead=False)
        else:
            H.getrf(A, nb, lookahead=False)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        print(json.dumps({"case": "phases", "n": n, "nb": nb, "emulated_update": bool(args.emulated), "wall_s": wall,
                          "phases_ms": H.phase_times(), "tflops": (2.0 / 3.0) * n ** 3 / wall / 1e12}))
        return 0
    raise SystemExit("unknown case %s" % args.case)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, choices=sorted(CONFIGS), default=1)
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--nb", type=int, default=None)
    ap.add_argument("--seed", type=int, default=42)
    ap.add_argument("--no-lookahead", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3, help="steps of the end-to-end (host buffer) measurement")
    ap.add_argument("--no-mxp", action="store_true", help="leave the mixed-precision block out of the default line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--with-fp64", action="store_true", help="config 3: also time the FP64 path on the same system")
    ap.add_argument("--mxp-precs", default=None, help="config 3: comma list of bf16,e4m3 (default both)")
    ap.add_argument("--warmup-n", type=int, default=0, help="run the warm-up steps on an N of this size instead")
    ap.add_argument("--oracle-residual", action="store_true", help="also check the residual with the CPU oracle")
    ap.add_argument("--case", default=None, help="single-kernel case: dgemm | ozaki | phases | peaks | adjoint | laswp | panel | mxp_gemm | mxp_once")
    ap.add_argument("--m", type=int, default=8192)
    ap.add_argument("--n-cols", type=int, default=None)
    ap.add_argument("--k", type=int, default=384)
    ap.add_argument("--slices", type=int, default=0, help="slices of the emulated FP64 update (0 = chosen per k)")
    ap.add_argument("--emulated", action="store_true", help="--case phases: the emulated FP64 update")
    ap.add_argument("--no-emulated", action="store_true", help="leave the emulated-update block out of the default line")
    args = ap.parse_args(argv)
    if args.case:
        return run_case(args)
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps; the number is not a valid bench line", file=sys.stderr)
    cfg = dict(CONFIGS[args.config])
    if args.n:
        cfg["n"] = args.n
    if args.nb:
        cfg["nb"] = args.nb
    if args.impl == "reference":
        return run_reference(args, cfg)
    if args.config == 3:
        return run_mxp(args, cfg)
    return run_ours(args, cfg)


if __name__ == "__main__":
    sys.exit(main())
