"""Benchmark: seconds of one tiled BLR-QR factorization (blr_qr) of the
65536 x 32768 Yukawa kernel matrix (b = 512), with the fraction of the
roofline reached by the factorization kernel, the residual and
orthogonality of the result, an end-to-end number through host buffers,
and the CPU oracle timed on a bounded sample.  The headline is the
mixed-precision factorization; at N = 1 the FP64 factorization of the same
matrix at the same tolerance is timed beside it (both meet
||A - QR||/||A|| <= 10 tol, the stated residual).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision mixed|fp64] [--tol 1e-5] [--size full|small]

N > 1 runs N independent replicas (one per GPU, launched by torchrun); the
single-matrix factorization does not shard.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import collections
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "BLR-QR sec & %roofline at 65k x 32k; mixed vs FP64 GPU at stated ||A-QR||/||A||"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Arithmetic peaks of the pipes this path runs on, measured on a GB300 of
# this pool (one GPU, CUDA events, best of 5-8):
#   FP64: a DFMA throughput loop (16 independent register chains per thread,
#         152 x 8 CTAs of 256 threads): 1.255 TFLOP/s (cuBLAS DGEMM 8192^3:
#         1.10);
#   FP32 SIMT: the same loop in FFMA: 76.7 TFLOP/s;
#   TF32 tensor: torch.matmul of 8192^3 float32 with TF32 allowed (cuBLAS):
#         1033 TFLOP/s; a 3xTF32 product issues three MMAs, so the rate of
#         algorithmic flops is a third of it.
FP64_PEAK_TFLOPS = 1.255
FP32_PEAK_TFLOPS = 76.7
TF32_PEAK_TFLOPS = 1033.0
TC_KINDS = (2, 3, 5, 6, 7)   # update kinds applied on the tensor cores (see roofline)
# DRAM traffic of the factorization kernel: a summary of one ncu capture
# (profiles/), valid while the kernel sources it names are unchanged.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_factor_mixed_traffic_yukawa3d.md")


def csrc_digest() -> str:
    """sha256 (16 hex digits) of the CUDA sources the factorization kernel is
    built from: every file of csrc/ but blr_solve.cu, which holds only the
    kernels that use a finished factor (Q application, solves, products)."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2208_06194_gb300", "csrc")
    for name in sorted(os.listdir(d)):
        if name == "blr_solve.cu":
            continue
        with open(os.path.join(d, name), "rb") as fh:
            h.update(name.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def dram_traffic(flops_counted: float):
    """Bytes of DRAM traffic per launch, scaled from the committed ncu
    capture by counted flops; None when the kernel changed since."""
    try:
        text = open(TRAFFIC_FILE).read()
    except OSError:
        return None, "no capture"
    fields = dict(line.strip("- ").split(": ", 1) for line in text.splitlines()
                  if line.startswith("- ") and ": " in line)
    if fields.get("csrc_sha16") != csrc_digest():
        return None, "the kernel changed since the committed capture"
    per_flop = float(fields["dram_bytes_per_counted_flop"])
    return per_flop * flops_counted, f"scaled by counted flops from {fields.get('workload', '?')}"


def roofline(st, k_sec, prec_is_fp64):
    """Roofline of the factorization kernel for its own mix of work.
    FP64: every counted flop on the FP64 ALUs.  Mixed: the updates that run
    on the tensor cores at the 3xTF32 rate, every other counted flop at the
    FP32 SIMT rate; the bound is the sum of the two times and the peak is
    total flops / bound."""
    flops = st["flops"][4]
    achieved = flops / k_sec / 1e12
    if prec_is_fp64:
        peak = FP64_PEAK_TFLOPS
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None,
                "peak_note": "FP64 ALU, measured DFMA throughput 1.255 TFLOP/s (of measured)",
                "kernel": "k_factor (persistent scheduler)", "flops_counted": flops}
    p_tc = TF32_PEAK_TFLOPS / 3.0
    # updates whose reflector block is applied on the tensor cores: Y~ dense
    # with a dense R_kj or A_ij, and Y~ low-rank with a dense R_kj (their
    # rounded additions, a small share, are counted at the tensor rate too,
    # which can only lower the reported fraction)
    f_tc = sum(st["tpmqrt_kind_flops"][v] for v in TC_KINDS)
    t_bound = f_tc / (p_tc * 1e12) + (flops - f_tc) / (FP32_PEAK_TFLOPS * 1e12)
    peak = flops / t_bound / 1e12
    traffic, traffic_note = dram_traffic(flops)
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": t_bound / k_sec,
            "traffic": traffic, "traffic_note": traffic_note,
            "peak_note": (f"mix of this run: {f_tc / 1e12:.1f} TFLOP at the 3xTF32 rate ({p_tc:.0f} TFLOP/s = "
                          f"measured TF32 {TF32_PEAK_TFLOPS:.0f} / 3) + {(flops - f_tc) / 1e12:.1f} TFLOP at the "
                          f"measured FP32 SIMT rate ({FP32_PEAK_TFLOPS:.1f} TFLOP/s); peak = flops / summed bound "
                          f"time (of measured)"),
            "kernel": "k_factor (persistent scheduler)", "flops_counted": flops,
            "tensor_part": {"tflop": f_tc / 1e12,
                            "cta_seconds": sum(st["tpmqrt_kind_seconds"][v] for v in TC_KINDS)}}

SIZES = {
    "full": dict(m=65536, n=32768, b=512, seed_x=301, seed_y=302),
    "small": dict(m=8192, n=4096, b=512, seed_x=301, seed_y=302),
    # the 131072 x 65536 kernel matrix of the differentiable least-squares
    # workload (points seeds 501/502, right-hand sides seed 503), at b = 512
    "target": dict(m=131072, n=65536, b=512, seed_x=501, seed_y=502),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--tol", type=float, default=1e-5)
    # dense threshold per path (a low-rank result above it is stored dense):
    # measured best at 65536 x 32768, tol 1e-5.  Mixed: 16 3.57 s, 24 3.71,
    # 32 3.92, 48 4.25, 64 4.75 (dense and low-rank-reflector updates with a
    # dense R run on the tensor cores, the other low-rank work as FP32 SIMT
    # code, so dense pays from low ranks on).  FP64: 96 57.4 s, 128 51.0,
    # 160 54.8.
    ap.add_argument("--dense-rank", type=int, default=0, help="0: 16 for mixed, 128 for fp64")
    ap.add_argument("--dense-rank-fp64", type=int, default=128)
    ap.add_argument("--size", default="full", choices=list(SIZES))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare-fp64", action="store_true",
                    help="skip the FP64 factorization timed beside the mixed one (N = 1)")
    ap.add_argument("--lstsq-rhs", type=int, default=0,
                    help="with the FP64 factor (the FP64 leg, or the main one with --precision fp64): also "
                         "solve min ||A~ X - B|| for this many N(0,1) right-hand sides (seed 503) with one "
                         "refinement step, timed")
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed FP64 factorizations (median)")
    ap.add_argument("--fp64-warmup", type=int, default=1)
    ap.add_argument("--scratch-b2", type=int, default=0, help="per-CTA scratch in units of b*b doubles")
    ap.add_argument("--workload", default="yukawa", choices=["yukawa", "batched"],
                    help="batched: 64 uneven Laplace 3D matrices in one graph-captured launch")
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--ill-conditioned", action="store_true",
                    help="columns scaled by a geometric sequence from 1 to 1e-10 (Res and Orth reported)")
    ap.add_argument("--autotune-cache", default=None)
    return ap.parse_args()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- helpers
def kernel_matrix_times(pr, z, torch, dev):
    """A Z for the uncompressed kernel matrix, evaluated on the GPU in row
    blocks (check only; not part of the timed path)."""
    x = torch.from_numpy(pr.x).to(dev)
    y = torch.from_numpy(pr.y).to(dev)
    if pr.col_scale is not None:
        z = z * torch.from_numpy(pr.col_scale).to(dev)[:, None]
    out = torch.empty((pr.m, z.shape[1]), dtype=torch.float64, device=dev)
    for r0 in range(0, pr.m, 2048):
        d = torch.cdist(x[:, r0:r0 + 2048].T, y.T)
        a = torch.exp(-d) / (d + 1e-3)
        out[r0:r0 + 2048] = a @ z
    return out


def probes(blr, fac, a_clone, pr, torch, dev, k=16, seed=5):
    """Res against A~ and A and Orth, estimated with k Gaussian probes:
    E||M Z||_F^2 = k ||M||_F^2 for Z with N(0,1) entries."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    m, n = pr.m, pr.n
    z = torch.randn((n, k), generator=g, dtype=torch.float64)
    zf = blr.to_fortran(z)
    rz = blr.blr_apply_r(fac, zf)
    qrz = blr.fortran_empty(m, k)
    qrz.zero_()
    qrz[:n] = rz
    blr.blr_apply_qt(fac, qrz, trans=1)
    atz = blr.blr_matmul(a_clone, zf)
    az = kernel_matrix_times(pr, z.to(dev), torch, dev)
    res_at = float(torch.linalg.norm(qrz - atz) / torch.linalg.norm(atz))
    res_a = float(torch.linalg.norm(qrz - az) / torch.linalg.norm(az))
    qz = blr.fortran_empty(m, k)
    qz.zero_()
    qz[:n] = zf
    blr.blr_apply_qt(fac, qz, trans=1)
    blr.blr_apply_qt(fac, qz, trans=0)
    orth = float(torch.linalg.norm(qz[:n] - zf) / np.sqrt(k) / np.sqrt(n)) if k else None
    return res_a, res_at, orth


def lstsq_check(blr, fac, a_t, pr, k, torch, seed=503):
    """X = argmin ||A~ X - B||_F for k N(0,1) right-hand sides with one step
    of refinement (blr_lstsq), timed with CUDA events; the residual and the
    optimality of X (Q_1^T r = 0, i.e. A~^T r = R^T Q_1^T r = 0)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    bmat = blr.to_fortran(torch.randn((pr.m, k), generator=g, dtype=torch.float64))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    x = blr.blr_lstsq(fac, bmat, a_orig=a_t, refine_steps=1)
    e1.record()
    e1.synchronize()
    r = bmat - blr.blr_matmul(a_t, x)
    qtr = blr.fortran_empty(pr.m, k)
    qtr.copy_(r)
    blr.blr_apply_qt(fac, qtr, trans=0)
    rn = float(torch.linalg.norm(r))
    return {"rhs": k, "seconds": e0.elapsed_time(e1) * 1e-3, "refine_steps": 1,
            "residual_rel": rn / float(torch.linalg.norm(bmat)),
            "optimality": float(torch.linalg.norm(qtr[:pr.n])) / rn}


_SAMPLE = {}


def dense_equivalent(m: int, n: int, seconds: float) -> dict:
    """Context only: the rate a dense Householder QR of the same m x n
    matrix would need to finish in `seconds` ((2 m n^2 - 2 n^3 / 3) flop)."""
    flop = 2.0 * m * n * n - 2.0 * n ** 3 / 3.0
    return {"tflops": flop / seconds / 1e12, "flop": flop,
            "note": "context only: (2mn^2 - 2n^3/3) / time, the work of a dense Householder QR"}


def tpmqrt_kinds(st, prec_is_fp64=False):
    """Trapezoidal updates by operand kinds (D dense, L low-rank) of Y~_ik,
    R_kj and A_ij: count, summed CTA-seconds, counted GFLOP, and the rate
    while they run as a fraction of one SM's share of the pipe they run on
    (3xTF32 tensor, FP32 SIMT or FP64; one CTA per SM)."""
    out = {}
    for v in range(8):
        n = st["tpmqrt_kind"][v]
        if n:
            name = "Y{} R{} A{}".format(*("D" if v & bit else "L" for bit in (4, 2, 1)))
            cta_s, fl = st["tpmqrt_kind_seconds"][v], st["tpmqrt_kind_flops"][v]
            if prec_is_fp64:
                pipe, peak = "fp64", FP64_PEAK_TFLOPS
            elif v in TC_KINDS:
                pipe, peak = "3xtf32", TF32_PEAK_TFLOPS / 3.0
            else:
                pipe, peak = "fp32", FP32_PEAK_TFLOPS
            rate = fl / cta_s / 1e9 if cta_s > 0 else 0.0
            out[name] = {"n": n, "cta_s": round(cta_s, 3), "gflop": round(fl / 1e9, 1),
                         "gflops_per_sm": round(rate, 1), "pipe": pipe,
                         "frac_of_sm_peak": float(f"{rate / (peak * 1e3 / 152):.4g}")}
    return out


def _task_counts(p: int, q: int) -> dict:
    return {"geqrt": q, "larfb": q * (q - 1) // 2,
            "tsqrt": sum(p - k - 1 for k in range(q)),
            "tpmqrt": sum((p - k - 1) * (q - k - 1) for k in range(q))}


def _host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_factor_time(m: int, n: int, b: int, tol: float, dense_rank: int, seeds: tuple) -> dict:
    """The oracle as it stands on one whole matrix of the benchmark's
    generator: compression (not timed), then Algorithm 4 timed in full, with
    the time of every task recorded by type."""
    from oracle import blr_qr as O
    from paper_2208_06194_gb300 import workloads as W
    key = (m, n, b, tol, dense_rank, seeds)
    if key not in _SAMPLE:
        pr = W.yukawa3d(m, n, b, *seeds)
        _SAMPLE[key] = O.compress(pr.tile, m // b, n // b, b, eps=tol, dense_rank=dense_rank)
    times = {"geqrt": [], "larfb": [], "tsqrt": [], "tpmqrt": []}

    def timed(name, fn):
        def w(*a, **k):
            t0 = time.perf_counter()
            out = fn(*a, **k)
            times[name].append(time.perf_counter() - t0)
            return out
        return w

    saved = (O.geqrt, O.larfb, O.tsqrt, O.tpmqrt)
    O.geqrt, O.larfb, O.tsqrt, O.tpmqrt = (timed("geqrt", O.geqrt), timed("larfb", O.larfb),
                                           timed("tsqrt", O.tsqrt), timed("tpmqrt", O.tpmqrt))
    t0 = time.perf_counter()
    try:
        O.blr_qr(_SAMPLE[key], tol)
    finally:
        O.geqrt, O.larfb, O.tsqrt, O.tpmqrt = saved
    wall = time.perf_counter() - t0
    return {"workload": f"yukawa3d {m}x{n} b={b} tol={tol:g} dense threshold {dense_rank}", "seconds": wall,
            "mean_task_s": {t: (statistics.mean(v) if v else 0.0) for t, v in times.items()},
            "tasks": {t: len(v) for t, v in times.items()}}


def extrapolate(sample: dict, p: int, q: int) -> float:
    """Mean oracle time per task type of a fully timed run x the task counts
    of a p x q tile DAG (the work outside the tasks is negligible)."""
    counts = _task_counts(p, q)
    return sum(counts[t] * sample["mean_task_s"][t] for t in counts)


def cpu_baseline(pr_args, tol, dense_rank):
    """The oracle on the host cores, timed in full on two smaller matrices of
    the same generator, tolerance and dense threshold (4096 x 2048 and
    8192 x 4096), and on the 2048 x 1024 fixed-rank workload.  The value for
    the 65536 x 32768 factorization is extrapolated from the 8192 x 4096 run
    (mean time per task type x the full task counts: at this threshold
    nearly every tile of both is dense, so a task costs the same in both);
    the same extrapolation from 4096 x 2048 to 8192 x 4096 is checked
    against the timed run."""
    from oracle import blr_qr as O
    from paper_2208_06194_gb300 import workloads as W
    b = pr_args["b"]
    seeds = (pr_args["seed_x"], pr_args["seed_y"])
    small = oracle_factor_time(4096, 2048, b, tol, dense_rank, seeds)
    mid = oracle_factor_time(8192, 4096, b, tol, dense_rank, seeds)
    predicted_mid = extrapolate(small, 8192 // b, 4096 // b)
    p, q = pr_args["m"] // b, pr_args["n"] // b
    est = extrapolate(mid, p, q)
    pr1 = W.inv1d_2048x1024()
    a1 = O.compress(pr1.tile, 16, 8, 128, fixed_rank=8)
    t0 = time.perf_counter()
    O.blr_qr(a1, 1e-14)
    cfg1 = time.perf_counter() - t0
    cores = _host_cores()
    return {"value": est, "unit": "s", "cores": cores, "kind": "oracle", "method": "extrapolated",
            "threads": os.environ.get("OMP_NUM_THREADS", f"numpy BLAS default ({cores} host cores)"),
            "sample": (f"oracle Algorithm 4 timed in full on {mid['workload']} ({mid['seconds']:.1f} s, "
                       f"{sum(mid['tasks'].values())} tasks); its mean time per task type x the task counts "
                       f"of the {pr_args['m']}x{pr_args['n']} factorization"),
            "timed_full": [{"workload": small["workload"], "seconds": small["seconds"]},
                           {"workload": mid["workload"], "seconds": mid["seconds"]},
                           {"workload": "inv1d 2048x1024 b=128 fixed rank 8 (rec 1e-14)", "seconds": cfg1}],
            "extrapolation_check": {"from": small["workload"], "to": mid["workload"],
                                    "predicted_s": predicted_mid, "timed_s": mid["seconds"],
                                    "error": predicted_mid / mid["seconds"] - 1.0}}


# ----------------------------------------------------------------------------- main
def run_reference(args, rank, world):
    """Reference arm: the oracle (the only reference there is) on the host.
    Each step times the oracle in full on the 4096 x 2048 matrix of the same
    generator, tolerance and dense threshold and extrapolates it to the
    benchmark's size (mean time per task type x the full task counts)."""
    if rank != 0:
        return
    s = SIZES[args.size]
    b = s["b"]
    vals, last = [], None
    for it in range(args.warmup + args.steps):
        last = oracle_factor_time(4096, 2048, b, args.tol, args.dense_rank, (s["seed_x"], s["seed_y"]))
        if it >= args.warmup:
            vals.append(extrapolate(last, s["m"] // b, s["n"] // b))
    v = statistics.median(vals)
    cores = _host_cores()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args), "global_batch": 1, "dense_rank": args.dense_rank},
            "cpu_baseline": {"kind": "oracle", "method": "extrapolated", "cores": cores, "value": v, "unit": "s",
                             "sample": (f"per step: oracle Algorithm 4 timed in full on {last['workload']} "
                                        f"({last['seconds']:.1f} s); mean time per task type x the task counts of "
                                        f"the {s['m']}x{s['n']} factorization")},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def replica_seeds(size: dict, rank: int) -> tuple[int, int]:
    """Point-set seeds of rank `rank`'s replica: independent problems of the
    same shape on every GPU (the factorization does not shard)."""
    return size["seed_x"] + 1000 * rank, size["seed_y"] + 1000 * rank


def max_over_ranks(value: float, world: int, dist, device) -> float:
    """The job's step time: the slowest rank's (the bench contract)."""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(t_step: float, world: int) -> float:
    """Seconds per factorization over the whole job: world replicas, each a
    full factorization, finish in max-over-ranks time t_step."""
    return t_step / max(world, 1)


def workload_name(args):
    s = SIZES[args.size]
    return (f"yukawa3d {s['m']}x{s['n']} b={s['b']} tol={args.tol:g} RCB-ordered points "
            f"seeds {s['seed_x']}/{s['seed_y']}" + (", columns scaled 1..1e-10" if args.ill_conditioned else ""))


def run_batched(args, rank, world):
    """The batched uneven workload: args.batch Laplace 3D matrices (m from
    {4096, ..., 16384}, n = m/2, tol 1e-6, mixed precision) with tile sizes
    and dense threshold chosen by the autotuner, factored by ONE persistent
    launch replayed from a CUDA graph; the sum of separate blr_qr launches
    of the same matrices is timed beside it."""
    import torch
    import torch.distributed as dist
    from paper_2208_06194_gb300 import autotune, blr
    from paper_2208_06194_gb300 import workloads as W
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl")
    tol, prec = 1e-6, blr.BLR_PREC_MIXED
    probs = W.batched_laplace3d(args.batch, 401 + 1000 * rank)
    tuned = autotune.tune(probs, "laplace3d", tol, prec, cache_path=args.autotune_cache)
    mats = []
    for (m, n, sx, sy), bb in zip(probs, tuned["b"]):
        pr = W.kernel_problem("laplace3d", m, n, bb, sx, sy)
        o = blr.blr_opts_default(b=bb, tol=tol, precision=prec, dense_rank=tuned["dense_rank"])
        mats.append(blr.blr_compress_kernel(pr.x, pr.y, "laplace3d", o))
    opts = blr.blr_opts_default(b=512, tol=tol, precision=prec, dense_rank=tuned["dense_rank"])
    plan = blr.BatchPlan(mats, opts)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            plan.launch(stream=stream.cuda_stream)
            plan.finish(stream=stream.cuda_stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            plan.launch(stream=stream.cuda_stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        clocks = ClockSampler(local)
        clocks.start()
        times = []
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            graph.replay()
            e1.record(stream)
            e1.synchronize()
            plan.finish(stream=stream.cuda_stream)
            times.append(e0.elapsed_time(e1) * 1e-3)
        clk = clocks.stop()
    t_batch = max_over_ranks(statistics.median(times), world, dist, dev)
    st = blr.blr_stats(plan.factor(0))
    # the same matrices one launch each (device time of each blr_qr)
    t_sep = 0.0
    for mm in mats:
        f = blr.blr_qr(blr.blr_matrix_clone(mm), opts)
        t_sep += blr.blr_stats(f)["seconds"]
        f.destroy()
    del graph
    plan.destroy()
    if rank == 0:
        line = {"metric": f"BLR-QR of a batch of {args.batch} uneven Laplace 3D matrices, one persistent launch",
                "value": job_value(t_batch, world), "unit": "s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_batch * 1e3, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64 panels + 3xtf32/f32 updates", "data": "synthetic",
                "config": {"workload": f"{args.batch} x laplace3d, m in 4096..16384, n = m/2, tol {tol:g}",
                           "global_batch": args.batch * world, "tile_sizes": dict(collections.Counter(tuned["b"])),
                           "dense_rank": tuned["dense_rank"], "launch": "CUDA graph replay of blr_batch_plan_launch",
                           "l2": "inputs larger than L2"},
                "separate_launches_seconds": t_sep, "batch_speedup": t_sep / t_batch,
                "tasks": st["tasks"], "flops_counted": st["flops"][4], "autotune": tuned["table"],
                "clocks": clk, "gpu_launches": args.steps}
        print(json.dumps(line), flush=True)
    for mm in mats:
        mm.destroy()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.dense_rank == 0:
        args.dense_rank = 16 if args.precision == "mixed" else 128
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batched":
        run_batched(args, rank, world)
        return
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2208_06194_gb300 import blr
    from paper_2208_06194_gb300 import workloads as W
    s = SIZES[args.size]
    pr = W.yukawa3d(s["m"], s["n"], s["b"], *replica_seeds(s, rank), ill_conditioned=args.ill_conditioned)
    prec = blr.BLR_PREC_MIXED if args.precision == "mixed" else blr.BLR_PREC_FP64
    opts = blr.blr_opts_default(b=s["b"], tol=args.tol, precision=prec, dense_rank=args.dense_rank,
                                scratch_b2=args.scratch_b2)
    a0 = blr.blr_compress_kernel(pr.x, pr.y, "yukawa3d", opts, col_scale=pr.col_scale)
    st_a = blr.blr_stats(a0)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def one_step(o, src=None):
        a = blr.blr_matrix_clone(a0 if src is None else src)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f = blr.blr_qr(a, o)
        e1.record(stream)
        e1.synchronize()
        return f, e0.elapsed_time(e1) * 1e-3

    for _ in range(args.warmup):
        f, _t = one_step(opts)
        f.destroy()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    times, kern, fac = [], [], None
    for it in range(args.steps):
        if fac is not None:
            fac.destroy()
        fac, t = one_step(opts)
        times.append(t)
        kern.append(blr.blr_stats(fac)["seconds"])
    barrier()
    clk = clocks.stop()
    st = blr.blr_stats(fac)
    t_step = max_over_ranks(statistics.median(times), world, dist, dev)
    res_a, res_at, orth = probes(blr, fac, a0, pr, torch, dev)
    ls_main = None
    if args.lstsq_rhs > 0 and prec == blr.BLR_PREC_FP64:
        ls_main = lstsq_check(blr, fac, a0, pr, args.lstsq_rhs, torch)
    fac.destroy()
    if args.size == "target":
        # 68.7 GB of tiles per copy: free the mixed path's input before the
        # FP64 leg compresses its own (the end-to-end leg is skipped here)
        a0.destroy()
        args.no_e2e = True

    # FP64 comparison at the same tolerance (mixed runs only)
    fp64 = None
    if not args.no_compare_fp64 and prec == blr.BLR_PREC_MIXED and world == 1:
        o64 = blr.blr_opts_default(b=s["b"], tol=args.tol, precision=blr.BLR_PREC_FP64,
                                   dense_rank=args.dense_rank_fp64, scratch_b2=args.scratch_b2)
        a64 = blr.blr_compress_kernel(pr.x, pr.y, "yukawa3d", o64, col_scale=pr.col_scale)   # its own threshold
        for _ in range(args.fp64_warmup):
            f64, _t = one_step(o64, a64)
            f64.destroy()
        t64s, f64 = [], None
        for _ in range(max(1, args.fp64_steps)):
            if f64 is not None:
                f64.destroy()
            f64, t64 = one_step(o64, a64)
            t64s.append(t64)
        t64 = statistics.median(t64s)
        r64 = probes(blr, f64, a64, pr, torch, dev)
        st64 = blr.blr_stats(f64)
        ls = lstsq_check(blr, f64, a64, pr, args.lstsq_rhs, torch) if args.lstsq_rhs > 0 else None
        a64.destroy()
        fp64 = {"seconds": t64, "seconds_all": t64s, "warmup": args.fp64_warmup,
                "res_A": r64[0], "res_At": r64[1], "orth": r64[2],
                "gflops_counted": st64["flops"][4] / 1e9,
                "roofline": roofline(st64, statistics.median(t64s), True),
                "meets_10tol": bool(r64[0] <= 10 * args.tol), "mixed_speedup": t64 / t_step,
                "dense_rank": args.dense_rank_fp64, "lstsq": ls}
        f64.destroy()

    # end to end through host buffers: import (H2D) + blr_qr + export (D2H)
    e2e = None
    if not args.no_e2e:
        ranks_h, tiles_h = blr.blr_matrix_export(a0)
        pin_t = torch.from_numpy(tiles_h).pin_memory()
        pin_r = torch.from_numpy(ranks_h).pin_memory()
        out_t = torch.empty_like(pin_t).pin_memory()
        out_r = torch.empty_like(pin_r).pin_memory()
        nt_blocks = sum(pr.m // s["b"] - k for k in range(pr.n // s["b"]))
        out_T = torch.empty(nt_blocks * 32 * s["b"], dtype=torch.float64).pin_memory()
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        a = blr.blr_matrix_import(pr.m, pr.n, s["b"], pin_r.numpy(), pin_t.numpy())
        f = blr.blr_qr(a, opts)
        blr.lib().blr_matrix_export(f.handle, 1, out_r.numpy().ctypes.data_as(blr._IP),
                                    out_t.numpy().ctypes.data_as(blr._DP), blr._stream(None))
        blr.lib().blr_factor_export_t(f.handle, out_T.numpy().ctypes.data_as(blr._DP), blr._stream(None))
        t1.record(stream)
        t1.synchronize()
        f.destroy()
        e2e_s = t0.elapsed_time(t1) * 1e-3
        h2d = pin_t.numel() * 8 + pin_r.numel() * 4
        d2h = out_t.numel() * 8 + out_r.numel() * 4 + out_T.numel() * 8
        e2e = {"value": e2e_s / max(world, 1), "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(s, args.tol, args.dense_rank)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    k_sec = statistics.median(kern)
    line = {
        "metric": METRIC, "value": job_value(t_step, world), "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == 0 else "f64 panels + 3xtf32/f32 updates",
        "data": "synthetic",
        "config": {"workload": workload_name(args), "global_batch": world, "precision": args.precision,
                   "dense_rank": args.dense_rank, "parallelism": "replicas" if world > 1 else "single",
                   "l2": f"inputs larger than L2 ({s['m'] * s['n'] * 8 / 1e9:.0f} GB of tiles per step)"},
        "res_A": res_a, "res_At": res_at, "orth": orth,
        "ranks": {"before": {"n_dense": st_a["n_dense"], "mean": st_a["mean_rank"], "max": st_a["max_rank"]},
                  "after": {"n_dense": st["n_dense"], "mean": st["mean_rank"], "max": st["max_rank"]}},
        "kernel_seconds": k_sec,
        "prep_pool": {"slots": st.get("prep_slots"), "misses": st.get("prep_misses")},
        "task_cta_seconds": dict(zip(["geqrt", "larfb", "tsqrt", "tpmqrt"], st["task_seconds"])),
        "tpmqrt_kinds": tpmqrt_kinds(st, prec == blr.BLR_PREC_FP64),
        "dense_equivalent": dense_equivalent(s["m"], s["n"], t_step),
        "roofline": roofline(st, k_sec, prec == blr.BLR_PREC_FP64),
        "clocks": clk,
        "gpu_launches": args.steps,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "fp64": fp64,
        "lstsq": ls_main,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
