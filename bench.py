#!/usr/bin/env python3
"""Benchmark of the OCSC hot path on GB300.

Headline ("images/s at fixed objective vs the plain path"): the batched online
pass on the paper-like workload -- 100x100 synthetic images zero-padded to a
128x128 circular domain, K = 100 filters 11x11, lambda = rho = 1, 50
code-ADMM and 10 dictionary-ADMM iterations -- at mini-batch 64.  One step =
one mini-batch through the whole hot path: FFT of the 64 images, their code
ADMM, the rank-64 history fold, the per-frequency factorisation and DictOCSC.
Metric: images/s.  Beside it: the plain per-image path (mini-batch 1) on the
same workload, and the held-out objective each reaches (the batched path must
reach the plain path's held-out objective within 1 %).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): each rank runs an independent OCSC stream on its own GPU
(replicas; the online dictionary is one sequential state, so the method has no
data-parallel split without changing it).  Time = max over ranks.
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

WORKLOAD = "plain_100in128_k100"
METRIC = "OCSC images/s at fixed objective vs plain path (100x100 in 128x128, K=100, 11x11, mini-batch 64)"
UNIT = "images/s"

# Arithmetic peaks of GB300 derived from unit counts and the maximum SM clock:
# FP64 152 SMs x 2 FMA/clk x 2 flop x 2070 MHz; FP32 152 SMs x 128 lanes x
# 2 flop (FMA) x 2070 MHz.  No driver measurement of either exists; an FMA
# probe on the box measured 73.8 TFLOP/s FP32 at ~1.98 GHz.
SMS = 152
FP64_FMA_PER_CLK_SM = 2
FP32_LANES_SM = 128
SM_MAX_MHZ = 2070.0
FP64_PEAK_TFLOPS = SMS * FP64_FMA_PER_CLK_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
FP32_PEAK_TFLOPS = SMS * FP32_LANES_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
FP32_PROBE_TFLOPS = 73.8
HBM_FALLBACK_GBS = 6800.0


def hbm_peak():
    """Measured copy bandwidth (GB/s) and where it comes from."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "of measured (MEASURED_PEAKS.json hbm_gbs: STREAM-style copy)"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "of fallback (6.8 TB/s, one earlier GB300 measurement)"


# DRAM bytes from ncu captures (profiles/), per unit of work, valid only while
# the kernel's source file is the one captured (sha1 of the file).
#   code_plane: the code128 profile case (the headline launch: 64 images of
#   the headline workload, a middle iteration) -> bytes per image; traffic
#   grows in proportion to the images of a launch (one CTA per image and
#   filter).
#   fold_factor: the fold128 profile case (the headline workload's factor at
#   mini-batch 1) -> bytes per launch at B = 1.
TRAFFIC_CAPTURES = {
    "code_plane": {"bytes": (889656576 + 787825152) / 64, "per": "image", "file": "plane_bodies.cuh",
                   "source_sha1": "7b34b11f81e6fb0ad083a4a77310677caef3084c"},
    "fold_factor": {"bytes": 349984000 + 626438656, "per": "launch at mini-batch 1", "file": "dict_update.cu",
                    "source_sha1": "3d5927605a4f02d7384b7ebd12d46785e836a2f2"},
}


def captured_traffic(kernel, units=1):
    import hashlib

    cap = TRAFFIC_CAPTURES.get(kernel)
    if cap is None:
        return None
    path = os.path.join(ROOT, "paper_1706_06972_gb300", "csrc", cap["file"])
    with open(path, "rb") as f:
        sha = hashlib.sha1(f.read()).hexdigest()
    return cap["bytes"] * units if sha == cap["source_sha1"] else None


def fold_factor_fp64_flops(K: int, F: int) -> float:
    """Flops of one fold_factor launch (all F frequencies) counted as FP64
    work: right-looking complex Cholesky (K^3/6 complex MACs + column scaling)
    and the forward substitution of the right-hand side, at 8 flops per
    complex MAC."""
    chol = 8.0 * (K - 1) * K * (K + 1) / 6.0 + 1.0 * K * (K - 1)
    solves = 8.0 * K * (K - 1) / 2.0
    return F * (chol + solves)


def fold_factor_method_flops(K: int, F: int, B: int) -> float:
    """The method's work in one fold_factor launch, as Sec. III-C counts it:
    per frequency a K x K complex Cholesky and the triangular inverse of its
    factor, (8/3) K^3 real flops (4/3 K^3 each), plus the rank-B fold of the
    history, 8 K^2 B flops (one complex outer product per sample)."""
    return F * (8.0 / 3.0 * K ** 3 + 8.0 * K * K * B)


# FP32 flops (FMA = 2) of one double-float complex multiply-subtract: four
# error-free real multiply-accumulates of 1 FMUL + 3 FFMA + 8 FADD each.
DF_CMAC_FLOPS = 4 * (1 + 3 * 2 + 8)


def fold_factor_df_flops(K: int, F: int) -> float:
    """FP32 flops of one fold_factor launch as the kernel executes it: the
    Cholesky's (K^3 - K)/6 trailing complex MACs and the K(K-1)/2 of the
    right-hand side in double-float (DF_CMAC_FLOPS each), the K(K-1)/2 column
    scalings (two pair products and four renormalisations, 32 flops), and
    X = L^-1 in FP32 ((K^3 - K)/6 complex MACs, 8 flops each)."""
    trail = (K ** 3 - K) / 6.0
    tri = K * (K - 1) / 2.0
    return F * (DF_CMAC_FLOPS * (trail + tri) + 32.0 * tri + 8.0 * trail)


def tri_stride(K: int) -> int:
    t = K * (K + 1) // 2
    return t + (t & 1)


def code_plane_bytes(K: int, N: int, B: int, Jz: int, want_u: bool) -> float:
    """Algorithmic HBM bytes of the Jz code_plane launches of one coding call
    (N <= 128) for B images, from the ADMM of Sec. II-C.1 as fused: per image
    and filter, W^ = F(U - Gamma) read and written between iterations (F
    complex bins each way, none read on the first iteration, none written on
    the last), Gamma read (not on the first) and written (P floats), Z~ of the
    last iteration written (F bins) and U written once if requested; per image
    and launch the multipliers r (F bins); per launch the dictionary spectrum
    D~ (K F bins)."""
    F, P = N * (N // 2 + 1), N * N
    per = (Jz - 1) * F * 8 * 2 + (Jz - 1) * P * 4 + Jz * P * 4 + F * 8 + (P * 4 if want_u else 0)
    return B * K * per + Jz * (B * F * 8 + K * F * 8)


def code_resid_bytes(K: int, N: int, B: int, Jz: int) -> float:
    """Algorithmic HBM bytes of the code_resid launches of one coding call:
    per launch after the first, W^ of every image and filter (F bins), and per
    launch D~ (K F bins), |d|^2 (F floats), x~ and r of every image."""
    F = N * (N // 2 + 1)
    return (Jz - 1) * B * K * F * 8 + Jz * (K * F * 8 + F * 4 + B * F * 16)


def dstep_bytes(K: int, N: int) -> float:
    """One dstep launch: X = L^-1 (packed, F frequencies) and five K x F
    spectra (y, V^, theta^ read; D~ and D~ + theta^ written)."""
    F = N * (N // 2 + 1)
    return F * tri_stride(K) * 8 + 5 * K * F * 8


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", gpu_id],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# oracle legs (CPU baseline and reference arm): the FP64 oracle as it stands
# ---------------------------------------------------------------------------

def _oracle_child(n_images: int, first: int, update: int) -> None:
    """Run in a subprocess: time the oracle coding images first..first+n-1
    (Jz iterations each) and, if update, one dictionary update folding them."""
    import numpy as np

    import oracle
    from workloads import WORKLOADS

    w = WORKLOADS[WORKLOAD]
    st = oracle.init_state(w.filters0().astype(np.float64), 128, 128, w.lam, w.rho)
    codes, res = [], []
    for i in range(first, first + n_images):
        img = w.image(i)
        t0 = time.perf_counter()
        res.append(oracle.code(st, img, w.Jz))
        codes.append(time.perf_counter() - t0)
    upd = None
    if update:
        t0 = time.perf_counter()
        oracle.update_dict(st, res, w.Jd)
        upd = time.perf_counter() - t0
    print(json.dumps({"code_seconds": codes, "update_seconds": upd}))


def run_oracle(n_images: int, first: int = 0, update: bool = True, threads: int = 1) -> dict:
    t = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t, CUDA_VISIBLE_DEVICES="")
    res = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-child", str(n_images), str(first),
                          str(int(update))], capture_output=True, text=True, env=env, cwd=ROOT)
    if res.returncode != 0:
        raise RuntimeError(f"oracle leg failed:\n{res.stderr[-2000:]}")
    return json.loads(res.stdout.strip().splitlines()[-1])


def oracle_rate(batch: int, threads: int, budget_s: float, max_images: int):
    """The oracle on a bounded sample of the headline workload: one image coded
    and folded by one dictionary update, then as many more images coded (no
    update) as the budget allows.  Per-image cost of the mini-batch-`batch`
    form = mean coding time + update time / batch."""
    first = run_oracle(1, 0, True, threads)
    codes = list(first["code_seconds"])
    upd = first["update_seconds"]
    more = int((budget_s - codes[0] - upd) // max(codes[0], 1e-3))
    more = max(0, min(more, max_images - 1))
    if more > 0:
        codes += run_oracle(more, 1, False, threads)["code_seconds"]
    per_image = sum(codes) / len(codes) + upd / batch
    sample = (f"{len(codes)} image(s) of {WORKLOAD} coded (Jz = 50) and one dictionary update (Jd = 10) "
              f"timed; per image = mean coding time + update time / {batch}; FP64 NumPy")
    return {"value": 1.0 / per_image, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
            "code_seconds_per_image": sum(codes) / len(codes), "update_seconds": upd}


def config_dict(extra=None):
    from workloads import WORKLOADS

    w = WORKLOADS[WORKLOAD]
    c = {"workload": WORKLOAD + " at mini-batch 64", "images": "100x100 zero-padded to 128x128 (FFT 128)",
         "n_images_stream": w.n_images, "K": w.K, "filter": f"{w.M}x{w.M}", "lambda": w.lam,
         "rho": w.rho, "batch": 64, "Jz": w.Jz, "Jd": w.Jd,
         "l2": "no flush: each step streams ~2 GB of code-ADMM workspace and the 336 MB history and "
               "factor (> 129 MB L2)"}
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------------------------
# multi-rank helpers
# ---------------------------------------------------------------------------

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device=None):
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------

def reference_arm(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    cpu = oracle_rate(64, 1, 150.0, max(args.steps, 1))
    value = cpu["value"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": 0, "ms_per_step": 1e3 * 64 / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict({"reference": "FP64 NumPy oracle of the paper's Algorithm 3, one host thread",
                               "parallelism": "single GPU", "graphs": False}),
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def test_objective(pkg, learner, w, dev, n_test=8):
    """Test-set evaluation of Sec. IV on held-out images coded with the current
    dictionary (samples are dropped, not folded): mean objective of eq. (ocsc0)
    and mean PSNR of the reconstruction, the peak being each image's range
    (max - min; the images are contrast-normalised floats, not 8-bit)."""
    import torch

    vals, psnrs = [], []
    for i in range(n_test):
        x = torch.from_numpy(w.image(1_000_000 + i)).to(dev)
        u = learner.code([x])
        vals.append(learner.objective([x], u)[0])
        psnrs.append(learner.psnr([x], u, peak=float(x.max() - x.min()))[0])
        learner.drop_pending()
    return sum(vals) / len(vals), sum(psnrs) / len(psnrs)


def make_learner(pkg, w, stream, B, graphs=0, **opts):
    return pkg.OCSC(w.K, w.M, w.lam, w.rho, stream=stream, fft_size=128, pad=w.pad, Jz=w.Jz, Jd=w.Jd,
                    max_batch=B, graphs=graphs, **opts)


def run_steps(learner, xs, B, first, n):
    """n online steps of mini-batch B: code (codes kept inside the library
    only: the step's product is the dictionary) and update."""
    for t in range(first, first + n):
        learner.code(xs[t * B:(t + 1) * B], want_codes=False)
        learner.update_dict()


def event_time(stream, fn):
    import torch

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def plain_leg(pkg, w, dev, stream, args):
    """The plain per-image path (mini-batch 1) on the headline workload: its
    images/s, and the roofline of its dominant kernel fold_factor."""
    import torch

    W, n = 3, args.plain_steps
    xs = [torch.from_numpy(w.image(5_000_000 + i)).to(dev) for i in range(W + n)]
    lr = make_learner(pkg, w, stream, 1, graphs=args.graphs)
    lr.set_dict(w.filters0(), normalize=True)
    run_steps(lr, xs, 1, 0, W)
    lr.sync()
    lr.profile(["fold_factor"])
    lr.profile_read(["fold_factor"])
    secs = event_time(stream, lambda: run_steps(lr, xs, 1, W, n))
    ms, launches = lr.profile_read(["fold_factor"])["fold_factor"]
    lr.profile([])
    lr.close()
    F = 128 * 65
    avg_s = ms / 1e3 / max(launches, 1)
    return {"batch": 1, "steps": n, "value": n / secs, "unit": UNIT, "ms_per_step": 1e3 * secs / n,
            "fold_factor": alu_roofline(w.K, F, 1, avg_s, launches)}


def alu_roofline(K, F, B, avg_s, launches):
    """fold_factor against the FP32 pipe it runs on, with the method's work
    (fold_factor_method_flops) as the numerator; the executed double-float
    instruction stream's flops give the issue efficiency beside it."""
    meth = fold_factor_method_flops(K, F, B)
    df = fold_factor_df_flops(K, F)
    achieved = meth / avg_s / 1e12
    return {"kernel": "fold_factor (per-frequency fold + Cholesky in double-float on the FP32 pipe + FP32 L^-1)",
            "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_PEAK_TFLOPS, "traffic": captured_traffic("fold_factor") if B == 1 else None,
            "peak_note": "FP32 pipe, derived: 152 SMs x 128 lanes x 2 flop x 2070 MHz (no driver measurement; "
                         f"an FMA probe measured {FP32_PROBE_TFLOPS} TFLOP/s at ~1.98 GHz)",
            "work": "method flops (8/3) K^3 F + 8 K^2 B F (Cholesky + triangular inverse + fold)",
            "flops_per_launch": meth, "avg_ms": avg_s * 1e3, "launches": launches,
            "issue_efficiency": {"df_flops_per_launch": df, "achieved": df / avg_s / 1e12,
                                 "frac": df / avg_s / 1e12 / FP32_PEAK_TFLOPS,
                                 "note": "FP32 flops of the double-float instruction stream executed"}}


def hbm_entry(name, bytes_per_launch, avg_s, launches, peak, peak_note, traffic=None):
    achieved = bytes_per_launch / avg_s / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_note": peak_note, "bytes_per_launch": bytes_per_launch,
            "avg_ms": avg_s * 1e3, "launches": launches, "traffic": traffic}


def persistent_leg(pkg, w, dev, stream, args):
    """The headline step (mini-batch 64 on the headline workload) with the
    persistent coder: the 50 code-ADMM iterations of each mini-batch in one
    cooperative launch instead of 100 launches; images/s beside the headline's
    per-iteration launches, on the same images."""
    import torch

    B, W, n = args.batch, 2, args.persistent_steps
    xs = [torch.from_numpy(w.image(i)).to(dev) for i in range((W + n) * B)]
    lr = make_learner(pkg, w, stream, B, persistent=1)
    lr.set_dict(w.filters0(), normalize=True)
    run_steps(lr, xs, B, 0, W)
    lr.sync()
    lr.profile(["persist"])
    lr.profile_read(["persist"])
    secs = event_time(stream, lambda: run_steps(lr, xs, B, W, n))
    ms, launches = lr.profile_read(["persist"])["persist"]
    lr.close()
    return {"batch": B, "steps": n, "value": B * n / secs, "unit": UNIT, "ms_per_step": 1e3 * secs / n,
            "persist_ms_per_launch": ms / max(launches, 1), "launches": launches}


def fixed_objective_leg(pkg, w, dev, stream, args):
    """"At fixed objective" (Sec. IV's test objective on held-out images): a
    plain learner (mini-batch 1) trains on n images; its held-out objective is
    the target.  A batched learner (mini-batch 64) trains on the same image
    stream and its held-out objective is evaluated after every mini-batch; the
    leg reports how many images it needed to reach the target within 1 %."""
    import torch

    B, n, cap = args.batch, args.quality_images, args.quality_images * 4
    xs = [torch.from_numpy(w.image(3_000_000 + i)).to(dev) for i in range(cap)]
    lp = make_learner(pkg, w, stream, 1)
    lp.set_dict(w.filters0(), normalize=True)
    run_steps(lp, xs, 1, 0, n)
    target, p_plain = test_objective(pkg, lp, w, dev)
    lp.close()
    lq = make_learner(pkg, w, stream, B)
    lq.set_dict(w.filters0(), normalize=True)
    reached, trace = None, []
    for t in range(cap // B):
        run_steps(lq, xs, B, t, 1)
        f, p = test_objective(pkg, lq, w, dev)
        trace.append(round(f, 4))
        if reached is None and f <= target * 1.01:
            reached = (t + 1) * B
        if reached is not None and (t + 1) * B >= n:
            break
    lq.close()
    return {"plain_images": n, "target_objective": target, "plain_test_psnr_db": p_plain,
            "band": 0.01, "batched_images_to_target": reached, "batched_objective_after": trace[-1],
            "batched_test_psnr_db": p, "batched_objective_trace": trace, "test_images": 8,
            "test_coding": f"Jz = {w.Jz} iterations per held-out image"}


def mixed_leg(pkg, dev, stream, args):
    """Uneven sizes: images of side 64 / 128 / 256 padded by 10 to FFT 128 /
    256 / 512, K = 100 filters 11x11, mini-batches of 64 mixed images; one
    learner with three size classes (consensus dictionary step).  Three ways of
    issuing the coding of a mini-batch, timed on the same batches: per-iteration
    launches, the same replayed from CUDA graphs, and the persistent coder (all
    Jz iterations of the mini-batch in one cooperative launch)."""
    import torch
    from workloads import WORKLOADS

    w = WORKLOADS["batched_mixed_k100"]
    B = w.batch
    nb = args.mixed_steps
    xs = [torch.from_numpy(w.image(i)).to(dev) for i in range(B * (nb + 2))]
    sides = [int(x.shape[0]) for x in xs]
    kinds = ["image_spectrum", "code_resid", "code_plane", "fold_factor", "dstep", "persist"]
    out = {"workload": "batched_mixed_k100", "batch": B, "steps": nb}
    for name, opts in (("per_iteration", {}), ("graphs", {"graphs": 1}), ("persistent", {"persistent": 1})):
        learner = pkg.OCSC(w.K, w.M, w.lam, w.rho, stream=stream, fft_sizes=[128, 256, 512], pad=w.pad,
                           Jz=w.Jz, Jd=w.Jd, max_batch=B, **opts)
        learner.set_dict(w.filters0(), normalize=True)
        for t in range(2):   # the second batch captures the graphs of the graph variant
            learner.code(xs[t * B:(t + 1) * B], want_codes=False)
            learner.update_dict()
        learner.sync()
        if name != "graphs":
            learner.profile(kinds)
            learner.profile_read(kinds)
        secs = event_time(stream, lambda: run_steps(learner, xs, B, 2, nb))
        prof = learner.profile_read(kinds) if name != "graphs" else {}
        learner.close()
        out[name] = {"value": B * nb / secs, "unit": UNIT, "ms_per_batch": 1e3 * secs / nb,
                     "ms_per_batch_by_kernel": {k: v[0] / nb for k, v in prof.items() if v[1]}}
    timed = sides[2 * B:]
    out["value"] = out["persistent"]["value"]
    out["sides_in_timed_batches"] = {str(sd): timed.count(sd) for sd in sorted(set(timed))}
    return out


def precision_leg(pkg, dev, stream, args):
    """Precision variants of the history fold on the full precision workload
    (256 x 256 images padded by 32 to FFT 288, K = 256 filters 11 x 11,
    mini-batch 128): throughput of the all-FP32 path and of the BF16
    tensor-core fold, and how far the BF16 dictionary and objective move from
    the FP32 path's (the errors of each path against the FP64 oracle are
    measured by the parity tests)."""
    import numpy as np
    import torch

    from workloads import WORKLOADS

    w = WORKLOADS["precision_256_k256"]
    B, N, nb = w.batch, 288, args.precision_steps
    xs = [torch.from_numpy(w.image(i)).to(dev) for i in range(B * (nb + 1))]
    test = [torch.from_numpy(w.image(w.n_images - 1 - i)).to(dev) for i in range(4)]
    kinds = ["image_spectrum", "code_resid", "code_plane", "history_tc", "fold_factor", "dstep"]
    out = {"workload": "precision_256_k256", "fft": N, "K": w.K, "batch": B, "steps": nb}
    dicts, objs = {}, {}
    for prec in (0, 1):
        lr = pkg.OCSC(w.K, w.M, w.lam, w.rho, stream=stream, fft_size=N, pad=w.pad, Jz=w.Jz, Jd=w.Jd,
                      max_batch=B, precision=prec)
        lr.set_dict(w.filters0(), normalize=True)
        lr.code(xs[:B], want_codes=False)
        lr.update_dict()
        lr.sync()
        lr.profile(kinds)
        lr.profile_read(kinds)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for t in range(1, nb + 1):
            lr.code(xs[t * B:(t + 1) * B], want_codes=False)
            lr.update_dict()
        e1.record(stream)
        e1.synchronize()
        secs = e0.elapsed_time(e1) / 1e3
        prof = lr.profile_read(kinds)
        dicts[prec] = lr.get_dict().astype(np.float64)
        us = lr.code(test)
        objs[prec] = float(np.mean(lr.objective(test, us)))
        lr.drop_pending()
        lr.close()
        out["fp32" if prec == 0 else "bf16_tc"] = {
            "value": B * nb / secs, "unit": UNIT, "ms_per_batch": 1e3 * secs / nb,
            "ms_per_batch_by_kernel": {k: v[0] / nb for k, v in prof.items() if v[1]}}
        torch.cuda.empty_cache()
    out["bf16_vs_fp32_full_size"] = {
        "dictionary_rel": float(np.linalg.norm(dicts[1] - dicts[0]) / np.linalg.norm(dicts[0])),
        "objective_rel": abs(objs[1] - objs[0]) / abs(objs[0]),
        "test_images": len(test)}
    return out


def recursion_leg(pkg, w, dev, stream, args):
    """The recursion variant of the history (eq. C_update: C^p kept in FP64 and
    updated in O(K^2) per sample, the ADMM penalty rho / t that matches its
    decaying ridge) against the per-sample factorisation, both under the
    paper's rho P, on the headline workload (B = 1): images/s, per-kernel ms
    per sample (the recursion's fold is timed as fold_factor), and the held-out
    objective and PSNR after the same samples."""
    import torch

    W, n = 3, args.recursion_steps
    xs = [torch.from_numpy(w.image(i)).to(dev) for i in range(W + n)]
    kinds = ["image_spectrum", "code_resid", "code_plane", "fold_factor", "dstep", "vstep_cols",
             "vstep_project", "vstep_spectrum", "dict_norms"]
    out = {"workload": WORKLOAD, "rho_convention": "paper (rho P)", "steps": n}
    for hist, name in ((0, "factor"), (1, "recursion")):
        lr = pkg.OCSC(w.K, w.M, w.lam, w.rho, stream=stream, fft_size=128, pad=w.pad, Jz=w.Jz, Jd=w.Jd,
                      max_batch=1, graphs=args.graphs, history=hist, rho_convention=1)
        lr.set_dict(w.filters0(), normalize=True)
        for i in range(W):
            lr.code([xs[i]], want_codes=False)
            lr.update_dict()
        lr.sync()
        lr.profile(kinds)
        lr.profile_read(kinds)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(W, W + n):
            lr.code([xs[i]], want_codes=False)
            lr.update_dict()
        e1.record(stream)
        e1.synchronize()
        secs = e0.elapsed_time(e1) / 1e3
        prof = lr.profile_read(kinds)
        lr.profile([])
        obj, psnr = test_objective(pkg, lr, w, dev)
        lr.close()
        out[name] = {"value": n / secs, "unit": UNIT, "ms_per_step": 1e3 * secs / n,
                     "ms_per_step_by_kernel": {k: v[0] / n for k, v in prof.items() if v[1]},
                     "test_objective": obj, "test_psnr_db": psnr, "samples_seen": W + n}
        torch.cuda.empty_cache()
    return out


SERVING_CLASSES = (96, 128, 144, 192, 256, 288, 384, 512, 576)


def serving_leg(pkg, dev, stream, args):
    """Continuous batching of single-image requests (side log-uniform in
    [64, 512], FFT class the smallest even 2^a 3^b >= side + 10: 96, 128, 144,
    192, 256, 288, 384, 512, 576; K = 100, residuals checked every 5
    iterations, cap 500, dictionary update every 64 completions, 8 GiB
    admission budget).  Main series at tolerance 1e-2, which the fixed-rho ADMM
    reaches within the cap on these images (~230 iterations for a 100 x 100
    image at rho = lambda = 1), so requests finish at different iterations and
    free their slots early: saturated throughput, then Poisson arrivals at 25 /
    50 / 90 % of it with p50 / p99 latency (arrival to completion, host clock)
    and the fraction of requests stopped by the tolerance.  A short saturated
    run at tolerance 1e-4 shows the cap-bound case."""
    import math
    import random

    import torch
    from workloads import WORKLOADS

    w = WORKLOADS["serving_k100"]
    n_req = args.serve_requests
    loads = (0.25, 0.5, 0.9)
    total = n_req * (1 + len(loads)) + args.serve_cap_requests
    xs = [torch.from_numpy(w.image(i)).to(dev) for i in range(total)]
    lr = pkg.OCSC(w.K, w.M, w.lam, w.rho, stream=stream, fft_sizes=list(SERVING_CLASSES), pad=w.pad,
                  Jz=50, Jd=w.Jd, max_batch=w.batch)
    lr.set_dict(w.filters0(), normalize=True)
    outs = []
    for x in xs:
        n = lr.padded_size(x.shape[0], x.shape[1])
        outs.append(torch.empty((w.K, n, n), device=dev))

    def run(srv, ids, arrivals):
        pos = {rid: k for k, rid in enumerate(ids)}
        t0 = time.perf_counter()
        nxt, done, lat, iters = 0, 0, [], []
        while done < len(ids):
            now = time.perf_counter() - t0
            while nxt < len(ids) and arrivals[nxt] <= now:
                srv.submit(ids[nxt], xs[ids[nxt]], out=outs[ids[nxt]])
                nxt += 1
            active, queued = srv.step() if (nxt > done) else (0, 0)
            t_done = time.perf_counter() - t0
            for d in srv.poll():
                lat.append(t_done - arrivals[pos[d["id"]]])
                iters.append(d["iters"])
                done += 1
            if active == 0 and queued == 0 and nxt < len(ids):
                wait = arrivals[nxt] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
        return time.perf_counter() - t0, lat, iters

    def pct(lat, q):
        lat = sorted(lat)
        return 1e3 * lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)]

    def summary(iters, cap):
        return {"mean_iters": sum(iters) / len(iters),
                "stopped_by_tol": sum(1 for i in iters if i < cap) / len(iters)}

    cap = w.Jz
    torch.cuda.synchronize(dev)
    srv = pkg.Server(lr, tol=args.serve_tol, check_every=5, max_iters=cap, update_every=w.batch, learn=1,
                     mem_budget=8 << 30)
    ids = list(range(n_req))
    secs, lat, iters = run(srv, ids, [0.0] * n_req)
    sat = n_req / secs
    res = {"workload": "serving_k100", "tol": args.serve_tol, "max_iters": cap, "requests_per_load": n_req,
           "saturated": {"rps": sat, "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99), **summary(iters, cap)},
           "loads": []}
    rng = random.Random(5)
    for j, f in enumerate(loads):
        lam = f * sat
        arr, t = [], 0.0
        for _ in range(n_req):
            t += rng.expovariate(lam)
            arr.append(t)
        ids = list(range(n_req * (j + 1), n_req * (j + 2)))
        secs, lat, iters = run(srv, ids, arr)
        res["loads"].append({"offered": f, "offered_rps": lam, "achieved_rps": n_req / secs,
                             "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99), **summary(iters, cap)})
    srv.close()
    if args.serve_cap_requests > 0:
        srv = pkg.Server(lr, tol=1e-4, check_every=5, max_iters=cap, update_every=w.batch, learn=1,
                         mem_budget=8 << 30)
        base = n_req * (1 + len(loads))
        ids = list(range(base, base + args.serve_cap_requests))
        secs, lat, iters = run(srv, ids, [0.0] * len(ids))
        res["tol_1e-4_saturated"] = {"requests": len(ids), "rps": len(ids) / secs, "p50_ms": pct(lat, 0.5),
                                     **summary(iters, cap)}
        srv.close()
    res["dict_version"] = lr.counters()["dict_updates"]
    lr.close()
    return res


def ours_arm(args):
    import torch
    import torch.distributed as dist

    world, rank, local = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    from paper_1706_06972_gb300 import build as _build

    if rank == 0:
        _build.build()
    barrier(dev)
    import paper_1706_06972_gb300 as pkg
    from workloads import WORKLOADS

    w = WORKLOADS[WORKLOAD]
    N, B = 128, args.batch
    K, W, E = args.steps, args.warmup, args.e2e_steps
    base = rank * (W + K) * B
    x_dev = [torch.from_numpy(w.image(base + i)).to(dev) for i in range((W + K) * B)]
    stream = torch.cuda.current_stream(dev)
    learner = make_learner(pkg, w, stream, B)
    learner.set_dict(w.filters0(), normalize=True)
    run_steps(learner, x_dev, B, 0, W)
    learner.sync()
    torch.cuda.synchronize(dev)
    barrier(dev)

    timed_kinds = ["code_plane", "fold_factor"]
    learner.profile(timed_kinds)
    learner.profile_read(timed_kinds)
    c0 = learner.counters()
    gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    sampler = ClockSampler(gpu_id)
    time.sleep(0.3)
    torch.cuda.synchronize(dev)
    barrier(dev)
    t_local = event_time(stream, lambda: run_steps(learner, x_dev, B, W, K))
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    barrier(dev)
    t_max = max_over_ranks(t_local, dev)
    c1 = learner.counters()
    prof = learner.profile_read(timed_kinds)
    learner.profile([])
    learner.sync()

    # Per-kernel breakdown on a few extra steps (all kernel classes timed).
    breakdown = {}
    if args.breakdown_steps > 0:
        learner.profile()
        learner.profile_read()
        run_steps(learner, x_dev, B, W, args.breakdown_steps)
        rd = learner.profile_read()
        learner.profile([])
        tot = sum(v[0] for v in rd.values()) or 1.0
        breakdown = {k: {"ms_per_step": v[0] / args.breakdown_steps,
                         "launches_per_step": v[1] / args.breakdown_steps, "share": v[0] / tot}
                     for k, v in rd.items() if v[1]}

    # End to end through the public API: each step copies its 64 images from
    # pinned host memory and reads the updated dictionary back.
    e2e = None
    if E > 0:
        host = [torch.from_numpy(w.image(10_000_000 + base + i)).pin_memory() for i in range(B * E)]
        xd = [torch.empty_like(host[0], device=dev) for _ in range(B)]
        D_dev = torch.empty((w.K, w.M, w.M), device=dev)
        D_host = torch.empty((w.K, w.M, w.M)).pin_memory()
        torch.cuda.synchronize(dev)
        barrier(dev)

        def e2e_steps():
            for t in range(E):
                for i in range(B):
                    xd[i].copy_(host[t * B + i], non_blocking=True)
                learner.code(xd, want_codes=False)
                learner.update_dict()
                learner.dict_device(out=D_dev)
                D_host.copy_(D_dev, non_blocking=True)

        te = max_over_ranks(event_time(stream, e2e_steps), dev)
        e2e = {"value": world * B * E / te, "unit": UNIT, "h2d_bytes_per_step": int(B * host[0].numel() * 4),
               "d2h_bytes_per_step": int(D_host.numel() * 4), "steps": E}
    tuned = learner.tuning(N)  # launch shapes the autotuner chose
    learner.close()
    legs = set(args.legs.split(","))
    plain = plain_leg(pkg, w, dev, stream, args) if "plain" in legs and args.plain_steps > 0 else None
    fixed = fixed_objective_leg(pkg, w, dev, stream, args) if "fixed" in legs and args.quality_images > 0 else None
    persist = persistent_leg(pkg, w, dev, stream, args) if "persistent" in legs and args.persistent_steps > 0 else None
    mixed = mixed_leg(pkg, dev, stream, args) if args.mixed_steps > 0 and "mixed" in legs else None
    serving = serving_leg(pkg, dev, stream, args) if args.serve_requests > 0 and "serving" in legs else None
    precision = precision_leg(pkg, dev, stream, args) if args.precision_steps > 0 and "precision" in legs else None
    recursion = recursion_leg(pkg, w, dev, stream, args) if args.recursion_steps > 0 and "recursion" in legs else None

    if rank != 0:
        return
    value = world * K * B / t_max
    F = N * (N // 2 + 1)
    peak, peak_note = hbm_peak()
    rooflines = {}
    ms, n = prof["code_plane"]
    if n:
        rooflines["code_plane"] = hbm_entry("code_plane", code_plane_bytes(w.K, N, B, w.Jz, False) / w.Jz,
                                            ms / 1e3 / n, n, peak, peak_note, captured_traffic("code_plane", B))
    ms, n = prof["fold_factor"]
    if n:
        rooflines["fold_factor"] = alu_roofline(w.K, F, B, ms / 1e3 / n, n)
    if breakdown.get("code_resid"):
        b = breakdown["code_resid"]
        n = b["launches_per_step"]
        rooflines["code_resid"] = hbm_entry("code_resid", code_resid_bytes(w.K, N, B, w.Jz) / w.Jz,
                                            b["ms_per_step"] / 1e3 / n, n * args.breakdown_steps, peak, peak_note)
    if breakdown.get("dstep"):
        b = breakdown["dstep"]
        n = b["launches_per_step"]
        rooflines["dstep"] = hbm_entry("dstep", dstep_bytes(w.K, N), b["ms_per_step"] / 1e3 / n,
                                       n * args.breakdown_steps, peak, peak_note)
    shares = {k: breakdown.get(k, {}).get("share", 0.0) for k in rooflines}
    top = max(shares, key=shares.get) if shares and max(shares.values()) > 0 else "code_plane"
    roofline = rooflines.get(top)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = oracle_rate(B, 1, args.cpu_budget, 64)
        if args.cpu_all_cores:
            cpu["all_cores"] = oracle_rate(B, os.cpu_count() or 1, args.cpu_budget, 64)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": 1e3 * t_max / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f32x2", "data": "synthetic",
        "config": config_dict({"parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                               "graphs": False, "tuned": tuned}),
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        "gpu_launches": int(c1["kernel_launches"] - c0["kernel_launches"]),
        "plain_path": plain,
        "vs_plain_path": (value / plain["value"]) if plain else None,
        "fixed_objective": fixed,
        "persistent_coder": persist,
        "rooflines": rooflines,
        "kernel_breakdown": breakdown,
        "mixed_sizes": mixed,
        "serving": serving,
        "precision": precision,
        "recursion": recursion,
    }
    print(json.dumps(line))


PROFILE_CASES = {
    # name: (K, M, FFT size, images, image side, Jz, history precision[, history variant[, update]])
    "large512": (32, 11, 512, 4, 400, 10, 0),
    "large256": (32, 11, 256, 8, 200, 10, 0),
    "code128": (100, 11, 128, 64, 100, 10, 0),
    # K = 256 dictionary step (tensor-core fold, blocked FP64 factor, substitution
    # D-step) on the FFT 64 grid: 2112 frequencies, ~1.7 GB of history and factor.
    "bigk64": (256, 11, 64, 8, 53, 5, 1),
    # Recursion variant of the history (eq. C_update) at the headline sizes:
    # K = 100, FFT 128, one sample per update; C is 672 MB of double-float.
    "rec128": (100, 11, 128, 1, 100, 5, 0, 1),
    # The factorisation (fold_factor) at the headline sizes: K = 100, FFT 128.
    "fold128": (100, 11, 128, 1, 100, 5, 0, 0, 1),
    # The same with the headline's mini-batch of 64 samples folded per update.
    "fold128b64": (100, 11, 128, 64, 100, 2, 0, 0, 1),
}


def profile_case(name: str) -> None:
    """A small coding run for ncu captures of one kernel family (a few GB on
    the device at most, working set still larger than L2)."""
    import torch

    import paper_1706_06972_gb300 as pkg
    from paper_1706_06972_gb300 import build as _build
    from workloads import make_image, raw_filters

    _build.build()
    K, M, N, n, side, Jz, prec, *rest = PROFILE_CASES[name]
    hist = rest[0] if rest else 0
    upd = prec or hist or (len(rest) > 1 and rest[1])
    lr = pkg.OCSC(K, M, 1.0, 1.0, fft_size=N, pad=M - 1, Jz=Jz, Jd=2, max_batch=n, precision=prec,
                  history=hist, rho_convention=1 if hist else 0)
    lr.set_dict(raw_filters(K, M, 3), normalize=True)
    xs = [torch.from_numpy(make_image(side, side, 100 + i)).cuda() for i in range(n)]
    for rep in range(2):
        lr.code(xs, want_codes=False)
        if upd:
            lr.update_dict()
        else:
            lr.drop_pending()
    lr.sync()
    lr.close()
    print(json.dumps({"profile_case": name, "K": K, "N": N, "images": n, "Jz": Jz, "ok": True}))


def main():
    if len(sys.argv) > 1 and sys.argv[1] == "--oracle-child":
        _oracle_child(int(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4]))
        return
    if len(sys.argv) > 2 and sys.argv[1] == "--profile-case":
        profile_case(sys.argv[2])
        return
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--batch", type=int, default=64, help="mini-batch of the headline step")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--breakdown-steps", type=int, default=3)
    ap.add_argument("--plain-steps", type=int, default=30, help="timed samples of the plain (B = 1) leg")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=40.0, help="seconds of oracle work per CPU leg")
    ap.add_argument("--cpu-all-cores", type=int, default=1, help="1: also time the oracle with all host cores")
    ap.add_argument("--graphs", type=int, default=1,
                    help="1: ocsc_code replays a CUDA graph per chunk shape (plain and recursion legs)")
    ap.add_argument("--precision-steps", type=int, default=2,
                    help="timed batches of 128 per variant in the precision leg (0: skip)")
    ap.add_argument("--recursion-steps", type=int, default=40,
                    help="timed samples of each history variant in the recursion leg (0: skip)")
    ap.add_argument("--persistent-steps", type=int, default=10,
                    help="timed mini-batches of the persistent-coder leg (0: skip)")
    ap.add_argument("--legs", default="plain,fixed,persistent,mixed,serving,precision,recursion",
                    help="comma list of the extra legs to run besides the headline")
    ap.add_argument("--mixed-steps", type=int, default=2,
                    help="timed batches of the uneven-size leg (0: skip)")
    ap.add_argument("--serve-requests", type=int, default=400,
                    help="requests per load level of the serving leg (0: skip)")
    ap.add_argument("--serve-tol", type=float, default=1e-2, help="residual tolerance of the serving series")
    ap.add_argument("--serve-cap-requests", type=int, default=64,
                    help="requests of the tolerance-1e-4 saturated serving run (0: skip)")
    ap.add_argument("--quality-images", type=int, default=256,
                    help="images of the plain learner for the fixed-objective target (0: skip)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours_arm(args)


if __name__ == "__main__":
    main()
