#!/usr/bin/env python3
"""Benchmark of the OCSC hot path on GB300.

Workload: the plain online pass at paper-like scale -- 100x100 synthetic
images zero-padded to a 128x128 circular domain, K = 100 filters 11x11,
lambda = rho = 1, mini-batch 1, 50 code-ADMM and 10 dictionary-ADMM iterations
per sample.  One step = one sample through the whole hot path: FFT, code ADMM,
history fold, FP64 per-frequency Cholesky, DictOCSC.  Metric: images/s.

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
METRIC = "OCSC images/s, plain online pass (100x100 in 128x128, K=100, 11x11, B=1)"
UNIT = "images/s"

# Arithmetic peaks of GB300 derived from unit counts and the maximum SM clock:
# FP64 152 SMs x 2 FMA/clk x 2 flop x 2070 MHz; FP32 152 SMs x 128 lanes x
# 2 flop (FMA) x 2070 MHz.
SMS = 152
FP64_FMA_PER_CLK_SM = 2
FP32_LANES_SM = 128
SM_MAX_MHZ = 2070.0
FP64_PEAK_TFLOPS = SMS * FP64_FMA_PER_CLK_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
FP32_PEAK_TFLOPS = SMS * FP32_LANES_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12


# DRAM bytes per fold_factor launch from an ncu capture of this workload
# (profiles/fold_factor_plain_100in128_k100.md), valid only while the kernel
# source is the one captured (sha1 of dict_update.cu).
TRAFFIC_CAPTURE = {"bytes": 350.423040e6 + 625.118720e6,
                   "source_sha1": "5aace13e6608b8694365c38ae4152e912b1af9d3"}


def captured_traffic():
    import hashlib

    path = os.path.join(ROOT, "paper_1706_06972_gb300", "csrc", "dict_update.cu")
    with open(path, "rb") as f:
        sha = hashlib.sha1(f.read()).hexdigest()
    return TRAFFIC_CAPTURE["bytes"] if sha == TRAFFIC_CAPTURE["source_sha1"] else None


def fold_factor_fp64_flops(K: int, F: int) -> float:
    """Algorithmic flops of one fold_factor launch (all F frequencies) counted
    as FP64 work: right-looking complex Cholesky (K^3/6 complex MACs + column
    scaling) and the forward substitution of the right-hand side, at 8 flops
    per complex MAC."""
    chol = 8.0 * (K - 1) * K * (K + 1) / 6.0 + 1.0 * K * (K - 1)
    solves = 8.0 * K * (K - 1) / 2.0
    return F * (chol + solves)


# FP32 flops (FMA = 2) of one double-float complex multiply-subtract: four
# error-free real multiply-accumulates of 1 FMUL + 3 FFMA + 8 FADD each.
DF_CMAC_FLOPS = 4 * (1 + 3 * 2 + 8)


def fold_factor_df_flops(K: int, F: int) -> float:
    """Algorithmic FP32 flops of one fold_factor launch as the kernel computes
    it: the Cholesky's (K^3 - K)/6 trailing complex MACs and the K(K-1)/2 of the
    right-hand side in double-float (DF_CMAC_FLOPS each), the K(K-1)/2 column
    scalings (two pair products and four renormalisations, 32 flops), and
    X = L^-1 in FP32 ((K^3 - K)/6 complex MACs, 8 flops each)."""
    trail = (K ** 3 - K) / 6.0
    tri = K * (K - 1) / 2.0
    return F * (DF_CMAC_FLOPS * (trail + tri) + 32.0 * tri + 8.0 * trail)


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
# oracle legs (CPU baseline and reference arm): FP64 oracle, one thread
# ---------------------------------------------------------------------------

def _oracle_child(n_images: int, first: int) -> None:
    """Run in a subprocess: time the oracle on images first..first+n-1."""
    import numpy as np

    import oracle
    from workloads import WORKLOADS

    w = WORKLOADS[WORKLOAD]
    st = oracle.init_state(w.filters0().astype(np.float64), 128, 128, w.lam, w.rho)
    times = []
    for i in range(first, first + n_images):
        img = w.image(i)
        t0 = time.perf_counter()
        res = oracle.code(st, img, w.Jz)
        oracle.update_dict(st, [res], w.Jd)
        times.append(time.perf_counter() - t0)
    print(json.dumps({"seconds": times}))


def run_oracle(n_images: int, first: int = 0) -> list:
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    res = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-child", str(n_images),
                          str(first)], capture_output=True, text=True, env=env, cwd=ROOT)
    if res.returncode != 0:
        raise RuntimeError(f"oracle leg failed:\n{res.stderr[-2000:]}")
    return json.loads(res.stdout.strip().splitlines()[-1])["seconds"]


def config_dict(extra=None):
    from workloads import WORKLOADS

    w = WORKLOADS[WORKLOAD]
    c = {"workload": WORKLOAD, "images": "100x100 zero-padded to 128x128 (FFT 128)",
         "n_images_stream": w.n_images, "K": w.K, "filter": f"{w.M}x{w.M}", "lambda": w.lam,
         "rho": w.rho, "batch": w.batch, "Jz": w.Jz, "Jd": w.Jd,
         "l2": "no flush: each step streams the 336 MB history and writes the 336 MB factor (> 129 MB L2)"}
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
    budget_s = 150.0
    first = run_oracle(1, 0)
    steps = max(1, min(args.steps, int(budget_s // max(first[0], 1e-3))))
    times = first if steps == 1 else first + run_oracle(steps - 1, 1)
    total = sum(times)
    value = steps / total
    sample = f"first {steps} image(s) of the {WORKLOAD} stream, code + dictionary update each"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": 0, "ms_per_step": 1e3 * total / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict({"reference": "FP64 NumPy oracle of the paper's Algorithm 3, one host thread"}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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


def batched_leg(pkg, w, dev, stream, args):
    """Mini-batch B = 64 on the same workload: throughput, and the held-out
    objective after the same images against the plain B = 1 path."""
    import torch

    B = args.batch
    N = 128
    mk = lambda bsz: pkg.OCSC(w.K, w.M, w.lam, w.rho, stream=stream, fft_size=N, pad=w.pad, Jz=w.Jz,
                              Jd=w.Jd, max_batch=max(bsz, 1), graphs=args.graphs)
    # throughput (two warm-up batches: the second captures the coding graph)
    lb = mk(B)
    lb.set_dict(w.filters0(), normalize=True)
    base = 2_000_000
    nb = args.batched_steps
    xs = [torch.from_numpy(w.image(base + i)).to(dev) for i in range(B * (nb + 1))]
    us = [torch.empty((w.K, N, N), device=dev) for _ in range(B)]
    for _ in range(2):
        lb.code(xs[:B], out=us)
        lb.update_dict()
    lb.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for t in range(1, nb + 1):
        lb.code(xs[t * B:(t + 1) * B], out=us)
        lb.update_dict()
    e1.record(stream)
    e1.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    lb.close()
    out = {"batch": B, "steps": nb, "value": B * nb / secs, "unit": UNIT, "ms_per_batch": 1e3 * secs / nb}
    # same images, plain vs batched, then the held-out objective
    if args.quality_images > 0:
        n = args.quality_images // B * B
        train = [torch.from_numpy(w.image(3_000_000 + i)).to(dev) for i in range(n)]
        lp = mk(1)
        lp.set_dict(w.filters0(), normalize=True)
        for x in train:
            lp.code([x], want_codes=False)
            lp.update_dict()
        f_plain, p_plain = test_objective(pkg, lp, w, dev)
        lp.close()
        lq = mk(B)
        lq.set_dict(w.filters0(), normalize=True)
        for t in range(0, n, B):
            lq.code(train[t:t + B], want_codes=False)
            lq.update_dict()
        f_batch, p_batch = test_objective(pkg, lq, w, dev)
        lq.close()
        out.update({"quality_train_images": n, "test_objective_plain": f_plain,
                    "test_objective_batched": f_batch, "objective_gap": (f_batch - f_plain) / abs(f_plain),
                    "test_psnr_plain_db": p_plain, "test_psnr_batched_db": p_batch, "test_images": 8})
    return out


def mixed_leg(pkg, dev, stream, args):
    """Uneven sizes: images of side 64 / 128 / 256 padded by 10 to FFT 128 /
    256 / 512, K = 100 filters 11x11, mini-batches of 64 mixed images; one
    learner with three size classes (consensus dictionary step)."""
    import torch
    from workloads import WORKLOADS

    w = WORKLOADS["batched_mixed_k100"]
    B = w.batch
    learner = pkg.OCSC(w.K, w.M, w.lam, w.rho, stream=stream, fft_sizes=[128, 256, 512], pad=w.pad,
                       Jz=w.Jz, Jd=w.Jd, max_batch=B)
    learner.set_dict(w.filters0(), normalize=True)
    nb = args.mixed_steps
    xs = [torch.from_numpy(w.image(i)).to(dev) for i in range(B * (nb + 1))]
    sides = [int(x.shape[0]) for x in xs]
    learner.code(xs[:B], want_codes=False)
    learner.update_dict()
    learner.sync()
    kinds = ["image_spectrum", "code_resid", "code_plane", "fold_factor", "dstep"]
    learner.profile(kinds)
    learner.profile_read(kinds)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for t in range(1, nb + 1):
        learner.code(xs[t * B:(t + 1) * B], want_codes=False)
        learner.update_dict()
    e1.record(stream)
    e1.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    prof = learner.profile_read(kinds)
    learner.close()
    timed = sides[B:]
    return {"workload": "batched_mixed_k100", "batch": B, "steps": nb, "value": B * nb / secs, "unit": UNIT,
            "ms_per_batch": 1e3 * secs / nb,
            "sides_in_timed_batches": {str(sd): timed.count(sd) for sd in sorted(set(timed))},
            "ms_per_batch_by_kernel": {k: v[0] / nb for k, v in prof.items()}}


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
    192, 256, 288, 384, 512, 576; K = 100, tolerance 1e-4 checked every 5
    iterations, cap 500, dictionary update every 64 completions, 8 GiB
    admission budget): saturated throughput, then Poisson arrivals at 25 / 50 /
    90 % of it with p50 / p99 latency (arrival to completion, host clock)."""
    import math
    import random

    import torch
    from workloads import WORKLOADS

    w = WORKLOADS["serving_k100"]
    lr = pkg.OCSC(w.K, w.M, w.lam, w.rho, stream=stream, fft_sizes=list(SERVING_CLASSES), pad=w.pad,
                  Jz=50, Jd=w.Jd, max_batch=w.batch)
    lr.set_dict(w.filters0(), normalize=True)
    n_req = args.serve_requests
    loads = (0.25, 0.5, 0.9)
    total = n_req * (1 + len(loads))
    xs = [torch.from_numpy(w.image(i)).to(dev) for i in range(total)]
    outs = []
    for x in xs:
        n = lr.padded_size(x.shape[0], x.shape[1])
        outs.append(torch.empty((w.K, n, n), device=dev))
    srv = pkg.Server(lr, tol=1e-4, check_every=5, max_iters=w.Jz, update_every=w.batch, learn=1,
                     mem_budget=8 << 30)

    def run(ids, arrivals):
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
                k = ids.index(d["id"])
                lat.append(t_done - arrivals[k])
                iters.append(d["iters"])
                done += 1
            if active == 0 and queued == 0 and nxt < len(ids):
                wait = arrivals[nxt] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
        return time.perf_counter() - t0, lat, iters

    torch.cuda.synchronize(dev)
    ids = list(range(n_req))
    secs, lat, iters = run(ids, [0.0] * n_req)
    sat = n_req / secs
    res = {"workload": "serving_k100", "requests_per_load": n_req, "saturated_rps": sat,
           "saturated_mean_iters": sum(iters) / len(iters), "loads": []}
    rng = random.Random(5)
    for j, f in enumerate(loads):
        lam = f * sat
        arr, t = [], 0.0
        for _ in range(n_req):
            t += rng.expovariate(lam)
            arr.append(t)
        ids = list(range(n_req * (j + 1), n_req * (j + 2)))
        secs, lat, iters = run(ids, arr)
        lat.sort()
        p = lambda q: 1e3 * lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)]
        res["loads"].append({"offered": f, "offered_rps": lam, "achieved_rps": n_req / secs,
                             "p50_ms": p(0.50), "p99_ms": p(0.99), "mean_iters": sum(iters) / len(iters)})
    res["dict_version"] = lr.counters()["dict_updates"]
    srv.close()
    lr.close()
    return res


def ours_arm(args):
    import numpy as np
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
    N = 128
    K, W, E = args.steps, args.warmup, args.e2e_steps
    base = rank * (W + K + E)
    imgs = [w.image(base + i) for i in range(W + K + E)]
    x_dev = [torch.from_numpy(im).to(dev) for im in imgs[:W + K]]
    x_host = [torch.from_numpy(im).pin_memory() for im in imgs[W + K:]]
    stream = torch.cuda.current_stream(dev)
    learner = pkg.OCSC(w.K, w.M, w.lam, w.rho, stream=stream, fft_size=N, pad=w.pad, Jz=w.Jz,
                       Jd=w.Jd, max_batch=1, graphs=args.graphs)
    learner.set_dict(w.filters0(), normalize=True)
    u_dev = torch.empty((w.K, N, N), device=dev, dtype=torch.float32)

    for i in range(W):
        learner.code([x_dev[i]], out=[u_dev])
        learner.update_dict()
    learner.sync()
    torch.cuda.synchronize(dev)
    barrier(dev)

    learner.profile(["fold_factor"])
    learner.profile_read(["fold_factor"])
    c0 = learner.counters()
    gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    sampler = ClockSampler(gpu_id)
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    barrier(dev)
    ev0.record(stream)
    for i in range(W, W + K):
        learner.code([x_dev[i]], out=[u_dev])
        learner.update_dict()
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    barrier(dev)
    t_local = ev0.elapsed_time(ev1) / 1e3
    t_max = max_over_ranks(t_local, dev)
    c1 = learner.counters()
    prof = learner.profile_read(["fold_factor"])["fold_factor"]
    learner.profile([])
    learner.sync()
    tuning = learner.tuning(N)

    # Per-kernel breakdown on a few extra steps (context only, not the headline).
    breakdown = {}
    if args.breakdown_steps > 0:
        learner.profile()
        learner.profile_read()
        for i in range(args.breakdown_steps):
            learner.code([x_dev[W + (i % max(K, 1))]], out=[u_dev])
            learner.update_dict()
        rd = learner.profile_read()
        learner.profile([])
        tot = sum(v[0] for v in rd.values()) or 1.0
        breakdown = {k: {"ms_per_step": v[0] / args.breakdown_steps, "launches_per_step": v[1] / args.breakdown_steps,
                         "share": v[0] / tot} for k, v in rd.items()}

    # End to end through the public API with host buffers.
    e2e = None
    if E > 0:
        xd = torch.empty((imgs[0].shape[0], imgs[0].shape[1]), device=dev, dtype=torch.float32)
        u_host = torch.empty((w.K, N, N), dtype=torch.float32).pin_memory()
        torch.cuda.synchronize(dev)
        barrier(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(E):
            xd.copy_(x_host[i], non_blocking=True)
            learner.code([xd], out=[u_dev])
            learner.update_dict()
            u_host.copy_(u_dev, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        te = max_over_ranks(e0.elapsed_time(e1) / 1e3, dev)
        e2e = {"value": world * E / te, "unit": UNIT, "h2d_bytes_per_step": int(xd.numel() * 4),
               "d2h_bytes_per_step": int(u_host.numel() * 4), "steps": E}
    learner.close()
    legs = set(args.legs.split(","))
    batched = batched_leg(pkg, w, dev, stream, args) if args.batched_steps > 0 and "batched" in legs else None
    mixed = mixed_leg(pkg, dev, stream, args) if args.mixed_steps > 0 and "mixed" in legs else None
    serving = serving_leg(pkg, dev, stream, args) if args.serve_requests > 0 and "serving" in legs else None
    precision = precision_leg(pkg, dev, stream, args) if args.precision_steps > 0 and "precision" in legs else None
    recursion = recursion_leg(pkg, w, dev, stream, args) if args.recursion_steps > 0 and "recursion" in legs else None

    if rank != 0:
        return
    value = world * K / t_max
    F = N * (N // 2 + 1)
    flops = fold_factor_df_flops(w.K, F)
    avg_s = prof[0] / 1e3 / max(prof[1], 1)
    achieved = flops / avg_s / 1e12
    fp64_eq = fold_factor_fp64_flops(w.K, F) / avg_s / 1e12
    roofline = {"kernel": "fold_factor (per-frequency Cholesky in double-float on the FP32 pipe)", "bound": "alu",
                "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_PEAK_TFLOPS,
                "traffic": args.traffic if args.traffic is not None else captured_traffic(),
                "peak_note": "FP32 pipe: 152 SMs x 128 lanes x 2 flop (FMA) x 2070 MHz (derived); "
                             "work = the double-float algorithm's FP32 flops",
                "fp64_equivalent": {"achieved": fp64_eq, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                    "frac": fp64_eq / FP64_PEAK_TFLOPS,
                                    "note": "the same factorisation counted as FP64 work against the FP64 pipe"},
                "launches": prof[1], "avg_ms": avg_s * 1e3, "flops_per_launch": flops}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        secs = run_oracle(1, 0)
        cpu = {"value": 1.0 / secs[0], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"image 0 of {WORKLOAD}: code (50 it) + dictionary update (10 it), FP64 NumPy, 1 thread",
               "seconds": secs[0]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": 1e3 * t_max / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f32x2", "data": "synthetic",
        "config": config_dict({"parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                               "graphs": bool(args.graphs), "tuned_tiles": tuning}),
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        "gpu_launches": int(c1["kernel_launches"] - c0["kernel_launches"]),
        "kernel_breakdown": breakdown,
        "batched": batched,
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
    "code128": (100, 11, 128, 16, 100, 10, 0),
    # K = 256 dictionary step (tensor-core fold, blocked FP64 factor, substitution
    # D-step) on the FFT 64 grid: 2112 frequencies, ~1.7 GB of history and factor.
    "bigk64": (256, 11, 64, 8, 53, 5, 1),
    # Recursion variant of the history (eq. C_update) at the headline sizes:
    # K = 100, FFT 128, one sample per update; C is 672 MB of double-float.
    "rec128": (100, 11, 128, 1, 100, 5, 0, 1),
    # The factorisation (fold_factor) at the headline sizes: K = 100, FFT 128.
    "fold128": (100, 11, 128, 1, 100, 5, 0, 0, 1),
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
        _oracle_child(int(sys.argv[2]), int(sys.argv[3]))
        return
    if len(sys.argv) > 2 and sys.argv[1] == "--profile-case":
        profile_case(sys.argv[2])
        return
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--breakdown-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--graphs", type=int, default=1,
                    help="1: ocsc_code replays a CUDA graph per chunk shape (plain and batched legs)")
    ap.add_argument("--precision-steps", type=int, default=2,
                    help="timed batches of 128 per variant in the precision leg (0: skip)")
    ap.add_argument("--recursion-steps", type=int, default=40,
                    help="timed samples of each history variant in the recursion leg (0: skip)")
    ap.add_argument("--legs", default="plain,batched,mixed,serving,precision,recursion",
                    help="comma list of legs to run (profiling runs pick one); the headline needs plain")
    ap.add_argument("--batch", type=int, default=64, help="mini-batch of the batched leg")
    ap.add_argument("--batched-steps", type=int, default=4, help="timed batches of the batched leg (0: skip)")
    ap.add_argument("--mixed-steps", type=int, default=2,
                    help="timed batches of the uneven-size leg (0: skip)")
    ap.add_argument("--serve-requests", type=int, default=96,
                    help="requests per load level of the serving leg (0: skip)")
    ap.add_argument("--quality-images", type=int, default=256,
                    help="images for the plain-vs-batched held-out objective (0: skip)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per fold_factor launch from an ncu capture of this kernel")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours_arm(args)


if __name__ == "__main__":
    main()
