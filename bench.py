#!/usr/bin/env python
"""Benchmark of the SOR-SVD hot path on GB300 (one JSON line on stdout).

A step is one whole SOR-SVD solve (Algorithm 3: Omega, q+1 power passes with
re-orthonormalisation, CholeskyQR of both sketches, core product Q1^T A Q2,
Jacobi SVD of the core, output assembly) on a synthetic matrix already
resident in HBM.  Default workload: bf16 A 65536 x 16384 = U diag(exp(-i/64))
V^T (i <= 1024, Haar U and V), k = 256, p = 10, q = 2, with the precision
comparison of the metric beside it: the same stored matrix solved as BF16,
BF16 + REFINE and FP32 (fp32-accurate split-TF32 tensor-core products),
each timed and scored by ||A - U S V^T||_F / sigma_{k+1}.  ``--workload
cfg2`` runs the fp32 20000 x 10000 matrix U diag(1/i) V^T (Haar U, V of
width 500) + 1e-3 N(0,1), k = 100, p = 10, q = 1.

``value`` is whole-job TFLOP/s with the operation count of the paper's eq.
(C_SOR-SVD+PM) (2q+3) l C_mult + 2 l (m+n)(l+k) + 2 l^2 (m+l), C_mult = 2mn.
``e2e`` is the same metric through the public API with the matrix in pinned
host memory (``sorsvd_run_host``): the host-to-device copy of A and the
device-to-host copy of U, S, V are inside the timed region.  The timed
region records CUDA events around the passes over A only (the roofline's
kernel); the per-class times come from a few extra untimed steps with events
around every launch.  Multi-GPU runs (torchrun) solve one independent
replica per rank (the path has no exchange step): scaling is weak.

``--impl reference`` times the binary64 CPU oracle on the host cores instead
(rank 0 only), on a row-sample of the same workload (sized so that a step
takes a few seconds of CPU time).
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "SOR-SVD TFLOP/s & % roofline; BF16 vs FP32 time at equal relative error"

WORKLOADS = {
    "cfg2": dict(m=20000, n=10000, k=100, p=10, q=1, dtype="f32", width=500, noise=1e-3, spectrum="poly1",
                 desc="fp32 A 20000x10000 = U diag(1/i) V^T (Haar U, V of width 500) + 1e-3 N(0,1); "
                      "k=100, p=10, q=1"),
    "cfg3": dict(m=65536, n=16384, k=256, p=10, q=2, dtype="bf16", width=1024, noise=0.0, spectrum="exp64",
                 desc="bf16 A 65536x16384 = U diag(exp(-i/64))_{i<=1024} V^T (Haar); k=256, p=10, q=2"),
    "cfg1": dict(m=1000, n=1000, k=20, p=5, q=1, dtype="f64", width=1000, noise=0.0, spectrum="cfg1",
                 desc="fp64 A 1000x1000, sigma_i = 1 (i<=20), 10^{-(i-20)/10}; k=20, p=5, q=1"),
    "cfg4": dict(batch=512, p=8, q=1, dtype="tf32",
                 desc="512 fp32 matrices, m log-uniform [256, 4096], n log-uniform [128, 2048], k uniform 8..64, "
                      "p=8, q=1, sigma_i = i^-2 over min(m, n) (Haar factors); batched plan replayed as a CUDA graph"),
    "cfg5": dict(batch=8, m=25344, n=400, rank=5, k=5, p=5, q=1, dtype="f32",
                 desc="RPCA (inexact ALM, SOR-SVD low-rank step) of 8 problems X = L + S, 25344x400 fp32, "
                      "L rank 5 (Gaussian factors), S 5% support, |S| uniform [1, 10]; k=5, p=5, q=1; "
                      "tol 1e-7, <= 50 iterations, fp32 SOR-SVD with a binary64 finish"),
}


# (rows, columns) of the oracle's sample of a workload: the cpu_baseline leg
# (one solve, ~10-30 s) and the reference arm (one solve per step, W + K
# steps within a few minutes).  The oracle's Householder QR of an n x 266
# sketch costs ~10 s at n = 16384, so the 65536 x 16384 workload is sampled
# in both dimensions.
CPU_SAMPLE = {"cfg2": (20000, 10000), "cfg3": (8192, 4096), ("cfg3", "reference"): (3072, 2048),
              "cfg1": (1000, 1000)}


def flops(m, n, k, p, q):
    """eq. (C_SOR-SVD+PM) with C_mult = 2mn."""
    l = k + p
    return float((2 * q + 3) * l * 2 * m * n + 2 * l * (m + n) * (l + k) + 2 * l * l * (m + l))


def sigma_of(w):
    from paper_1804_00462_gb300 import inputs
    if w["spectrum"] == "poly1":
        return inputs.sigma_poly(w["width"])
    if w["spectrum"] == "exp64":
        return inputs.sigma_exp(w["width"], 64.0)
    return inputs.sigma_cfg1(w["width"])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except Exception:
            return None
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows)}


def build_input(w, seed, device):
    import torch
    from paper_1804_00462_gb300 import inputs
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f64": torch.float32}[w["dtype"]]
    At = inputs.spectral_torch(w["m"], w["n"], sigma_of(w), seed, device=device, noise=w["noise"], out_dtype=tdt)
    if w["dtype"] == "f64":
        At = At.double()
    return At            # (n, m) contiguous = column-major A


def traffic_from_profiles(kernel_key: str):
    """dram bytes per launch from a committed ncu summary, if it still matches the source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    ent = d.get(kernel_key)
    if not ent:
        return None
    # every source file that defines the kernel, hashed in the listed order
    srcs = ent.get("sources") or [ent["source"]]
    try:
        hh = hashlib.sha256()
        for src in srcs:
            hh.update(open(os.path.join(ROOT, src), "rb").read())
        h = hh.hexdigest()[:16]
    except Exception:
        return None
    return ent["bytes_per_launch"] if h == ent.get("source_sha256_16") else None


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over all ranks (a job's step time is its slowest
    rank's); x itself on a single rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_tflops(flops_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput: the work of every rank over the job's step time."""
    return flops_per_rank * world / (ms * 1e-3) / 1e12


def run_ours(args, w, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1804_00462_gb300 import native

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    m, n, k, p, q, dt = w["m"], w["n"], w["k"], w["p"], w["q"], w["dtype"]
    At = build_input(w, seed=rank, device=dev)
    A = At.T
    od = native.out_dtype(native.dtype_code(dt))
    U = native.colmajor_empty(m, k, od, dev)
    S = torch.empty(k, dtype=od, device=dev)
    V = native.colmajor_empty(n, k, od, dev)
    ws = native.alloc_workspace(m, n, k, p, dt, 0, dev)
    stream = torch.cuda.current_stream()

    def step(seed):
        native.run(A, k, p, q, seed=seed, dtype=dt, workspace=ws, out=(U, S, V))

    for i in range(args.warmup):
        step(i)
    st, info = native.get_status(ws)
    if st != 0:
        raise RuntimeError(f"device status after warm-up: {native.status_string(st)}")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # --- timed region (kernel-only: A resident in HBM; A is 800 MB > L2, so
    # no L2 flush is needed between steps) ---
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    lc0 = native.launch_count()
    # CUDA events around the passes over A only (the roofline's kernel): an
    # event pair around every launch would itself add to the step time
    pass_classes = ("pass", "pass_split", "core_pass")
    native.profile_begin(pass_classes)
    with ClockSampler(local_rank) as clk:
        t_wall = time.perf_counter()
        ev0.record(stream)
        for i in range(args.steps):
            step(1000 + i)
        ev1.record(stream)
        barrier()
        t_wall = time.perf_counter() - t_wall
    prof = native.profile_end()
    launches = native.launch_count() - lc0
    ms = ev0.elapsed_time(ev1) / args.steps
    # every launch class, from a few more (untimed) steps with events around
    # each launch
    prof_steps = max(1, min(args.steps, 5))
    native.profile_begin()
    for i in range(prof_steps):
        step(3000 + i)
    all_prof = native.profile_end()
    barrier()
    clocks = clk.summary()
    ms = max_over_ranks(ms, world, dev)
    F = flops(m, n, k, p, q)
    value = job_tflops(F, world, ms)

    # --- end to end through the public API: A in pinned host memory, U S V
    # back to pinned host memory; sorsvd_run_host copies A in column blocks
    # (overlapped with Omega and the transposed copy) and the factors back ---
    esz = A.element_size()
    hostA = torch.empty(At.shape, dtype=At.dtype, pin_memory=True)
    hostA.copy_(At)
    hU = torch.empty(k, m, dtype=od, pin_memory=True)
    hS = torch.empty(k, dtype=od, pin_memory=True)
    hV = torch.empty(k, n, dtype=od, pin_memory=True)
    ws_host = native.alloc_workspace(m, n, k, p, dt, native.FLAG_HOST_IO, dev)
    e_steps = max(3, min(args.steps, 10))

    def e2e_step(seed):
        native.run_host(hostA.T, k, p, q, seed=seed, dtype=dt, workspace=ws_host, out=(hU.T, hS, hV.T))

    e2e_step(0)
    barrier()
    ev0.record(stream)
    for i in range(e_steps):
        e2e_step(2000 + i)
    ev1.record(stream)
    barrier()
    e_ms = max_over_ranks(ev0.elapsed_time(ev1) / e_steps, world, dev)
    h2d = m * n * esz
    d2h = (m * k + k + n * k) * torch.empty(0, dtype=od).element_size()

    # --- roofline of the dominant pass over A (the contraction the
    # throughput is about); every class's time is reported beside it ---
    pk, pk_src = peaks()
    pass_classes = ("pass", "pass_split", "core_pass")
    dom = max(pass_classes, key=lambda c: prof[c][0])
    dom_ms, dom_n = prof[dom]
    per_launch_ms = dom_ms / max(dom_n, 1)
    l = k + p
    algo_flops = 2.0 * m * n * l
    acc_e = 8 if dt == "f64" else 4
    algo_bytes = m * n * esz + (m + n) * l * acc_e
    achieved_gbs = algo_bytes / (per_launch_ms * 1e-3) / 1e9
    tc_peak = {"bf16": pk["bf16_tflops_sustained"], "f16": pk["bf16_tflops_sustained"],
               "tf32": 0.5 * pk["bf16_tflops_sustained"], "f32": 0.5 * pk["bf16_tflops_sustained"]}
    if dt == "f64":
        # CUDA-core binary64 passes: the part's nominal FP64 rate
        roofline = {"bound": "alu", "kernel": f"gemm_kernel ({dom})", "achieved": algo_flops / (per_launch_ms * 1e-3) / 1e12,
                    "peak": 1.25, "unit": "TFLOP/s", "peak_source": "nominal FP64 rate of GB300 (1.25 TFLOP/s)"}
        roofline["frac"] = roofline["achieved"] / roofline["peak"]
    else:
        mma = 3.0 if dom == "pass_split" or (dom == "core_pass" and dt == "f32") else 1.0
        # 16-bit sketches wider than 128 columns run on CTA pairs (SORSVD_TC_PAIR=0: single CTAs)
        npad = (l + 15) // 16 * 16
        pair = dt in ("bf16", "f16") and 128 < npad <= 512 and os.environ.get("SORSVD_TC_PAIR", "1") != "0"
        kname = "tc_pair_kernel" if pair else "tc_gemm_kernel"
        roofline = {"bound": "hbm", "kernel": f"{kname} ({dom})", "achieved": achieved_gbs,
                    "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": achieved_gbs / pk["hbm_gbs"],
                    "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({pk_src})",
                    "algorithmic_bytes_per_launch": algo_bytes,
                    "tensor_view": {"mma_tflops": mma * algo_flops / (per_launch_ms * 1e-3) / 1e12,
                                    "peak_tflops": tc_peak[dt], "frac": mma * algo_flops / (per_launch_ms * 1e-3) / 1e12 / tc_peak[dt],
                                    "peak_source": "bf16 sustained x 0.5 (nominal TF32:BF16 ratio)" if dt in ("f32", "tf32") else "bf16 sustained"}}
    roofline.update({"launch_ms": per_launch_ms, "launches": dom_n,
                     "traffic": traffic_from_profiles(f"{dom}:{args.workload}")})
    out = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": dt, "data": "synthetic (seeded, built on the GPU)",
           "config": {"workload": f"{args.workload}: {w['desc']}", "m": m, "n": n, "k": k, "p": p, "q": q,
                      "flops_per_step": F, "l2": "inputs larger than L2 (A is %d MB)" % (m * n * esz // 2**20),
                      "parallelism": f"replicas x{world}"},
           "e2e": {"value": job_tflops(F, world, e_ms), "unit": "TFLOP/s", "ms_per_step": e_ms,
                   "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
           "gpu_launches": launches, "roofline": roofline, "clocks": clocks,
           "kernel_ms_per_step": {c: round(v[0] / prof_steps, 4) for c, v in all_prof.items()},
           "launches_per_step": {c: v[1] / prof_steps for c, v in all_prof.items()},
           "jacobi_sweeps": (info >> 8) & 0xFF,
           "wall_s_timed": t_wall}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, args.cpu_rows, args.cpu_cols)
    if not args.no_compare_precisions and dt in ("bf16", "f16"):
        out["precision_comparison"] = compare_precisions(w, A, At, k, p, q, max(3, min(args.steps, 5)))
    return out


def compare_precisions(w, A, At, k, p, q, steps):
    """Time and accuracy of the 16-bit path (with and without REFINE) and of
    the fp32 path on the same stored matrix: the fp32 run factors the 16-bit
    values widened exactly to fp32, so both approximate the same A.
    Accuracy: ||A - U S V^T||_F / sigma_{k+1}, sigma_{k+1} of the construction
    (the storage rounding moves it by ~2^-9 relative)."""
    import torch
    from paper_1804_00462_gb300 import native
    sig = sigma_of(w)
    s_k1 = float(sig[k]) if k < len(sig) else float("nan")
    A32t = At.float()                      # (n, m) row-major = A column-major, exact widening
    res = {}
    for name, mat, dt, fl in (("bf16", A, w["dtype"], 0), ("bf16_refine", A, w["dtype"], native.FLAG_REFINE),
                              ("f32", A32t.T, "f32", 0)):
        ws = native.alloc_workspace(w["m"], w["n"], k, p, dt, fl)
        out = native.run(mat, k, p, q, seed=0, dtype=dt, flags=fl, workspace=ws)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for i in range(steps):
            out = native.run(mat, k, p, q, seed=i, dtype=dt, flags=fl, workspace=ws)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        U, S, V = out
        # ||A - U S V^T||_F by row blocks of A (fp32 on the GPU)
        err2 = 0.0
        for c0 in range(0, w["n"], 2048):
            c1 = min(w["n"], c0 + 2048)
            blk = A32t[c0:c1].T - (U * S[None, :]) @ V[c0:c1].T
            err2 += float((blk.double() ** 2).sum())
        st, _ = native.get_status(ws)
        res[name] = {"ms": ms, "err_over_sigma_k1": err2 ** 0.5 / s_k1, "status": st}
        del ws
    res["speedup_bf16_vs_f32"] = res["f32"]["ms"] / res["bf16"]["ms"]
    res["speedup_bf16_refine_vs_f32"] = res["f32"]["ms"] / res["bf16_refine"]["ms"]
    # "equal relative error": the two errors within 1 % of each other
    ef = res["f32"]["err_over_sigma_k1"]
    for name in ("bf16", "bf16_refine"):
        res[name]["err_rel_to_f32"] = res[name]["err_over_sigma_k1"] / ef - 1.0
        res[name]["equal_error_within_1pct"] = abs(res[name]["err_over_sigma_k1"] / ef - 1.0) <= 0.01
    res["note"] = ("same stored matrix; err = ||A - U S V^T||_F / sigma_{k+1}; the Eckart-Young floor "
                   "is ||sigma_{k+1:}||_2 / sigma_{k+1}")
    res["eckart_young_floor"] = float((sig[k:] ** 2).sum() ** 0.5 / s_k1)
    return res


def _timed(args, world, fn, stream):
    """W warm-up calls, then K timed calls between CUDA events (max over ranks)."""
    import torch
    import torch.distributed as dist
    for i in range(args.warmup):
        fn(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        for i in range(args.steps):
            fn(1000 + i)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world, "cuda")
    return ms, clk.summary()


def run_batched(args, w, rank, world, local_rank):
    """Batched SOR-SVD: one step = the whole 512-problem batch (graph replay)."""
    import torch
    from paper_1804_00462_gb300 import inputs, native
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    sizes = inputs.batched_sizes(w["batch"], seed=0)
    As = [inputs.batched_matrix_torch(m, n, seed=1000 * (rank + 1) + b, device=dev,
                                      dtype=torch.float32) for b, (m, n, k) in enumerate(sizes)]
    ks = [k for _, _, k in sizes]
    plan = native.BatchedPlan(As, ks, w["p"], w["q"], seeds=list(range(len(sizes))), dtype=w["dtype"],
                              use_graph=True)
    stream = torch.cuda.current_stream()
    lc0 = native.launch_count()
    ms, clocks = _timed(args, world, lambda i: plan.launch(), stream)
    launches = (native.launch_count() - lc0) // (args.steps + args.warmup) * args.steps
    st = plan.status()
    if any(st):
        raise RuntimeError(f"device status: {[native.status_string(c) for c in st if c][:3]}")
    F = sum(flops(m, n, k, w["p"], w["q"]) for m, n, k in sizes)
    value = job_tflops(F, world, ms)
    # end to end: pinned host matrices -> device, solve, U S V -> host
    hostA = [a.T.contiguous().cpu().pin_memory() for a in As]
    hU = [torch.empty(u.shape[1], u.shape[0], pin_memory=True) for u in plan.U]
    hV = [torch.empty(v.shape[1], v.shape[0], pin_memory=True) for v in plan.V]
    hS = [torch.empty(s.shape, pin_memory=True) for s in plan.S]

    def e2e(i):
        for a, h in zip(As, hostA):
            a.T.copy_(h, non_blocking=True)
        plan.launch()
        for u, h in zip(plan.U, hU):
            h.copy_(u.T, non_blocking=True)
        for v, h in zip(plan.V, hV):
            h.copy_(v.T, non_blocking=True)
        for s_, h in zip(plan.S, hS):
            h.copy_(s_, non_blocking=True)

    eargs = argparse.Namespace(warmup=1, steps=max(3, min(args.steps, 5)))
    e_ms, _ = _timed(eargs, world, e2e, stream)
    h2d = sum(a.numel() * 4 for a in As)
    d2h = sum(u.numel() * 4 + v.numel() * 4 + s_.numel() * 4 for u, v, s_ in zip(plan.U, plan.V, plan.S))
    total_bytes = sum(m * n * 4 for m, n, _ in sizes)
    tiles = plan.tiles
    plan.close()
    return {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded, built on the GPU)",
            "config": {"workload": f"{args.workload}: {w['desc']}", "batch": len(sizes),
                       "autotuned_tiles": tiles, "flops_per_step": F,
                       "a_bytes": total_bytes, "l2": "inputs larger than L2 (%d MB of A)" % (total_bytes // 2**20),
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": job_tflops(F, world, e_ms), "unit": "TFLOP/s", "ms_per_step": e_ms,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches), "clocks": clocks,
            "roofline": {"bound": "hbm", "kernel": "whole batch (all stages)",
                         "achieved": (2 * w["q"] + 3) * total_bytes / (ms * 1e-3) / 1e9,
                         "peak": peaks()[0]["hbm_gbs"], "unit": "GB/s",
                         "frac": (2 * w["q"] + 3) * total_bytes / (ms * 1e-3) / 1e9 / peaks()[0]["hbm_gbs"],
                         "note": "algorithmic bytes = (2q+3) reads of every A over the whole step",
                         "traffic": None}}


def run_rpca(args, w, rank, world, local_rank):
    """RPCA: one step = 8 problems solved to tol (synchronous loop)."""
    import numpy as np
    import torch
    from paper_1804_00462_gb300 import inputs, native
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    Xs = []
    for b in range(w["batch"]):
        X, _, _ = inputs.rpca_problem(m=w["m"], n=w["n"], rank=w["rank"], seed=100 * (rank + 1) + b)
        Xs.append(torch.from_numpy(np.ascontiguousarray(X.T.astype(np.float32))).to(dev).T)
    ws = torch.empty(native.rpca_workspace_size(Xs, w["k"], w["p"], dtype=w["dtype"]), dtype=torch.uint8,
                     device=dev)
    info = {}

    def step(i):
        Ls, Ss, its, xis, _ = native.rpca(Xs, w["k"], w["p"], w["q"], seeds=[i * 8 + b for b in range(len(Xs))],
                                          dtype=w["dtype"], workspace=ws)
        info["its"], info["xis"] = its, xis

    lc0 = native.launch_count()
    stream = torch.cuda.current_stream()
    ms, clocks = _timed(args, world, step, stream)
    launches = (native.launch_count() - lc0) // (args.steps + args.warmup) * args.steps
    sweeps = sum(info["its"])
    return {"metric": "RPCA time to tolerance (8 problems)", "value": ms, "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded, built on the host)",
            "config": {"workload": f"{args.workload}: {w['desc']}", "iterations": info["its"],
                       "final_xi": info["xis"], "l2": "each X is 40.5 MB; 8 problems x (X, S, Y, G) exceed L2",
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": ms, "unit": "ms", "ms_per_step": ms, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 16 * w["batch"] * sweeps // max(len(info["its"]), 1),
                    "note": "the loop is host-driven: the per-iteration residual read-back is inside the timing"},
            "gpu_launches": int(launches), "clocks": clocks, "roofline": None}


def oracle_sample(w, rows, cols):
    """The workload's recipe at rows x cols (the same spectrum, cut to the
    sample's rank), stored in the workload's dtype and widened exactly."""
    import numpy as np
    from paper_1804_00462_gb300 import inputs
    m_s, n_s = min(rows, w["m"]), min(cols or w["n"], w["n"])
    r = min(w["width"], m_s, n_s)
    A64, _, _, _ = inputs.noisy_poly(m_s, n_s, r, w["noise"], seed=0) if w["spectrum"] == "poly1" \
        else inputs.spectral(m_s, n_s, sigma_of(w)[:r], 0)
    _, exact = inputs.to_storage(A64, w["dtype"])
    return np.ascontiguousarray(exact), m_s, n_s


def cpu_baseline(w, rows, cols):
    """The binary64 oracle timed on the host on a sample of the workload."""
    import oracle
    exact, m_s, n_s = oracle_sample(w, rows, cols)
    t = time.perf_counter()
    oracle.sorsvd(exact, w["k"], w["p"], w["q"], 0, omega_dtype=w["dtype"])
    t = time.perf_counter() - t
    F = flops(m_s, n_s, w["k"], w["p"], w["q"])
    return {"value": F / t / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"one solve of the same recipe at {m_s}x{n_s} (of {w['m']}x{w['n']}), "
                      f"k={w['k']}, p={w['p']}, q={w['q']}; numpy BLAS threads",
            "seconds": t}


def run_reference(args, w, rank, world):
    """The oracle (binary64, host cores) as the reference arm."""
    if rank != 0:
        return None
    import oracle
    exact, m_s, n_s = oracle_sample(w, args.cpu_rows, args.cpu_cols)
    for i in range(args.warmup):
        oracle.sorsvd(exact, w["k"], w["p"], w["q"], i, omega_dtype=w["dtype"])
    t = time.perf_counter()
    for i in range(args.steps):
        oracle.sorsvd(exact, w["k"], w["p"], w["q"], 1000 + i, omega_dtype=w["dtype"])
    t = (time.perf_counter() - t) / args.steps
    F = flops(m_s, n_s, w["k"], w["p"], w["q"])
    v = F / t / 1e12
    sample = (f"each step one oracle solve of the same recipe at {m_s}x{n_s} (of {w['m']}x{w['n']}), "
              f"k={w['k']}, p={w['p']}, q={w['q']}")
    return {"metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded, built on the host)",
            "config": {"workload": f"{args.workload}: {w['desc']}", "m": w["m"], "n": w["n"], "k": w["k"],
                       "p": w["p"], "q": w["q"], "sample_rows": m_s, "sample_cols": n_s},
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=tuple(WORKLOADS), default="cfg3")
    ap.add_argument("--cpu-rows", type=int, default=None,
                    help="rows of the oracle's sample (default: per workload, a few seconds of CPU work)")
    ap.add_argument("--cpu-cols", type=int, default=None, help="columns of the oracle's sample")
    ap.add_argument("--shrink", type=int, default=1,
                    help="single-matrix workloads: divide m and n by this factor (a smaller case of the same "
                         "recipe for profiler captures; not a bench line of the workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare-precisions", action="store_true",
                    help="16-bit workloads: skip the BF16 / BF16+REFINE / FP32 comparison on the same matrix")
    args = ap.parse_args()
    samp = CPU_SAMPLE.get((args.workload, args.impl), CPU_SAMPLE.get(args.workload, (20000, None)))
    if args.cpu_rows is None:
        args.cpu_rows = samp[0]
    if args.cpu_cols is None:
        args.cpu_cols = samp[1]
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.gpus != world and rank == 0:
        # one rank per GPU: --gpus N is launched by torchrun with N ranks;
        # the line reports the ranks that actually ran
        print(f"bench.py: --gpus {args.gpus} but {world} rank(s) running; n_gpus reports {world}",
              file=sys.stderr, flush=True)
    w = dict(WORKLOADS[args.workload])
    if args.shrink > 1 and "m" in w and args.workload not in ("cfg4", "cfg5"):
        w["m"] //= args.shrink
        w["n"] //= args.shrink
        w["desc"] = f"{w['desc']} [rows and columns divided by {args.shrink}: {w['m']}x{w['n']}]"
    if args.impl == "reference" and args.workload in ("cfg4", "cfg5"):
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the oracle on the "
                              "single-matrix workloads (cfg1-cfg3) only"}), flush=True)
        return
    if args.impl == "reference":
        out = run_reference(args, w, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if args.workload == "cfg4":
        out = run_batched(args, w, rank, world, local_rank)
    elif args.workload == "cfg5":
        out = run_rpca(args, w, rank, world, local_rank)
    else:
        out = run_ours(args, w, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
