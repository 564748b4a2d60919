"""Benchmark of the batched block-diagonal least-squares solve on GB300.

Workload (default): 1,000,000 independent blocks, rows ~ U{2..16}, cols ~ U{1..min(rows,6)},
N(0,1) entries, one right-hand side per block, FP32 Householder QR with extended-precision
refinement (adaptive: each block stops when its correction is below 1e-6 of its solution,
at most 2 steps).  One "solve" = factor + Q^T b + back-substitution + refinement of all
1,000,000 blocks (one kernel launch).  The relative error of the solution against the FP64
oracle is measured on every block in the same run; plain FP32 (no refinement) is
timed beside it for comparison.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank solves its own 1,000,000 blocks
(independent problems, no collective on the data path: weak scaling); the timing is the
max over ranks.  `--impl reference` times the CPU FP64 oracle on a bounded sample of the
same workload (the paper's own Eigen code is not available).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LM-step QR solves/s and HBM-roofline % at rel err ≤1e-5 vs FP64 oracle"
UNIT = "solves/s"
K_BLOCKS = 1_000_000
WORKLOAD = "batched block-diagonal QR solve: 1,000,000 blocks n~U{2..16}, m~U{1..min(n,6)}, FP32-refined"
KERNEL = "block_task_kernel + block_task_refine_kernel (one solve)"
KERNEL_SRCS = [os.path.join(ROOT, "paper_1802_03773_gb300", "csrc", f)
               for f in ("block_tasks.cuh", "block_tasks.cu", "block_tasks_f32sel.cu", "block_tasks_f32selw.cu",
                         "block_tasks_refine.cu", "device_util.cuh", "internal.h")]


def workload_config(args):
    """The workload as both arms report it (identical dictionaries)."""
    return {"workload": WORKLOAD, "blocks_per_gpu": K_BLOCKS, "precision": args.precision,
            "refine_steps": args.refine_steps if args.precision == "fp32_refined" else 0,
            "l2": "inputs 2 x 158 MB alternated between steps (each larger than the 129 MB L2)",
            "parallelism": "independent blocks, one replica per GPU, no collective"}


def dist_env():
    from paper_1802_03773_gb300.replicas import dist_env as env
    return env()


def algorithmic_bytes(d, elem=4, with_qtb=False):
    """Bytes the fused solve must move: read J, b; write factor, tau, p (and Q^T b)."""
    nm = int(d["val_off"][-1])
    n = int(d["row_off"][-1])
    m = int(d["col_off"][-1])
    return elem * (2 * nm + n + 2 * m + (n if with_qtb else 0))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def recorded_traffic(mapping=None):
    """DRAM bytes of one solve (the launches of its kernels) under the given block mapping (the
    autotuner's text form) from the committed ncu summary, if it was taken on the current kernel
    source and that mapping (else None)."""
    p = os.path.join(ROOT, "profiles", "block_task_kernel_1m_blocks.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    sha = hashlib.sha256()
    for f in KERNEL_SRCS:
        sha.update(open(f, "rb").read())
    h = sha.hexdigest()
    if rec.get("kernel_source_sha256") != h:
        return None
    v = rec.get("dram_bytes_per_launch", {}).get(mapping)
    return sum(v.values()) if isinstance(v, dict) else None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
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
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def cpu_oracle_sample(d, seconds):
    """Time the FP64 oracle (per-block Householder QR solve) on the first blocks of the workload."""
    from oracle import householder as hh
    t0 = time.perf_counter()
    k = 0
    while True:
        n, m = int(d["n"][k]), int(d["m"][k])
        v0, r0 = int(d["val_off"][k]), int(d["row_off"][k])
        A = np.asarray(d["vals"][v0:v0 + n * m], dtype=np.float64).reshape(m, n).T
        b = np.asarray(d["b"][r0:r0 + n], dtype=np.float64)
        hh.lstsq(A, b)
        k += 1
        el = time.perf_counter() - t0
        if el >= seconds or k >= d["K"]:
            break
    return k, el


def every_block_error(d, p):
    """Error of p against the oracle's FP64 solution of every block (the per-block Householder
    solve taken over stacks of one shape): aggregate, worst block, blocks above 1e-5."""
    from oracle import householder as hh
    n = d["n"].astype(np.int64)
    m = d["m"].astype(np.int64)
    key = n * 16 + m
    err = np.zeros(d["K"])
    num = den = 0.0
    for k in np.unique(key):
        sel = np.nonzero(key == k)[0]
        nn, mm = int(n[sel[0]]), int(m[sel[0]])
        vo = d["val_off"][sel][:, None] + np.arange(nn * mm)[None, :]
        A = np.asarray(d["vals"], dtype=np.float64)[vo].reshape(-1, mm, nn).transpose(0, 2, 1)
        ro = d["row_off"][sel][:, None] + np.arange(nn)[None, :]
        co = d["col_off"][sel][:, None] + np.arange(mm)[None, :]
        x = hh.lstsq_stack(A, np.asarray(d["b"], dtype=np.float64)[ro])
        e = np.asarray(p, dtype=np.float64)[co] - x
        num += float((e * e).sum())
        den += float((x * x).sum())
        err[sel] = np.linalg.norm(e, axis=1) / np.linalg.norm(x, axis=1)
    return {"rel_err": (num / den) ** 0.5, "max_block_rel_err": float(err.max()),
            "blocks_above_1e-5": int((err > 1e-5).sum()), "blocks_checked": int(d["K"]),
            "oracle": "per-block Householder QR in float64, every block"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from workloads import batched_blocks
    d = batched_blocks(K=K_BLOCKS)
    per_step = float(os.environ.get("QRKIT_REF_STEP_SECONDS", "4"))
    for _ in range(args.warmup):
        cpu_oracle_sample(d, min(per_step, 1.0))
    blocks = 0
    el = 0.0
    for _ in range(args.steps):
        k, t = cpu_oracle_sample(d, per_step)
        blocks += k
        el += t
    value = blocks / el / K_BLOCKS
    cores = 1
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * el / args.steps, "blocks_per_step": blocks / args.steps,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{blocks} blocks of the 1,000,000-block workload in {args.steps} "
                                       f"steps of ~{per_step:.0f} s, per-block Householder QR solve "
                                       "(numpy, float64), extrapolated to whole 1,000,000-block solves"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _time(stream, fn, reps, warm=2):
    """Average milliseconds of fn() over reps runs (CUDA events on the launching stream)."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(warm):
            fn()
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        stream.synchronize()
    return e0.elapsed_time(e1) / reps


def _curvefit_batch(ctx, specs, dev, stream):
    """Curve-fit problems with their data synthesised on the GPU: data = curve(t_true) + noise,
    the curve evaluated by the library's own model (qrkit_lm_residual with zero data)."""
    import torch
    from workloads import curvefit_problem
    draws = [curvefit_problem(npoints=n, Kc=kc, seed_offset=sd) for n, kc, sd in specs]
    npts = [dr["npoints"] for dr in draws]
    kcs = [dr["Kc"] for dr in draws]
    xt = np.concatenate([dr["t_true"] for dr in draws] + [dr["P_true"].reshape(-1) for dr in draws])
    x0 = np.concatenate([dr["t_true"] + dr["dt"] for dr in draws] +
                        [(dr["P_true"] + dr["dP"]).reshape(-1) for dr in draws])
    noise = np.concatenate([dr["noise"] for dr in draws]).reshape(-1)
    with torch.cuda.stream(stream):
        zero = torch.zeros(2 * sum(npts), dtype=torch.float64, device=dev)
        ctx.lm_plan(npts, kcs, zero)
        f = torch.empty_like(zero)
        ctx.lm_residual(torch.from_numpy(xt).to(dev), f)
        data = (f + torch.from_numpy(noise).to(dev)).contiguous()
        stream.synchronize()
        ctx.lm_plan(npts, kcs, data)
        x = torch.from_numpy(x0).to(dev)
    return x, x0, data, npts, kcs


def _curvefit_problems(specs, dev, stream):
    """Per-problem host arrays (data (P, 2), x0 = [t | control points]) of curve-fit problems,
    the data synthesised on the GPU by the library's own model."""
    from paper_1802_03773_gb300 import Context
    ctx = Context(dev.index, stream=stream, precision="fp64")
    _, x0, data, npts, kcs = _curvefit_batch(ctx, specs, dev, stream)
    dh = data.cpu().numpy().reshape(-1, 2)
    ctx.close()
    NP = sum(npts)
    out, p, c = [], 0, NP
    for n, kc in zip(npts, kcs):
        out.append((dh[p:p + n], np.concatenate([x0[p:p + n], x0[c:c + 2 * kc]])))
        p += n
        c += 2 * kc
    return out


def _convergence(h, times, target, iters):
    """Problems whose best cost reaches target, iterations and wall-clock latency to get there."""
    from paper_1802_03773_gb300 import learned
    it = learned.iterations_to(h, target)
    ok = np.isfinite(it)
    r = {"reached": int(ok.sum()), "of": int(it.size),
         "iterations_mean_all": float(np.where(ok, it, iters + 1).mean())}
    if ok.any():
        its = it[ok].astype(int)
        lat = times[its - 1]
        r.update({"iterations_p50": float(np.percentile(its, 50)), "iterations_p99": float(np.percentile(its, 99)),
                  "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99))})
    return r


def _curvefit_cond(dev, stream):
    """cond(J) of a scaled replica of the curve fit (2,000 points, 64 control points) at its start
    point, from the singular values of the dense Jacobian the library linearises (numpy SVD), and
    of the damped [J; lambda^(1/2) D] over the lambda sweep."""
    import torch
    from paper_1802_03773_gb300 import Context
    ctx = Context(dev.index, stream=stream, precision="fp64")
    x, x0, data, npts, kcs = _curvefit_batch(ctx, [(2000, 64, 0)], dev, stream)
    NP, s = npts[0], 2 * kcs[0]
    with torch.cuda.stream(stream):
        Jl = torch.empty(2 * NP, dtype=torch.float64, device=dev)
        Sl = torch.empty(16 * NP, dtype=torch.float64, device=dev)
        st = torch.empty(NP, dtype=torch.int32, device=dev)
        ctx.lm_linearize(torch.from_numpy(x0).to(dev), Jl, Sl, None, st)
        stream.synchronize()
    ctx.close()
    Jb, Sb, stt = Jl.cpu().numpy().reshape(NP, 2), Sl.cpu().numpy().reshape(NP, 8, 2), st.cpu().numpy()
    A = np.zeros((2 * NP, NP + s))
    for i in range(NP):
        A[2 * i:2 * i + 2, i] = Jb[i]
        for t in range(8):
            if stt[i] + t < s:
                A[2 * i:2 * i + 2, NP + stt[i] + t] = Sb[i, t]
    sv = np.linalg.svd(A, compute_uv=False)
    D = np.sqrt((A * A).sum(axis=0))
    D[D == 0] = 1.0
    damped = {}
    for lam in (1e-6, 1e-3, 1.0, 1e2):
        sd = np.linalg.svd(np.vstack([A, np.sqrt(lam) * np.diag(D)]), compute_uv=False)
        damped[f"{lam:g}"] = float(sd[0] / sd[-1])
    return {"points": NP, "control_points": kcs[0], "cond_J": float(sv[0] / sv[-1]), "cond_damped": damped}


def other_workloads(dev, stream, only=None):
    """The remaining configurations, each timed briefly (CUDA events, after warm-up); `only`
    restricts the run to the workloads whose key starts with it."""
    import torch
    from paper_1802_03773_gb300 import Context, qrkit
    from workloads import banded_batch_shapes, banded_problem, block_angular_dense
    out = {}
    peaks, peak_kind = measured_peaks()
    want = lambda key: only is None or key.startswith(only) or only.startswith(key)
    if want("peaks_probe"):
        # the rates no library measures: FMA throughput of the CUDA cores and the dense TF32 rate
        # of the tensor cores, by the library's own probe kernels
        out["peaks_probe"] = {"unit": "TFLOP/s",
                              "fp32_fma": qrkit.peak_probe(dev.index, "fp32"),
                              "fp64_fma": qrkit.peak_probe(dev.index, "fp64"),
                              "tf32_tensor_dense": qrkit.peak_probe(dev.index, "tf32")}
    if want("more_1m"):
        # Moré's two factorizations on the 1M-block workload: stage 1 once (undamped fused QR, its
        # Q^T b kept), then stage 2 per damping value ([R_i; lambda^(1/2) D_i] per block)
        from workloads import batched_blocks
        res = {}
        for prec, dt in (("fp32", np.float32), ("fp64", np.float64)):
            d = batched_blocks(K=K_BLOCKS, dtype=dt)
            ctx = Context(dev.index, stream=stream, precision=prec)
            ctx.plan_blocks(d["n"], d["m"])
            J = torch.from_numpy(d["vals"]).to(dev)
            b = torch.from_numpy(d["b"]).to(dev)
            p1 = torch.empty(int(d["col_off"][-1]), dtype=J.dtype, device=dev)
            q = torch.empty(int(d["row_off"][-1]), dtype=J.dtype, device=dev)
            torch.cuda.synchronize()
            t1 = _time(stream, lambda: ctx.factor_solve(J, b, p1, q, refine_steps=0), 5)
            t2 = _time(stream, lambda: ctx.more_solve(q, p1, None, 1e-2), 10)
            ctx.sync_status()
            # the trust-region lambda for a radius a tenth of the undamped step's scaled length
            # (host clock: the iteration reads three sums back per pass)
            ctx.more_solve(q, p1, None, 0.0)
            gn = float(torch.linalg.vector_norm(p1.double()).item())
            ctx.more_trust_region(q, p1, 0.1 * gn)   # warm
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            reps = 5
            for _ in range(reps):
                lam_tr, it_tr = ctx.more_trust_region(q, p1, 0.1 * gn)
            t_tr = (time.perf_counter() - t0) / reps * 1e3
            ctx.sync_status()
            res[prec] = {"ms_stage1_factor_qtb_solve": t1, "ms_stage2_per_lambda": t2,
                         "lambda_trials_per_s": 1000.0 / t2,
                         "trust_region": {"radius": "0.1 ||p_GN||_2, inside the undamped step's scaled length ||D p_GN||",
                                          "ms": t_tr, "passes": it_tr + 1, "lambda": lam_tr}}
            ctx.close()
            del J, b, p1, q
        out["more_two_step_1m_blocks"] = {
            "workload": "1,000,000 blocks as the headline; stage 2 with D = column norms, lambda 1e-2", **res}
    if want("dense_hcat_batch"):
        # the dense horizontal concatenation over 4096 seeds: independent FP64 solves spread over
        # 32 streams (one context each), eager launches
        nstreams, nseeds = 32, 4096
        ctxs, data = [], []
        streams = [torch.cuda.Stream(dev) for _ in range(nstreams)]
        for k in range(nstreams):
            c = Context(dev.index, stream=streams[k], precision="fp64")
            c.plan_blocks(np.full(200, 4), np.full(200, 2), qrkit.COUPLED_DENSE, shared_cols=30)
            ctxs.append(c)
        for sd in range(nseeds):
            d = block_angular_dense(seed_offset=1000 + sd)
            data.append((torch.from_numpy(np.ascontiguousarray(d["blocks"].transpose(0, 2, 1).reshape(-1))).to(dev),
                         torch.from_numpy(np.asarray(d["S"]).T.reshape(-1).copy()).to(dev),
                         torch.from_numpy(np.asarray(d["b"])).to(dev),
                         torch.empty(430, dtype=torch.float64, device=dev)))
        torch.cuda.synchronize()

        def run_all():
            for sd in range(nseeds):
                k = sd % nstreams
                J, S, b, pp = data[sd]
                with torch.cuda.stream(streams[k]):
                    ctxs[k].factor(J, S, None, 1e-2)
                    ctxs[k].solve(b, pp, refine_steps=0)
        run_all()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run_all()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        for c in ctxs:
            c.sync_status()
            c.close()
        out["dense_hcat_200x(4x2)_s30_fp64_batch_4096"] = {
            "workload": "4096 seeds of J = [blkdiag(200 blocks 4x2) | S 800x30], lambda 1e-2, D = norms, FP64, "
                        "32 streams", "value": nseeds / el, "unit": "solves/s", "ms_total": 1000.0 * el}
        del data
    if want("dense_hcat_200x"):
        # dense horizontal concatenation, one LM-step solve in FP64
        d = block_angular_dense()
        K, n, m, s = d["K"], d["n"], d["m"], d["s"]
        ctx = Context(dev.index, stream=stream, precision="fp64")
        ctx.plan_blocks(np.full(K, n), np.full(K, m), qrkit.COUPLED_DENSE, shared_cols=s)
        J = torch.from_numpy(np.concatenate([d["blocks"][i].T.reshape(-1) for i in range(K)])).to(dev)
        S = torch.from_numpy(np.asarray(d["S"]).T.reshape(-1).copy()).to(dev)
        b = torch.from_numpy(np.asarray(d["b"])).to(dev)
        pd = torch.empty(K * m + s, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()   # inputs copied on the default stream before the context's stream reads them

        def dense_solve():
            ctx.factor(J, S, None, d["lam"])
            ctx.solve(b, pd, refine_steps=0)
        ms = _time(stream, dense_solve, 100)
        ctx.sync_status()
        l0 = ctx.launch_count
        with torch.cuda.stream(stream):
            dense_solve()
        launches = ctx.launch_count - l0
        # the same solve captured once in a CUDA graph and replayed (this small solve is bound by
        # the launches of its ~60 short kernels)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            dense_solve()
        ms_graph = _time(stream, graph.replay, 200)
        ctx.sync_status()
        out["dense_hcat_200x(4x2)_s30_fp64"] = {
            "workload": "J = [blkdiag(200 blocks 4x2) | S 800x30], columns scaled 1..1e3, lambda 1e-2, D = norms",
            "value": 1000.0 / ms_graph, "unit": "solves/s", "us_per_solve_graph": 1000.0 * ms_graph,
            "us_per_solve_eager": 1000.0 * ms, "launches_per_solve": launches}
        ctx.close()
    if want("dense_hcat_100k"):
        # dense hcat at the tensor-core size: 100,000 blocks 4x2, S 400,000 x 128, FP32-refined
        d = block_angular_dense(K=100_000, n=4, m=2, s=128, scale_decades=2.0, dtype=np.float32)
        K, n, m, s = d["K"], d["n"], d["m"], d["s"]
        ctx = Context(dev.index, stream=stream, precision="fp32_refined")
        ctx.plan_blocks(np.full(K, n), np.full(K, m), qrkit.COUPLED_DENSE, shared_cols=s)
        J = torch.from_numpy(np.concatenate([d["blocks"][i].T.reshape(-1) for i in range(K)])).to(dev)
        S = torch.from_numpy(np.asarray(d["S"]).T.reshape(-1).copy()).to(dev)
        b = torch.from_numpy(np.asarray(d["b"])).to(dev)
        pl = torch.empty(K * m + s, dtype=torch.float32, device=dev)
        torch.cuda.synchronize()
        tf = _time(stream, lambda: ctx.factor(J, S, None, d["lam"]), 5)
        ts = _time(stream, lambda: ctx.solve(b, pl, refine_steps=1), 5)
        ctx.sync_status()
        Mred = K * n + s
        flops = 2.0 * Mred * s * s   # useful flops of the reduced block's Householder QR (leading term)
        out["dense_hcat_100k_blocks_s128_fp32_refined"] = {
            "workload": "J = [blkdiag(100,000 blocks 4x2) | S 400,000 x 128], lambda 1e-2, D = norms; "
                        "reduced block by 4 column panels of 32 (TSQR each, tcgen05 3xTF32 updates)",
            "ms_factor": tf, "ms_solve_refined_1": ts, "value": 1000.0 / (tf + ts), "unit": "solves/s",
            "reduced_block_tflops_useful": flops / (tf * 1e-3) / 1e12}
        ctx.close()
        del J, S, b
    if want("dense_wide") or only == "dense_wide_small":
        # wider reduced blocks: s = 256 and 512 by 32-column panels, each a TSQR
        # whose tiles' Q^T reaches the later columns through the tensor cores (tcgen05, 3xTF32).
        # "dense_wide_small" (20,000 blocks, s = 512, asked for by name only) is the profiling case.
        small = only == "dense_wide_small"
        for s in ((512,) if small else (256, 512)):
            K = 20_000 if small else 100_000
            d = block_angular_dense(K=K, n=4, m=2, s=s, scale_decades=2.0, dtype=np.float32)
            n, m = d["n"], d["m"]
            ctx = Context(dev.index, stream=stream, precision="fp32_refined")
            ctx.plan_blocks(np.full(K, n), np.full(K, m), qrkit.COUPLED_DENSE, shared_cols=s)
            J = torch.from_numpy(np.concatenate([d["blocks"][i].T.reshape(-1) for i in range(K)])).to(dev)
            S = torch.from_numpy(np.asarray(d["S"]).T.reshape(-1).copy()).to(dev)
            b = torch.from_numpy(np.asarray(d["b"])).to(dev)
            pl = torch.empty(K * m + s, dtype=torch.float32, device=dev)
            del d
            torch.cuda.synchronize()
            tf = _time(stream, lambda: ctx.factor(J, S, None, 1e-2), 2 if small else 5)
            ts = _time(stream, lambda: ctx.solve(b, pl, refine_steps=1), 2 if small else 5)
            ctx.sync_status()
            l0 = ctx.launch_count
            with torch.cuda.stream(stream):
                ctx.factor(J, S, None, 1e-2)
            launches = ctx.launch_count - l0
            Mred = K * n + s
            flops = 2.0 * Mred * s * s - 2.0 * s ** 3 / 3.0   # Householder QR of the Mred x s reduced block
            out[f"dense_wide_{K // 1000}k_blocks_s{s}_fp32_refined"] = {
                "workload": f"J = [blkdiag({K:,} blocks 4x2) | S {K * n:,} x {s}], lambda 1e-2, D = norms; reduced "
                            f"block by {s // 32} column panels of 32 (TSQR each, tcgen05 3xTF32 updates)",
                "ms_factor": tf, "ms_solve_refined_1": ts, "value": 1000.0 / (tf + ts), "unit": "solves/s",
                "reduced_block_tflops_useful": flops / (tf * 1e-3) / 1e12, "launches_per_factor": launches}
            ctx.close()
            del J, S, b
            torch.cuda.empty_cache()
    if want("ba_"):
        # BA-shaped system (bundle adjustment, Sec. 6.2): 100,000 points, each seen by 2-6 of 14
        # cameras (9 parameters each, 126 columns padded to 128, a multiple of the panel width), damped
        from workloads import ba_system
        d = ba_system(P=100_000, C=14, s_pad=128, dtype=np.float32)
        K, s = d["K"], d["s"]
        ctx = Context(dev.index, stream=stream, precision="fp32_refined")
        ctx.plan_blocks(d["n"], np.full(K, 3), qrkit.COUPLED_DENSE, shared_cols=s)
        J = torch.from_numpy(np.concatenate([blk.T.reshape(-1) for blk in d["blocks"]])).to(dev)
        S = torch.from_numpy(np.asarray(d["S"]).T.reshape(-1).copy()).to(dev)
        b = torch.from_numpy(np.asarray(d["b"])).to(dev)
        pl = torch.empty(3 * K + s, dtype=torch.float32, device=dev)
        torch.cuda.synchronize()
        tf = _time(stream, lambda: ctx.factor(J, S, None, d["lam"]), 5)
        ts = _time(stream, lambda: ctx.solve(b, pl, refine_steps=1), 5)
        ctx.sync_status()
        rows = int(np.sum(d["n"]))
        out["ba_100k_points_14_cameras_fp32_refined"] = {
            "workload": f"BA-shaped: 100,000 points x 2-6 observations ({rows} rows) of 14 cameras "
                        f"(9 parameters each, S {rows} x 128 dense with the camera blocks), lambda 1e-3, D = norms",
            "ms_factor": tf, "ms_solve_refined_1": ts, "value": 1000.0 / (tf + ts), "unit": "solves/s"}
        ctx.close()
        del J, S, b, d
    if want("ellipse_fit"):
        # the surface fitting benchmark's shape: one LM-step system of an ellipse fit to N points
        # (N blocks 2x1 + 5 dense shared columns), N over the paper's sweep, FP64
        from workloads import ellipse_system
        per_n = {}
        for N in (500, 2000, 10_000, 100_000, 500_000):
            d = ellipse_system(N=N)
            ctx = Context(dev.index, stream=stream, precision="fp64")
            ctx.plan_blocks(np.full(N, 2), np.full(N, 1), qrkit.COUPLED_DENSE, shared_cols=5)
            J = torch.from_numpy(np.ascontiguousarray(d["blocks"].reshape(-1))).to(dev)
            S = torch.from_numpy(np.asarray(d["S"]).T.reshape(-1).copy()).to(dev)
            b = torch.from_numpy(np.asarray(d["b"])).to(dev)
            pe = torch.empty(N + 5, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()

            def ellipse_solve():
                ctx.factor(J, S, None, d["lam"])
                ctx.solve(b, pe, refine_steps=0)
            ms = _time(stream, ellipse_solve, 20)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                ellipse_solve()
            ms_graph = _time(stream, graph.replay, 50)
            ctx.sync_status()
            per_n[str(N)] = {"us_per_solve_eager": 1000.0 * ms, "us_per_solve_graph": 1000.0 * ms_graph}
            ctx.close()
            del graph, J, S, b, pe
        out["ellipse_fit_system_fp64"] = {
            "workload": "one LM-step system of an ellipse fit: blkdiag(N blocks 2x1) | S 2N x 5, lambda 1e-3, "
                        "D = norms, factor + solve, FP64; N = 500 .. 500,000",
            "value": 1e6 / per_n["500000"]["us_per_solve_graph"], "unit": "solves/s at N = 500,000",
            "per_n": per_n}
    if want("curvefit"):
        # curve fit, 200,000 points, 2048 control points: LM iterations and fixed-lambda solves
        cf = {}
        for prec in ("fp32_refined", "fp32", "fp64"):
            ctx = Context(dev.index, stream=stream, precision=prec)
            x, x0, data, npts, kcs = _curvefit_batch(ctx, [(200_000, 2048, 0)], dev, stream)
            st = ctx.lm_states(1e-3)
            ctx.lm_run(x, st, max_iter=2, ftol=0.0, refine_steps=1, use_graph=True)
            it = 10
            st = ctx.lm_states(1e-3)
            ms = _time(stream, lambda: ctx.lm_run(x, st, max_iter=it, ftol=0.0, refine_steps=1, use_graph=True), 1,
                       warm=0) / it
            cf[f"lm_iteration_{prec}"] = {"ms": ms, "iterations_per_s": 1000.0 / ms}
            if prec == "fp32_refined":
                # the linearised system at the start point, solved for several lambda by QR and by
                # the normal equations (Cholesky)
                NP = npts[0]
                with torch.cuda.stream(stream):
                    Jl = torch.empty(2 * NP, dtype=torch.float32, device=dev)
                    Sl = torch.empty(16 * NP, dtype=torch.float32, device=dev)
                    bl = torch.empty(2 * NP, dtype=torch.float32, device=dev)
                    stl = torch.empty(NP, dtype=torch.int32, device=dev)
                    xs = torch.from_numpy(x0).to(dev)
                    ctx.lm_linearize(xs, Jl, Sl, bl, stl)
                    stream.synchronize()
                    starts = stl.cpu().numpy()
                sctx = Context(dev.index, stream=stream, precision=prec)
                sctx.plan_blocks(np.full(NP, 2), np.full(NP, 1), qrkit.COUPLED_WINDOW, shared_cols=2 * kcs[0], window=8,
                                 window_start=starts)
                pq = torch.empty(NP + 2 * kcs[0], dtype=torch.float32, device=dev)
                # the FP64 solve of the same float-rounded system is the accuracy reference
                dctx = Context(dev.index, stream=stream, precision="fp64")
                dctx.plan_blocks(np.full(NP, 2), np.full(NP, 1), qrkit.COUPLED_WINDOW, shared_cols=2 * kcs[0],
                                 window=8, window_start=starts)
                Jd, Sd, bd = Jl.double(), Sl.double(), bl.double()
                pd = torch.empty(NP + 2 * kcs[0], dtype=torch.float64, device=dev)
                per_lam = {}
                for lam in (1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 1e-1, 1.0, 1e1, 1e2):
                    def qr():
                        sctx.factor(Jl, Sl, None, lam)
                        sctx.solve(bl, pq, refine_steps=1)
                    tq = _time(stream, qr, 5)
                    eq = pq.double()
                    tc = _time(stream, lambda: sctx.normal_solve(Jl, Sl, bl, pq, None, lam), 5)
                    ec = pq.double()

                    def f64():
                        dctx.factor(Jd, Sd, None, lam)
                        dctx.solve(bd, pd, refine_steps=0)
                    td = _time(stream, f64, 3)
                    stream.synchronize()
                    ref = pd.clone()
                    rel = lambda v: float(torch.linalg.norm(v - ref) / torch.linalg.norm(ref))
                    per_lam[f"{lam:g}"] = {"qr_fp32_refined_solves_per_s": 1000.0 / tq,
                                           "cholesky_fp32_solves_per_s": 1000.0 / tc,
                                           "qr_fp64_solves_per_s": 1000.0 / td,
                                           "rel_err_qr_fp32_refined": rel(eq), "rel_err_cholesky_fp32": rel(ec)}
                sctx.sync_status()
                dctx.sync_status()
                sctx.close()
                dctx.close()
                cf["fixed_lambda_solves"] = per_lam
                cf["fixed_lambda_note"] = ("relative errors against the FP64 QR solve of the same float-rounded "
                                           "system (the FP64 path matches the oracle to 1e-12 in the tests)")
                cf["cond_J_replica"] = _curvefit_cond(dev, stream)
            ctx.sync_status()
            ctx.close()
        out["curvefit_200k_points_2048_control_points"] = {
            "workload": "open uniform cubic B-spline, 200,000 points (2x1 blocks), 4096 shared columns in windows of 8",
            **cf}
    if want("curvefit_convergence"):
        # the same 200,000-point fit solved to convergence, FP32 QR with refinement against plain
        # FP64 QR on the same GPU: wall-clock time (one iteration per call, the state read back each
        # time) until the cost is within 1e-6 of the best FP64 cost
        runs = {}
        for prec in ("fp32_refined", "fp64"):
            ctx = Context(dev.index, stream=stream, precision=prec)
            x, x0, data, npts, kcs = _curvefit_batch(ctx, [(200_000, 2048, 0)], dev, stream)
            st = ctx.lm_states(1e-3)
            costs, times = [], []
            t0 = time.perf_counter()
            for it in range(120):
                ctx.lm_run(x, st, max_iter=1, ftol=0.0, refine_steps=1, use_graph=True)
                times.append(1000.0 * (time.perf_counter() - t0))
                costs.append(st[0].cost_new if st[0].accepted else st[0].cost)
            ctx.sync_status()
            runs[prec] = (np.minimum.accumulate(np.array(costs)), np.array(times))
            ctx.close()
        best = runs["fp64"][0][-1]
        res = {}
        for prec, (c, t) in runs.items():
            hit = np.nonzero(c <= best * (1.0 + 1e-6))[0]
            res[prec] = {"final_cost": float(c[-1]), "ms_per_iteration": float(t[-1] / len(t)),
                         "iterations_to_1e-6": int(hit[0] + 1) if hit.size else None,
                         "ms_to_1e-6": float(t[hit[0]]) if hit.size else None}
        out["curvefit_200k_convergence_fp32_refined_vs_fp64"] = {
            "workload": "200,000-point curve fit, 2048 control points, Nielsen damping, up to 120 iterations",
            "target": "cost <= (1 + 1e-6) x the best FP64 cost", **res}
    if want("banded_1e6"):
        # banded + vertical concatenation: one instance of 1,000,000 columns, 4,000,000 rows
        bp = banded_problem(n=1_000_000, rows_per_col=4, w=8, seed_offset=0)
        ctx = Context(dev.index, stream=stream, precision="fp32_refined")
        ctx.plan_banded([1_000_000], rows_per_col=4, window=8)
        Jb = torch.from_numpy(np.ascontiguousarray(bp["vals"].reshape(-1))).to(dev)
        bb = torch.from_numpy(bp["b"]).to(dev)
        xb = torch.empty(1_000_000, dtype=torch.float32, device=dev)
        torch.cuda.synchronize()
        t0 = _time(stream, lambda: ctx.factor_solve(Jb, bb, xb, None, lam=1e-3, refine_steps=0), 5)
        t2 = _time(stream, lambda: ctx.factor_solve(Jb, bb, xb, None, lam=1e-3, refine_steps=2), 5)
        ctx.sync_status()
        alg = 4 * (Jb.numel() + bb.numel() + xb.numel())
        out["banded_1e6_cols_4e6_rows"] = {
            "workload": "J 4,000,000 x 1,000,000, row i on columns floor(i/4)..+7, lambda 1e-3, D = norms",
            "value": 1000.0 / t2, "unit": "solves/s", "ms_refined_2": t2, "ms_no_refinement": t0,
            "roofline": {"bound": "hbm", "algorithmic_bytes": alg, "achieved": alg / (t0 * 1e-3) / 1e9,
                         "peak": peaks["hbm_gbs"], "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": alg / (t0 * 1e-3) / 1e9 / peaks["hbm_gbs"],
                         "note": "factor + solve without refinement; algorithmic bytes = read J and b, write x"}}
        ctx.close()
        del Jb, bb, xb
    if want("banded_batch"):
        # the batch of banded instances at full size: 4096 instances, n ~ U{1000..100000}, 4n rows
        # each (about 2e8 columns, 8e8 rows, 30 GB of J and b drawn on the device), parallel
        # solver, FP32 refined; timed eagerly and as one captured CUDA graph
        from workloads.device import banded_batch_device
        cols = banded_batch_shapes()
        t0 = time.perf_counter()
        db = banded_batch_device(cols, seed_offset=10, device=dev)
        ctx = Context(dev.index, stream=stream, precision="fp32_refined")
        ctx.plan_banded(list(cols), rows_per_col=4, window=8, solver=2)
        plan_s = time.perf_counter() - t0
        Jv, bv = db["vals"].reshape(-1), db["b"]
        xv = torch.empty(int(np.sum(cols)), dtype=torch.float32, device=dev)
        torch.cuda.synchronize()
        solve = lambda: ctx.factor_solve(Jv, bv, xv, None, lam=1e-3, refine_steps=2)
        tb = _time(stream, solve, 3)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            solve()
        tg = _time(stream, graph.replay, 3)
        ctx.sync_status()
        nb = 4 * (int(db["row0"][-1]) * 9 + int(np.sum(cols)))   # read J (w values) and b per row, write x
        out["banded_batch_4096_instances"] = {
            "workload": f"4096 banded instances, n ~ U{{1000..100000}} (total {int(np.sum(cols))} columns, "
                        f"{int(db['row0'][-1])} rows), lambda 1e-3, D = norms, 2 refinement steps",
            "value": 4096 * 1000.0 / tg, "unit": "instances/s", "ms_graph": tg, "ms_eager": tb,
            "plan_and_generate_s": plan_s,
            "hbm_frac_of_measured": nb / (tg * 1e-3) / 1e9 / peaks["hbm_gbs"],
            "note": "hbm fraction counts one read of J and b and one write of x per solve"}
        ctx.close()
        del db, Jv, bv, xv, graph
        torch.cuda.empty_cache()
    if want("batched_lm"):
        # batched LM: 1024 curve-fit problems, points ~ U{500..20000}, control points ~ U{16..256}
        g = np.random.default_rng(5)
        specs = [(int(g.integers(500, 20001)), int(g.integers(16, 257)), 100 + i) for i in range(1024)]
        ctx = Context(dev.index, stream=stream, precision="fp32_refined")
        x, x0, data, npts, kcs = _curvefit_batch(ctx, specs, dev, stream)
        st = ctx.lm_states(1e-3)
        ctx.lm_run(x, st, max_iter=2, ftol=0.0, refine_steps=1, use_graph=True)
        st = ctx.lm_states(1e-3)
        it = 5
        ms = _time(stream, lambda: ctx.lm_run(x, st, max_iter=it, ftol=0.0, refine_steps=1, use_graph=True), 1,
                   warm=0) / it
        ctx.sync_status()
        out["batched_lm_1024_curvefit_problems"] = {
            "workload": f"1024 problems, {sum(npts)} points in total, Nielsen damping, CUDA-graph iterations",
            "value": 1000.0 / ms, "unit": "LM iterations/s (all problems)", "ms_per_iteration": ms}
        ctx.close()
    if want("batched_lm_convergence"):
        # the same kind of batch solved towards convergence with Nielsen's rule and with the learned
        # damping policy (trained here on 128 smaller problems); the FP64 optimum of every problem
        # comes from FP64 LM polishing the better final point of the two runs
        from paper_1802_03773_gb300 import learned
        from workloads import mlp_init
        g = np.random.default_rng(7)
        specs = [(int(g.integers(500, 20001)), int(g.integers(16, 257)), 3000 + i) for i in range(1024)]
        batch = learned.Batch(_curvefit_problems(specs, dev, stream))
        tspecs = [(int(g.integers(500, 3001)), int(g.integers(16, 65)), 9000 + i) for i in range(128)]
        t0 = time.perf_counter()
        params, nsamples, _ = learned.train_policy(learned.Batch(_curvefit_problems(tspecs, dev, stream)),
                                                   mlp_init(7), device=dev.index)
        train_s = time.perf_counter() - t0
        iters = 150
        hn, _, tn, xn = learned.run(batch, iters=iters, with_times=True, device=dev.index)
        hm, _, tm, xm = learned.run(batch, iters=iters, params=params, with_times=True, device=dev.index)
        use_m = hm[-1] < hn[-1]
        xb = xn.copy()
        for k in np.nonzero(use_m)[0]:
            t_sl = slice(batch.p0[k], batch.p0[k + 1])
            c_sl = slice(batch.NP + batch.c0[k], batch.NP + batch.c0[k + 1])
            xb[t_sl], xb[c_sl] = xm[t_sl], xm[c_sl]
        h64, _ = learned.run(batch, iters=40, precision="fp64", x0=xb, device=dev.index)
        opt = np.minimum(h64[-1], np.minimum(hn[-1], hm[-1]))
        res = {"workload": f"1024 problems, {batch.NP} points, Kc ~ U{{16..256}}, FP32-refined, {iters} iterations",
               "policy_training_s": train_s, "training_samples": int(nsamples),
               "ms_per_iteration": {"nielsen": float(tn[-1] / iters), "mlp": float(tm[-1] / iters)}}
        for tol in (1e-6, 1e-3):
            res[f"within_{tol:g}_of_fp64_optimum"] = {
                "nielsen": _convergence(hn, tn, opt * (1.0 + tol), iters),
                "mlp": _convergence(hm, tm, opt * (1.0 + tol), iters)}
        # the two smallest problems, for the oracle's own FP64 LM in the CPU leg
        small = np.argsort([n for n, _, _ in specs])[:2]
        probs = _curvefit_problems([specs[k] for k in small], dev, stream)
        res["_oracle_check"] = [(probs[j][0], probs[j][1], float(opt[k])) for j, k in enumerate(small)]
        out["batched_lm_convergence_1024"] = res
    return out


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_1802_03773_gb300 import Context
    from workloads import batched_blocks

    d = batched_blocks(K=K_BLOCKS, seed_offset=rank)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    ctx = Context(local, stream=stream, precision=args.precision)
    ctx.plan_blocks(d["n"], d["m"])
    # two resident copies of the inputs, alternated between steps (each 158 MB > 129 MB L2)
    Js = [torch.from_numpy(d["vals"]).to(dev) for _ in range(2)]
    bs = [torch.from_numpy(d["b"]).to(dev) for _ in range(2)]
    ncols = int(d["col_off"][-1])
    p = torch.empty(ncols, device=dev, dtype=torch.float32)
    torch.cuda.synchronize()   # inputs copied on the default stream before the context's stream reads them
    refine = args.refine_steps

    # the block-to-warp mapping, chosen by the library's autotuner on these inputs (or given)
    if args.tuning:
        tuned = args.tuning.replace(",", " ")
        ctx.apply_tuning(tuned)
    else:
        tuned = ctx.autotune(Js[0], bs[0], p, refine_steps=refine)

    def step(i):
        ctx.factor_solve(Js[i & 1], bs[i & 1], p, None, refine_steps=refine)

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            step(i)
    ctx.sync_status()
    launches0 = ctx.launch_count
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.25)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        step(i)
        ev[i][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    kern_ms = [a.elapsed_time(b) for a, b in ev]
    launches = ctx.launch_count - launches0
    ctx.sync_status()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        from paper_1802_03773_gb300.replicas import max_over_ranks
        total_ms = max_over_ranks(total_ms, dev)

    # end-to-end through the public API with host buffers: every step copies its J and b from
    # pinned host memory and reads its p back, all inside the timed region; the copy of step
    # i + 1 runs on its own stream into the other of two device input sets while step i solves
    hJ = torch.from_numpy(d["vals"]).pin_memory()
    hb = torch.from_numpy(d["b"]).pin_memory()
    hps = [torch.empty(ncols, dtype=torch.float32).pin_memory() for _ in range(2)]
    ps = [p, torch.empty_like(p)]
    cs = torch.cuda.Stream(dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]

    def e2e_step(i):
        k = i & 1
        cs.wait_event(freed[k])          # the solve that last read input set k is done
        with torch.cuda.stream(cs):
            Js[k].copy_(hJ, non_blocking=True)
            bs[k].copy_(hb, non_blocking=True)
        copied[k].record(cs)
        stream.wait_event(copied[k])
        with torch.cuda.stream(stream):
            ctx.factor_solve(Js[k], bs[k], ps[k], None, refine_steps=refine)
            freed[k].record(stream)
            hps[k].copy_(ps[k], non_blocking=True)

    for i in range(3):
        e2e_step(i)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cs.wait_event(e0)
    for i in range(args.steps):
        e2e_step(i)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    ctx.sync_status()

    # the host link the inputs cross: copy engine and kernel zero-copy reads of pinned memory
    from paper_1802_03773_gb300 import qrkit as _qk
    cg, kg = _qk.host_link_probe(local, 1 << 30)
    link_bytes = hJ.numel() * 4 + hb.numel() * 4 + hps[0].numel() * 4
    link = {"copy_gbs": cg, "kernel_read_gbs": kg,
            "achieved_gbs": link_bytes / (e2e_ms * 1e-3) / 1e9,
            "frac_of_copy_rate": link_bytes / (e2e_ms * 1e-3) / 1e9 / cg,
            "note": "both directions' bytes per step over the time of a step; the copy rate is one direction"}

    p_host = p.cpu().numpy()
    # the other precision mode, timed the same way for a few steps
    refined = None
    if not args.no_refined:
        other = "fp32" if args.precision == "fp32_refined" else "fp32_refined"
        rctx = Context(local, stream=stream, precision=other)
        rctx.plan_blocks(d["n"], d["m"])
        # its own mapping: the headline's choice fits the headline's kernels, not these
        if args.tuning:
            rctx.apply_tuning(tuned)
        else:
            other_tuned = rctx.autotune(Js[0], bs[0], torch.empty_like(p), refine_steps=args.refine_steps)
        pr = torch.empty_like(p)
        with torch.cuda.stream(stream):
            for i in range(10):   # a fresh context: its buffers and kernels warmed like the headline's
                rctx.factor_solve(Js[i & 1], bs[i & 1], pr, None, refine_steps=args.refine_steps)
            stream.synchronize()
            r0 = torch.cuda.Event(enable_timing=True)
            r1 = torch.cuda.Event(enable_timing=True)
            nref = max(10, min(args.steps, 40))
            r0.record(stream)
            for i in range(nref):
                rctx.factor_solve(Js[i & 1], bs[i & 1], pr, None, refine_steps=args.refine_steps)
            r1.record(stream)
            stream.synchronize()
        rctx.sync_status()
        rms = r0.elapsed_time(r1) / nref
        pr_host = pr.cpu().numpy()
        refined = {"precision": other, "value": ws * 1000.0 / rms, "unit": UNIT, "ms_per_step": rms,
                   "autotuned": tuned if args.tuning else other_tuned,
                   "refine_steps": args.refine_steps if other == "fp32_refined" else 0}
        rctx.close()
    extra = None
    if rank == 0 and not args.no_workloads:
        extra = other_workloads(dev, stream)
    if rank != 0:
        ctx.close()
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    if args.no_cpu_baseline and extra:
        extra.get("batched_lm_convergence_1024", {}).pop("_oracle_check", None)
    ms_per_step = total_ms / args.steps
    value = ws * 1000.0 / ms_per_step
    peaks, peak_kind = measured_peaks()
    alg = algorithmic_bytes(d)
    kavg = sum(kern_ms) / len(kern_ms)
    achieved = alg / (kavg * 1e-3) / 1e9
    traffic = recorded_traffic(tuned)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args),
        "blocks_per_s": value * K_BLOCKS, "autotuned": tuned,
        "roofline": {"bound": "hbm", "kernel": KERNEL, "achieved": achieved,
                     "peak": peaks["hbm_gbs"], "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                     "algorithmic_bytes_per_launch": alg, "avg_launch_ms": kavg},
        "e2e": {"value": ws * 1000.0 / e2e_ms, "unit": UNIT,
                "h2d_bytes_per_step": int(hJ.numel() * 4 + hb.numel() * 4),
                "d2h_bytes_per_step": int(hps[0].numel() * 4),
                "overlap": "copy of step i + 1 on its own stream during the solve of step i",
                "host_link": link},
        "gpu_launches": launches,
        "clocks": clk,
        "accuracy": None,
        "other_precision": refined,
        "workloads": extra,
    }
    if ws == 1 and not args.no_cpu_baseline:
        # the oracle leg: its timing on a sample, and the error of this run's solutions on
        # sampled blocks against it
        secs = float(os.environ.get("QRKIT_CPU_BASELINE_SECONDS", "12"))
        k, el = cpu_oracle_sample(d, secs)
        line["cpu_baseline"] = {
            "value": k / el / K_BLOCKS, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {k} blocks of the workload ({el:.1f} s), per-block Householder QR "
                      "solve in numpy float64, extrapolated to whole 1,000,000-block solves"}
        line["accuracy"] = every_block_error(d, p_host)
        chk = (extra or {}).get("batched_lm_convergence_1024", {}).pop("_oracle_check", None)
        if chk:
            # the FP64 optimum of sampled problems from the oracle's own LM (Nielsen rule, FP64)
            from oracle import lm as olm
            rows = []
            for data_k, x0_k, opt_k in chk:
                t0 = time.perf_counter()
                stt = olm.lm_run(x0_k, data_k, lam0=1e-3, max_iter=150, ftol=1e-14)
                rows.append({"points": int(data_k.shape[0]), "oracle_cost": float(stt.cost),
                             "library_optimum": opt_k, "rel_diff": (opt_k - stt.cost) / stt.cost,
                             "oracle_iterations": int(stt.it), "oracle_s": time.perf_counter() - t0})
            line["workloads"]["batched_lm_convergence_1024"]["fp64_optimum_vs_oracle"] = rows
        if refined is not None:
            racc = every_block_error(d, pr_host)
            refined["rel_err_sampled"] = racc["rel_err"]
            refined["max_block_rel_err"] = racc["max_block_rel_err"]
    ctx.close()
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--refine-steps", type=int, default=2)
    ap.add_argument("--precision", default="fp32_refined", choices=["fp32_refined", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-refined", action="store_true")
    ap.add_argument("--no-workloads", action="store_true")
    ap.add_argument("--tuning", default=None,
                    help="apply this block mapping (text form of the autotuner's choice, commas for spaces) "
                         "instead of autotuning")
    ap.add_argument("--only-workload", default=None,
                    help="run only this other workload (key prefix) and print its result; for profiling")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.only_workload:
        import torch
        dev = torch.device("cuda", 0)
        print(json.dumps(other_workloads(dev, torch.cuda.Stream(dev), args.only_workload)), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
