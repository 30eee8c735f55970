"""Benchmark: 3D cubic-quintic CGL, periodic, Fourier 128^3, complex128,
tau = 0.005, fourth-order splitting (split4); Strang and RK4 alongside.

A bench step is one cgl_step call advancing the 128^3 field by `--chunk`
time steps (default 50) on the GPU.  value = grid points x time steps / s.
Inputs are resident in HBM; L2 (129 MB) is flushed by writing a 256 MiB
buffer between timed iterations, outside the timed events.

--impl reference times the FP64 CPU oracle on the same workload (a bounded
sample: one time step per bench step) and prints the same JSON line.

Multi-GPU (torchrun, N > 1): every rank advances its own replica of the
workload (the method has no exchange step); value sums the ranks' grid-point
steps over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2403_02816_gb300 import inputs as I  # noqa: E402

METRIC = "grid-pt·steps/s at fixed rel. L2 error vs FP64 oracle; % tensor/HBM roofline"
UNIT = "grid-pt·steps/s"

# FP64 peak of the GB300: 1.25 TFLOP/s nominal (dense FP64) at the 2070 MHz
# maximum SM clock over 152 SMs, i.e. 2 FP64 FMA per clock per SM.
FP64_FMA_PER_CLK_PER_SM = 2
N_SM = 152
SM_MAX_MHZ = 2070.0
# The paper's 3D cubic-quintic periodic 128^3 split4 run (Sec. 4.3 table): 900
# steps in 842.6 s, i.e. 128^3 * 900 / 842.6 grid-pt.steps/s (context only).
PAPER_E4_SPLIT4 = 128 ** 3 * 900 / 842.6
# FP32: 128 FP32 FMA per clock per SM.
FP32_PEAK_TFLOPS = N_SM * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12


def fp64_peak_tflops(sm_mhz=SM_MAX_MHZ):
    return N_SM * FP64_FMA_PER_CLK_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chunk", type=int, default=50, help="time steps per bench step")
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--scheme", default="split4")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--workload", default="periodic128",
                    choices=["periodic128", "periodic256_f32", "neumann256", "stencil256", "batch512", "corrector",
                             "coupled700x350"],
                    help="periodic128: the headline 3D periodic workload; periodic256_f32: the same "
                         "problem at 256^3 in complex64 (HBM roofline, cuFFT yardstick); neumann256: the 3D "
                         "Neumann precision study (FP64 / FP32 / BF16x3 tensor cores)")
    ap.add_argument("--t1-steps", type=int, default=100, help="neumann256: steps of the T=1 error run")
    ap.add_argument("--precisions", default="bf16x3,f32,f64tc,f64",
                    help="neumann256: comma-separated precisions to run (errors need f64)")
    ap.add_argument("--corr-traj", type=int, default=96, help="corrector: training trajectories")
    ap.add_argument("--corr-iters", type=int, default=3000, help="corrector: training iterations")
    ap.add_argument("--corr-test", type=int, default=8, help="corrector: held-out trajectories")
    ap.add_argument("--corr-sub", type=int, default=8, help="corrector: fine steps per coarse step")
    ap.add_argument("--corr-coarse-steps", type=int, default=312, help="corrector: coarse steps per trajectory")
    return ap.parse_args()


def profiled_traffic(summary, sources):
    """Per-launch DRAM bytes recorded by an ncu capture in profiles/<summary>,
    or None when the kernel sources changed since the capture."""
    import hashlib
    try:
        text = open(os.path.join(ROOT, "profiles", summary)).read()
    except OSError:
        return None
    h = hashlib.sha256()
    for s in sources:
        with open(os.path.join(ROOT, "paper_2403_02816_gb300", "csrc", s), "rb") as f:
            h.update(f.read())
    val = sha = None
    for line in text.splitlines():
        if line.startswith("traffic_bytes_per_launch:"):
            val = float(line.split(":")[1])
        if line.startswith("source_sha256_16:"):
            sha = line.split(":")[1].split()[0]
    return val if (val is not None and sha == h.hexdigest()[:16]) else None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def timed_steps(step_fn, K, chunk, warmup, flush, stream, each=None):
    """ms per time step: `warmup` (at least 3) untimed calls of one step, then
    K calls of `chunk` steps, each bracketed by CUDA events on `stream` with
    L2 flushed (outside the events) before it.  `each` (a list), if given,
    receives every timed call's ms per time step, so that an outlier shows."""
    import torch
    for _ in range(max(warmup, 3)):
        step_fn(1)
    torch.cuda.synchronize()
    ms = 0.0
    for _ in range(K):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step_fn(chunk)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        ms += t
        if each is not None:
            each.append(t / chunk)
    return ms / (K * chunk)


def neumann256_study(dev, flush, K, warmup, chunk, t1_steps, n=256, precisions=("bf16x3", "f32", "f64")):
    """3D cubic Neumann n^3, Lawson4, tau = 0.01 in each precision: ms per
    time step, per-kernel timing of one step, and the error after t1_steps
    steps from the initial data against the FP64 path."""
    import torch
    from paper_2403_02816_gb300 import native as nat
    w = I.workload_3d_neumann(n)
    U0 = I.u0_3d_neumann(w)
    N = w.prob.N
    stream = torch.cuda.current_stream()
    res, prof, finals = {}, {}, {}
    for prec in precisions:
        dt = torch.complex128 if prec in ("f64", "f64tc") else torch.complex64
        with nat.Plan(w.prob, w.tau, "lawson4", prec) as plan:
            u = nat.to_device(U0, dt, dev)
            each = []
            ms = timed_steps(lambda k: plan.step(u, k), K if prec != "f64" else 1, chunk, warmup, flush, stream, each)
            res[prec] = {"grid_pt_steps_per_s": N / (ms / 1e3), "ms_per_time_step": ms,
                         "ms_per_time_step_each_call": each,
                         "launches_per_step": plan.info()["launches_per_step"]}
            prof[prec] = plan.profile(u, 1)
            v = nat.to_device(U0, dt, dev)
            plan.step(v, t1_steps)
            torch.cuda.synchronize()
            res[prec]["device_status"] = plan.device_status()
            finals[prec] = v
    ref = finals.get("f64")
    for prec in precisions:
        if prec == "f64" or ref is None:
            continue
        e2, einf, nf = nat.cgl_rel_error(finals[prec].to(torch.complex128), ref, nat.CGL_F64)
        res[prec]["rel_l2_vs_f64_at_T"] = e2
        res[prec]["rel_inf_vs_f64_at_T"] = einf
        res[prec]["speedup_vs_f64"] = res[prec]["grid_pt_steps_per_s"] / res["f64"]["grid_pt_steps_per_s"]
    return w, res, prof


def mma_roofline(prof_bf16):
    """tcgen05 mode pass of the BF16x3 path: issued tensor flops over its
    per-launch CUDA-event time, against the measured BF16 peak."""
    peaks = measured_peaks()
    mma = [r for r in prof_bf16 if r["name"] == "mma_mode_bf16x3"][0]
    achieved = mma["flops"] / (mma["total_ms"] / 1e3) / 1e12
    peak = float(peaks.get("bf16_tflops", 1948.7))
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "kernel": "mma_mode_bf16x3", "launches_profiled": mma["launches"],
            "avg_launch_ms": mma["total_ms"] / mma["launches"],
            "flops_counted": "issued: 6 split products x 8 n real flops per point per mode",
            "algorithmic_frac": achieved / 6 / peak,
            "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst, of measured)",
            "share": mma["total_ms"] / sum(r["total_ms"] for r in prof_bf16),
            "frac_of_sustained": achieved / float(peaks.get("bf16_tflops_sustained", 1712.8))}


def oz_roofline(prof_oz):
    """tcgen05 pass of the FP64-accurate path: issued tensor flops (28 digit
    products) over its per-launch CUDA-event time, against the measured BF16
    peak; the share of the step it takes."""
    peaks = measured_peaks()
    k = [r for r in prof_oz if r["name"] == "oz_mode_f64tc"][0]
    achieved = k["flops"] / (k["total_ms"] / 1e3) / 1e12
    peak = float(peaks.get("bf16_tflops", 1948.7))
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "kernel": "oz_mode_f64tc", "launches_profiled": k["launches"],
            "avg_launch_ms": k["total_ms"] / k["launches"],
            "flops_counted": "issued: 28 digit products x 8 n real flops per point per mode",
            "algorithmic_fp64_tflops": achieved / 28,
            "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst, of measured)",
            "share": k["total_ms"] / sum(r["total_ms"] for r in prof_oz)}


def batch512_study(dev, flush, K, warmup, chunk, t1_steps, precisions=("bf16x3", "f32", "f64"), single=False):
    """The 512-instance batch, Lawson4, tau = 0.01: ms per time step of each
    precision, the per-instance errors after t1_steps steps against the FP64
    batch, and (single=True) the plain method, one FP64 plan per instance."""
    import torch
    from paper_2403_02816_gb300 import native as nat
    count = 512
    probs = I.batched_problems(count)
    fields = [I.u0_bumps(p, np.random.Generator(np.random.PCG64(I.SEED_BASE + 3 + 1000 * i)))
              for i, p in enumerate(probs)]
    total = sum(p.N for p in probs)
    stream = torch.cuda.current_stream()
    # algorithmic flops per Lawson4 step: 2 sweeps x 2 fields x 8 n_mu N per mode,
    # plus g (15), the first-sweep combination (46) and the last (19) per point
    flops_step = sum(4 * 8 * (p.n[0] + p.n[1]) * p.N + (15 + 46 + 19) * p.N for p in probs)
    # tensor-core flops issued per step: 6 split products of each mode product
    tensor_flops_step = sum(6 * 4 * 8 * (p.n[0] + p.n[1]) * p.N for p in probs)
    res, finals = {}, {}
    for prec in precisions:
        t0 = time.perf_counter()
        with nat.Batch(probs, 0.01, "lawson4", prec) as b:
            create_s = time.perf_counter() - t0
            u = b.pack(fields, dev)
            each = []
            ms = timed_steps(lambda k: b.step(u, k), K if prec != "f64" else max(1, K // 2), chunk, warmup, flush,
                             stream, each)
            res[prec] = {"grid_pt_steps_per_s": total / (ms / 1e3), "ms_per_time_step": ms,
                         "ms_per_time_step_each_call": each,
                         "create_s": create_s, "launches_per_step": b.launches_per_step,
                         "achieved_tflops": flops_step / (ms / 1e3) / 1e12}
            v = b.pack(fields, dev)
            b.step(v, t1_steps)
            torch.cuda.synchronize()
            res[prec]["device_status"] = b.device_status()
            finals[prec] = b.unpack(v)
    if "bf16x3" in res:
        res["bf16x3"]["achieved_tensor_tflops"] = tensor_flops_step / (res["bf16x3"]["ms_per_time_step"] / 1e3) / 1e12
    if single:
        plans = [nat.Plan(p, 0.01, "lawson4", "f64") for p in probs]
        us = [nat.to_device(U, torch.complex128, dev) for U in fields]

        def seq(k):
            for pl, uu in zip(plans, us):
                pl.step(uu, k)
        ms = timed_steps(seq, 1, chunk, warmup, flush, stream)
        res["single_plans_f64"] = {"grid_pt_steps_per_s": total / (ms / 1e3), "ms_per_time_step": ms,
                                   "achieved_tflops": flops_step / (ms / 1e3) / 1e12}
        for pl in plans:
            pl.close()
    errs = {}
    if "f64" in finals:
        for prec in finals:
            if prec == "f64":
                continue
            e2 = [float(np.linalg.norm(a - r) / np.linalg.norm(r)) for a, r in zip(finals[prec], finals["f64"])]
            ei = [float(np.abs(a - r).max() / np.abs(r).max()) for a, r in zip(finals[prec], finals["f64"])]
            errs[prec] = {"rel_l2_max": max(e2), "rel_l2_median": float(np.median(e2)), "rel_inf_max": max(ei),
                          "rel_inf_median": float(np.median(ei)), "steps": t1_steps}
    return {"instances": count, "total_points": total, "flops_step": flops_step,
            "tensor_flops_step": tensor_flops_step}, res, errs


def run_batch512(args):
    """512 independent 2D cubic / cubic-quintic instances (grids 48..256 per
    direction, Dirichlet/Neumann mixes, random parameters and bumps),
    Lawson4, tau = 0.01: batched launches (BF16x3 on the tensor cores, FP32
    and FP64 SIMT) against the plain method (one FP64 plan per instance,
    stepped one after another), and the complex64 batches' errors after
    `--t1-steps` steps against the FP64 batch."""
    import torch
    from paper_2403_02816_gb300 import native as nat

    dev = torch.device("cuda", 0)
    nat.load()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    chunk = args.chunk
    with Clocks(0) as clk:
        info, res, errs = batch512_study(dev, flush, args.steps, args.warmup, chunk, args.t1_steps, single=True)
    f32, bf = res["f32"], res["bf16x3"]
    peaks = measured_peaks()
    tpeak = float(peaks.get("bf16_tflops", 1948.7))
    line = {
        "metric": METRIC, "value": bf["grid_pt_steps_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": bf["ms_per_time_step"] * chunk, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3", "data": "synthetic",
        "config": {"workload": "batched_512x2d_lawson4_c64", "instances": info["instances"],
                   "total_points": info["total_points"], "tau": 0.01, "time_steps_per_bench_step": chunk,
                   "T_steps_for_error": args.t1_steps, "l2": "flushed (256 MiB write) between timed iterations"},
        "results": res, "per_instance_errors_vs_f64": errs,
        "speedup_batched_bf16x3_vs_single_f64": bf["grid_pt_steps_per_s"] /
        res["single_plans_f64"]["grid_pt_steps_per_s"],
        "speedup_batched_f32_vs_single_f64": f32["grid_pt_steps_per_s"] / res["single_plans_f64"]["grid_pt_steps_per_s"],
        "speedup_batched_f64_vs_single_f64": res["f64"]["grid_pt_steps_per_s"] /
        res["single_plans_f64"]["grid_pt_steps_per_s"],
        "roofline": {"bound": "tensor", "kernel": "mma_group_kernel", "achieved": bf["achieved_tensor_tflops"],
                     "peak": tpeak, "unit": "TFLOP/s", "frac": bf["achieved_tensor_tflops"] / tpeak,
                     "traffic": None, "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst, of measured)",
                     "note": "issued tensor flops over the whole-step time (all launches, pointwise stages "
                             "included): a lower bound for the grouped pass"},
        "roofline_f32_simt": {"bound": "alu", "kernel": "batched_mode_pass_kernel<float>",
                              "achieved": f32["achieved_tflops"], "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                              "frac": f32["achieved_tflops"] / FP32_PEAK_TFLOPS,
                              "peak_source": "derived: 152 SM x 128 FP32 FMA/clk x 2 flop x 2070 MHz",
                              "note": "whole-step time, all passes"},
        "clocks": clk.summary(),
    }
    print(json.dumps(line))


def run_corrector(args):
    """Learned corrector on the 2D periodic cubic CGL 128^2: data from the fine
    method (Lawson4, complex128, tau = 0.002), corrections F^8(u_n) - C(u_n)
    with a complex128 coarse Lawson4 step (tau = 0.016), training of the
    6-layer CNN on the tensor-core kernels, and held-out trajectories run to
    t = 4.992 with the corrected coarse step against the fine method."""
    import torch
    from paper_2403_02816_gb300 import learned as Lm
    from paper_2403_02816_gb300 import native as nat

    nat.load()
    ntraj, iters, batch = args.corr_traj, args.corr_iters, 32
    sub, csteps = args.corr_sub, args.corr_coarse_steps
    data = Lm.Dataset(ntraj=ntraj, snaps=8, sub=sub, coarse_steps=csteps)
    corr = nat.Corrector(Lm.N, Lm.N, 32, 6, max_batch=batch)
    losses, train_s = Lm.train(corr, data, iters=iters, batch=batch, lr=3e-4, log_every=max(1, iters // 4))
    # throughput of one corrected coarse step vs 8 fine steps (one instance, 128^2)
    p = Lm.problem((1.0, 0.5, 0.5, -1.0, 1.0))
    rng = np.random.default_rng(0)
    U0 = I.u0_bumps(p, rng)
    stream = torch.cuda.current_stream()
    with nat.Plan(p, Lm.FINE_TAU, "lawson4", "f64") as fine, nat.Plan(p, Lm.FINE_TAU * sub, "lawson4", "f64") as crs:
        uf = nat.to_device(U0, torch.complex128)
        uc = nat.to_device(U0, torch.complex128).reshape(1, Lm.N, Lm.N)
        prev = torch.empty_like(uc)
        prm = torch.tensor([[1.0, 0.5, 0.5, -1.0, 1.0]], dtype=torch.float32, device="cuda")
        reps = 50

        def corrected(k):
            for _ in range(k):
                prev.copy_(uc)
                crs.step(uc, 1)
                corr.apply_c128(uc, prev, prm, uc)

        ms = {}
        for fn, key in ((lambda k: fine.step(uf, sub * k), "fine_steps_f64"),
                        (lambda k: crs.step(uc, k), "coarse_step_f64"), (corrected, "corrected_coarse_step")):
            fn(3)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(reps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms[key] = e0.elapsed_time(e1) / reps
    rows = Lm.evaluate(corr, ntraj=args.corr_test, seed=Lm.SEED + 7777, sub=sub, coarse_steps=csteps)
    e_c = float(np.mean([r["coarse"] for r in rows]))
    e_l = float(np.mean([r["corrected"] for r in rows]))
    held = Lm.Dataset(ntraj=args.corr_test, snaps=8, seed=Lm.SEED + 7777, sub=sub, coarse_steps=csteps)
    one_step = {}
    for name, ds in (("train_pairs", data), ("held_out_pairs", held)):
        g = Lm.one_step_gains(corr, ds)
        one_step[name] = {"gain_mean": float(g.mean()), "gain_median": float(np.median(g)),
                          "fraction_improved": float(np.mean(g > 1))}
    npts = Lm.N * Lm.N
    t_corr = ms["corrected_coarse_step"]
    line = {
        "metric": METRIC, "value": npts / (t_corr / 1e3), "unit": UNIT, "n_gpus": 1, "steps": reps,
        "warmup": 3, "ms_per_step": t_corr, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+bf16", "data": "synthetic",
        "config": {"workload": "learned_corrector_2d_periodic_128^2", "fine_tau": Lm.FINE_TAU,
                   "coarse_tau": Lm.FINE_TAU * sub, "fine_steps_per_coarse": sub, "train_trajectories": ntraj,
                   "pairs": data.size, "iterations": iters, "batch": batch, "test_trajectories": args.corr_test,
                   "t_final": csteps * sub * Lm.FINE_TAU, "coarse_precision": "complex128",
                   "output_scale": "per sample: RMS coarse increment x dataset RMS ratio"},
        "correction_rms": data.correction_rms, "relative_rms": data.relative_rms,
        "dataset_seconds": data.seconds, "train_seconds": train_s,
        "train_samples_per_s": iters * batch / train_s, "losses": losses, "ms": ms,
        "speedup_corrected_vs_fine_f64": ms["fine_steps_f64"] / t_corr,
        "held_out_rel_l2_vs_fine": {"coarse": e_c, "corrected": e_l, "gain": e_c / e_l, "target_gain": 5.0,
                                    "rows": rows},
        "one_step_gain_vs_fine": one_step,
    }
    print(json.dumps(line))


def run_neumann256(args):
    """3D cubic Neumann 256^3, Lawson4, tau = 0.01: throughput of each
    precision and its relative L2 error at T = steps * tau against the FP64
    path (itself held to 1e-11 of the FP64 oracle by the parity tests)."""
    import torch
    from paper_2403_02816_gb300 import native as nat

    dev = torch.device("cuda", 0)
    nat.load()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    chunk = args.chunk
    with Clocks(0) as clk:
        w, res, prof = neumann256_study(dev, flush, args.steps, args.warmup, chunk, args.t1_steps,
                                        n=args.n if args.n != 128 else 256,
                                        precisions=tuple(args.precisions.split(",")))
    head = "bf16x3" if "bf16x3" in res else next(iter(res))
    rooflines = {}
    if "bf16x3" in prof:
        rooflines["roofline"] = mma_roofline(prof["bf16x3"])
        rooflines["roofline"]["traffic"] = profiled_traffic("mma_mode_bf16x3_ncu_neumann256.md",
                                                            ["mma_mode.cu", "tc_ptx.cuh", "cgl_internal.cuh"])
    if "f64tc" in prof:
        rooflines["roofline_f64tc"] = oz_roofline(prof["f64tc"])
    simt = {}
    for prec, name, peak in (("f64", "mode_pass_f64", fp64_peak_tflops()), ("f32", "mode_pass_f32", FP32_PEAK_TFLOPS)):
        if prec in prof:
            k = [r for r in prof[prec] if r["name"] == name][0]
            tf = k["flops"] / (k["total_ms"] / 1e3) / 1e12
            simt[name] = {"achieved_tflops": tf, "frac_of_peak": tf / peak}
    line = {
        "metric": METRIC, "value": res[head]["grid_pt_steps_per_s"], "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": res[head]["ms_per_time_step"] * chunk,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": head, "data": "synthetic",
        "config": {"workload": w.name, "scheme": "lawson4", "tau": w.tau, "grid": list(w.prob.n),
                   "time_steps_per_bench_step": chunk, "T": args.t1_steps * w.tau,
                   "l2": "flushed (256 MiB write) between timed iterations"},
        "precisions": res, "simt_kernels": simt, "kernels": prof, "clocks": clk.summary(),
    }
    line.update(rooflines)
    print(json.dumps(line))


# the paper's coupled run (Sec. 4.5): split4 with 500 steps to T = 3 on
# N = 700 x 350 took 85.5 s (MATLAB FP64 on a 6-core laptop CPU)
PAPER_COUPLED_SPLIT4 = 700 * 350 * 500 / 85.5


def run_coupled(args):
    """Coupled two-field cubic-quintic system on the paper's 700 x 350
    periodic grid (Sec. 4.5, its parameters and a soliton-pair initial
    state), tau = 3/500 (its coarsest split4 step): split4, Lawson4 (if4),
    Strang and Lawson2 (if2) in FP64 and FP32 (grid points N = 700 x 350 per
    time step, as the paper counts
    degrees of freedom), per-kernel timing of the mixed-radix FFT passes,
    the FP64 split4 result against the oracle after two steps, end to end
    through host buffers, and the oracle on one host core (one step, also
    the parity check of one GPU step)."""
    import torch
    from oracle import coupled_oracle as C
    from paper_2403_02816_gb300 import native as nat

    dev = torch.device("cuda", 0)
    nat.load()
    p = I.coupled_problem()
    W0 = I.coupled_u0(p)
    N = p.N
    tau, chunk = 3.0 / 500, args.chunk
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res, prof = {}, None
    launches = 0
    with Clocks(0) as clk:
        for prec in ("f64", "f32"):
            dt = torch.complex128 if prec == "f64" else torch.complex64
            for scheme in ("split4", "lawson4", "strang", "lawson2"):
                with nat.CoupledPlan(p, tau, scheme, prec) as plan:
                    w = nat.to_device_pair(W0, dt, dev)
                    for _ in range(max(args.warmup, 3)):
                        plan.step(w, chunk)
                    torch.cuda.synchronize()
                    ms = 0.0
                    for _ in range(args.steps):
                        flush.fill_(1.0)
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        plan.step(w, chunk)
                        e1.record(stream)
                        torch.cuda.synchronize()
                        ms += e0.elapsed_time(e1)
                    ms /= args.steps * chunk
                    res["%s_%s" % (scheme, prec)] = {"grid_pt_steps_per_s": N / (ms / 1e3), "ms_per_time_step": ms,
                                                     "launches_per_step": plan.info()["launches_per_step"],
                                                     "device_status": plan.device_status()}
                    if prec == "f64" and scheme == "split4":
                        launches = plan.info()["launches_per_step"] * chunk * args.steps
                        prof = plan.profile(w, 1)
    # explicit RK4 at the paper's finest RK4 step (3/2562, inside its stability limit)
    with nat.CoupledPlan(p, 3.0 / 2562, "rk4", "f64") as plan:
        w = nat.to_device_pair(W0, torch.complex128, dev)
        for _ in range(max(args.warmup, 3)):
            plan.step(w, chunk)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.step(w, chunk * args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / (chunk * args.steps)
        res["rk4_f64_tau_3/2562"] = {"grid_pt_steps_per_s": N / (ms / 1e3), "ms_per_time_step": ms,
                                     "launches_per_step": plan.info()["launches_per_step"],
                                     "device_status": plan.device_status()}
    head = res["split4_f64"]
    dom = max(prof, key=lambda r: r["total_ms"])
    achieved = dom["flops"] / (dom["total_ms"] / 1e3) / 1e12
    peak = fp64_peak_tflops()
    # cpu_baseline leg: one FP64 split4 step of the oracle on one host core,
    # its result also compared with one GPU step
    with nat.CoupledPlan(p, tau, "split4", "f64") as plan:
        w = nat.to_device_pair(W0, torch.complex128, dev)
        plan.step(w, 1)
        got = nat.from_device_pair(w)
    t0 = time.perf_counter()
    ref = C.integrate(C.CoupledProblem(p.n, p.lo, p.hi, p.a0, p.a1, p.b1, p.a2, p.a3, p.b3, p.a4, p.b4, p.a5),
                      W0, tau, 1, "split4")
    cpu_s = time.perf_counter() - t0
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    # end to end through the C ABI with pinned host buffers (u and v)
    with nat.CoupledPlan(p, tau, "split4", "f64") as plan:
        host = torch.from_numpy(np.ascontiguousarray(np.stack([W0[0].T, W0[1].T]))).pin_memory()
        plan.step_host(host, 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            plan.step_host(host, chunk)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
    line = {
        "metric": METRIC, "value": head["grid_pt_steps_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": head["ms_per_time_step"] * chunk, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "coupled_cubicquintic_periodic_700x350_c128", "scheme": "split4", "tau": tau,
                   "grid": list(p.n), "fields": 2, "time_steps_per_bench_step": chunk,
                   "l2": "flushed (256 MiB write) between timed iterations",
                   "data": "the paper's parameters; soliton pair from the Gaussian seed of its 1D relaxation run"},
        "results": res,
        "rel_l2_vs_oracle_1step": err,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None, "kernel": dom["name"] + " (mixed radix 700 = 4.5.5.7, 350 = 2.5.5.7)",
                     "launches_profiled": dom["launches"], "avg_launch_ms": dom["total_ms"] / dom["launches"],
                     "flops_counted": "5 n log2 n per transform, 6 per symbol multiply, nonlinear operators",
                     "peak_source": "derived: 152 SM x 2 FP64 FMA/clk x 2 flop x 2070 MHz",
                     "share": dom["total_ms"] / sum(r["total_ms"] for r in prof)},
        "cpu_baseline": {"value": N / cpu_s, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "1 split4 time step of the 700x350 coupled system (numpy FP64, single thread)"},
        "e2e": {"value": N * chunk * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 2 * N * 16,
                "d2h_bytes_per_step": 2 * N * 16},
        "gpu_launches": launches,
        "paper_context": {"note": "the paper's split4 run on this grid (500 steps, 85.5 s; MATLAB FP64 on a 6-core "
                                  "laptop CPU)", "grid_pt_steps_per_s": PAPER_COUPLED_SPLIT4,
                          "ratio": head["grid_pt_steps_per_s"] / PAPER_COUPLED_SPLIT4},
        "kernels": prof, "clocks": clk.summary(),
    }
    print(json.dumps(line))


def run_periodic_f32(args):
    """3D cubic-quintic periodic 256^3 (the 128^3 workload's parameters and
    initial data on a finer grid), split4, tau = 0.005, in complex64 and in
    complex128: throughput, the FP32 FFT pass against the HBM roofline, the
    FP32 result's relative L2 error against the FP64 path after `chunk`
    steps, and cuFFT (torch.fft) applying the same linear flow as a
    yardstick."""
    import torch
    from paper_2403_02816_gb300 import native as nat

    dev = torch.device("cuda", 0)
    nat.load()
    n = args.n if args.n != 128 else 256
    w = I.workload_3d_periodic(n)
    U0 = I.u0_3d_periodic(w)
    N = w.prob.N
    chunk = args.chunk
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(fn, K, W):
        for _ in range(W):
            fn()
        torch.cuda.synchronize()
        ms = 0.0
        for _ in range(K):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        return ms / K

    res, finals, prof = {}, {}, {}
    W = max(args.warmup, 3)
    with Clocks(0) as clk:
        for prec in ("f32", "f64"):
            dt = torch.complex64 if prec == "f32" else torch.complex128
            with nat.Plan(w.prob, w.tau, args.scheme, prec) as plan:
                u = nat.to_device(U0, dt, dev)
                ms = timed(lambda: plan.step(u, chunk), args.steps if prec == "f32" else 2, W)
                res[prec] = {"grid_pt_steps_per_s": N * chunk / (ms / 1e3), "ms_per_time_step": ms / chunk}
                prof[prec] = plan.profile(u, 1)
                v = nat.to_device(U0, dt, dev)
                plan.step(v, chunk)
                torch.cuda.synchronize()
                res[prec]["device_status"] = plan.device_status()
                finals[prec] = v
                if prec == "f32":
                    # yardstick: the linear flow exp(tau K) u by this library and by cuFFT
                    y = nat.to_device(U0, dt, dev)
                    ours_ms = timed(lambda: plan.linear_flow(y, 1.0), 10, W)
                    E = None
                    for mu in range(3):
                        f = torch.from_numpy(plan.factor(1.0, mu) * w.prob.n[mu]).to(dev, torch.complex64)
                        shape = [1, 1, 1]
                        shape[2 - mu] = -1
                        E = f.view(shape) if E is None else E * f.view(shape)
                    x = nat.to_device(U0, dt, dev)
                    z = torch.empty_like(x)

                    def lib_flow():
                        torch.fft.ifftn(E * torch.fft.fftn(x), out=z)

                    lib_ms = timed(lib_flow, 10, W)
                    yy = nat.to_device(U0, dt, dev)
                    plan.linear_flow(yy, 1.0)
                    lib_flow()
                    torch.cuda.synchronize()
                    agree = float(torch.linalg.vector_norm(yy - z) / torch.linalg.vector_norm(z))
                    res["linear_flow_yardstick"] = {
                        "ours_ms": ours_ms, "cufft_fftn_mul_ifftn_ms": lib_ms, "ours_over_cufft_speed": lib_ms / ours_ms,
                        "rel_l2_ours_vs_cufft": agree}
    e2, einf, _ = nat.cgl_rel_error(finals["f32"].to(torch.complex128), finals["f64"], nat.CGL_F64)
    res["f32"]["rel_l2_vs_f64"] = e2
    res["f32"]["rel_inf_vs_f64"] = einf
    res["f32"]["speedup_vs_f64"] = res["f32"]["grid_pt_steps_per_s"] / res["f64"]["grid_pt_steps_per_s"]
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6790.0))
    k = [r for r in prof["f32"] if r["name"] == "fft_pass_f32"][0]
    achieved = k["bytes"] / (k["total_ms"] / 1e3) / 1e9
    traffic = None
    if n == 256 and args.scheme == "split4":
        traffic = profiled_traffic("fft4_pass_f32_dram_split4_256cubed.md", ["fft.cu", "cgl_internal.cuh"])
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "kernel": "fft_pass_f32", "launches_profiled": k["launches"],
                "avg_launch_ms": k["total_ms"] / k["launches"],
                "bytes_counted": "8 B per complex64 value of every field read or written by the pass",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                "share": k["total_ms"] / sum(r["total_ms"] for r in prof["f32"])}
    line = {
        "metric": METRIC, "value": res["f32"]["grid_pt_steps_per_s"], "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": W, "ms_per_step": res["f32"]["ms_per_time_step"] * chunk,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "scheme": args.scheme, "tau": w.tau, "grid": list(w.prob.n),
                   "time_steps_per_bench_step": chunk, "l2": "flushed (256 MiB write) between timed iterations"},
        "precisions": res, "roofline": roofline, "kernels": prof, "clocks": clk.summary(),
    }
    print(json.dumps(line))


def run_stencil256(args):
    """Runge-Kutta (RK4, eq. RK4) on the 3D Neumann 256^3 finite-difference
    problem (the precision-study workload's grid and parameters) with a step
    below RK4's stability limit: each stage is one launch of the eq. kronsumv
    stencil fused with the stage epilogue, an HBM-bound kernel; FP64 and FP32."""
    import torch
    from paper_2403_02816_gb300 import native as nat

    dev = torch.device("cuda", 0)
    nat.load()
    w = I.workload_3d_neumann(256)
    U0 = I.u0_3d_neumann(w)
    N = w.prob.N
    tau = 2e-4  # below 2.8 / |lambda_max(K)| for this grid
    chunk = args.chunk
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6790.0))
    res, prof = {}, {}
    with Clocks(0) as clk:
        for prec in ("f64", "f32"):
            dt = torch.complex128 if prec == "f64" else torch.complex64
            with nat.Plan(w.prob, tau, "rk4", prec) as plan:
                u = nat.to_device(U0, dt, dev)
                for _ in range(max(args.warmup, 3)):
                    plan.step(u, 1)
                torch.cuda.synchronize()
                ms = 0.0
                for _ in range(args.steps):
                    flush.fill_(1.0)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    plan.step(u, chunk)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms += e0.elapsed_time(e1)
                res[prec] = {"grid_pt_steps_per_s": N * chunk * args.steps / (ms / 1e3),
                             "ms_per_time_step": ms / (chunk * args.steps), "device_status": plan.device_status()}
                prof[prec] = plan.profile(u, 1)
    rl = {}
    for prec in ("f64", "f32"):
        k = [r for r in prof[prec] if r["name"].startswith("kron_stencil")][0]
        gbs = k["bytes"] / (k["total_ms"] / 1e3) / 1e9
        rl[prec] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                    "kernel": k["name"], "launches_profiled": k["launches"],
                    "avg_launch_ms": k["total_ms"] / k["launches"],
                    "bytes_counted": "per stage: the stage argument, 3 extra inputs and 1-2 outputs per point"}
    line = {
        "metric": METRIC, "value": res["f32"]["grid_pt_steps_per_s"], "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": res["f32"]["ms_per_time_step"] * chunk,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "3d_cubic_neumann_fd2_256^3_rk4", "scheme": "rk4", "tau": tau, "grid": [256] * 3,
                   "time_steps_per_bench_step": chunk, "l2": "flushed (256 MiB write) between timed iterations"},
        "precisions": res, "roofline": rl["f32"], "roofline_f64": rl["f64"], "kernels": prof, "clocks": clk.summary(),
    }
    print(json.dumps(line))


def measured_fma_peaks():
    """FP64 / FP32 FMA throughput measured by the library's microbenchmark."""
    from paper_2403_02816_gb300 import native as nat
    return {"f64_tflops": nat.cgl_measure_fma_peak("f64", 4096), "f32_tflops": nat.cgl_measure_fma_peak("f32", 65536)}


class Clocks:
    """Sample SM clocks and throttle reasons with nvidia-smi while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
                self.lines = [l for l in out.splitlines() if l.strip()]
            except Exception:
                self.proc.kill()

    def summary(self):
        if not getattr(self, "lines", None):
            return None
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        # samples under load: the upper half of the clock samples
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_worker(n, scheme, nsteps, barrier, queue):
    """One process of the all-cores oracle baseline: build the workload,
    wait for the others, time `nsteps` oracle steps."""
    w = I.workload_3d_periodic(n)
    U0 = I.u0_3d_periodic(w)
    barrier.wait()
    secs, _ = cpu_oracle_steps(w, U0, scheme, nsteps)
    queue.put(secs)


def cpu_oracle_all_cores(n, scheme, nsteps, procs):
    """The oracle on every host core at once: `procs` spawned processes (one
    numpy thread each) each time `nsteps` steps of the full field after a
    common barrier; throughput = procs * N * nsteps / slowest process."""
    import multiprocessing as mp
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(procs), ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(n, scheme, nsteps, barrier, queue)) for _ in range(procs)]
    for q in ps:
        q.start()
    secs = [queue.get(timeout=600) for _ in ps]
    for q in ps:
        q.join()
    N = n ** 3
    return procs * N * nsteps / max(secs), max(secs)


def dirichlet64_gpu(dev, flush, K, warmup):
    """The 2D Dirichlet 64^2 parity workload (FP64, tau = 0.01, 200 steps of
    Strang and of Lawson4) on the GPU: ms per time step and the final fields."""
    import torch
    from paper_2403_02816_gb300 import native as nat
    w = I.workload_2d_dirichlet(64)
    U0 = I.u0_2d_dirichlet(w)
    stream = torch.cuda.current_stream()
    res, finals = {}, {}
    for scheme in ("strang", "lawson4"):
        with nat.Plan(w.prob, w.tau, scheme, "f64") as plan:
            u = nat.to_device(U0, torch.complex128, dev)
            ms = timed_steps(lambda k: plan.step(u, k), K, 200, warmup, flush, stream)
            res[scheme] = {"grid_pt_steps_per_s": w.prob.N / (ms / 1e3), "ms_per_time_step": ms,
                           "launches_per_step": plan.info()["launches_per_step"]}
            v = nat.to_device(U0, torch.complex128, dev)
            plan.step(v, 200)
            torch.cuda.synchronize()
            res[scheme]["device_status"] = plan.device_status()
            finals[scheme] = nat.from_device(v)
    return w, U0, res, finals


def oracle_problem(p):
    from oracle import cgl_oracle as O
    return O.OracleProblem(p.n, p.bc, p.lo, p.hi, p.a1, p.b1, p.a2, p.a3, p.b3, p.a4, p.b4)


def cpu_oracle_steps(w, U0, scheme, nsteps):
    """Time `nsteps` oracle steps on the full workload (bounded sample)."""
    from oracle import cgl_oracle as O
    L = O.LinearOperator(oracle_problem(w.prob), w.tau)
    step = O.SCHEMES[scheme]
    U = U0.copy()
    t0 = time.perf_counter()
    for _ in range(nsteps):
        U = step(L, U)
    return time.perf_counter() - t0, U


def over_ranks(ms_local, units_local, dist=None, device="cpu"):
    """Whole-job timing of replicas (one per rank): the slowest rank's time and
    the work of all ranks, value = total units / slowest time.  `dist` is
    torch.distributed with an initialised process group, or None for one
    process."""
    import torch
    t = torch.tensor([float(ms_local), float(units_local)], dtype=torch.float64, device=device)
    if dist is not None:
        ms_t = t[:1].clone()
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
        u_t = t[1:].clone()
        dist.all_reduce(u_t, op=dist.ReduceOp.SUM)
        ms_max, units = float(ms_t.item()), float(u_t.item())
    else:
        ms_max, units = float(ms_local), float(units_local)
    return ms_max, units, units / (ms_max / 1e3)


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on every host core (one process
    per core, each advancing its own copy of the full field by one time step
    per bench step, after `--warmup` untimed steps)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = I.workload_3d_periodic(args.n)
    N = w.prob.N
    procs = os.cpu_count() or 1
    value, secs = cpu_oracle_all_cores(args.n, args.scheme, max(args.warmup, 0) + args.steps, procs)
    # the warm-up steps run inside the same timed loop; the rate counts all steps
    steps_run = max(args.warmup, 0) + args.steps
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / steps_run,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "scheme": args.scheme, "tau": w.tau, "grid": list(w.prob.n),
                   "time_steps_per_bench_step": 1, "l2": "input larger than L2 not needed (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                         "sample": "%d time steps of %s on the full %s field in each of %d processes at once "
                                   "(numpy, FP64, one thread each)"
                                   % (steps_run, args.scheme, "x".join(map(str, w.prob.n)), procs)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "neumann256":
        run_neumann256(args)
        return
    if args.workload == "coupled700x350":
        run_coupled(args)
        return
    if args.workload == "periodic256_f32":
        run_periodic_f32(args)
        return
    if args.workload == "stencil256":
        run_stencil256(args)
        return
    if args.workload == "batch512":
        run_batch512(args)
        return
    if args.workload == "corrector":
        run_corrector(args)
        return

    import torch
    from paper_2403_02816_gb300 import native as nat

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    nat.load()
    w = I.workload_3d_periodic(args.n)
    U0 = I.u0_3d_periodic(w)
    N = w.prob.N
    chunk = args.chunk
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(plan, u, K, W):
        for _ in range(W):
            plan.step(u, chunk)
        barrier()
        evs = []
        for _ in range(K):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.step(u, chunk)
            e1.record(stream)
            evs.append((e0, e1))
        barrier()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        return ms

    plan = nat.Plan(w.prob, w.tau, args.scheme, "f64")
    u = nat.to_device(U0, torch.complex128, dev)
    with Clocks(local) as clk:
        ms = timed(plan, u, args.steps, max(args.warmup, 3))
    clocks = clk.summary()
    ms_max, units, value = over_ranks(ms, N * chunk * args.steps, dist, device=dev)
    status = plan.device_status()

    # per-kernel timing for the roofline (CUDA events around every launch)
    prof = plan.profile(u, 2)
    dom = max(prof, key=lambda r: r["total_ms"])
    share = dom["total_ms"] / sum(r["total_ms"] for r in prof)
    # the dominant kernel's time inside the replayed graph: its share (from
    # the per-launch events of cgl_profile_step) of the graph-timed step
    graph_ms_per_time_step = ms_max / (args.steps * chunk)
    achieved = (dom["flops"] / 2) / (share * graph_ms_per_time_step / 1e3) / 1e12
    achieved_events = dom["flops"] / (dom["total_ms"] / 1e3) / 1e12
    peak = fp64_peak_tflops()
    traffic = None
    if args.n == 128 and args.scheme == "split4":
        traffic = profiled_traffic("fft_pass_f64_dram_split4_128cubed.md", ["fft.cu", "cgl_internal.cuh"])
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": dom["name"], "launches_profiled": dom["launches"],
                "avg_launch_ms": share * graph_ms_per_time_step * 2 / dom["launches"],
                "timing": "share of the graph-timed step (CUDA events around the replayed graphs)",
                "achieved_per_launch_events": achieved_events,
                "peak_source": "derived: 152 SM x 2 FP64 FMA/clk x 2 flop x 2070 MHz (1.25 TFLOP/s nominal FP64)",
                "share": share}
    fma = measured_fma_peaks()
    roofline["peak_fma_microbenchmark"] = fma["f64_tflops"]
    roofline["frac_of_fma_microbenchmark"] = achieved / fma["f64_tflops"]

    # end to end through the C ABI with host buffers (pinned)
    host = torch.from_numpy(np.ascontiguousarray(U0.T)).pin_memory()
    plan.step_host(host, 1)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        plan.step_host(host, chunk)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": N * chunk * args.steps * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": N * 16, "d2h_bytes_per_step": N * 16}

    info = plan.info()
    extras = {}
    if not args.no_extras:
        for s in ("strang", "rk4", "lawson4", "strang3t", "split4_3t"):
            if s == args.scheme:
                continue
            with nat.Plan(w.prob, w.tau, s, "f64") as p2:
                u2 = nat.to_device(U0, torch.complex128, dev)
                ms2 = timed(p2, u2, 2, 1)
                extras[s] = N * chunk * 2 / (ms2 / 1e3)
        extras[args.scheme] = value / world

    workloads = {}
    c0 = None
    if not args.no_extras and rank == 0:
        with Clocks(local) as clk2:
            c0 = dirichlet64_gpu(dev, flush, 3, 3)
            workloads["dirichlet64_fd2_c128"] = {"config": c0[0].name, "tau": c0[0].tau, "steps": 200,
                                                 "precision": "f64", "schemes": c0[2]}
            wn, res_n, prof_n = neumann256_study(dev, flush, 3, 3, 10, 100,
                                                 precisions=("bf16x3", "f32", "f64tc", "f64"))
            rl = mma_roofline(prof_n["bf16x3"])
            rl["traffic"] = profiled_traffic("mma_mode_bf16x3_ncu_neumann256.md",
                                             ["mma_mode.cu", "tc_ptx.cuh", "cgl_internal.cuh"])
            workloads["neumann256_lawson4"] = {"config": wn.name, "tau": wn.tau, "T": 100 * wn.tau,
                                               "precisions": res_n, "roofline_tcgen05": rl,
                                               "roofline_f64tc": oz_roofline(prof_n["f64tc"])}
            info_b, res_b, errs_b = batch512_study(dev, flush, 3, 3, 10, 200)
            tpeak = float(measured_peaks().get("bf16_tflops", 1948.7))
            workloads["batch512_lawson4"] = {
                "config": "batched_512x2d_lawson4_c64", "tau": 0.01, "instances": info_b["instances"],
                "total_points": info_b["total_points"], "precisions": res_b, "per_instance_errors_vs_f64": errs_b,
                "tensor_frac_whole_step": res_b["bf16x3"]["achieved_tensor_tflops"] / tpeak}
        workloads["clocks"] = clk2.summary()

    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        secs, Uref = cpu_oracle_steps(w, U0, args.scheme, 1)
        procs = os.cpu_count() or 1
        all_value, all_secs = cpu_oracle_all_cores(args.n, args.scheme, 2, procs)
        cpu = {"value": all_value, "unit": UNIT, "cores": procs, "kind": "oracle",
               "sample": "2 time steps of %s on the full %s field in each of %d processes at once (numpy FP64, "
                         "one thread each)" % (args.scheme, "x".join(map(str, w.prob.n)), procs),
               "value_1_core": N / secs,
               "sample_1_core": "1 time step of %s on the full %s field (numpy FP64, single thread)"
                                % (args.scheme, "x".join(map(str, w.prob.n)))}
        if c0 is not None:
            # the 64^2 Dirichlet workload's whole run in the oracle: its time
            # and the GPU's relative L2 / inf differences from it
            from oracle import cgl_oracle as O
            w0, U00, _, finals0 = c0
            op0 = oracle_problem(w0.prob)
            for scheme in ("strang", "lawson4"):
                t0 = time.perf_counter()
                ref0 = O.integrate(op0, U00, w0.tau, 200, scheme)
                dt0 = time.perf_counter() - t0
                g0 = finals0[scheme]
                sc = workloads["dirichlet64_fd2_c128"]["schemes"][scheme]
                sc["rel_l2_vs_oracle"] = float(np.linalg.norm(g0 - ref0) / np.linalg.norm(ref0))
                sc["rel_inf_vs_oracle"] = float(np.abs(g0 - ref0).max() / np.abs(ref0).max())
                sc["oracle_grid_pt_steps_per_s_1_core"] = w0.prob.N * 200 / dt0
        with nat.Plan(w.prob, w.tau, args.scheme, "f64") as p3:
            u3 = nat.to_device(U0, torch.complex128, dev)
            p3.step(u3, 1)
            torch.cuda.synchronize()
            g3 = nat.from_device(u3)
            parity = float(np.linalg.norm(g3 - Uref) / np.linalg.norm(Uref))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "scheme": args.scheme, "tau": w.tau, "grid": list(w.prob.n),
                       "time_steps_per_bench_step": chunk, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "flushed (256 MiB write) between timed iterations"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": info["launches_per_step"] * chunk * args.steps,
            "clocks": clocks, "device_status": status,
            "rel_l2_vs_oracle_1step": parity, "schemes_grid_pt_steps_per_s": extras, "workloads": workloads,
            "paper_context": {
                "note": "the paper's nearest run (3D cubic-quintic, periodic Fourier 128^3, split4; other domain "
                        "and parameters, so not vs_baseline); MATLAB FP64 on a 6-core laptop CPU",
                "grid_pt_steps_per_s": PAPER_E4_SPLIT4, "ratio": value / PAPER_E4_SPLIT4},
            "kernels": prof,
        }
        print(json.dumps(line))
    plan.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
