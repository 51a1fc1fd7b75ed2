#!/usr/bin/env python3
"""Throughput of the photoionization KIFMM on one GB300 (S_ph points per second).

Workload (default): 128^3 cell centres of a 1 cm cube (2,097,152 points), Gaussian
source 1e22 exp(-|r - c|^2 / (0.1 cm)^2), p = 760 Torr, p_O2 = 0.2 p = 152 Torr,
surface order m0 = 6, leaf size 64. One step = one evaluation of S for the whole
field (every phase of the evaluation: weights, S2M, M2M, M2L, S2L/L2L, local and
W-list evaluation, near-field P2P, self term, reordering) in the mixed-precision
form; the plan (tree, lists, operators) is built once before timing, as in a time
loop on a fixed mesh. The mixed result is checked against the FP64 form (gate:
rel-L2 <= 1e-6) before timing.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica of the workload on its GPU
(the single-field path has no data-parallel split without a tree exchange).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 512 << 20
SM_COUNT = 152
# MUFU results per SM per clock of GB300, measured once with a microbenchmark of independent
# dependency chains (8 per thread, 4 blocks of 256 threads per SM, CUDA events): ex2.approx.ftz.f32
# 30.15 and rsqrt.approx.ftz.f32 15.15 results per SM per clock
EX2_PER_SM_CLK = 30.2
RSQ_PER_SM_CLK = 15.2
PAIRS_PER_SM_CLK = 1.0 / (2.0 / EX2_PER_SM_CLK + 1.0 / RSQ_PER_SM_CLK)   # one rsqrt + two ex2 per pair
FP64_TFLOPS = 1.25      # GB300 FP64 (nominal; FMA chains measured 1.01, the FP64 GEMM 1.13 TFLOP/s)


METRIC = "S_ph points/s at rel-L2<=1e-6 (FP64 vs mixed KIFMM)"

# DRAM bytes (read + write) per launch from the ncu captures summarised under profiles/, valid while the kernel's
# sources are the ones that were captured (else the roofline's traffic is null). The 96^3 capture has
# the far-field structure of the 128^3 workload (same M2L launch); the 64^3 capture has its per-leaf
# shape, and the pair kernel's traffic is compulsory and scales with the point count (x 8 for 128^3).
PROFILED_TRAFFIC = {
    "M2L": {"bytes": 165.548e6 + 12.911e6, "per_point_scaled": False,
            "src": {"paper_2006_03515_gb300/csrc/m2l_tc.cu":
                    "b8ad63f18f5197f235580d11661f1bafca743abe240f207bc031e4042d8595d5"},
            "profile": "profiles/k_m2l_tc_uniform96.md"},
    "P2P": {"bytes": 14.20e6, "per_point_scaled": True, "n_profiled": 64 ** 3,
            "src": {"paper_2006_03515_gb300/csrc/eval.cu":
                    "27add4c5c6f89bc5081df57c5cc3f95224a7882530864fae517b59636790b1c6"},
            "profile": "profiles/k_p2p_mixed_uniform64.md"},
    "NEAR": {"bytes": 3.958e6, "per_point_scaled": True, "n_profiled": 64 ** 3,
             "src": {"paper_2006_03515_gb300/csrc/m2l_tc.cu":
                     "b8ad63f18f5197f235580d11661f1bafca743abe240f207bc031e4042d8595d5",
                     "paper_2006_03515_gb300/csrc/near_tc.cu":
                     "46fa6d5f4f4f0e56deeea2645bf8112cb643b02e5a7550efca2993006487a7eb"},
             "profile": "profiles/k_m2l_tc_near_uniform64.md"},
}


def profiled_traffic(key, npts, workload_is_128_uniform):
    """Traffic per launch for the bench's workload, or None when the kernel changed or the
    capture does not describe this workload."""
    import hashlib
    e = PROFILED_TRAFFIC.get(key)
    if e is None or not workload_is_128_uniform:
        return None
    try:
        for src, sha in e["src"].items():
            with open(os.path.join(ROOT, src), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != sha:
                    return None
    except OSError:
        return None
    return e["bytes"] * (npts / e["n_profiled"] if e["per_point_scaled"] else 1.0)


def workload_name(args):
    rep = "m0=%d" % args.m0 if args.repr == "surface" else "Chebyshev p=%d" % args.m0
    return ("uniform %d^3 cell centres, 1 cm cube, Gaussian 1e22 exp(-r^2/0.1^2), p=%g Torr, pO2=%g, %s, "
            "leaf %d, %s" % (args.n, args.p, 0.2 * args.p, rep, args.leaf, args.precision))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=128, help="grid cells per axis")
    ap.add_argument("--m0", type=int, default=6)
    ap.add_argument("--leaf", type=int, default=64)
    ap.add_argument("--p", type=float, default=760.0, help="gas pressure (Torr); p_O2 = 0.2 p")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--repr", default="surface", choices=["surface", "cheb"],
                    help="far-field representation of the timed plan (cheb: --m0 is the Chebyshev order p)")
    ap.add_argument("--no-cheb", action="store_true", help="skip the Chebyshev-representation measurement")
    ap.add_argument("--cheb-p", type=int, default=8, help="Chebyshev order of that measurement")
    ap.add_argument("--no-radii", action="store_true", help="skip the figure-radii (1.2 / 2.6) measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-workload measurement")
    ap.add_argument("--batch-fields", type=int, default=64, help="fields of the batched workload")
    ap.add_argument("--batch-lanes", type=int, default=8, help="concurrent lanes of the batched workload")
    ap.add_argument("--batch-target", type=float, default=3e-3,
                    help="accuracy target (rel-L2 against the direct sum) of the batch's autotuner")
    ap.add_argument("--cpu-n", type=int, default=64, help="grid of the bounded CPU-oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 gate and FP64 timing")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate measurement")
    ap.add_argument("--no-streamer", action="store_true", help="skip the streamer time-loop measurement")
    ap.add_argument("--sd-n", type=int, default=128, help="streamer grid: n x n x 2n cells of the 0.5 x 0.5 x 1 cm gap")
    ap.add_argument("--sd-steps", type=int, default=10, help="timed streamer steps")
    ap.add_argument("--no-configs", action="store_true", help="skip the other target settings")
    ap.add_argument("--streamer-only", action="store_true",
                    help="measure only the streamer time loop (one JSON object; for its launch list)")
    ap.add_argument("--surrogate-only", action="store_true",
                    help="measure only the surrogate and print its record (profiling runs)")
    ap.add_argument("--sno-n", type=int, default=64, help="surrogate grid cells per axis")
    ap.add_argument("--sno-batch", type=int, default=32, help="surrogate inference batch (fields per forward pass)")
    ap.add_argument("--sno-fields", type=int, default=256, help="KIFMM-labelled training fields")
    ap.add_argument("--sno-heldout", type=int, default=128, help="held-out fields of the surrogate")
    ap.add_argument("--sno-train-s", type=float, default=15.0, help="surrogate training budget per model (s)")
    ap.add_argument("--sno-lr", type=float, default=1e-5, help="Adam learning rate from the far-part start")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms, ws):
    """The slowest rank's time (ms): the whole job ends when it does."""
    if ws <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t[0])


def whole_job_rate(npts, ws, ms):
    """Points per second of all ranks together: every rank evaluates its own npts-point
    field (replicas, weak scaling) in ms."""
    return ws * npts / (ms * 1e-3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = self.rows
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_sample(n_cpu, m0, leaf, a, b, C):
    """The oracle (plain CPU KIFMM, FP64) on an n_cpu^3 sample of the same workload
    (same cube, source, pressure, m0 and leaf size); returns points/s of its
    evaluation and the thread count it used."""
    import numpy as np
    from oracle import direct as D
    from oracle import kifmm as KF
    from paper_2006_03515_gb300 import workloads as W
    pts, h, I = W.config_uniform(n_cpu)
    p = KF.plan(pts, h, leaf, m0, a, b)
    t0 = time.perf_counter()
    KF.evaluate(p, I, C)
    dt = time.perf_counter() - t0
    return len(pts) / dt, D.c_threads(), dt


def run_reference(args):
    """The oracle as it stands, timed on this machine's host cores."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import build as ob
    from oracle import direct as D
    from oracle import kernel as K
    from oracle import kifmm as KF
    from paper_2006_03515_gb300 import workloads as W
    ob.build()
    a, b = K.absorption_coefficients(0.2 * args.p)
    C = K.source_scale(args.p)
    n = 32
    pts, h, I = W.config_uniform(n)
    p = KF.plan(pts, h, args.leaf, args.m0, a, b)
    for _ in range(args.warmup):
        KF.evaluate(p, I, C)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        KF.evaluate(p, I, C)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = len(pts) / (ms * 1e-3)
    sample = ("oracle KIFMM evaluation (FP64, numpy + C/OpenMP) on a %d^3 sample of the workload "
              "(same 1 cm cube, source, pressure, m0=%d, leaf %d); plan excluded" % (n, args.m0, args.leaf))
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": "points/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args), "sample": "uniform %d^3 cell centres of the same cube" % n,
                       "n_points": len(pts), "l2": "host run (no GPU)", "parallelism": "single"},
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": D.c_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def radii_bench(args, dev, stream, dpts, hval, dI, C, a, b, flush, peaks):
    """The same workload with the surfaces at the radii drawn in Fig. fmulloc, 1.2 / 2.6 box
    half-widths (the default is 1.05 / 2.95), mixed form: kept rank, plan time, evaluation
    time (CUDA events, L2 flushed between steps), phase times, the M2L rate, and the mixed
    result against one FP64 evaluation of the same radii."""
    import torch
    from paper_2006_03515_gb300 import kifmm
    radii = (1.2, 2.6)
    npts = dpts.shape[0]
    t0 = time.perf_counter()
    pl = kifmm.Plan(dpts, hval, args.leaf, args.m0, a, b, precision="mixed", stream=stream, surface_radii=radii)
    torch.cuda.synchronize(dev)
    plan_s = time.perf_counter() - t0
    S = torch.empty_like(dI)
    for _ in range(3):
        pl.eval(dI, S, C=C)
    steps = max(3, min(args.steps, 10))
    ms, phase_sum = [], None
    for k in range(steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pl.eval(dI, S, C=C)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        ph = pl.phase_times()
        phase_sum = ph if phase_sum is None else [x + y for x, y in zip(phase_sum, ph)]
    info = pl.info()
    phases = ["scatter", "S2M", "M2M+UC2UE", "M2L", "S2L+L2L+DC2DE", "L2P+M2P", "P2P"]
    ph_ms = {k: v / steps for k, v in zip(phases, phase_sum)}
    f16_peak = peaks.get("bf16_tflops", 1947.8)
    m2l_ach = info["m2l_flops"] / (ph_ms["M2L"] * 1e-3) / 1e12
    t = sum(ms) / len(ms)
    out = {"radii": list(radii), "precision": "mixed", "rank_min": info["pinv_rank_min"], "plan_s": plan_s,
           "ms": t, "points_per_s": npts / (1e-3 * t), "phase_ms": ph_ms,
           "m2l": {"path": "tcgen05 FP16x3" if info["m2l_tensor"] else "SIMT FP32", "tflops": m2l_ach,
                   "frac": m2l_ach / (f16_peak / 3.0), "flops": info["m2l_flops"]},
           "near_tensor": bool(info["near_tensor"]), "lattice_far": bool(info["lattice_far"])}
    if not args.no_fp64:
        p64 = kifmm.Plan(dpts, hval, args.leaf, args.m0, a, b, precision="fp64", stream=stream, surface_radii=radii)
        S64 = p64.eval(dI, C=C)
        torch.cuda.synchronize(dev)
        out["gate_rel_l2_mixed_vs_fp64"] = float(torch.linalg.norm(S - S64) / torch.linalg.norm(S64))
        p64.close()
        del S64
    pl.close()
    torch.cuda.empty_cache()
    return out


def cheb_bench(args, dev, stream, dpts, hval, dI, C, a, b, flush, peaks):
    """The same workload with the Chebyshev-node representation (order args.cheb_p), mixed
    form: plan time, evaluation time (CUDA events, L2 flushed between steps), phase times,
    the M2L rate, and the mixed result against one FP64 evaluation of the same plan."""
    import torch
    from paper_2006_03515_gb300 import kifmm
    npts = dpts.shape[0]
    t0 = time.perf_counter()
    pl = kifmm.Plan(dpts, hval, args.leaf, args.cheb_p, a, b, precision="mixed", stream=stream, repr="cheb")
    torch.cuda.synchronize(dev)
    plan_s = time.perf_counter() - t0
    S = torch.empty_like(dI)
    for _ in range(3):
        pl.eval(dI, S, C=C)
    steps = max(3, min(args.steps, 10))
    ms, phase_sum = [], None
    for k in range(steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pl.eval(dI, S, C=C)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        ph = pl.phase_times()
        phase_sum = ph if phase_sum is None else [x + y for x, y in zip(phase_sum, ph)]
    info = pl.info()
    phases = ["scatter", "P2M", "M2M", "M2L", "X+L2L", "L2P+W", "P2P"]
    ph_ms = {k: v / steps for k, v in zip(phases, phase_sum)}
    m2l_ach = info["m2l_flops"] / (ph_ms["M2L"] * 1e-3) / 1e12
    out = {"p": args.cheb_p, "nodes": info["surface_points"], "precision": "mixed", "plan_s": plan_s,
           "ms": sum(ms) / len(ms), "points_per_s": npts / (1e-3 * sum(ms) / len(ms)), "phase_ms": ph_ms,
           "m2l": {"path": "tcgen05 FP16x3" if info["m2l_tensor"] else "SIMT FP32", "tflops": m2l_ach,
                   "flops": info["m2l_flops"]}}
    if not args.no_fp64:
        p64 = kifmm.Plan(dpts, hval, args.leaf, args.cheb_p, a, b, precision="fp64", stream=stream, repr="cheb")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        S64 = p64.eval(dI, C=C)
        e1.record(stream)
        e1.synchronize()
        out["fp64_ms"] = e0.elapsed_time(e1)
        out["gate_rel_l2_mixed_vs_fp64"] = float(torch.linalg.norm(S - S64) / torch.linalg.norm(S64))
        p64.close()
        del S64
    pl.close()
    torch.cuda.empty_cache()
    return out


def _timed_eval(plan, dI, S, C, flush, stream, steps=5):
    """Median evaluation time (ms) over `steps` runs, CUDA events on the plan's stream, L2
    flushed between runs."""
    import torch
    for _ in range(2):
        plan.eval(dI, S, C=C)
    ms = []
    for k in range(steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.eval(dI, S, C=C)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms)


def configs_bench(args, dev, stream, flush):
    """Time and accuracy of the other target settings (not headlines): the 128^3 Gaussian
    field at 76 and 7.6 Torr (m0 = 6) and at 760 Torr with m0 = 4 and 8, and the adaptive
    3,219,819-point refined grid (760 Torr, p_O2 150, channel + head + noise). Each entry: the
    mixed form's median time and rate, the FP64 form's time, the mixed-vs-FP64 gate, and the
    rel-L2 of both forms against the whole discrete sum (the oracle's FFT convolution on the
    uniform grid; on the refined grid the oracle's direct sum at 4096 sampled targets, half of
    them among the fine cells)."""
    import numpy as np
    import torch
    from oracle import build as ob
    from oracle import direct as D
    from paper_2006_03515_gb300 import kifmm
    from paper_2006_03515_gb300 import workloads as W
    ob.build()
    out = {}

    def one(pts, hval, I, leaf, m0, p, p_o2, ref_fn):
        a, b = kifmm.absorption(p_o2)
        C = kifmm.scale_c(p)
        dpts, dI = torch.as_tensor(pts, device=dev), torch.as_tensor(I, device=dev)
        hv = torch.as_tensor(hval, device=dev) if isinstance(hval, np.ndarray) else hval
        pm = kifmm.Plan(dpts, hv, leaf, m0, a, b, precision="mixed", stream=stream)
        Sm = torch.empty_like(dI)
        ms = _timed_eval(pm, dI, Sm, C, flush, stream)
        p64 = kifmm.Plan(dpts, hv, leaf, m0, a, b, precision="fp64", stream=stream)
        S64 = torch.empty_like(dI)
        ms64 = _timed_eval(p64, dI, S64, C, flush, stream, steps=2)
        torch.cuda.synchronize(dev)
        gate = float(torch.linalg.norm(Sm - S64) / torch.linalg.norm(S64))
        idx, ref, kind = ref_fn(a, b, C)
        sm, s64 = Sm.cpu().numpy(), S64.cpu().numpy()
        if idx is not None:
            sm, s64 = sm[idx], s64[idx]
        rec = {"points": len(pts), "leaf": leaf, "m0": m0, "p_torr": p, "p_o2": p_o2, "ms": ms,
               "points_per_s": len(pts) / (1e-3 * ms), "fp64_ms": ms64, "gate_rel_l2_mixed_vs_fp64": gate,
               "rel_l2_vs_direct_sum": float(np.linalg.norm(sm - ref) / np.linalg.norm(ref)),
               "fp64_rel_l2_vs_direct_sum": float(np.linalg.norm(s64 - ref) / np.linalg.norm(ref)),
               "reference": kind, "near_tensor": bool(pm.info()["near_tensor"])}
        pm.close()
        p64.close()
        del Sm, S64, dI, dpts
        torch.cuda.empty_cache()
        return rec

    pts, h, I = W.config_uniform(128)
    for p, m0 in [(760.0, 4), (760.0, 8), (76.0, 6), (7.6, 6)]:
        def ref_fn(a, b, C):
            return None, D.fft_uniform(I.reshape(128, 128, 128), h[0], a, b, C).ravel(), "whole discrete sum (FFT)"
        out["uniform128_p%g_m0%d" % (p, m0)] = one(pts, float(h[0]), I, 64, m0, p, 0.2 * p, ref_fn)
    pts, h, I = W.config_adaptive()
    fine = np.nonzero(h < h.max())[0]
    rng = np.random.Generator(np.random.PCG64(2006))
    idx = np.sort(np.concatenate([rng.choice(len(pts), 2048, replace=False), rng.choice(fine, 2048, replace=False)]))

    def ref_ad(a, b, C):
        return idx, D.direct_sum(pts, h, I, a, b, C, targets=idx), "direct sum at 4096 sampled targets (2048 fine)"
    out["adaptive_3219819"] = one(pts, h, I, 64, 6, 760.0, 150.0, ref_ad)
    return out


def batch_bench(args, dev, stream, flush):
    """The batched workload: args.batch_fields streamer fields of uneven sizes (uniform grids
    of 80^3-158^3 cells, 0.5-4 M points, two channels each, 760 or 76 Torr, seed-drawn),
    evaluated as one CUDA-graph batch, back to back on one stream and on concurrent lanes;
    CUDA events on the launching stream, L2 flushed between steps, the lanes' results checked
    against the sequential ones. Leaf size and surface order come from the accuracy-targeted
    autotuner (kifmm_tune, target args.batch_target against the direct sum), run once per
    pressure on the first field of that pressure, mixed form. Plans pad each grid with
    zero-weight cells to a multiple of 8 cells per axis under the root at the grid's corner
    (kifmm_opts.pad_lattice), so that every field runs the lattice paths; the rate counts the
    fields' own points only."""
    import torch
    from paper_2006_03515_gb300 import kifmm
    from paper_2006_03515_gb300 import workloads as W
    fields = []
    for k in range(args.batch_fields):
        pts, h, I, p = W.two_channel_field(k)
        n = round(len(pts) ** (1 / 3))
        fields.append((torch.as_tensor(pts, device=dev), float(h[0]), torch.as_tensor(I, device=dev), p, n))
    Is = [f[2] for f in fields]
    Cs = [kifmm.scale_c(f[3]) for f in fields]
    npts = sum(int(x.shape[0]) for x in Is)
    steps = max(3, min(args.steps, 5))
    out = {"fields": len(fields), "points": npts, "sizes": [f[4] for f in fields],
           "pressures_torr": [f[3] for f in fields], "capture": True, "target": args.batch_target}
    # autotuner, once per pressure
    t0 = time.perf_counter()
    tuned = {}
    for f in fields:
        if f[3] in tuned:
            continue
        a, b = kifmm.absorption(0.2 * f[3])
        best, tab = kifmm.tune(f[0], f[1], f[2], a, b, leaf=(64,), order=(4, 6, 8), target=args.batch_target,
                               reps=2, stream=stream, pad_lattice=True)
        tuned[f[3]] = best
        out.setdefault("tuned", {})["%g Torr" % f[3]] = {"field_points": int(f[0].shape[0]), "best": best,
                                                         "candidates": tab}
    out["tune_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    plans = []
    for f in fields:
        bt = tuned[f[3]]
        plans.append(kifmm.Plan(f[0], f[1], bt["leaf"], bt["order"], *kifmm.absorption(0.2 * f[3]),
                                precision="mixed", stream=stream, pad_lattice=True))
    torch.cuda.synchronize(dev)
    out["plan_s"] = time.perf_counter() - t0
    infos = [pl.info() for pl in plans]
    out["lattice_fields"] = sum(1 for inf in infos if inf["near_tensor"])
    out["padding_cells"] = sum(inf["n_padding"] for inf in infos)

    def timed(lanes):
        Ss = [torch.empty_like(x) for x in Is]
        for _ in range(3):
            kifmm.eval_batch(plans, Is, Ss, C=Cs, capture=True, lanes=lanes)
        ms = []
        for k in range(steps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            kifmm.eval_batch(plans, Is, Ss, C=Cs, capture=True, lanes=lanes)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        for pl in plans:
            pl.check()
        t = statistics.median(ms)
        return {"ms": t, "points_per_s": npts / (1e-3 * t)}, Ss

    out["lanes1"], s1 = timed(1)
    key = "lanes%d" % args.batch_lanes
    out[key], sl = timed(args.batch_lanes)
    diffs = [float(torch.linalg.norm(x - y) / torch.linalg.norm(y)) for x, y in zip(sl, s1)]
    out["lanes_match_sequential"] = bool(all(d <= 1e-12 for d in diffs))
    out["lanes_max_rel_diff"] = max(diffs)   # (0: every field bit-identical to its sequential result)
    out["speedup_lanes"] = out["lanes1"]["ms"] / out[key]["ms"]
    for pl in plans:
        pl.close()
    del s1, sl, plans
    torch.cuda.empty_cache()
    return out


def streamer_bench(args, dev, stream):
    """The streamer time loop of Sec. 5 (Eq. (eM)): the double-headed streamer initial condition
    (two Gaussians of 1e14 cm^-3, width 0.03 cm, at (0.22, 0.25, 0.41) and (0.28, 0.25, 0.59)
    cm) in the 0.5 x 0.5 x 1 cm gap at 52 kV, 760 Torr, p_O2 150 Torr, on n x n x 2n cubic
    cells, time step 2.5e-3 ns (the paper's), Heun's method with S_ph from the mixed-form FMM
    on a plan of the grid built once (twice per step), the Poisson equation by multigrid to a
    relative residual of 1e-8. Timed: steps after two warm-up steps (CUDA events); the FMM's
    share from the same number of stand-alone evaluations; and the local evaluation (S_ph over
    the central sub-box of half the gap's width and 0.6 of its height, sources above 1e-4 of
    the largest)."""
    import numpy as np
    import torch
    from paper_2006_03515_gb300 import kifmm
    n = args.sd_n
    nx, ny, nz, h = n, n, 2 * n, 0.5 / n
    g = [(np.arange(m) + 0.5) * h for m in (nx, ny, nz)]
    zz, yy, xx = np.meshgrid(g[2], g[1], g[0], indexing="ij")
    pts = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    c = pts.reshape(nz, ny, nx, 3)

    def gauss(x0):
        return np.exp(-((c - np.asarray(x0)) ** 2).sum(-1) / 0.03 ** 2)
    n0 = torch.as_tensor(1e14 * (gauss((0.22, 0.25, 0.41)) + gauss((0.28, 0.25, 0.59))), device=dev)
    a, b = kifmm.absorption(150.0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"grid": [nx, ny, nz], "cells": nx * ny * nz, "h_cm": h, "dt_ns": 2.5e-3, "steps": args.sd_steps,
           "photo": "mixed KIFMM, m0 6, leaf 64, lattice-padded plan, twice per step"}

    def run(plan, region=None, threshold=0.0, Si_eval=None):
        kw = {} if region is None else {"region": region}
        sd = kifmm.Streamer(nx, ny, nz, h, plan=plan, stream=stream, threshold=threshold, **kw)
        sd.set(n0, n0)
        sd.step(2.5e-12, 2)
        stream.synchronize()
        e0.record(stream)
        sd.step(2.5e-12, args.sd_steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / args.sd_steps
        if plan is not None and region is None:   # one more step: the profiled range (ncu --profile-from-start off)
            torch.cuda.profiler.start()
            sd.step(2.5e-12, 1)
            stream.synchronize()
            torch.cuda.profiler.stop()
        inf = sd.info()
        ne, npi, _, _ = sd.get()
        ok = bool(torch.isfinite(ne).all() and torch.isfinite(npi).all())
        sd.close()
        return {"ms_per_step": ms, "cells_per_s": nx * ny * nz / (ms * 1e-3), "mg_levels": inf["mg_levels"],
                "mg_cycles_last": inf["last_cycles"], "mg_residual_last": inf["last_residual"], "finite": ok}

    t0 = time.perf_counter()
    plan = kifmm.Plan(torch.as_tensor(pts, device=dev), h, 64, 6, a, b, precision="mixed", stream=stream,
                      pad_lattice=True)
    stream.synchronize()
    out["plan_s"] = time.perf_counter() - t0
    out["full"] = run(plan)
    # the FMM's share: two evaluations per step, timed alone on the same plan
    Si = torch.rand(nx * ny * nz, dtype=torch.float64, device=dev)
    S = torch.empty_like(Si)
    for _ in range(2):
        plan.eval(Si, S)
    e0.record(stream)
    for _ in range(2 * args.sd_steps):
        plan.eval(Si, S)
    e1.record(stream)
    e1.synchronize()
    out["fmm_ms_per_step"] = e0.elapsed_time(e1) / args.sd_steps
    out["fmm_share"] = out["fmm_ms_per_step"] / out["full"]["ms_per_step"]
    plan.close()
    # local evaluation over the central sub-box
    reg = (nx // 4, 3 * nx // 4, ny // 4, 3 * ny // 4, int(0.2 * nz), int(0.8 * nz))
    rp = pts.reshape(nz, ny, nx, 3)[reg[4]:reg[5], reg[2]:reg[3], reg[0]:reg[1]].reshape(-1, 3)
    lplan = kifmm.Plan(torch.as_tensor(rp, device=dev), h, 64, 6, a, b, precision="mixed", stream=stream,
                       pad_lattice=True)
    out["local"] = run(lplan, region=reg, threshold=1e-4)
    out["local"]["region"] = list(reg)
    lplan.close()
    out["none"] = run(None)   # without photoionization: the transport and Poisson alone
    torch.cuda.empty_cache()
    return out


def surrogate_bench(args, dev, stream, peaks):
    """The learned surrogate on the n^3 grid (width 32, 12 modes, 4 layers, projection 64,
    BF16 spectral weights): amplitude-normalised linear form (u = I / max I, S = C max I y),
    exact near part up to 7 cells, period 1.5 n; labels from the GPU KIFMM (surfaces at
    1.05 / 2.95 r, mixed form). Two models are trained for the same budget: one started at the
    far part's Fourier multiplier, one from a random start. Held-out fields: their rel-L2
    against the KIFMM labels, and photo_solve's judged error and fallback at 1e-2; time per
    field of the batched forward pass (batch 32) and of photo_solve, against kifmm_eval per
    field on the same grid (one field, and 8 fields as one captured batch on 8 lanes), and of
    photo_solve_batch over 32 held-out fields (one forward pass, 32 judges)."""
    import numpy as np
    import torch
    from paper_2006_03515_gb300 import kifmm, surrogate
    from paper_2006_03515_gb300 import workloads as W
    n, width, modes, layers, proj, B = args.sno_n, 32, 12, 4, 64, args.sno_batch
    modes = min(modes, n // 2)
    plan, pts, C = surrogate.grid_plan(n, leaf=64, m0=6, p_torr=760.0, p_o2=150.0, stream=stream,
                                       surface_radii=(1.05, 2.95))
    fmm, _, _ = surrogate.grid_plan(n, leaf=64, m0=6, p_torr=760.0, p_o2=150.0, stream=stream)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    U, T = surrogate.make_dataset(plan, pts, C, count=args.sno_fields, seed=2006)
    Uh, Th = surrogate.make_dataset(plan, pts, C, count=args.sno_heldout, seed=100000)
    torch.cuda.synchronize(dev)
    gen_s = time.perf_counter() - t0
    out = {"grid": "%d^3" % n, "width": width, "modes": modes, "layers": layers, "proj": proj,
           "weights": "BF16 spectral (FP32 master), FP32 accumulation", "near_part_cells": [3.0, 7.0],
           "period": (3 * n) // 2, "train_fields": args.sno_fields, "heldout_fields": args.sno_heldout,
           "labels": "GPU KIFMM, mixed, m0 6, leaf 64, surfaces 1.05 / 2.95 r", "datagen_s": gen_s}

    tb = min(8, B)   # training and held-out batches (within the model's batch)

    def held(M):
        e = np.array(surrogate.rel_errors(M, Uh, Th, batch=tb))
        return {"mean": float(e.mean()), "p90": float(np.percentile(e, 90)), "max": float(e.max())}

    def train(M, budget, lr):
        t1 = time.perf_counter()
        steps, hist = 0, []
        while time.perf_counter() - t1 < budget:
            hist += surrogate.train(M, U, T, steps=20, batch=tb, lr=lr, seed=steps)
            steps += 20
        torch.cuda.synchronize(dev)
        return {"steps": steps, "s": time.perf_counter() - t1, "fields_per_s": tb * steps / (time.perf_counter() - t1),
                "loss_first": float(np.mean(hist[:5])), "loss_last": float(np.mean(hist[-5:]))}

    # random start, trained for the budget
    M = kifmm.SNO(n, width, modes, layers, proj, max_batch=B, stream=stream)
    surrogate.configure(M, plan)
    M.init_params(seed=1)
    out["random_init"] = {"lr": 1e-3, "train": train(M, args.sno_train_s, 1e-3), "heldout_rel_l2_vs_kifmm": held(M)}
    # far-part start, trained for the same budget: the model kept
    surrogate.init_far(M, seed=1)
    out["far_init"] = {"untrained": held(M)}
    out["far_init"]["lr"] = args.sno_lr
    out["far_init"]["train"] = train(M, args.sno_train_s, args.sno_lr)
    ho = held(M)
    out["far_init"]["heldout_rel_l2_vs_kifmm"] = ho
    out["heldout_rel_l2_vs_kifmm"] = ho["mean"]
    out["heldout_rel_l2_vs_kifmm_max"] = ho["max"]
    # judged surrogate-first solves on the held-out fields (the FMM plan of the time loop)
    S = torch.empty(n ** 3, dtype=torch.float64, device=dev)
    fbs, errs = [], []
    for k in range(args.sno_heldout):
        I = torch.as_tensor(W.surrogate_field(pts, 100000 * 1000003 + k), device=dev)
        _, fb, e = kifmm.photo_solve(fmm, M, I, S, C=C, tol=1e-2, k_samples=256, seed=k + 1)
        fbs.append(fb)
        errs.append(e)
    out["photo_solve"] = {"tol": 1e-2, "k_samples": 256, "fallback_rate": float(np.mean(fbs)),
                          "judged_rel_l2_mean": float(np.mean(errs)), "judged_rel_l2_max": float(np.max(errs))}
    # timings: batched forward, photo_solve per field, kifmm_eval per field (one field; a batch)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ub = Uh[:B].contiguous() if Uh.shape[0] >= B else U[:B].contiguous()
    yb = torch.empty_like(ub)
    for _ in range(3):
        M.forward(ub, yb)
    torch.cuda.synchronize(dev)
    torch.cuda.profiler.start()         # the timed forward passes are the profiled range
    e0.record(stream)
    reps = 5
    for _ in range(reps):
        M.forward(ub, yb)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.profiler.stop()
    fwd_ms = e0.elapsed_time(e1) / reps
    I = torch.as_tensor(W.surrogate_field(pts, 7), device=dev)
    for _ in range(2):
        kifmm.photo_solve(fmm, M, I, S, C=C, tol=1e-2)
    e0.record(stream)
    for _ in range(reps):
        kifmm.photo_solve(fmm, M, I, S, C=C, tol=1e-2)
    e1.record(stream)
    e1.synchronize()
    ps_ms = e0.elapsed_time(e1) / reps
    # batched surrogate-first solves: B held-out fields on B plans of the grid (judge at 256 targets)
    bplans = [fmm] + [surrogate.grid_plan(n, leaf=64, m0=6, p_torr=760.0, p_o2=150.0, stream=stream)[0]
                      for _ in range(B - 1)]
    bIs = [torch.as_tensor(W.surrogate_field(pts, 100000 * 1000003 + k), device=dev) for k in range(B)]
    bSs = [torch.empty_like(x) for x in bIs]
    for _ in range(2):
        kifmm.photo_solve_batch(bplans, M, bIs, bSs, C=[C] * B, tol=1e-2, k_samples=256, seed=1)
    e0.record(stream)
    for _ in range(reps):
        _, bfb, berr = kifmm.photo_solve_batch(bplans, M, bIs, bSs, C=[C] * B, tol=1e-2, k_samples=256, seed=1)
    e1.record(stream)
    e1.synchronize()
    psb_ms = e0.elapsed_time(e1) / reps / B
    for pl in bplans[1:]:
        pl.close()
    del bIs, bSs
    for _ in range(2):
        fmm.eval(I, S, C=C)
    e0.record(stream)
    for _ in range(reps):
        fmm.eval(I, S, C=C)
    e1.record(stream)
    e1.synchronize()
    fmm_ms = e0.elapsed_time(e1) / reps
    plans = [fmm] + [surrogate.grid_plan(n, leaf=64, m0=6, p_torr=760.0, p_o2=150.0, stream=stream)[0]
                     for _ in range(7)]
    Is = [I.clone() for _ in plans]
    Ss = [torch.empty_like(I) for _ in plans]
    for _ in range(3):
        kifmm.eval_batch(plans, Is, Ss, C=[C] * 8, capture=True, lanes=8)
    e0.record(stream)
    for _ in range(reps):
        kifmm.eval_batch(plans, Is, Ss, C=[C] * 8, capture=True, lanes=8)
    e1.record(stream)
    e1.synchronize()
    fmm_b_ms = e0.elapsed_time(e1) / reps / 8
    n3 = n ** 3
    K = (2 * modes) * (2 * modes) * modes
    alg_bytes = 4.0 * B * n3 * (2 + width * (2 + 2 * layers)) + layers * 2 * K * width * width * 2
    hbm = peaks.get("hbm_gbs", 6686.0)
    fwd_gbs = alg_bytes / (fwd_ms * 1e-3) / 1e9
    out.update({"forward_ms_batch32": fwd_ms, "forward_ms_per_field": fwd_ms / B,
                "photo_solve_ms_per_field": ps_ms, "kifmm_eval_ms_per_field": fmm_ms,
                "photo_solve_batch32_ms_per_field": psb_ms,
                "photo_solve_batch32_fallbacks": int(sum(bfb)), "photo_solve_batch32_judged_max": float(max(berr)),
                "kifmm_eval_batch8_ms_per_field": fmm_b_ms,
                "points_per_s": B * n3 / (fwd_ms * 1e-3), "params": M.num_params(),
                "roofline": {"bound": "hbm", "achieved": fwd_gbs, "peak": hbm, "unit": "GB/s", "frac": fwd_gbs / hbm,
                             "traffic": None, "algorithmic_bytes": alg_bytes}})
    for pl in plans:
        pl.close()
    M.close()
    plan.close()
    del U, T, Uh, Th
    torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.streamer_only:
        import torch
        from paper_2006_03515_gb300 import build as pb
        pb.build()
        dev = torch.device("cuda", 0)
        stream = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(stream):
            rec = streamer_bench(args, dev, stream)
        print(json.dumps({"streamer": rec}), flush=True)
        return 0
    if args.surrogate_only:
        import torch
        from paper_2006_03515_gb300 import build as pb
        pb.build()
        dev = torch.device("cuda", 0)
        stream = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(stream):
            rec = surrogate_bench(args, dev, stream, measured_peaks())
        print(json.dumps({"surrogate": rec}), flush=True)
        return 0
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2006_03515_gb300 import build as pb
    from paper_2006_03515_gb300 import kifmm, workloads
    pb.build()
    os.environ["KIFMM_TIMING"] = "1"

    p_o2 = 0.2 * args.p
    a, b = kifmm.absorption(p_o2)
    C = kifmm.scale_c(args.p)
    pts, h, I = workloads.config_uniform(args.n)
    npts = len(pts)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        dpts = torch.as_tensor(pts, device=dev)
        dI = torch.as_tensor(I, device=dev)
        S = torch.empty_like(dI)
        t0 = time.perf_counter()
        plan = kifmm.Plan(dpts, float(h[0]), args.leaf, args.m0, a, b, precision=args.precision, stream=stream,
                          repr=args.repr)
        torch.cuda.synchronize(dev)
        plan_s = time.perf_counter() - t0
        info = plan.info()
        gate = None
        fp64 = None
        if not args.no_fp64 and args.precision == "mixed":
            p64 = kifmm.Plan(dpts, float(h[0]), args.leaf, args.m0, a, b, precision="fp64", stream=stream,
                             repr=args.repr)
            S64 = p64.eval(dI, C=C)
            plan.eval(dI, S, C=C)
            torch.cuda.synchronize(dev)
            gate = float(torch.linalg.norm(S - S64) / torch.linalg.norm(S64))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t64 = []
            for _ in range(2):
                e0.record(stream)
                p64.eval(dI, S64, C=C)
                e1.record(stream)
                e1.synchronize()
                t64.append(e0.elapsed_time(e1))
            fp64 = {"points_per_s": npts / (1e-3 * min(t64)), "ms": min(t64)}
            p64.close()
            del S64
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        for _ in range(args.warmup):
            plan.eval(dI, S, C=C)
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.25)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        phase_sum = None
        torch.cuda.synchronize(dev)
        torch.cuda.profiler.start()         # the timed region is the profiled range (ncu --profile-from-start off)
        for k in range(args.steps):
            flush.fill_(float(k))           # L2 flush between timed steps (outside the events)
            starts[k].record(stream)
            plan.eval(dI, S, C=C)
            ends[k].record(stream)
            ends[k].synchronize()
            ph = plan.phase_times()
            phase_sum = ph if phase_sum is None else [x + y for x, y in zip(phase_sum, ph)]
        torch.cuda.synchronize(dev)
        torch.cuda.profiler.stop()
        clk = clocks.stop()
        launches_per_step = plan.info()["eval_launches"]
        step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        ms = max_over_ranks(sum(step_ms) / len(step_ms), ws)
        value = whole_job_rate(npts, ws, ms)

        # end to end through the public API with host buffers (pinned), copies inside the timed region
        hI = torch.empty(npts, dtype=torch.float64, pin_memory=True)
        hS = torch.empty(npts, dtype=torch.float64, pin_memory=True)
        hI.copy_(torch.as_tensor(I))
        hIn, hSn = hI.numpy(), hS.numpy()
        e2e_ms = []
        for k in range(max(3, args.steps // 2) + 2):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            plan.eval_host(hIn, hSn, C=C)
            e1.record(stream)
            e1.synchronize()
            if k >= 2:
                e2e_ms.append(e0.elapsed_time(e1))
        e2e_val = whole_job_rate(npts, ws, max_over_ranks(sum(e2e_ms) / len(e2e_ms), ws))
        e2e_ok = bool(np.allclose(hSn, S.cpu().numpy(), rtol=1e-12, atol=0))   # split partial sums add atomically

        # the lattice near field alone: its sums overlap the far field on their own stream in
        # the timed plan, so its roofline is timed on a plan that keeps them on the plan's stream
        near_alone_ms = None
        if info.get("near_tensor"):
            os.environ["KIFMM_NEAR_STREAM"] = "same"
            try:
                pn = kifmm.Plan(dpts, float(h[0]), args.leaf, args.m0, a, b, precision=args.precision,
                                stream=stream, repr=args.repr)
            finally:
                del os.environ["KIFMM_NEAR_STREAM"]
            for _ in range(2):
                pn.eval(dI, S, C=C)
            acc = []
            for k in range(5):
                flush.fill_(float(k))
                pn.eval(dI, S, C=C)
                torch.cuda.synchronize(dev)
                acc.append(pn.phase_times()[6])
            near_alone_ms = sum(acc) / len(acc)
            pn.close()

    # (an eighth entry: the near sums' span on their own stream, overlapping the far field;
    # P2P is then the join and the output combination)
    phases = ["scatter", "S2M", "M2M+UC2UE", "M2L", "S2L+L2L+DC2DE", "L2P+M2P", "P2P", "near sums (own stream)"]
    ph_ms = {k: v / args.steps for k, v in zip(phases, phase_sum)}
    near_ms = near_alone_ms if near_alone_ms else ph_ms["P2P"] + ph_ms.get("near sums (own stream)", 0.0)
    dom = max((k for k in ph_ms if k != "near sums (own stream)"), key=ph_ms.get)
    peaks = measured_peaks()
    sm_clk = 2070.0
    # rooflines of the three heavy kernels; the dominant one is "roofline"
    p2p_ach = info["p2p_pairs"] / (ph_ms["P2P"] * 1e-3) / 1e9
    if clk.get("sm_mhz"):
        sm_clk = float(clk["sm_mhz"])
    p2p_peak = SM_COUNT * PAIRS_PER_SM_CLK * sm_clk * 1e6 / 1e9
    std = (args.n == 128 and args.m0 == 6 and args.leaf == 64 and args.p == 760.0 and args.precision == "mixed"
           and args.repr == "surface")
    f16_peak = peaks.get("bf16_tflops", 1947.8)   # dense FP16 and BF16 share the tensor rate
    m2l_ach = info["m2l_flops"] / (ph_ms["M2L"] * 1e-3) / 1e12
    up_ach = info["upward_flops"] / (ph_ms["M2M+UC2UE"] * 1e-3) / 1e12
    up_mma = info.get("upward_mma_flops", 0.0) / (ph_ms["M2M+UC2UE"] * 1e-3) / 1e12
    roofs = {
        "P2P": {"kernel": "k_p2p_mixed (near-field pair sum, FP32)", "bound": "alu", "achieved": p2p_ach,
                "peak": p2p_peak, "unit": "Gpair/s", "frac": p2p_ach / p2p_peak,
                "traffic": profiled_traffic("P2P", npts, std),
                "peak_source": "derived from measured MUFU rates: 152 SMs x 1/(2/30.2 + 1/15.2) pairs/clk x "
                               "median SM clock under load"},
        "M2L": {"kernel": "k_m2l_tc (tcgen05 kind::f16, 3-term FP16 split with power-of-two scaling, "
                          "coefficient basis)", "bound": "tensor", "achieved": m2l_ach,
                "peak": f16_peak / 3.0, "unit": "TFLOP/s", "frac": m2l_ach / (f16_peak / 3.0),
                "traffic": profiled_traffic("M2L", npts, std),
                "peak_source": "of measured: bf16_tflops (dense FP16 = BF16 rate) / 3 MMAs per product"},
        "upward": ({"kernel": "k_pinv_oz (UC2UE pseudo-inverse c = Sigma^+ U^T chk to FP64 accuracy by exact "
                             "6-bit integer slices on the FP16 tensor cores; the phase also holds the slicing and the "
                             "FP32 M2M translations)", "bound": "tensor", "achieved": up_mma, "peak": f16_peak,
                   "unit": "TFLOP/s", "frac": up_mma / f16_peak, "traffic": None, "fp64_equivalent_tflops": up_ach,
                   "peak_source": "of measured: bf16_tflops (dense FP16 = BF16 rate); achieved = executed slice-product "
                                  "flop over the whole upward phase"}
                   if info.get("upward_mma_flops", 0.0) > 0 else
                   {"kernel": "k_apply<double> (UC2UE pseudo-inverse on the FP64 pipe)", "bound": "alu",
                    "achieved": up_ach, "peak": FP64_TFLOPS, "unit": "TFLOP/s", "frac": up_ach / FP64_TFLOPS,
                    "traffic": None, "peak_source": "GB300 FP64 nominal 1.25 TFLOP/s"}),
    }
    if info.get("near_tensor"):   # uniform lattice: near field as 27 per-offset matrices on the tensor cores
        nf_ach = 2.0 * info["p2p_pairs"] / (near_ms * 1e-3) / 1e12
        roofs["P2P"] = {"kernel": "k_m2l_tc on the 27 near-offset kernel matrices (R = 64 cells per leaf; timed "
                                  "on a plan that runs the weight split, the contraction and the output "
                                  "combination on its own stream, not overlapping the far field)",
                        "bound": "tensor", "achieved": nf_ach, "peak": f16_peak / 3.0, "unit": "TFLOP/s",
                        "frac": nf_ach / (f16_peak / 3.0), "traffic": profiled_traffic("NEAR", npts, std),
                        "pairs_per_s": info["p2p_pairs"] / (near_ms * 1e-3),
                        "ms": near_ms,
                        "peak_source": "of measured: bf16_tflops (dense FP16 = BF16 rate) / 3 MMAs per product; "
                                       "achieved = 2 flop per near pair over the whole near-field phase"}
    if not info["m2l_tensor"]:   # SIMT M2L (FP64 form, or a coefficient count the tensor path does not take)
        fp_peak = (SM_COUNT * 128 * 2 * sm_clk * 1e6 / 1e12 if args.precision == "mixed" else FP64_TFLOPS)
        roofs["M2L"] = {"kernel": "k_m2l (SIMT, %s)" % ("FP32" if args.precision == "mixed" else "FP64"),
                        "bound": "alu", "achieved": m2l_ach, "peak": fp_peak, "unit": "TFLOP/s",
                        "frac": m2l_ach / fp_peak, "traffic": None,
                        "peak_source": ("152 SMs x 128 FP32 FMA lanes x 2 x median SM clock under load"
                                        if args.precision == "mixed" else "GB300 FP64 nominal 1.25 TFLOP/s")}
    key = "P2P" if dom == "P2P" else ("M2L" if dom == "M2L" else "upward")
    roof = dict(roofs[key])
    gpu_launches = launches_per_step * args.steps
    line = {"metric": METRIC, "value": value, "unit": "points/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": workload_name(args),
                       "n_points": npts, "l2": "512 MB buffer written between timed steps",
                       "parallelism": "replicas" if ws > 1 else "single"},
            "gate_rel_l2_mixed_vs_fp64": gate, "fp64": fp64, "plan_s": plan_s,
            "phase_ms": ph_ms, "roofline": roof, "rooflines": roofs, "clocks": clk, "gpu_launches": gpu_launches,
            "e2e": {"value": e2e_val, "unit": "points/s", "h2d_bytes_per_step": npts * 8,
                    "d2h_bytes_per_step": npts * 8, "matches_device_result": e2e_ok}}
    if std:   # the headline form's own accuracy against the whole discrete sum (oracle FFT convolution)
        try:
            from oracle import direct as D
            ref = D.fft_uniform(I.reshape(args.n, args.n, args.n), float(h[0]), a, b, C).ravel()
            got = S.cpu().numpy()
            line["rel_l2_vs_direct_sum"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
            del ref, got
        except Exception as exc:
            line["rel_l2_vs_direct_sum"] = {"error": "%s: %s" % (type(exc).__name__, exc)}
    if not args.no_configs and std:
        try:
            with torch.cuda.stream(stream):
                line["configs"] = configs_bench(args, dev, stream, flush)
        except Exception as exc:    # the headline line is printed whatever happens here
            line["configs"] = {"error": "%s: %s" % (type(exc).__name__, exc)}
    if not args.no_cheb and args.repr == "surface":
        try:
            with torch.cuda.stream(stream):
                line["cheb"] = cheb_bench(args, dev, stream, dpts, float(h[0]), dI, C, a, b, flush, peaks)
        except Exception as exc:    # the headline line is printed whatever happens here
            line["cheb"] = {"error": "%s: %s" % (type(exc).__name__, exc)}
    if not args.no_radii and args.repr == "surface":
        try:
            with torch.cuda.stream(stream):
                line["radii"] = radii_bench(args, dev, stream, dpts, float(h[0]), dI, C, a, b, flush, peaks)
        except Exception as exc:    # the headline line is printed whatever happens here
            line["radii"] = {"error": "%s: %s" % (type(exc).__name__, exc)}
    if not args.no_batch and args.repr == "surface":
        try:
            with torch.cuda.stream(stream):
                line["batch"] = batch_bench(args, dev, stream, flush)
        except Exception as exc:    # the headline line is printed whatever happens here
            line["batch"] = {"error": "%s: %s" % (type(exc).__name__, exc)}
    if not args.no_surrogate:
        try:
            with torch.cuda.stream(stream):
                line["surrogate"] = surrogate_bench(args, dev, stream, peaks)
        except Exception as exc:    # the headline line is printed whatever happens here
            line["surrogate"] = {"error": "%s: %s" % (type(exc).__name__, exc)}
    if not args.no_streamer:
        try:
            with torch.cuda.stream(stream):
                line["streamer"] = streamer_bench(args, dev, stream)
        except Exception as exc:    # the headline line is printed whatever happens here
            line["streamer"] = {"error": "%s: %s" % (type(exc).__name__, exc)}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from oracle import build as ob
        ob.build()
        v, cores, dt = cpu_sample(args.cpu_n, args.m0, args.leaf, a, b, C)
        line["cpu_baseline"] = {"value": v, "unit": "points/s", "cores": cores, "kind": "oracle",
                                "sample": "oracle KIFMM evaluation (FP64, numpy + C/OpenMP) of a %d^3 sample of "
                                          "the workload (%.1f s); plan excluded" % (args.cpu_n, dt)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
