#!/usr/bin/env python
"""Throughput of generalized Nystrom (GN) on one GB300 per rank.

Workload: A = W1 diag(i^-2) W2^T + 1e-8 N (2000 modes), 32768 x 16384, sketch
sizes r = 1000, l = 500 (Gaussian X, Y), the mixed-precision path: A, X, Y in
BF16 (tensor-core sketch, FP32 accumulation), FP64 core.  One step = one
approximation in the paper's output form (Algorithm 2 and the text after it:
AX, Y^T A, Q, R): the sketch launch, the core product C = (Y^T A) X on the
tensor cores (three bf16 slices of Y^T A), Householder QR of C in FP64 and the
Section 5.1.2 detector / Section 5.1.1 truncation (mode AUTO).

Steps run on --inflight handles (default 5), each with its own CUDA stream,
workspace and outputs: step i's core is enqueued without a host wait
(GN_CORE_DEFER) and finished once the next steps are enqueued, so one step's
latency-bound FP64 core overlaps the following steps' sketches and cores.  The K
steps are timed --reps times (default 3), each repetition exactly K steps between
a barrier and device synchronizations; the median repetition is the value and
all of them are in the line.  The latency of a single approximation (one in
flight) is reported beside it.

Prints ONE JSON line (rank 0).  Also reported, outside the timed region: the
measured FP8 (e4m3) and FP64 peaks, the split-BF16 and e4m3 paths, the plain
FP64 GPU path, the error of each precision against the FP64 GPU path on the
same quantized sketches (and on the same stored A), factor formation, the
20000 x 10000 and 1000 x 500 FP64 cases with HMT beside GN, the Section 6
sketch-state operations, r = 2000, the adjoint, the batched path, and the FP64
CPU oracle timed on one whole approximation of the same matrix.

--impl reference times the FP64 CPU oracle alone (the reference arm): every
timed step is one whole approximation of the full matrix.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import signal
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import gn_synth  # noqa: E402

METRIC = "GN approximations/s (32768x16384, r=1000, l=500, BF16 tensor-core sketch + FP64 core)"
UNIT = "approximations/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gn", choices=["gn", "reference"])
    ap.add_argument("--m", "--rows", type=int, default=32768)
    ap.add_argument("--n", "--cols", type=int, default=16384)
    ap.add_argument("--r", "--sketch-r", type=int, default=1000,
                    help="r (l = r / 2); --rows, --cols, --sketch-r: spellings that launchers do not take for their own options")
    ap.add_argument("--inflight", type=int, default=5, help="approximations in flight (handles / streams)")
    ap.add_argument("--no-extras", action="store_true", help="skip the side measurements and the CPU baseline")
    ap.add_argument("--op", default="bf16", choices=["bf16", "e4m3"],
                    help="sketch operand type of the timed step (e4m3: per-128x128-tile scales)")
    ap.add_argument("--prio", type=int, default=0,
                    help="stream priority of the approximations' streams (0 default, -1 high)")
    ap.add_argument("--h2d-streams", type=int, default=1, help="host-to-device copy streams of the e2e loop")
    ap.add_argument("--e2e-sets", type=int, default=0, help="device buffer sets of the e2e loop (0: in-flight + ahead)")
    ap.add_argument("--e2e-ahead", type=int, default=2, help="steps whose input copies are queued ahead in the e2e loop")
    ap.add_argument("--e2e-reps", type=int, default=5, help="timed repetitions of the e2e loop (the median is reported)")
    ap.add_argument("--reps", type=int, default=3, help="timed repetitions of the K steps (the median is reported)")
    ap.add_argument("--only", default=None, choices=["batched", "adjoint", "fp64_cases"],
                    help="run one side measurement alone and print its JSON (for profiling it)")
    return ap.parse_args()


def config_dict(a, precision=None):
    precision = precision or getattr(a, "op", "bf16")
    return {
        "workload": f"GN dense {a.m}x{a.n} low-rank+noise (i^-2, 2000 modes, 1e-8 noise), r={a.r}, "
                    f"l={a.r // 2}, Gaussian sketches, {precision} operands, FP64 core, mode AUTO",
        "m": a.m, "n": a.n, "r": a.r, "l": a.r // 2,
        "inflight": getattr(a, "inflight", 1),
        "l2": "inputs larger than L2 (A alone is %.2f GB in BF16)" % (2.0 * a.m * a.n / 1e9),
        "parallelism": "replicas" if a.gpus > 1 else "single GPU",
    }


# --------------------------------------------------------------------------- peaks
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _best_ms(fn, reps, stream):
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def measure_dtype_peaks(dev, stream):
    """The FP8 (e4m3, per-tensor scales, cuBLASLt through torch._scaled_mm) and
    FP64 (torch.matmul) peaks on this GPU, measured the way MEASURED_PEAKS.json
    measures BF16: best of several CUDA-event timed square products."""
    out = {}
    with torch.cuda.stream(stream):
        try:
            n = 8192
            a = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn)
            b = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn).t()
            one = torch.tensor(1.0, device=dev)
            f = lambda: torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
            f()
            ms = _best_ms(f, 10, stream)
            out["e4m3_tflops"] = 2.0 * n ** 3 / (ms / 1e3) / 1e12
            out["e4m3_how"] = "torch._scaled_mm e4m3 8192^3, per-tensor scales, bf16 out, best of 10"
            del a, b
        except Exception as ex:  # pragma: no cover
            out["e4m3_tflops"] = None
            out["e4m3_how"] = f"not measured: {type(ex).__name__}: {ex}"
        n = 4096
        a = torch.randn(n, n, device=dev, dtype=torch.float64)
        b = torch.randn(n, n, device=dev, dtype=torch.float64)
        f = lambda: torch.matmul(a, b)
        f()
        ms = _best_ms(f, 4, stream)
        out["fp64_tflops"] = 2.0 * n ** 3 / (ms / 1e3) / 1e12
        out["fp64_how"] = "torch.matmul float64 4096^3, best of 4"
        del a, b
    torch.cuda.synchronize()
    return out


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if "Active" in v and "Not" not in v:
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_id_for_smi(local_rank):
    try:
        u = torch.cuda.get_device_properties(local_rank).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            return vis.split(",")[local_rank]
        return local_rank


# --------------------------------------------------------------------------- CPU oracle
def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count()


def oracle_step(A, X, Y, r):
    """One whole approximation by the FP64 CPU oracle (sketch of the full A,
    then the core: C, Householder QR, detector, truncation); returns seconds
    and the split."""
    from oracle import gn_oracle as O
    t0 = time.perf_counter()
    AX, YtA = O.sketch(A, X, Y)
    t1 = time.perf_counter()
    O.core(YtA, X, 10 * 2.0 ** -53, O.AUTO, eps_relative=True, diag_iters=6)
    t2 = time.perf_counter()
    return t2 - t0, t1 - t0, t2 - t1


def run_reference(a, rank, world):
    """The reference arm: the FP64 CPU oracle on the host cores.  Each timed
    step is one whole approximation of the full 32768 x 16384 matrix; the
    warm-up steps (nothing to compile or cache) run the oracle on a 512-row
    block so that the whole run stays within a few minutes."""
    if rank != 0:
        return
    from oracle import gn_oracle as O
    l = a.r // 2
    p = gn_synth.config3(r=a.r, m=a.m, n=a.n)
    A, X, Y = p.a.numpy(), p.x.numpy(), p.y.numpy()
    del p
    for _ in range(a.warmup):
        O.sketch(A[:512], X, Y[:512])
    times, splits = [], []
    t_all0 = time.perf_counter()
    for _ in range(a.steps):
        t, ts, tc = oracle_step(A, X, Y, a.r)
        times.append(t)
        splits.append((ts, tc))
    wall = time.perf_counter() - t_all0
    per = wall / a.steps
    v = 1.0 / per
    desc = (f"FP64 numpy oracle, one whole approximation per step on the full {a.m}x{a.n} matrix "
            f"(sketch {statistics.mean(s for s, _ in splits):.2f}s + {a.r + l}x{a.r} core "
            f"{statistics.mean(c for _, c in splits):.2f}s)")
    line = {
        "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "impl": "reference", "config": config_dict(a),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": blas_threads(), "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- GPU arm
def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
        backend = "nccl" if (a.impl == "gn" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    if a.impl == "reference":
        run_reference(a, rank, world)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    import paper_2009_11392_gb300 as gn

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if a.only:
        stream = torch.cuda.Stream(device=dev)
        torch.cuda.set_stream(stream)
        H = gn.Handle(stream)
        f = {"batched": lambda: batched_measurement(gn, H, stream, dev, steps=max(3, a.steps)),
             "adjoint": lambda: adjoint_measurement(gn, H, stream, dev),
             "fp64_cases": lambda: fp64_cases(gn, H, stream, dev)}[a.only]
        print(json.dumps({"only": a.only, "result": f()}), flush=True)
        return
    m, n, r = a.m, a.n, a.r
    l = r // 2
    nf = max(1, a.inflight)
    stream = torch.cuda.Stream(device=dev, priority=a.prio)
    torch.cuda.set_stream(stream)
    H = gn.Handle(stream)
    Hs = [H] + [gn.Handle(torch.cuda.Stream(device=dev, priority=a.prio)) for _ in range(nf - 1)]

    # ---- inputs (seeded, drawn on the device; FP64)
    p = gn_synth.config3(r=r, device=dev, m=m, n=n)
    A64, X64, Y64 = p.a, p.x, p.y
    # Section 4.1's eps = 10u, with u the unit roundoff of the arithmetic that
    # forms the core (FP32 accumulation here), relative to ||C||_2.
    eps = 10 * 2.0 ** -24
    mode = gn.AUTO | gn.EPS_RELATIVE

    # ---- a1: operand quantisation (reported separately)
    q0 = torch.cuda.Event(enable_timing=True)
    q1 = torch.cuda.Event(enable_timing=True)
    q0.record(stream)
    Ab = H.quantize(A64)
    q1.record(stream)
    Xb, Yb = H.quantize(X64), H.quantize(Y64)
    if a.op == "e4m3":   # the timed step's operands; the BF16 ones serve the side measurements
        q0.record(stream)
        Aop = H.quantize_e4m3(A64)
        q1.record(stream)
        Xop, Yop = H.quantize_e4m3(X64, data=False), H.quantize_e4m3(Y64, data=False)
    else:
        Aop, Xop, Yop = Ab, Xb, Yb
    torch.cuda.synchronize()
    quantize_ms = q0.elapsed_time(q1)

    wsd = gn.E4M3 if a.op == "e4m3" else gn.BF16X2
    bufs = [(Hj.workspace(m, n, r, l, wsd), torch.empty(m, r, dtype=torch.float32, device=dev),
             torch.empty(r + l, n, dtype=torch.float32, device=dev), gn.Core.empty(r, l, dev)) for Hj in Hs]
    ws, AX, YtA, core = bufs[0]

    def run_steps(k, use, evs=None):
        """k steps on the first `use` handles; step i's core is finished after
        step i + use - 1 is enqueued."""
        pend = []
        for i in range(k):
            j = i % use
            Hj = Hs[j]
            wsj, AXj, YtAj, cj = bufs[j]
            if evs is not None:
                evs[i][0].record(Hj.stream)
            Hj.sketch(Aop, Xop, Yop, AXj, YtAj, wsj)
            if evs is not None:
                evs[i][1].record(Hj.stream)
            Hj.core(YtAj, Xop, eps, mode | gn.CORE_DEFER, cj, wsj)
            pend.append((Hj, cj))
            if len(pend) >= use:
                h_, c_ = pend.pop(0)
                h_.core_finish(c_)
        for h_, c_ in pend:
            h_.core_finish(c_)

    def timed(k, use, evs=None):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(Hs[0].stream)
        for Hj in Hs[1:use]:
            Hj.stream.wait_event(t0)
        run_steps(k, use, evs)
        for Hj in Hs[1:use]:
            Hs[0].stream.wait_stream(Hj.stream)
        t1.record(Hs[0].stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1)

    run_steps(max(a.warmup, nf), nf)
    torch.cuda.synchronize()
    for Hj in Hs:
        if Hj.sync_status() != 0:
            raise RuntimeError("device status after warm-up")

    sampler = ClockSampler(gpu_id_for_smi(local))
    sampler.start()
    time.sleep(0.3)
    # a few timed repetitions of exactly K steps each (barrier and synchronize
    # around every one, max over ranks); the median one is reported, all of them
    # are in the line: a host-side stall of tens of ms otherwise decides a
    # region of ~0.1 s
    reps = []   # (elapsed ms, launches, mean sketch ms)
    for _ in range(max(1, a.reps)):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        launches0 = gn.kernel_launches()
        el = timed(a.steps, nf, evs)
        nl = gn.kernel_launches() - launches0
        sk = statistics.mean(e0.elapsed_time(e1) for e0, e1 in evs)
        if dist:
            t = torch.tensor([el], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        reps.append((el, nl, sk))
    clocks = sampler.stop()
    for Hj in Hs:
        if Hj.sync_status() != 0:
            raise RuntimeError("device status after timed steps")
    elapsed_ms, launches, sketch_ms = sorted(reps)[len(reps) // 2]
    per_step_ms = elapsed_ms / a.steps
    value = world * a.steps / (elapsed_ms / 1e3)

    # the same loop with one approximation in flight: the latency of one
    # approximation, and the sketch launch timed alone on the device
    evs1 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    latency_ms = timed(a.steps, 1, evs1) / a.steps
    sketch_alone_ms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in evs1)

    e2e = e2e_measurement(a, gn, Hs, nf, dev, m, n, r, l, Aop, Xop, Yop, Ab, Xb, Yb, bufs, eps, mode)

    peaks, peak_kind = measured_peaks()
    flops = 2.0 * m * n * (2 * r + l)
    dpk = measure_dtype_peaks(dev, stream) if rank == 0 else {}
    if a.op == "e4m3":
        peak = dpk.get("e4m3_tflops") or 2.0 * peaks["bf16_tflops"]
        pk = "e4m3 measured in this run (torch._scaled_mm)" if dpk.get("e4m3_tflops") else \
            f"2 x bf16 burst ({peak_kind}; nominal ratio)"
    else:
        peak = peaks["bf16_tflops"]
        pk = f"bf16 burst, {peak_kind} (MEASURED_PEAKS.json); the kernel runs at full clock inside a short timed region"
    a_bytes = m * n * (1 if a.op == "e4m3" else 2)
    roof_ms = max(a_bytes / (peaks["hbm_gbs"] * 1e9), flops / (peak * 1e12)) * 1e3
    achieved = flops / (sketch_ms / 1e3) / 1e12
    achieved_alone = flops / (sketch_alone_ms / 1e3) / 1e12

    core_info = {"eps_rel": eps, "eps_abs": core.eps_abs, "c_norm_est": core.c_norm_est,
                 "k": core.k, "sgn": core.sgn, "rinv_est": core.rinv_est}
    extras = {}
    if not a.no_extras and rank == 0:
        extras = side_measurements(a, gn, H, stream, dev, A64, X64, Y64, Ab, Xb, Yb, eps, mode, ws, AX, YtA, core,
                                   peaks, dpk)

    cpu = None
    if rank == 0 and not a.no_extras:
        try:
            Ah, Xh, Yh = A64.cpu().numpy(), X64.cpu().numpy(), Y64.cpu().numpy()
            t, ts, tc = oracle_step(Ah, Xh, Yh, r)
            del Ah, Xh, Yh
            cpu = {"value": 1.0 / t, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                   "sample": f"one whole approximation of the same {m}x{n} matrix by the FP64 numpy oracle "
                             f"(sketch {ts:.2f}s + {r + l}x{r} core {tc:.2f}s), not extrapolated"}
        except Exception as ex:  # pragma: no cover
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": f"failed: {ex}"}

    # DRAM bytes per launch from the committed ncu summary, valid only while the
    # kernel source is the one the counters were taken on.
    traffic = None
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tp):
        try:
            import hashlib
            t = json.load(open(tp)).get(f"sketch_{a.op}_{m}x{n}_r{r}")
            src = open(os.path.join(ROOT, "paper_2009_11392_gb300", "csrc", "gn_tc.cu"), "rb").read()
            if t and hashlib.sha256(src).hexdigest()[:16] == t["kernel_sha256_16"]:
                traffic = t["traffic_bytes"]
        except Exception:
            traffic = None

    if rank == 0:
        line = {
            "metric": METRIC if a.op == "bf16" else METRIC.replace("BF16", "e4m3 block-scaled"),
            "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": per_step_ms, "higher_is_better": True, "scaling": "weak",
            "reps": len(reps), "statistic": "median of the timed repetitions of K steps",
            "ms_per_step_reps": [el / a.steps for el, _, _ in reps],
            "vs_baseline": None, "dtype": a.op, "data": "synthetic (seeded low-rank + noise, Gaussian sketches)",
            "config": config_dict(a),
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "tc_multigemm_kernel (AX and Y^T A in one launch)",
                         "kernel_ms": sketch_ms, "algorithmic_flops": flops, "peak_kind": pk,
                         "kernel_ms_alone": sketch_alone_ms, "frac_alone": achieved_alone / peak,
                         "frac_vs_sustained": (achieved / peaks["bf16_tflops_sustained"]) if a.op == "bf16" else None,
                         "step_roofline_ms": roof_ms, "step_frac": roof_ms / per_step_ms,
                         "step_frac_latency": roof_ms / latency_ms},
            "latency_ms": latency_ms,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "quantize_ms": quantize_ms,
            "dtype_peaks": dpk,
        }
        line.update(core_info)
        line.update(extras)
        if "factors_ms" in extras:   # sketch + core + factors F (FP64 solve) and G
            line["all_in"] = {"approx_per_s": 1e3 / (latency_ms + extras["factors_ms"]),
                              "ms": latency_ms + extras["factors_ms"], "inflight": 1}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def e2e_measurement(a, gn, Hs, nf, dev, m, n, r, l, Aop, Xop, Yop, Ab, Xb, Yb, bufs, eps, mode):
    """End to end through the API with host buffers: every step copies its own
    inputs in from pinned host memory and its results (AX, Y^T A, Q, R) out.
    nf + ahead device buffer sets; the input copies of the next `ahead` steps
    are queued on the host-to-device stream(s) and the results go out on one
    device-to-host stream while the steps compute on the nf handles."""
    ahead = max(1, a.e2e_ahead)
    nset = max(a.e2e_sets, nf + ahead)   # a set's previous step is complete before its next copy is queued
    if a.op == "e4m3":
        srcs = [Aop.data, Aop.data_t, Xop.data_t, Yop.data_t, Aop.scale, Xop.scale, Yop.scale]
        hosts = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True).copy_(t) for t in srcs]

        def make_in():
            d = [torch.empty_strided(t.shape, t.stride(), dtype=t.dtype, device=dev) for t in srcs]
            return d, (gn.E4M3Mat(m, n, d[4], d[0], d[1]), gn.E4M3Mat(n, r, d[5], None, d[2]),
                       gn.E4M3Mat(m, r + l, d[6], None, d[3]))
    else:
        srcs = [Ab, Xb, Yb]
        hosts = [torch.empty(t.shape, dtype=torch.bfloat16, pin_memory=True).copy_(t) for t in srcs]

        def make_in():
            d = [gn.padded(m, n, torch.bfloat16, dev), gn.padded(n, r, torch.bfloat16, dev),
                 gn.padded(m, r + l, torch.bfloat16, dev)]
            return d, tuple(d)
    ins = [make_in() for _ in range(nset)]
    outd = [(torch.empty(m, r, dtype=torch.float32, device=dev), torch.empty(r + l, n, dtype=torch.float32, device=dev),
             gn.Core.empty(r, l, dev)) for _ in range(nset)]
    outh = [[torch.empty(m, r, dtype=torch.float32, pin_memory=True),
             torch.empty(r + l, n, dtype=torch.float32, pin_memory=True),
             torch.empty(r + l, r, dtype=torch.float64, pin_memory=True),
             torch.empty(r, r, dtype=torch.float64, pin_memory=True)] for _ in range(nset)]
    h2d = sum(t.numel() * t.element_size() for t in hosts)
    d2h = sum(o.numel() * o.element_size() for o in outh[0])
    nh = max(1, a.h2d_streams)
    hs = [torch.cuda.Stream(device=dev) for _ in range(nh)]
    dstream = torch.cuda.Stream(device=dev)
    ev_in = [[torch.cuda.Event() for _ in range(nh)] for _ in range(nset)]
    ev_done = [torch.cuda.Event() for _ in range(nset)]
    ev_out = [torch.cuda.Event() for _ in range(nset)]
    step_handle = {}

    copy_ev = []   # per step: events around its input copies on the first copy stream

    def prefetch(i):
        b = i % nset
        for q in hs:
            q.wait_event(ev_done[b])              # the set's previous step has finished computing
        c0 = torch.cuda.Event(enable_timing=True)
        c0.record(hs[0])
        for d_, h_ in zip(ins[b][0], hosts):
            if h_.numel() * h_.element_size() >= (64 << 20) and h_.dim() >= 1 and h_.shape[0] >= nh:
                step = (h_.shape[0] + nh - 1) // nh   # row blocks, one per copy stream
                for qi, q in enumerate(hs):
                    with torch.cuda.stream(q):
                        d_[qi * step:(qi + 1) * step].copy_(h_[qi * step:(qi + 1) * step], non_blocking=True)
            else:
                with torch.cuda.stream(hs[0]):
                    d_.copy_(h_, non_blocking=True)
        for q, ev in zip(hs, ev_in[b]):
            ev.record(q)
        c1 = torch.cuda.Event(enable_timing=True)
        c1.record(hs[0])
        copy_ev.append((c0, c1))

    def enqueue(i):
        b, j = i % nset, i % nf
        Hj = Hs[j]
        wsj = bufs[j][0]
        Ad, Xd, Yd = ins[b][1]
        AXd, YtAd, cd = outd[b]
        for ev in ev_in[b]:
            Hj.stream.wait_event(ev)
        Hj.stream.wait_event(ev_out[b])           # the set's previous results are out
        Hj.sketch(Ad, Xd, Yd, AXd, YtAd, wsj)
        Hj.core(YtAd, Xd, eps, mode | gn.CORE_DEFER, cd, wsj)
        step_handle[i] = Hj

    def complete(i):
        b = i % nset
        Hj = step_handle.pop(i)
        AXd, YtAd, cd = outd[b]
        Hj.core_finish(cd)
        ev_done[b].record(Hj.stream)
        dstream.wait_event(ev_done[b])
        with torch.cuda.stream(dstream):
            for o, s_ in zip(outh[b], (AXd, YtAd, cd.Q, cd.R)):
                o.copy_(s_, non_blocking=True)
        ev_out[b].record(dstream)

    def run(k):
        # the copies of step i + ahead are queued before the host waits on an
        # older step: their buffer set was released by step i + ahead - nset
        # <= i - nf, whose done-event an earlier iteration recorded
        lag = nf - 1
        for i in range(min(ahead, k)):
            prefetch(i)
        for i in range(k):
            enqueue(i)
            if i + ahead < k:
                prefetch(i + ahead)
            if i - lag >= 0:
                complete(i - lag)
        for i in range(max(0, k - lag), k):
            complete(i)

    run(max(1, a.warmup))
    torch.cuda.synchronize()
    # the median of a few timed repetitions of the K steps: a rare host-side
    # stall of tens of ms (seen in about one run in six) otherwise decides the figure
    reps_ms, reps_copy, reps_idle = [], [], []
    for _ in range(max(1, a.e2e_reps)):
        copy_ev.clear()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(hs[0])
        for q in hs[1:] + [dstream] + [Hj.stream for Hj in Hs]:   # nothing of the timed steps starts before e0
            q.wait_stream(hs[0])
        run(a.steps)
        e1.record(dstream)                   # after the last step's results are out (which waits for all)
        torch.cuda.synchronize()
        reps_ms.append(e0.elapsed_time(e1) / a.steps)
        # the input copies of each step, and the host-to-device stream's idle time between them
        durs = sorted(c0.elapsed_time(c1) for c0, c1 in copy_ev)
        reps_copy.append(durs[len(durs) // 2])
        reps_idle.append(sum(max(0.0, copy_ev[t][1].elapsed_time(copy_ev[t + 1][0]))
                             for t in range(len(copy_ev) - 1)))
    ms = sorted(reps_ms)[len(reps_ms) // 2]
    # the host link's own rates on this machine (pinned, one stream each way), for reading the figure above
    big = hosts[0]
    dbig = ins[0][0][0]
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(hs[0])
    with torch.cuda.stream(hs[0]):
        dbig.copy_(big, non_blocking=True)
    c1.record(hs[0])
    torch.cuda.synchronize()
    h2d_gbs = big.numel() * big.element_size() / (c0.elapsed_time(c1) / 1e3) / 1e9
    c0.record(dstream)
    with torch.cuda.stream(dstream):
        big.copy_(dbig, non_blocking=True)
    c1.record(dstream)
    torch.cuda.synchronize()
    d2h_gbs = big.numel() * big.element_size() / (c0.elapsed_time(c1) / 1e3) / 1e9
    del ins, outd, outh, hosts
    torch.cuda.empty_cache()
    return {"value": 1e3 / ms, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": ms, "h2d_gbs_one_stream": h2d_gbs, "d2h_gbs_one_stream": d2h_gbs,
            "h2d_streams": nh, "buffer_sets": nset, "ahead": ahead,
            "reps": len(reps_ms), "statistic": "median", "ms_per_step_reps": reps_ms,
            "h2d_ms_per_step_median_reps": reps_copy, "h2d_idle_ms_reps": reps_idle,
            "copy_floor_ms": max(h2d / h2d_gbs, d2h / d2h_gbs) / 1e6}


# --------------------------------------------------------------------------- side measurements
def side_measurements(a, gn, H, stream, dev, A64, X64, Y64, Ab, Xb, Yb, eps, mode, ws, AX, YtA, core, peaks, dpk):
    """Outside the timed region: the precision contract, the FP64 path, factors,
    the FP64 cases with HMT, the Section 6 operations, r = 2000, the adjoint and
    the batched path."""
    m, n, r = a.m, a.n, a.r
    l = r // 2
    out = {}
    ev = lambda: torch.cuda.Event(enable_timing=True)
    F = torch.empty(m, r, dtype=torch.float64, device=dev)
    G = torch.empty(r, n, dtype=torch.float64, device=dev)
    e2 = torch.zeros(1, dtype=torch.float64, device=dev)
    normA = A64.norm().item()
    reps = max(3, a.steps // 2)

    def err_of(AXt, YtAt, c, Aref):
        H.factors(AXt, YtAt, c, F, G, ws)
        H.error_fro2(Aref, F[:, :c.k], G[:c.k], e2, ws)
        torch.cuda.synchronize()
        return math.sqrt(e2.item())

    # factors time (FP64 trsm + G) for the bf16 path
    H.sketch(Ab, Xb, Yb, AX, YtA, ws)
    H.core(YtA, Xb, eps, mode, core, ws)
    f0, f1 = ev(), ev()
    f0.record(stream)
    H.factors(AX, YtA, core, F, G, ws)
    f1.record(stream)
    torch.cuda.synchronize()
    out["factors_ms"] = f0.elapsed_time(f1)
    out["err_bf16"] = err_of(AX, YtA, core, A64)

    # ---- the plain FP64 GPU path (its own timing, on the unrounded Gaussian sketches)
    AX64 = torch.empty(m, r, dtype=torch.float64, device=dev)
    YtA64 = torch.empty(r + l, n, dtype=torch.float64, device=dev)
    c64 = gn.Core.empty(r, l, dev)
    ws64 = H.workspace(m, n, r, l, gn.F64)
    eps64 = 10 * 2.0 ** -53
    p0, p1, p2 = ev(), ev(), ev()
    p0.record(stream)
    H.sketch(A64, X64, Y64, AX64, YtA64, ws64)
    p1.record(stream)
    H.core(YtA64, X64, eps64, mode, c64, ws64)
    p2.record(stream)
    torch.cuda.synchronize()
    fp64_ms = p0.elapsed_time(p2)
    sk64 = p0.elapsed_time(p1)
    fl = 2.0 * m * n * (2 * r + l)
    fp64_peak = dpk.get("fp64_tflops")
    out["fp64_path"] = {"approx_per_s": 1e3 / fp64_ms, "ms_per_step": fp64_ms, "sketch_ms": sk64,
                        "sketch_tflops": fl / (sk64 / 1e3) / 1e12,
                        "sketch_frac": (fl / (sk64 / 1e3) / 1e12 / fp64_peak) if fp64_peak else None,
                        "peak_kind": "fp64 measured in this run (torch.matmul float64)",
                        "err": None}

    def fp64_err(Aexact, Xs, Ys, Aref):
        """FP64 GPU path (sketch, core, factors) on exact FP64 inputs; error vs Aref."""
        H.sketch(Aexact, Xs, Ys, AX64, YtA64, ws64)
        H.core(YtA64, Xs, eps64, mode, c64, ws64)
        H.factors(AX64, YtA64, c64, F, G, ws64)
        H.error_fro2(Aref, F[:, :c64.k], G[:c64.k], e2, ws64)
        torch.cuda.synchronize()
        return math.sqrt(e2.item())

    out["fp64_path"]["err"] = fp64_err(A64, X64, Y64, A64)

    # ---- precision contract: every mixed path against the FP64 GPU path on the
    # same quantized sketches (and, for parity, on the same stored A)
    Xq, Yq = Xb.double(), Yb.double()
    err_ref = fp64_err(A64, Xq, Yq, A64)
    prec = {"fp64_matched_err": err_ref,
            "reading": "ratio_vs_fp64 = err(mixed path, vs FP64 A) / err(FP64 path on the FP64 A with the same "
                       "quantized X, Y); parity_ratio = the same two paths on the stored (quantized) A, each "
                       "measured against that stored A; floor = ||A - A_stored||_F (storage error no rank-r "
                       "approximant removes)"}

    def contract(name, Astored64, Xs64, Ys64, mixed_err_vs_A, mixed_err_vs_Ast):
        ref_st = fp64_err(Astored64, Xs64, Ys64, Astored64)
        d = (A64 - Astored64).norm().item()
        prec[name] = {"err_vs_A": mixed_err_vs_A, "ratio_vs_fp64": mixed_err_vs_A / err_ref,
                      "err_vs_A_stored": mixed_err_vs_Ast, "fp64_on_A_stored_err": ref_st,
                      "parity_ratio": mixed_err_vs_Ast / ref_st, "floor_storage": d,
                      "floor_estimate": math.sqrt(err_ref ** 2 + d ** 2)}

    Ab64 = Ab.double()
    H.sketch(Ab, Xb, Yb, AX, YtA, ws)
    H.core(YtA, Xb, eps, mode, core, ws)
    e_a = err_of(AX, YtA, core, A64)
    e_s = err_of(AX, YtA, core, Ab64)
    contract("bf16", Ab64, Xq, Yq, e_a, e_s)
    del Ab64

    # split bf16 (hi + lo) path: throughput and the contract.  It aims at the FP64
    # path's error, so its accumulation is FP64-level: sketches in stored K parts
    # of 8192 summed in FP64, digit-sliced C, FP64 G (gn_set_fp64_accum).
    part_k = 8192
    H.set_fp64_accum(part_k)
    Ahi, Alo = H.quantize(A64, split=True)
    H.sketch(Ahi, Xb, Yb, AX, YtA, ws, A_lo=Alo)
    H.core(YtA, Xb, eps, mode, core, ws)
    torch.cuda.synchronize()
    k0, k1, s0, s1 = ev(), ev(), ev(), ev()
    s0.record(stream)
    for _ in range(reps):
        k0.record(stream)
        H.sketch(Ahi, Xb, Yb, AX, YtA, ws, A_lo=Alo)
        k1.record(stream)
        H.core(YtA, Xb, eps, mode, core, ws)
    s1.record(stream)
    torch.cuda.synchronize()
    split_ms = s0.elapsed_time(s1) / reps
    split_sketch_ms = k0.elapsed_time(k1)
    Asp64 = Ahi.double() + Alo.double()
    e_a = err_of(AX, YtA, core, A64)
    e_s = err_of(AX, YtA, core, Asp64)
    H.set_fp64_accum(0)
    fl2 = 2 * fl
    out["split_bf16"] = {"approx_per_s": 1e3 / split_ms, "ms_per_step": split_ms, "sketch_ms": split_sketch_ms,
                         "sketch_tflops": fl2 / (split_sketch_ms / 1e3) / 1e12, "err": e_a,
                         "fp64_accum_part_k": part_k, "g_fp64": True}
    contract("split_bf16", Asp64, Xq, Yq, e_a, e_s)
    del Ahi, Alo, Asp64

    # e4m3 path: one power-of-two scale per 128 x 128 tile, block-scaled MMAs
    q0, q1 = ev(), ev()
    q0.record(stream)
    A8 = H.quantize_e4m3(A64)
    X8 = H.quantize_e4m3(X64, data=False)
    Y8 = H.quantize_e4m3(Y64, data=False)
    q1.record(stream)
    ws8 = H.workspace(m, n, r, l, gn.E4M3)
    H.sketch(A8, X8, Y8, AX, YtA, ws8)
    H.core(YtA, X8, eps, mode, core, ws8)
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record(stream)
    for _ in range(reps):
        k0.record(stream)
        H.sketch(A8, X8, Y8, AX, YtA, ws8)
        k1.record(stream)
        H.core(YtA, X8, eps, mode, core, ws8)
    e1.record(stream)
    torch.cuda.synchronize()
    f8_ms = e0.elapsed_time(e1) / reps
    f8_sketch_ms = k0.elapsed_time(k1)
    peak8 = dpk.get("e4m3_tflops") or 2.0 * peaks["bf16_tflops"]
    A8v = A8.values()
    e_a = err_of(AX, YtA, core, A64)
    e_s = err_of(AX, YtA, core, A8v)
    out["fp8_e4m3"] = {"approx_per_s": 1e3 / f8_ms, "ms_per_step": f8_ms, "sketch_ms": f8_sketch_ms,
                       "sketch_tflops": fl / (f8_sketch_ms / 1e3) / 1e12,
                       "sketch_frac": fl / (f8_sketch_ms / 1e3) / 1e12 / peak8, "peak_tflops": peak8,
                       "peak_kind": ("e4m3 measured in this run (torch._scaled_mm)" if dpk.get("e4m3_tflops")
                                     else "2 x bf16 burst (nominal ratio)"),
                       "quantize_ms": q0.elapsed_time(q1), "k": core.k, "err": e_a}
    contract("e4m3", A8v, X8.values(), Y8.values(), e_a, e_s)
    prec["e4m3"]["sketches"] = "e4m3 X, Y (their own per-tile scales); ratio_vs_fp64 against the BF16-rounded ones"
    del A8, X8, Y8, ws8, A8v
    out["precision"] = prec
    out["norm_A_fro"] = normA
    del AX64, YtA64, c64, ws64
    torch.cuda.empty_cache()

    out["dct_sketch"] = dct_measurement(gn, H, stream, dev, a, A64, Ab, eps, mode, out["err_bf16"])
    out["fp64_cases"] = fp64_cases(gn, H, stream, dev)
    out["sparse_countsketch"] = sparse_measurement(gn, H, stream, dev)
    out["sgn_variants"] = variants_measurement(gn, H, stream, dev)
    out["oversampling_sweep"] = oversampling_sweep(gn, H, stream, dev)
    out["sketch_state_ops"] = sketch_state_ops(gn, H, stream, dev, a, Ab, Xb, Yb, eps, mode)
    out["r2000"] = r2000_measurement(gn, H, stream, dev, a, A64, Ab, eps, mode)
    out["adjoint"] = adjoint_measurement(gn, H, stream, dev)
    out["batched"] = batched_measurement(gn, H, stream, dev, steps=max(3, a.steps))
    return out


def dct_measurement(gn, H, stream, dev, a, A64, Ab, eps, mode, err_gauss):
    """The subsampled DCT sketches of Section 7's experiments on the bench
    matrix: X = D C^T S (n x r) and Y (m x (r + l)) made on the device from their
    draws (BF16), the tensor-core sketch with them, the core, and the error
    against the FP64 A beside the Gaussian sketches' error."""
    m, n, r = a.m, a.n, a.r
    l = r // 2
    sx, cx = gn_synth.dct_sketch_draws(n, r, seed=gn_synth.DEFAULT_SEED + 5)
    sy, cy = gn_synth.dct_sketch_draws(m, r + l, seed=gn_synth.DEFAULT_SEED + 6)
    sx, cx, sy, cy = sx.to(dev), cx.to(dev), sy.to(dev), cy.to(dev)
    gen_ms = _best_ms(lambda: (H.dct_sketch(n, sx, cx), H.dct_sketch(m, sy, cy)), 3, stream)
    Xd, Yd = H.dct_sketch(n, sx, cx), H.dct_sketch(m, sy, cy)
    ws = H.workspace(m, n, r, l, gn.BF16)
    AX = torch.empty(m, r, dtype=torch.float32, device=dev)
    YtA = torch.empty(r + l, n, dtype=torch.float32, device=dev)
    core = gn.Core.empty(r, l, dev)
    sk_ms = _best_ms(lambda: H.sketch(Ab, Xd, Yd, AX, YtA, ws), 3, stream)
    H.core(YtA, Xd, eps, mode, core, ws)
    F = torch.empty(m, r, dtype=torch.float64, device=dev)
    G = torch.empty(r, n, dtype=torch.float64, device=dev)
    e2 = torch.zeros(1, dtype=torch.float64, device=dev)
    H.factors(AX, YtA, core, F, G, ws)
    H.error_fro2(A64, F[:, :core.k], G[:core.k], e2, ws)
    torch.cuda.synchronize()
    err = math.sqrt(e2.item())
    peaks, _ = measured_peaks()
    fl = 2.0 * m * n * (2 * r + l)
    out = {"workload": f"{m}x{n}, r={r}, l={l}, subsampled DCT X, Y (BF16), FP64 core",
           "generate_ms": gen_ms, "sketch_ms": sk_ms, "sketch_tflops": fl / (sk_ms / 1e3) / 1e12,
           "sketch_frac": fl / (sk_ms / 1e3) / 1e12 / peaks["bf16_tflops"], "k": core.k, "err": err,
           "err_over_gaussian": err / err_gauss}
    del Xd, Yd, ws, AX, YtA, core, F, G
    torch.cuda.empty_cache()
    return out


def sparse_measurement(gn, H, stream, dev, m=178866, n=178866, r=200, l=100, k=50, per_row=5):
    """Section 7's sparse experiment with a seeded stand-in of the same size and
    density as its matrix (178866 x 178866, about a million nonzeros): the
    O(nnz) CountSketch sketches of the CSR matrix, the core product by
    CountSketch (C given to the core), the FP64 core, and the HBM bytes of the
    sketch step (CSR arrays read, outputs zeroed and updated)."""
    rows, cols, vals = gn_synth.sparse_lowrank_plus_noise(m, n, k, per_row)
    order = torch.argsort(rows * n + cols)
    rows, cols, vals = rows[order], cols[order], vals[order]
    key = rows * n + cols
    uniq, inv = torch.unique_consecutive(key, return_inverse=True)
    v = torch.zeros(uniq.numel(), dtype=torch.float64).index_add_(0, inv, vals)
    rr, cc = uniq // n, uniq % n
    crow = torch.zeros(m + 1, dtype=torch.int64)
    crow[1:] = torch.cumsum(torch.bincount(rr, minlength=m), 0)
    crow, col, val = crow.to(dev), cc.to(torch.int32).to(dev), v.to(dev)
    nnz = int(val.numel())
    bx, sx = (t.to(dev) for t in gn_synth.countsketch_draws(n, r, seed=gn_synth.DEFAULT_SEED + 7))
    by, sy = (t.to(dev) for t in gn_synth.countsketch_draws(m, r + l, seed=gn_synth.DEFAULT_SEED + 8))
    AX = torch.empty(m, r, dtype=torch.float64, device=dev)
    YtA = torch.empty(r + l, n, dtype=torch.float64, device=dev)
    core = gn.Core.empty(r, l, dev)
    ws = H.workspace(m, n, r, l, gn.F64)
    Xview = torch.empty(n, r, dtype=torch.float64, device=dev)   # shapes only: C is given, X is not read
    sk_ms = _best_ms(lambda: H.sketch_csr_countsketch(crow, col, val, (m, n), bx, sx, by, sy, AX, YtA), 3, stream)
    c_ms = _best_ms(lambda: H.countsketch_apply(YtA, bx, sx, core.C), 3, stream)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    H.core(YtA, Xview, 10 * 2.0 ** -53, gn.AUTO | gn.EPS_RELATIVE | gn.CORE_C_GIVEN, core, ws)
    t1.record(stream)
    torch.cuda.synchronize()
    core_ms = t0.elapsed_time(t1)
    peaks, _ = measured_peaks()
    bytes_ = 8 * (m + 1) + 4 * nnz + 8 * nnz + 8 * (m * r + (r + l) * n) * 2 + 8 * (n + m) * 2
    out = {"workload": f"sparse {m}x{n}, nnz={nnz} (seeded low-rank + noise stand-in), CountSketch r={r}, l={l}, FP64",
           "nnz": nnz, "sketch_ms": sk_ms, "core_product_ms": c_ms, "core_ms": core_ms, "k": core.k,
           "sketch_bytes": bytes_, "sketch_hbm_frac": bytes_ / (sk_ms / 1e3) / (peaks["hbm_gbs"] * 1e9),
           "approx_per_s": 1e3 / (sk_ms + c_ms + core_ms)}
    del AX, YtA, core, ws, crow, col, val
    torch.cuda.empty_cache()
    return out


def variants_measurement(gn, H, stream, dev, m=4096, n=2048, r=100, l=50):
    """Section 5.1.1's alternatives on one FP64 sketch state (W1 diag(i^-2) W2^T
    + 1e-8 noise): SGN with the SVD eps-pseudoinverse, raised singular values,
    pivoted QR with raised diagonal, raised diagonal, beside the library's
    QR-truncation core (AUTO); floor = 10 u ||C||_2 for all; time (after a
    warm-up) and error against A."""
    p = gn_synth.config2(m=m, n=n, r=r, l=l, device=dev)
    A, X, Y = p.a, p.x, p.y
    ws = H.workspace(m, n, r, l, gn.F64)
    AX = torch.empty(m, r, dtype=torch.float64, device=dev)
    YtA = torch.empty(r + l, n, dtype=torch.float64, device=dev)
    F = torch.zeros(m, r, dtype=torch.float64, device=dev)
    G = torch.zeros(r, n, dtype=torch.float64, device=dev)
    e2 = torch.zeros(1, dtype=torch.float64, device=dev)
    core = gn.Core.empty(r, l, dev)
    H.sketch(A, X, Y, AX, YtA, ws)
    H.core(YtA, X, 10 * 2.0 ** -53, gn.AUTO | gn.EPS_RELATIVE, core, ws)
    torch.cuda.synchronize()
    floor = core.eps_abs
    out = {"workload": f"{m}x{n}, r={r}, l={l}, FP64 sketches, floor = 10 u ||C||_2 = {floor:.3e}"}

    def err(k):
        H.error_fro2(A, F[:, :k], G[:k], e2, ws)
        torch.cuda.synchronize()
        return math.sqrt(e2.item())

    def tcore():
        H.core(YtA, X, 10 * 2.0 ** -53, gn.AUTO | gn.EPS_RELATIVE, core, ws)
        H.factors(AX, YtA, core, F, G, ws)
    ms = _best_ms(tcore, 3, stream)
    out["qr_truncation_auto"] = {"ms": ms, "k": core.k, "err": err(core.k)}
    for name, code in (("svd_truncate", gn.SVD_TRUNCATE), ("svd_raise", gn.SVD_RAISE),
                       ("rrqr_raise", gn.RRQR_RAISE), ("diag_raise", gn.DIAG_RAISE)):
        kk = [0]

        def run():
            kk[0] = H.factors_variant(AX, YtA, X, floor, code, F, G)
        ms = _best_ms(run, 3, stream)
        out[name] = {"ms": ms, "k": kk[0], "err": err(kk[0])}
    del A, X, Y, ws, AX, YtA, F, G, core
    torch.cuda.empty_cache()
    return out


def oversampling_sweep(gn, H, stream, dev, m=8192, n=4096, r=200):
    """The oversampling study of Section 5.2: the FP64 GN error ||A - F G||_F
    for l in {1, 2, 5, 10, 20, 50, 100, 200} at fixed r, beside HMT's error with
    the same X (W1 diag(i^-2) W2^T + 1e-8 noise)."""
    p = gn_synth.config2(m=m, n=n, r=r, l=r, device=dev)
    A, X = p.a, p.x
    Yfull = p.y
    e2 = torch.zeros(1, dtype=torch.float64, device=dev)
    res = {"workload": f"{m}x{n}, r={r}, FP64, Gaussian X, Y; errors ||A - Ahat||_F"}
    ws = H.workspace(m, n, r, r, gn.F64)
    Q = torch.empty(m, r, dtype=torch.float64, device=dev)
    B = torch.empty(r, n, dtype=torch.float64, device=dev)
    H.hmt(A, X, Q, B, ws)
    H.error_fro2(A, Q, B, e2, ws)
    torch.cuda.synchronize()
    res["hmt_err"] = math.sqrt(e2.item())
    errs = {}
    for l in (1, 2, 5, 10, 20, 50, 100, 200):
        Y = Yfull[:, :r + l].contiguous()
        AX = torch.empty(m, r, dtype=torch.float64, device=dev)
        YtA = torch.empty(r + l, n, dtype=torch.float64, device=dev)
        core = gn.Core.empty(r, l, dev)
        F = torch.empty(m, r, dtype=torch.float64, device=dev)
        G = torch.empty(r, n, dtype=torch.float64, device=dev)
        H.approx(A, X, Y, 10 * 2.0 ** -53, gn.AUTO | gn.EPS_RELATIVE, AX, YtA, core, F, G, ws)
        H.error_fro2(A, F[:, :core.k], G[:core.k], e2, ws)
        torch.cuda.synchronize()
        errs[str(l)] = {"err": math.sqrt(e2.item()), "over_hmt": math.sqrt(e2.item()) / res["hmt_err"], "k": core.k}
    res["gn"] = errs
    del A, X, Yfull, ws, Q, B
    torch.cuda.empty_cache()
    return res


def fp64_cases(gn, H, stream, dev):
    """The FP64 cases with the HMT baseline (Algorithm 1) beside GN on the same
    X: 1000 x 500 (sigma_i = 2^(-i/10), r = 20, l = 10, eps = 1e-15 ||A||) and
    20000 x 10000 (i^-2 over 2000 modes + 1e-8 noise, r = 500, l = 250).  GN
    time = sketch + core + factors (gn_approx); HMT = AX, its Householder QR and
    B = Q^T A (gn_hmt)."""
    res = {}
    for name, p, reps in (("1000x500_r20", gn_synth.config1(device=dev), 50),
                          ("20000x10000_r500", gn_synth.config2(device=dev), 3)):
        A, X, Y, r, l = p.a, p.x, p.y, p.r, p.l
        m, n = A.shape
        eps, mode = (p.eps, gn.AUTO) if p.eps > 0 else (10 * 2.0 ** -53, gn.AUTO | gn.EPS_RELATIVE)
        ws = H.workspace(m, n, r, l, gn.F64)
        AX = torch.empty(m, r, dtype=torch.float64, device=dev)
        YtA = torch.empty(r + l, n, dtype=torch.float64, device=dev)
        c = gn.Core.empty(r, l, dev)
        F = torch.empty(m, r, dtype=torch.float64, device=dev)
        G = torch.empty(r, n, dtype=torch.float64, device=dev)
        Q = torch.empty(m, r, dtype=torch.float64, device=dev)
        B = torch.empty(r, n, dtype=torch.float64, device=dev)
        e2 = torch.zeros(1, dtype=torch.float64, device=dev)

        def gn_run():
            H.approx(A, X, Y, eps, mode, AX, YtA, c, F, G, ws)

        def hmt_run():
            H.hmt(A, X, Q, B, ws)

        out = {}
        for nm, f in (("gn", gn_run), ("hmt", hmt_run)):
            f()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                f()
            e1.record(stream)
            torch.cuda.synchronize()
            out[nm + "_ms"] = e0.elapsed_time(e1) / reps
        H.error_fro2(A, F[:, :c.k], G[:c.k], e2, ws)
        torch.cuda.synchronize()
        out["gn_err"] = math.sqrt(e2.item())
        H.error_fro2(A, Q, B, e2, ws)
        torch.cuda.synchronize()
        out["hmt_err"] = math.sqrt(e2.item())
        out["gn_k"] = c.k
        out["gn_over_hmt_time"] = out["gn_ms"] / out["hmt_ms"]
        out["gn_over_hmt_err"] = out["gn_err"] / out["hmt_err"]
        res[name] = out
        del A, X, Y, AX, YtA, c, F, G, Q, B, ws, p
        torch.cuda.empty_cache()
    return res


def sketch_state_ops(gn, H, stream, dev, a, Ab, Xb, Yb, eps, mode):
    """Section 6 on the bench matrix (BF16 operands, FP32 sketches), each timed
    (CUDA events, best of 3) beside a fresh sketch of the enlarged or updated
    matrix: the streaming update A <- A + E, resampling r -> r + 100 (l + 50),
    1024 appended rows, 1024 appended columns, and A_hat W / W A_hat (64
    vectors) without forming A_hat."""
    m, n, r = a.m, a.n, a.r
    l = r // 2
    ws = H.workspace(m, n, r, l, gn.BF16)
    AX = torch.empty(m, r, dtype=torch.float32, device=dev)
    YtA = torch.empty(r + l, n, dtype=torch.float32, device=dev)
    core = gn.Core.empty(r, l, dev)
    H.sketch(Ab, Xb, Yb, AX, YtA, ws)
    H.core(YtA, Xb, eps, mode, core, ws)
    torch.cuda.synchronize()
    res = {}

    def best(f):
        f()
        return _best_ms(f, 3, stream)

    res["fresh_sketch_ms"] = best(lambda: H.sketch(Ab, Xb, Yb, AX, YtA, ws))
    # streaming update: E of the size of A
    Eb = H.quantize(gn_synth.gaussian((m, n), 5, 0, device=dev, dtype=torch.float32) * 1e-3)
    AXu, YtAu = AX.clone(), YtA.clone()
    wsu = H.update_workspace(m, n, r, l, gn.BF16, dev)
    res["update_ms"] = best(lambda: H.update(Eb, Xb, Yb, AXu, YtAu, wsu))
    del Eb, wsu
    # resampling r -> r + 100, l -> l + 50
    dr, dl = 100, 50
    Xd = H.quantize(gn_synth.gaussian((n, dr), 6, 0, device=dev))
    Yd = H.quantize(gn_synth.gaussian((m, dr + dl), 7, 0, device=dev))
    AXn = torch.empty(m, r + dr, dtype=torch.float32, device=dev)
    YtAn = torch.empty(r + l + dr + dl, n, dtype=torch.float32, device=dev)
    res["resample_ms"] = best(lambda: H.resample(Ab, Xd, Yd, AX, YtA, AXn, YtAn))
    Xn, Yn = gn.padded(n, r + dr, torch.bfloat16, dev), gn.padded(m, r + l + dr + dl, torch.bfloat16, dev)
    Xn[:, :r].copy_(Xb)
    Xn[:, r:].copy_(Xd)
    Yn[:, :r + l].copy_(Yb)
    Yn[:, r + l:].copy_(Yd)
    res["resample_fresh_sketch_ms"] = best(lambda: H.sketch(Ab, Xn, Yn, AXn, YtAn, ws))
    del Xd, Yd, AXn, YtAn, Xn, Yn
    # 1024 appended rows and 1024 appended columns
    mb = nb = 1024
    Br = H.quantize(gn_synth.gaussian((mb, n), 8, 0, device=dev, dtype=torch.float32))
    Yr = H.quantize(gn_synth.gaussian((mb, r + l), 9, 0, device=dev))
    AXr = torch.empty(m + mb, r, dtype=torch.float32, device=dev)
    YtAc = YtA.clone()
    res["append_rows_ms"] = best(lambda: H.append_rows(Br, Xb, Yr, AX, YtAc, AXr))
    Abig = gn.padded(m + mb, n, torch.bfloat16, dev)
    Abig[:m].copy_(Ab)
    Abig[m:].copy_(Br)
    Ybig = gn.padded(m + mb, r + l, torch.bfloat16, dev)
    Ybig[:m].copy_(Yb)
    Ybig[m:].copy_(Yr)
    wsb = H.workspace(m + mb, n, r, l, gn.BF16)
    res["append_rows_fresh_sketch_ms"] = best(lambda: H.sketch(Abig, Xb, Ybig, AXr, YtAc, wsb))
    del Br, Yr, AXr, Abig, Ybig, wsb
    Bc = H.quantize(gn_synth.gaussian((m, nb), 10, 0, device=dev, dtype=torch.float32))
    Xc = H.quantize(gn_synth.gaussian((nb, r), 11, 0, device=dev))
    YtAw = torch.empty(r + l, n + nb, dtype=torch.float32, device=dev)
    AXc = AX.clone()
    res["append_cols_ms"] = best(lambda: H.append_cols(Bc, Xc, Yb, AXc, YtA, YtAw))
    Awide = gn.padded(m, n + nb, torch.bfloat16, dev)
    Awide[:, :n].copy_(Ab)
    Awide[:, n:].copy_(Bc)
    Xw = gn.padded(n + nb, r, torch.bfloat16, dev)
    Xw[:n].copy_(Xb)
    Xw[n:].copy_(Xc)
    wsw = H.workspace(m, n + nb, r, l, gn.BF16)
    res["append_cols_fresh_sketch_ms"] = best(lambda: H.sketch(Awide, Xw, Yb, AXc, YtAw, wsw))
    del Bc, Xc, YtAw, AXc, Awide, Xw, wsw
    # A_hat W and W A_hat without forming A_hat (64 vectors)
    kw = 64
    W = gn_synth.gaussian((n, kw), 12, 0, device=dev)
    Wl = gn_synth.gaussian((kw, m), 13, 0, device=dev)
    o1 = torch.empty(m, kw, dtype=torch.float64, device=dev)
    o2 = torch.empty(kw, n, dtype=torch.float64, device=dev)
    res["apply_right_64_ms"] = best(lambda: H.apply(AX, YtA, core, W, o1, 0))
    res["apply_left_64_ms"] = best(lambda: H.apply(AX, YtA, core, Wl, o2, 1))
    res["workload"] = (f"{m}x{n}, r={r}, l={l}, BF16 operands: update E {m}x{n}; resample +{dr}/+{dl}; "
                       f"append {mb} rows / {nb} cols; apply with {kw} vectors")
    del W, Wl, o1, o2, AXu, YtAu, ws, AX, YtA, core
    torch.cuda.empty_cache()
    return res


def r2000_measurement(gn, H, stream, dev, a, A64, Ab, eps, mode, r=2000):
    """The same matrix with the larger sketch size, r = 2000, l = 1000 (BF16
    sketch + FP64 core of 3000 x 2000): approximations/s, the sketch rate and
    the error against the FP64 A."""
    m, n = a.m, a.n
    l = r // 2
    X64, Y64 = gn_synth.sketches(m, n, r, l, gn_synth.DEFAULT_SEED + 2, device=dev)
    Xb, Yb = H.quantize(X64), H.quantize(Y64)
    del X64, Y64
    ws = H.workspace(m, n, r, l, gn.BF16)
    AX = torch.empty(m, r, dtype=torch.float32, device=dev)
    YtA = torch.empty(r + l, n, dtype=torch.float32, device=dev)
    core = gn.Core.empty(r, l, dev)
    H.sketch(Ab, Xb, Yb, AX, YtA, ws)
    H.core(YtA, Xb, eps, mode, core, ws)
    torch.cuda.synchronize()
    reps = 3
    e0, e1, k0, k1 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
    e0.record(stream)
    for _ in range(reps):
        k0.record(stream)
        H.sketch(Ab, Xb, Yb, AX, YtA, ws)
        k1.record(stream)
        H.core(YtA, Xb, eps, mode, core, ws)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    sk = k0.elapsed_time(k1)
    fl = 2.0 * m * n * (2 * r + l)
    F = torch.empty(m, r, dtype=torch.float64, device=dev)
    G = torch.empty(r, n, dtype=torch.float64, device=dev)
    e2 = torch.zeros(1, dtype=torch.float64, device=dev)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    H.factors(AX, YtA, core, F, G, ws)
    f1.record(stream)
    H.error_fro2(A64, F[:, :core.k], G[:core.k], e2, ws)
    torch.cuda.synchronize()
    out = {"workload": f"{m}x{n}, r={r}, l={l}, bf16 operands, FP64 core, mode AUTO",
           "approx_per_s": 1e3 / ms, "ms_per_step": ms, "sketch_ms": sk,
           "sketch_tflops": fl / (sk / 1e3) / 1e12, "k": core.k, "factors_ms": f0.elapsed_time(f1),
           "err": math.sqrt(e2.item())}
    del Xb, Yb, ws, AX, YtA, core, F, G
    torch.cuda.empty_cache()
    return out


def adjoint_measurement(gn, H, stream, dev, m=4096, n=4096, r=256, l=128):
    """Forward (dense A_hat) and hand-written adjoint of <G, A_hat> on the
    4096 x 4096 FP32 case (sigma_i = i^-1.5 over 1024 modes + 1e-6 noise,
    r = 256, l = 128), each timed with CUDA events (best of 3 after a warm-up):
    the standalone backward, the backward from the forward's front, and forward
    plus that backward as one step."""
    p, G = gn_synth.config4(device=dev, m=m, n=n, r=r, l=l, dtype=torch.float32)
    A, X, Y = p.a, p.x, p.y
    ws = H.backward_workspace(m, n, r, l, gn.F32)
    Ah = torch.empty_like(A)
    dA = torch.empty_like(A)
    fwd = _best_ms(lambda: H.forward_dense(A, X, Y, Ah, ws), 4, stream)
    bwd = _best_ms(lambda: H.backward(A, X, Y, G, dA, ws), 4, stream)
    # the backward from the front the forward leaves in ws (as autograd runs it)
    H.forward_dense(A, X, Y, Ah, ws)
    bwd_saved = _best_ms(lambda: H.backward_saved(X, Y, G, dA, ws), 4, stream)

    def step():
        H.forward_dense(A, X, Y, Ah, ws)
        H.backward_saved(X, Y, G, dA, ws)

    fwd_bwd = _best_ms(step, 4, stream)
    return {"workload": f"{m}x{n} FP32, r={r}, l={l}, loss <G, A_hat>", "fwd_ms": fwd, "bwd_ms": bwd,
            "bwd_saved_ms": bwd_saved, "fwd_bwd_saved_ms": fwd_bwd, "grad_norm": float(dA.norm().item())}


def batched_measurement(gn, H, stream, dev, count=512, steps=10):
    """512 problems, m ~ U[256,4096], n ~ U[128,m], r ~ U{16..128}, l = r/2, each
    W1 diag(2^(-i/10)) W2^T + 1e-8 N with its own seed, BF16 operands; the four
    launches of gn_batched_run captured once in a CUDA graph and replayed."""
    shapes = gn_synth.batched_shapes(count)
    probs = []
    a_bytes = 0
    flops = 0.0
    for i, (m, n, r, l) in enumerate(shapes):
        p = gn_synth.config5_problem(i, (m, n, r, l), device=dev)
        d = {"A": H.quantize(p.a), "X": H.quantize(p.x), "Y": H.quantize(p.y)}
        del p
        d["AX"] = torch.empty(m, r, dtype=torch.float32, device=dev)
        d["YtA"] = torch.empty(r + l, n, dtype=torch.float32, device=dev)
        for nm, (a, b) in (("Q", (r + l, r)), ("R", (r, r)), ("Q2", (r, r)), ("R2", (r, r))):
            d[nm] = torch.empty(a, b, dtype=torch.float64, device=dev)
        d["k"] = torch.empty(1, dtype=torch.int32, device=dev)
        probs.append(d)
        a_bytes += 2 * m * n
        flops += 2.0 * m * n * (2 * r + l)
    ws = H.batched_prepare(probs)
    eps, mode = 10 * 2.0 ** -24, gn.AUTO | gn.EPS_RELATIVE
    H.batched_run(eps, mode, ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        H.batched_run(eps, mode, ws)
    e1.record(stream)
    torch.cuda.synchronize()
    fixed_ms = e0.elapsed_time(e1) / 3
    policy, tuned_ms = H.batched_tune(eps, mode, ws)   # re-prepares with the fastest tile policy
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        H.batched_run(eps, mode, ws)
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ks = [int(d["k"].item()) for d in probs]
    peaks, _ = measured_peaks()
    return {"workload": f"{count} problems, m~U[256,4096], n~U[128,m], r~U{{16..128}}, l=r/2, BF16, mode AUTO",
            "approx_per_s": count * 1e3 / ms, "ms_per_batch": ms, "cuda_graph": True, "launches_per_batch": 4,
            "tile_policy": policy, "tuned_ms_no_graph": tuned_ms, "fixed_rule_ms_no_graph": fixed_ms,
            "a_bytes": a_bytes, "hbm_floor_ms": a_bytes / (peaks["hbm_gbs"] * 1e9) * 1e3,
            "sketch_flops": flops, "truncated": sum(1 for k, (m, n, r, l) in zip(ks, shapes) if k < r)}


if __name__ == "__main__":
    main()
