#!/usr/bin/env python
"""Throughput of the test-side SCW pass of the tensor-based sketching method.

Metric: stream matrices per second through Algorithm 1 (QR form) with the
tensor sketch -- X = (S A)^T, thin QR, A Q, truncated rank-r SVD and the
error ||A - B||_F for every matrix -- BF16 path (tensor cores) with the plain
FP32 path timed beside it, valid at a relative Frobenius-error gap <= 1e-3
to the FP64 oracle (checked on a sample in the same run).

Default workload (one step = one batch): 500 synthetic 2048 x 2048 BF16
stream matrices per GPU, k = 40, r = 20, sketch trained on 1000 matrices of
the same stream.  Inputs stay resident in HBM (4.2 GB per step, far larger
than the 129 MB L2, so no flush is needed between steps).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import datetime
import faulthandler
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0,
                  "bf16_tflops_sustained": 1700.0}


# DRAM bytes (read + write) per 2048 x 2048 BF16 matrix of the tcgen05 sketch
# kernel with k = 40, from ncu on a 64-matrix launch (537.21 MB read, 33.25 MB
# written); re-measure whenever that kernel changes.
SKETCH_TRAFFIC_PER_MATRIX = (537.21e6 + 33.25e6) / 64

def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return PEAKS_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons around the timed
    region, each stamped by nvidia-smi itself.

    Samples whose stamp falls inside [mark(), mark_end()] are the timed
    region's.  A region shorter than a few sampling periods may hold none,
    so after mark_end() the caller keeps running the same (untimed) step
    until need_more() is false; those samples, taken with the GPU still on
    the same work right after the region, are reported separately."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 50
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # nvidia-smi takes a moment to start: wait for its first sample
        t0 = time.time()
        while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.01)

    def mark(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    @staticmethod
    def parse(item):
        """(unix time, sm MHz, max sm MHz, set of active reasons) or None for
        an (arrival time, line) pair; the time is nvidia-smi's own stamp,
        else the line's arrival."""
        arrived, line = item
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            return None
        try:
            sm, mx = float(parts[1]), float(parts[2])
        except ValueError:
            return None
        try:
            ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            ts = arrived
        active = {nm for nm, v in zip(ClockSampler.REASONS, parts[5:9])
                  if v.lower() == "active"}
        return ts, sm, mx, active

    def _after(self):
        return sum(1 for ln in list(self.lines)
                   if (p := self.parse(ln)) is not None and self.t1 is not None
                   and p[0] > self.t1)

    def need_more(self, want: int = 3, limit_s: float = 2.0) -> bool:
        """True while fewer than `want` samples have arrived after the
        region's end (for at most limit_s seconds)."""
        if self.proc is None or self.t1 is None:
            return False
        return self._after() < want and time.time() - self.t1 < limit_s

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return self.summary(self.lines, self.t0, self.t1)

    @classmethod
    def summary(cls, lines, t0, t1):
        inside, after = [], []
        for ln in lines:
            p = cls.parse(ln)
            if p is None or t0 is None or t1 is None or p[0] < t0:
                continue
            (inside if p[0] <= t1 else after).append(p)
        kept = inside if inside else after
        if not kept:
            return None
        reasons = sorted(set().union(*[p[3] for p in kept]))
        out = {"sm_mhz": statistics.median(p[1] for p in kept),
               "sm_max_mhz": max(p[2] for p in kept), "reasons": reasons,
               "samples": len(inside)}
        if not inside:
            out["samples_after_region"] = len(after)
            out["window"] = (f"the timed region ({1e3 * (t1 - t0):.0f} ms) was shorter than the "
                             f"{cls.PERIOD_MS} ms sampling period allowed for; samples taken "
                             "right after it, the same step still running untimed")
        return out


def stage(msg):
    print(f"[bench] {time.strftime('%H:%M:%S')} {msg}", file=sys.stderr, flush=True)


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return max(int(i.get("num_threads", 1)) for i in info)
    except Exception:
        pass
    return os.cpu_count() or 1


# --------------------------------------------------------------------------
def run_reference(args):
    """The FP64 oracle on the host cores, bounded samples of the workload."""
    import numpy as np
    import torch

    import oracle
    import synth
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    spec = synth.C3
    per_step = args.ref_sample
    n_train = 16
    tr = synth.stream(spec, "train", count=n_train, dtype=torch.float64).numpy()
    S, _, _, _ = oracle.train_sketch(list(tr), spec.k)
    S = S.astype(np.float32).astype(np.float64)
    te = synth.stream(spec, "test", count=per_step).double().numpy()  # BF16 values
    for _ in range(args.warmup):
        for A in te:
            oracle.scw(A, S, spec.r, dense=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for A in te:
            oracle.scw(A, S, spec.r, dense=False)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    cores = cpu_threads()
    sample = (f"{per_step} of the 500 test matrices (2048x2048, BF16 values in "
              f"float64) per step; sketch from {n_train} training matrices")
    line = {
        "impl": "reference",
        "metric": "stream matrices/s, rank-r SCW (BF16 vs FP32 path) at rel-err gap <=1e-3",
        "value": value, "unit": "matrices/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "C3 test pass: 2048x2048, k=40, r=20 (oracle sample)",
                   "m": spec.m, "n": spec.n, "k": spec.k, "r": spec.r},
        "cpu_baseline": {"value": value, "unit": "matrices/s", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "matrices/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
def _timed_plan(plan, steps, ws, dist, probe=True):
    """Executes a plan `steps` times between barriers; returns the total
    device time (CUDA events on the launching stream) and the per-execution
    sketch-pass times (event-record nodes inside the plan's graph)."""
    import torch
    evb = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    eve = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for e in evb + eve:
        e.record()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record()
    for i in range(steps):
        if probe:
            plan.set_probe(evb[i], eve[i])
        plan.execute()
    t_end.record()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    total_ms = t_start.elapsed_time(t_end)
    stage_ms = [b.elapsed_time(e) for b, e in zip(evb, eve)] if probe else []
    if probe:
        plan.set_probe(None, None)
    return total_ms, stage_ms


def _max_over_ranks(v, ws, dist):
    import torch
    t = torch.tensor([v], device="cuda", dtype=torch.float64)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sgemm_peak():
    """FP32 FMA peak of this GPU, measured: a CUDA-core SGEMM (cuBLAS,
    TF32 off) of 8192^3, best of 5, as the BF16 denominator is measured
    with a cuBLAS GEMM."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        n = 8192
        a = torch.randn(n, n, device="cuda")
        b = torch.randn(n, n, device="cuda")
        c = torch.empty(n, n, device="cuda")
        for _ in range(2):
            torch.matmul(a, b, out=c)
        best = 1e30
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        del a, b, c
        return 2.0 * n ** 3 / (best / 1e3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def device_median_ms(fn, reps):
    """Median over `reps` calls of fn's time between CUDA events on the
    current stream."""
    import torch
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return sorted(ts)[len(ts) // 2]


def fp8_training_gram(tsk, h, tr, G_bf16, k, peaks, peak_src):
    """The training Gram from E4M3 copies (per-row, per-8-matrix power-of-two
    scales): quantisation (into buffers allocated once; the call's host-side
    pointer copy and stream synchronisation included) and Gram timed on the
    device, the Gram against
    twice the measured BF16 peak (the nominal FP8 / BF16 tensor ratio), and
    the sketch it gives scored on the BF16 Gram: the fraction of the best
    captured energy trace(S G S^T) (Eq. 3.2) that it keeps."""
    import torch
    D, m, n = tr.shape
    mats = tr  # (D, m, n): the binding computes the matrices' addresses
    A8, scales = h.quantize_e4m3(mats)
    G8 = h.gram_e4m3(A8, scales, n)  # encodes and caches the tensor maps
    torch.cuda.synchronize()
    q_ms = device_median_ms(lambda: h.quantize_e4m3(mats, out=(A8, scales)), 3)
    g_ms = device_median_ms(lambda: h.gram_e4m3(A8, scales, n, out=G8), 3)
    flops = float(m) ** 2 * n * D
    tf = flops / (g_ms / 1e3) / 1e12
    peak = 2.0 * float(peaks.get("bf16_tflops", PEAKS_FALLBACK["bf16_tflops"]))
    S8, _, st8 = h.sketch_from_gram(G8, k, prec=tsk.FP32)
    Sb, _, stb = h.sketch_from_gram(G_bf16, k, prec=tsk.FP32)
    Gd = G_bf16.double()
    cap8 = float(torch.trace(S8.double() @ Gd @ S8.double().T))
    capb = float(torch.trace(Sb.double() @ Gd @ Sb.double().T))
    rel = float((G8 - Gd).abs().max() / Gd.diagonal().max())
    del A8, scales, G8
    qbytes = float(D) * m * n * (tr.element_size() + 1)  # A read once, E4M3 written
    qgbs = qbytes / (q_ms / 1e3) / 1e9
    hbm = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    return {"quantize_ms": q_ms, "gram_ms": g_ms, "status": [st8, stb],
            "quantize_roofline": {"bound": "hbm", "achieved": qgbs, "peak": hbm, "unit": "GB/s",
                                  "frac": qgbs / hbm, "bytes": qbytes},
            "gram_max_abs_diff_over_max_diag": rel,
            "captured_energy_vs_bf16_gram": cap8 / capb,
            "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                         "frac": tf / peak,
                         "peak_source": "2 x bf16_tflops (burst) of " + peak_src +
                                        " (nominal FP8 / BF16 ratio)", "flops": flops}}


def run_tsk(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2209_14637_gb300 as tsk
    import synth
    from paper_2209_14637_gb300 import build as _build

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    if rank == 0 or ws == 1:
        _build.build()
    if ws > 1:
        dist.barrier()
    peaks, peak_src = load_peaks()
    spec = synth.C3
    count = args.matrices if args.matrices > 0 else spec.n_test
    refine = {"always": tsk.REFINE_ALWAYS, "auto": tsk.REFINE_AUTO,
              "never": tsk.REFINE_NEVER}[args.refine]
    h = tsk.Handle(kernel=args.kernel, refine_q=refine)

    # ---- training side (timed separately, not part of the metric) --------
    from paper_2209_14637_gb300.dist import allreduce_gram, shard_range
    a, b = shard_range(args.train, ws, rank)
    stage(f"generating training matrices {a}..{b}")
    tr = synth.stream(spec, "train", device="cuda", start=a, count=b - a)
    torch.cuda.synchronize()
    stage("training the sketch")
    t0 = time.perf_counter()
    # mode-1 Gram of this rank's shard, summed over ranks (the one exchange
    # of the training side), then the leading eigenvectors on every rank
    G = h.gram(tr, mode=1)
    allreduce_gram(G)
    S, eig, st = h.sketch_from_gram(G, spec.k, prec=tsk.BF16)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    # the Gram (T1) once more, timed on the device (its tensor maps are
    # cached by the handle, so this is the kernel's time): a tensor-bound
    # SYRK of m^2 n multiply-adds' worth of flops per matrix (half of 2 m^2 n)
    mats = tr
    gram_ms = device_median_ms(lambda: h.gram(mats, mode=1, out=G), 3)
    gram_flops = float(spec.m) ** 2 * spec.n * (b - a)
    gram_tf = gram_flops / (gram_ms / 1e3) / 1e12
    gpeak = float(peaks.get("bf16_tflops", PEAKS_FALLBACK["bf16_tflops"]))
    train_info = {"matrices": b - a, "total_s": train_s, "gram_ms": gram_ms,
                  "gram_kernel": "tcgen05" if args.kernel != tsk.KERNEL_SIMT else "simt",
                  "roofline": {"bound": "tensor", "achieved": gram_tf, "peak": gpeak,
                               "unit": "TFLOP/s", "frac": gram_tf / gpeak,
                               "peak_source": "bf16_tflops (burst) of " + peak_src,
                               "flops": gram_flops}}
    if args.kernel != tsk.KERNEL_SIMT:
        train_info["fp8"] = fp8_training_gram(tsk, h, tr, G, spec.k, peaks, peak_src)
        # T1' (the mode-2 Gram sum_d A_d^T A_d, n x n, Eq. 3.6) on the same
        # matrices: the tensor-core kernel with MN-major operands
        G2 = h.gram(mats, mode=2)
        torch.cuda.synchronize()
        g2_ms = device_median_ms(lambda: h.gram(mats, mode=2, out=G2), 3)
        g2_flops = float(spec.n) ** 2 * spec.m * (b - a)
        g2_tf = g2_flops / (g2_ms / 1e3) / 1e12
        train_info["mode2"] = {"gram_ms": g2_ms,
                               "roofline": {"bound": "tensor", "achieved": g2_tf, "peak": gpeak,
                                            "unit": "TFLOP/s", "frac": g2_tf / gpeak,
                                            "peak_source": "bf16_tflops (burst) of " + peak_src,
                                            "flops": g2_flops}}
        del G2
    stage(f"training Gram: {train_info}")
    del tr, G
    torch.cuda.empty_cache()

    # ---- test side: this rank's shard of the stream (weak scaling) --------
    stage(f"trained in {train_s:.2f} s (status {st}); generating the test stream")
    te = synth.stream(spec, "test", device="cuda", start=rank * count, count=count)
    err = torch.empty(count, dtype=torch.float64, device="cuda")
    tune = None
    if not args.no_tune and te.dtype == torch.bfloat16 and args.kernel != tsk.KERNEL_SIMT:
        # the project's autotuner picks the sketch kernel's rows per CTA for
        # this workload's size class (untimed, before the plan is built)
        import tempfile
        h.autotune(te, S, spec.r)
        with tempfile.TemporaryDirectory() as td:
            h.autotune_save(os.path.join(td, "t.json"))
            with open(os.path.join(td, "t.json")) as f:
                tune = json.load(f)["classes"]
        stage(f"autotune: {tune}")
    plan = h.plan(te, S, spec.r, err)
    info = plan.info()
    plan_kind = "tcgen05" if te.dtype == torch.bfloat16 and args.kernel != tsk.KERNEL_SIMT else "simt"
    stage(f"plan ready: {info}")

    for _ in range(args.warmup):
        plan.execute()
    torch.cuda.synchronize()
    stage(f"timing the BF16 path (refine {args.refine})")
    clocks = ClockSampler(local)
    clocks.start()
    clocks.mark()
    total_ms, stage_ms = _timed_plan(plan, args.steps, ws, dist)
    clocks.mark_end()
    # untimed: the same step keeps the GPU busy until a few clock samples
    # have landed after the region (a short region may hold none)
    while clocks.need_more():
        plan.execute()
        torch.cuda.synchronize()
    clk = clocks.stop()
    assert h.sync_status() == 0
    max_ms = _max_over_ranks(total_ms, ws, dist)
    value = count * ws * args.steps / (max_ms / 1e3)
    ms_per_step = max_ms / args.steps
    stage_avg = statistics.mean(stage_ms)
    stage(f"bf16: {value:.1f} matrices/s, {ms_per_step:.3f} ms/step, sketch pass "
          f"{stage_avg:.3f} ms, clocks {clk}")
    alg_bytes = float(sum(te[i].numel() * te[i].element_size() for i in range(count)))
    achieved = alg_bytes / (stage_avg / 1e3) / 1e9
    peak = float(peaks["hbm_gbs"])

    def side_variant(hv, steps):
        """Matrices/s of the same workload through another handle setting."""
        pv = hv.plan(te, S, spec.r, torch.empty(count, dtype=torch.float64, device="cuda"))
        for _ in range(max(1, args.warmup)):
            pv.execute()
        ms, _ = _timed_plan(pv, steps, ws, dist, probe=False)
        ms = _max_over_ranks(ms, ws, dist)
        pv.close()
        return {"value": count * ws * steps / (ms / 1e3), "unit": "matrices/s",
                "ms_per_step": ms / steps, "steps": steps}

    variants = {}
    if not args.no_variants:
        # the adaptive refinement (only matrices whose rounding bound asks)
        ha = tsk.Handle(kernel=args.kernel, refine_q=tsk.REFINE_AUTO)
        variants["refine_auto"] = side_variant(ha, args.steps)
        ha.close()
        # the k x k steps in FP64 (Householder R factors + Jacobi SVD in double)
        hd = tsk.Handle(kernel=args.kernel, refine_q=refine, small_fp64=True)
        variants["small_fp64"] = side_variant(hd, max(1, min(args.steps, 5)))
        hd.close()
        stage(f"variants: {variants}")

    # ---- plain FP32 path on the same matrices ----------------------------
    fp32 = None
    sgemm = None
    if not args.no_fp32:
        stage("timing the FP32 path")
        te32 = te.float()
        err32 = torch.empty(count, dtype=torch.float64, device="cuda")
        h32 = tsk.Handle(refine_q=refine)
        plan32 = h32.plan(te32, S, spec.r, err32)
        for _ in range(max(1, args.warmup)):
            plan32.execute()
        steps32 = max(1, min(args.steps, 10))
        ms32, st32 = _timed_plan(plan32, steps32, ws, dist)
        ms32 = _max_over_ranks(ms32, ws, dist)
        sgemm = _sgemm_peak()
        sk32 = statistics.mean(st32)
        flops32 = 4.0 * spec.m * spec.n * spec.k * count
        fp32 = {"value": count * ws * steps32 / (ms32 / 1e3), "unit": "matrices/s",
                "ms_per_step": ms32 / steps32, "steps": steps32,
                "sketch_pass_ms": sk32,
                "roofline": {"bound": "alu", "achieved": flops32 / (sk32 / 1e3) / 1e12,
                             "peak": sgemm, "unit": "TFLOP/s",
                             "frac": flops32 / (sk32 / 1e3) / 1e12 / sgemm,
                             "peak_source": "FP32 SGEMM (cuBLAS, TF32 off) 8192^3 "
                                            "measured in this run",
                             "kernel": "CUDA-core sketch pass (X = A^T S^T, Y = A X)",
                             "flops": flops32}}
        stage(f"fp32: {fp32}")

    # ---- end to end through the public API with host buffers -------------
    e2e = None
    if not args.no_e2e:
        stage("end to end with host buffers")
        # The inputs live in page-locked host memory (cudaHostAlloc), filled
        # once outside the timed region.  Each step streams them to the
        # device in chunks on a copy stream and runs one plan per chunk as
        # soon as its chunk has landed, so the copy of chunk i + 1 overlaps
        # the SCW of chunk i; the errors come back to host memory.
        host = torch.empty(te.shape, dtype=te.dtype, pin_memory=True)
        host.copy_(te)
        err_host = torch.empty(count, dtype=torch.float64, pin_memory=True)
        nch = max(1, min(args.e2e_chunks, count))
        bnd = [count * i // nch for i in range(nch + 1)]
        cplans = [h.plan(te[bnd[i]:bnd[i + 1]], S, spec.r, err[bnd[i]:bnd[i + 1]])
                  for i in range(nch)]
        cs = torch.cuda.Stream()
        main_s = torch.cuda.current_stream()
        copied = [torch.cuda.Event() for _ in range(nch)]
        consumed = [torch.cuda.Event() for _ in range(nch)]
        for ev in consumed:
            ev.record(main_s)

        def e2e_step():
            for i in range(nch):
                cs.wait_event(consumed[i])  # the last step's SCW of chunk i has read it
                with torch.cuda.stream(cs):
                    te[bnd[i]:bnd[i + 1]].copy_(host[bnd[i]:bnd[i + 1]], non_blocking=True)
                copied[i].record(cs)
            for i in range(nch):
                main_s.wait_event(copied[i])
                cplans[i].execute()
                consumed[i].record(main_s)
            err_host.copy_(err, non_blocking=True)

        steps_e = max(1, min(args.steps, 5))
        e2e_step()
        torch.cuda.synchronize()
        stage("end to end: timed steps")
        if ws > 1:
            dist.barrier()
        a_ev = torch.cuda.Event(enable_timing=True)
        b_ev = torch.cuda.Event(enable_timing=True)
        a_ev.record()
        for _ in range(steps_e):
            e2e_step()
        b_ev.record()
        torch.cuda.synchronize()
        ms_e = _max_over_ranks(a_ev.elapsed_time(b_ev), ws, dist)
        e2e = {"value": count * ws * steps_e / (ms_e / 1e3), "unit": "matrices/s",
               "h2d_bytes_per_step": int(alg_bytes), "d2h_bytes_per_step": 8 * count,
               "steps": steps_e, "host_buffer": "page-locked (cudaHostAlloc)",
               "chunks": nch, "ms_per_step": ms_e / steps_e,
               "h2d_gbs": alg_bytes / (ms_e / steps_e) / 1e6}
        stage(f"e2e: {e2e}")
        for cp in cplans:
            cp.close()
        del host

    # ---- oracle on a bounded sample: CPU baseline and the error gap ------
    # The oracle trains its own sketch (16 training matrices) and runs SCW
    # on a sample of the test matrices; the GPU paths run the same sample
    # with that sketch (rounded to float32, the sketch type of the BF16 and
    # FP32 paths), so no oracle input comes from the GPU.
    cpu = None
    gap = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        stage("oracle sample on the host cores")
        import oracle
        tr_o = synth.stream(spec, "train", device="cuda", count=16)
        S_o, _, _, _ = oracle.train_sketch(list(tr_o.double().cpu().numpy()), spec.k)
        del tr_o
        S_o32 = torch.tensor(S_o, device="cuda", dtype=torch.float32)
        Sn = S_o32.double().cpu().numpy()
        idx = list(range(0, count, max(1, count // args.cpu_sample)))[:args.cpu_sample]
        mats = [te[i].double().cpu().numpy() for i in idx]
        t0 = time.perf_counter()
        ref = np.array([oracle.scw(A, Sn, spec.r, dense=False)["err"] for A in mats])
        dt = time.perf_counter() - t0
        cpu = {"value": len(mats) / dt, "unit": "matrices/s", "cores": cpu_threads(),
               "kind": "oracle",
               "sample": f"{len(mats)} of the {count} test matrices, FP64 numpy SCW"}
        sub = te[idx]
        gap = {}
        runs = [("bf16", dict(refine_q=refine), sub),
                ("bf16_small_fp64", dict(refine_q=refine, small_fp64=True), sub),
                ("bf16_refine_auto", dict(refine_q=tsk.REFINE_AUTO), sub),
                ("fp32", dict(refine_q=refine), sub.float())]
        got = {}
        for name, kw, A in runs:
            hv = tsk.Handle(kernel=args.kernel, **kw)
            o = hv.approx_batch(A, S_o32, spec.r)
            torch.cuda.synchronize()
            assert hv.sync_status() == 0
            got[name] = o["err"].cpu().numpy()
            gap[name] = float(np.max(np.abs(got[name] - ref) / ref))
            hv.close()
        # the k x k steps in FP32 against the same steps in FP64, on the
        # same BF16 panels
        gap["fp32_vs_fp64_kxk"] = float(np.max(np.abs(got["bf16"] - got["bf16_small_fp64"])
                                               / got["bf16_small_fp64"]))
        gap["checked"] = len(mats)
        gap["sketch"] = "oracle's, from 16 training matrices (FP64 Gram + eigh)"
        stage(f"oracle: {cpu}; gap {gap}")

    extra = {}
    if not args.no_extra:
        extra = run_extra_workloads(args, tsk, h, sgemm, peaks, ws, dist, rank)

    if rank == 0:
        traffic = None
        if plan_kind == "tcgen05" and (spec.m, spec.n, spec.k) == (2048, 2048, 40):
            traffic = SKETCH_TRAFFIC_PER_MATRIX * count
        line = {
            "metric": "stream matrices/s, rank-r SCW (BF16 vs FP32 path) at rel-err gap <=1e-3",
            "value": value, "unit": "matrices/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"C3 test pass: {count} stream matrices 2048x2048 BF16 "
                                   "per GPU, k=40, r=20, one refinement step on Q per "
                                   f"matrix (refine={args.refine}), sketch trained on "
                                   f"{args.train} matrices of the stream",
                       "m": spec.m, "n": spec.n, "k": spec.k, "r": spec.r,
                       "refine": args.refine,
                       "small_factors": "fp32 (Gram route); fp64 timed in small_fp64",
                       "matrices_per_step_per_gpu": count,
                       "l2": f"inputs ({alg_bytes / 1e9:.2f} GB per step) larger than "
                             "L2 (129 MB); no flush",
                       "sketch_kernel": plan_kind,
                       "autotune": tune},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": f"hbm_gbs of {peak_src}",
                         "kernel": "sketch pass (X = A^T S^T, Y = A X)",
                         "kernel_ms": stage_avg,
                         "algorithmic_bytes": alg_bytes,
                         "traffic": traffic,
                         "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum "
                                            "of one 64-matrix launch of this shape, scaled to "
                                            "this launch by the number of matrices"
                                            if traffic is not None else None)},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": info["launches"] * args.steps,
            "fp32_path": fp32,
            "variants": variants,
            "rel_err_gap": gap,
            "train_s": train_s,
            "train": train_info,
            "train_status": st,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if fp32 is not None:
        plan32.close()
        h32.close()
    plan.close()
    h.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def _optimal_errors(As, r):
    """||A - A_r||_F of the best rank-r approximation (Eckart-Young): the
    reference the test error (Eq. 4.1) is measured against.  A plain
    singular-value routine in float64 (reporting, not part of the path)."""
    import torch
    out = []
    for A in As:
        A64 = A.detach().to(torch.float64)
        try:
            s = torch.linalg.svdvals(A64)
        except Exception:  # no device linear-algebra library: use the host
            s = torch.linalg.svdvals(A64.cpu())
        out.append(float(torch.sqrt(torch.sum(s[r:] ** 2))))
    return out


def _test_error(errs, opt):
    """Eq. 4.1: the mean over the test set of (err - opt) / opt."""
    return float(sum((e - o) / o for e, o in zip(errs, opt)) / len(opt))


def run_extra_workloads(args, tsk, h, sgemm, peaks, ws, dist, rank):
    """The other workloads of the method, each under its own key: C2 (FP32,
    1024 x 768), C4 (512 ragged BF16 matrices in one plan), C5 (the learned
    refiner), the classical random sketches (Gaussian, sign) against the
    tensor sketch, and the training-fraction sweep."""
    import dataclasses

    import torch

    import synth
    out = {}
    peak_hbm = float(peaks["hbm_gbs"])

    def timed_value(plan, n, steps, probe=True):
        for _ in range(max(1, args.warmup)):
            plan.execute()
        ms, st = _timed_plan(plan, steps, ws, dist, probe=probe)
        ms = _max_over_ranks(ms, ws, dist)
        return n * ws * steps / (ms / 1e3), ms / steps, (statistics.mean(st) if st else None)

    # ---- C2: plain FP32 path, HSI shape --------------------------------
    spec2 = synth.C2
    stage("C2: training on 400 FP32 matrices")
    tr2 = synth.stream(spec2, "train", device="cuda")
    h2 = tsk.Handle(refine_q=tsk.REFINE_ALWAYS)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S2, _, _, st2 = h2.train_sketch(tr2, spec2.k)
    torch.cuda.synchronize()
    train2_s = time.perf_counter() - t0
    te2 = synth.stream(spec2, "test", device="cuda")
    err2 = torch.empty(spec2.n_test, dtype=torch.float64, device="cuda")
    p2 = h2.plan(te2, S2, spec2.r, err2)
    v2, ms2, sk2 = timed_value(p2, spec2.n_test, args.steps)
    flops2 = 4.0 * spec2.m * spec2.n * spec2.k * spec2.n_test
    opt2 = _optimal_errors(te2[:50], spec2.r)
    c2 = {"value": v2, "unit": "matrices/s", "ms_per_step": ms2, "dtype": "f32",
          "workload": "C2: 200 FP32 1024x768 matrices per step, k=20, r=10, sketch from "
                      "400 training matrices, one refinement step per matrix",
          "train_s": train2_s, "train_status": st2,
          "test_error_4_1": _test_error(err2[:50].tolist(), opt2),
          "roofline": ({"bound": "alu", "achieved": flops2 / (sk2 / 1e3) / 1e12,
                        "peak": sgemm, "unit": "TFLOP/s",
                        "frac": flops2 / (sk2 / 1e3) / 1e12 / sgemm,
                        "peak_source": "FP32 SGEMM (cuBLAS, TF32 off) measured in this run",
                        "kernel": "CUDA-core sketch pass", "flops": flops2}
                       if sgemm else None)}
    # NEXT-4: the data-oblivious sketches of classical SCW on the same matrices
    rnd = {"tensor": c2["test_error_4_1"]}
    for kind in ("gauss", "sign"):
        Sr = synth.random_sketch(kind, spec2.k, spec2.m, spec2.seed, device="cuda")
        e = h2.approx_batch(te2[:50], Sr, spec2.r)["err"]
        rnd[kind] = _test_error(e.tolist(), opt2)
    out["c2"] = c2
    out["random_sketch_test_error"] = dict(rnd, matrices=50, workload="C2")
    stage(f"C2: {c2}; random sketches {rnd}")
    p2.close()

    # two-sided sketching (Algorithms 3 and 5) on the same stream, k = l = 20:
    # a synthetic analogue of the paper's comparison of the two methods
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S2t, W2t, energy, sweeps, _ = h2.train_two_sided(tr2, spec2.k, spec2.k)
    torch.cuda.synchronize()
    train_two = time.perf_counter() - t0
    h2.approx_two_sided(te2, S2t, W2t, spec2.r)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = 5
    for _ in range(reps):
        e_two = h2.approx_two_sided(te2, S2t, W2t, spec2.r)["err"]
    torch.cuda.synchronize()
    test_two = (time.perf_counter() - t0) / reps
    out["two_sided"] = {
        "workload": "C2 stream: HOOI (HOSVD start) on the 400 training matrices, k = l = 20; "
                    "Algorithm 3 on the 200 test matrices, r = 10",
        "train_s": train_two, "hooi_sweeps": sweeps, "core_energy": energy,
        "test_s": test_two, "value": spec2.n_test / test_two, "unit": "matrices/s",
        "timing": "host wall clock around the blocking call (descriptor staging included)",
        "test_error_4_1": {"two_sided": _test_error(e_two[:50].tolist(), opt2),
                           "one_sided": c2["test_error_4_1"], "matrices": 50},
        "one_sided": {"train_s": train2_s, "test_s": spec2.n_test / v2}}
    stage(f"two-sided: {out['two_sided']}")
    del tr2

    # NEXT-3: training fraction (2 %, 20 %, 80 % of a 600-matrix C2 stream),
    # the Gram accumulated chunk by chunk as the stream arrives
    pool = dataclasses.replace(spec2, n_train=500, n_test=100)
    teP = synth.stream(pool, "test", device="cuda", count=50)
    optP = _optimal_errors(teP, pool.r)
    sweep = {}
    G = None
    done = 0
    for frac in (0.02, 0.2, 0.8):
        want = int(round(frac * 600))
        while done < want:
            c = min(want - done, 60)
            chunk = synth.stream(pool, "train", device="cuda", start=done, count=c)
            G = h2.gram([chunk[i] for i in range(c)], mode=1, out=G, accumulate=G is not None)
            done += c
        Sf, _, _ = h2.sketch_from_gram(G, pool.k, prec=tsk.FP32)
        e = h2.approx_batch(teP, Sf, pool.r)["err"]
        sweep[f"{int(frac * 100)}%"] = {"train_matrices": want,
                                        "test_error_4_1": _test_error(e.tolist(), optP)}
    out["sample_ratio"] = dict(sweep, test_matrices=50, stream=600, workload="C2 stream")
    stage(f"sample ratio: {out['sample_ratio']}")
    h2.close()
    del te2, teP
    torch.cuda.empty_cache()

    # ---- C4: 512 ragged BF16 matrices in one plan -----------------------
    stage("C4: generating 512 ragged matrices")
    items = synth.ragged_sizes(512)
    S4 = [synth.item_sketch(it, device="cuda") for it in items]
    r4 = [it.r for it in items]
    c4 = {"workload": "C4: 512 BF16 matrices per step, m in [256, 4096], n in [256, 2048] "
                      "log-uniform, k in {10, 20, 40}, r = k/2, one refinement step each",
          "unit": "matrices/s"}
    for pad in (True, False):
        A4 = synth.ragged_batch(items, device="cuda", pad_rows=pad)
        alg4 = float(sum(it.m * it.n * 2 for it in items))
        h4 = tsk.Handle(refine_q=tsk.REFINE_ALWAYS)
        if not args.no_tune:
            h4.autotune(A4, S4, r4)
        e4 = torch.empty(len(items), dtype=torch.float64, device="cuda")
        p4 = h4.plan(A4, S4, r4, e4)
        inf4 = p4.info()
        v4, ms4, sk4 = timed_value(p4, len(items), args.steps)
        key = "padded_rows" if pad else "contiguous_rows"
        c4[key] = {"value": v4, "ms_per_step": ms4, "sketch_pass_ms": sk4,
                   "launches": inf4["launches"],
                   "tensor_core_matrices": sum(it.m <= 4096 and it.k <= 48 for it in items),
                   "copied_to_aligned_rows": sum((A.stride(0) * 2) % 16 != 0
                                                 or A.data_ptr() % 16 != 0 for A in A4),
                   "roofline": {"bound": "hbm", "achieved": alg4 / (sk4 / 1e3) / 1e9,
                                "peak": peak_hbm, "unit": "GB/s",
                                "frac": alg4 / (sk4 / 1e3) / 1e9 / peak_hbm,
                                "algorithmic_bytes": alg4,
                                "kernel": "sketch pass"}}
        p4.close()
        h4.close()
        del A4
    out["c4"] = c4
    stage(f"C4: {c4}")
    del S4
    torch.cuda.empty_cache()

    # ---- C5: the learned refiner ------------------------------------------
    spec5 = synth.C5
    stage("C5: refiner")
    tr5 = synth.stream(spec5, "train", device="cuda")
    te5 = synth.stream(spec5, "test", device="cuda")
    h5 = tsk.Handle()
    S5, _, _, _ = h5.train_sketch(tr5, spec5.k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dS, hist = h5.refine_sketch(tr5[:350], tr5[350:], S5, spec5.r, steps=args.c5_steps,
                                batch=16, lr=1e-3, eval_every=100)
    torch.cuda.synchronize()
    dt5 = time.perf_counter() - t0
    opt5 = _optimal_errors(te5[:50], spec5.r)
    plain = h5.approx_batch(te5[:50], S5, spec5.r)["err"].tolist()
    refined = h5.approx_batch(te5[:50], S5 + dS, spec5.r)["err"].tolist()
    out["c5"] = {"workload": "C5: refiner S_theta = S_tensor + dS, 1024x768 FP32, k=20, "
                             f"r=10, SGD batch 16, lr 1e-3, {args.c5_steps} steps on 350 "
                             "training matrices, validation on 50",
                 "steps_per_s": args.c5_steps / dt5, "train_s": dt5,
                 "val_loss_first_best": [hist[0], min(hist)],
                 "held_out_test_error_4_1": {"tensor": _test_error(plain, opt5),
                                             "refined": _test_error(refined, opt5),
                                             "matrices": 50},
                 "held_out_mean_err": {"tensor": sum(plain) / 50, "refined": sum(refined) / 50,
                                       "optimal": sum(opt5) / 50}}
    stage(f"C5: {out['c5']}")
    h5.close()
    return out


def main():
    faulthandler.enable()
    faulthandler.dump_traceback_later(600, repeat=True)
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="tsk", choices=["tsk", "reference"])
    ap.add_argument("--kernel", type=int, default=0, help="0 auto, 1 simt, 2 tcgen05")
    ap.add_argument("--train", type=int, default=1000)
    ap.add_argument("--matrices", type=int, default=0,
                    help="stream matrices per step and GPU (default: the 500 of the "
                         "workload; smaller values are for profiling captures)")
    ap.add_argument("--cpu-sample", type=int, default=24)
    ap.add_argument("--ref-sample", type=int, default=4)
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-chunks", type=int, default=4,
                    help="chunks the end-to-end leg streams and computes in overlap")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the refine_auto and small_fp64 timings")
    ap.add_argument("--c5-steps", type=int, default=2000)
    ap.add_argument("--no-tune", action="store_true",
                    help="build the plans without running the sketch-shape autotuner")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the C2, C4 and C5 workloads")
    ap.add_argument("--refine", default="always", choices=["always", "auto", "never"],
                    help="refinement of Q on the headline path (the workload states one "
                         "step per matrix)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_tsk(args)


if __name__ == "__main__":
    sys.exit(main())
