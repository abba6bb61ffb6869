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
# kernel with k = 40, from ncu on a 64-matrix launch (537.21 MB read, 33.06 MB
# written); re-measure whenever that kernel changes.
SKETCH_TRAFFIC_PER_MATRIX = (537.21e6 + 33.06e6) / 64

def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return PEAKS_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

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
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "samples": len(sm), "reasons": sorted(reasons)}


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
    h = tsk.Handle(kernel=args.kernel)

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
    G = h.gram([tr[i] for i in range(tr.shape[0])], mode=1)
    allreduce_gram(G)
    S, eig, st = h.sketch_from_gram(G, spec.k, prec=tsk.BF16)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    # the Gram (T1) once more, timed on the device: a tensor-bound SYRK of
    # m^2 n multiply-adds' worth of flops per matrix (half of 2 m^2 n)
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record()
    h.gram([tr[i] for i in range(tr.shape[0])], mode=1, out=G)
    g1.record()
    torch.cuda.synchronize()
    gram_ms = g0.elapsed_time(g1)
    gram_flops = float(spec.m) ** 2 * spec.n * (b - a)
    gram_tf = gram_flops / (gram_ms / 1e3) / 1e12
    gpeak = float(peaks.get("bf16_tflops", PEAKS_FALLBACK["bf16_tflops"]))
    train_info = {"matrices": b - a, "total_s": train_s, "gram_ms": gram_ms,
                  "gram_kernel": "tcgen05" if args.kernel != tsk.KERNEL_SIMT else "simt",
                  "roofline": {"bound": "tensor", "achieved": gram_tf, "peak": gpeak,
                               "unit": "TFLOP/s", "frac": gram_tf / gpeak,
                               "peak_source": "bf16_tflops of " + peak_src,
                               "flops": gram_flops}}
    stage(f"training Gram: {train_info}")
    del tr, G
    torch.cuda.empty_cache()

    # ---- test side: this rank's shard of the stream (weak scaling) --------
    stage(f"trained in {train_s:.2f} s (status {st}); generating the test stream")
    te = synth.stream(spec, "test", device="cuda", start=rank * count, count=count)
    err = torch.empty(count, dtype=torch.float64, device="cuda")
    plan = h.plan(te, S, spec.r, err)
    info = plan.info()
    plan_kind = "tcgen05" if te.dtype == torch.bfloat16 and args.kernel != tsk.KERNEL_SIMT else "simt"
    stage(f"plan ready: {info}")

    def timed(plan_, steps, probe=True):
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
                plan_.set_probe(evb[i], eve[i])
            plan_.execute()
        t_end.record()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        total_ms = t_start.elapsed_time(t_end)
        stage_ms = [b.elapsed_time(e) for b, e in zip(evb, eve)] if probe else []
        if probe:
            plan_.set_probe(None, None)
        return total_ms, stage_ms

    for _ in range(args.warmup):
        plan.execute()
    torch.cuda.synchronize()
    stage("timing the BF16 path")
    clocks = ClockSampler(local)
    clocks.start()
    total_ms, stage_ms = timed(plan, args.steps)
    clk = clocks.stop()
    assert h.sync_status() == 0
    t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    value = count * ws * args.steps / (max_ms / 1e3)
    ms_per_step = max_ms / args.steps
    stage_avg = statistics.mean(stage_ms)
    stage(f"bf16: {value:.1f} matrices/s, {ms_per_step:.3f} ms/step, sketch pass "
          f"{stage_avg:.3f} ms, clocks {clk}")
    alg_bytes = float(sum(te[i].numel() * te[i].element_size() for i in range(count)))
    achieved = alg_bytes / (stage_avg / 1e3) / 1e9
    peak = float(peaks["hbm_gbs"])

    # ---- plain FP32 path on the same matrices ----------------------------
    fp32 = None
    if not args.no_fp32:
        stage("timing the FP32 path")
        te32 = te.float()
        err32 = torch.empty(count, dtype=torch.float64, device="cuda")
        h32 = tsk.Handle()
        plan32 = h32.plan(te32, S, spec.r, err32)
        for _ in range(max(1, args.warmup)):
            plan32.execute()
        steps32 = max(1, min(args.steps, 10))
        ms32, st32 = timed(plan32, steps32)
        t = torch.tensor([ms32], device="cuda", dtype=torch.float64)
        if ws > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms32 = float(t.item())
        fp32 = {"value": count * ws * steps32 / (ms32 / 1e3), "unit": "matrices/s",
                "ms_per_step": ms32 / steps32, "steps": steps32,
                "sketch_pass_ms": statistics.mean(st32)}
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
        main = torch.cuda.current_stream()
        copied = [torch.cuda.Event() for _ in range(nch)]
        consumed = [torch.cuda.Event() for _ in range(nch)]
        for ev in consumed:
            ev.record(main)

        def e2e_step():
            for i in range(nch):
                cs.wait_event(consumed[i])  # the last step's SCW of chunk i has read it
                with torch.cuda.stream(cs):
                    te[bnd[i]:bnd[i + 1]].copy_(host[bnd[i]:bnd[i + 1]], non_blocking=True)
                copied[i].record(cs)
            for i in range(nch):
                main.wait_event(copied[i])
                cplans[i].execute()
                consumed[i].record(main)
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
        ms_e = a_ev.elapsed_time(b_ev)
        t = torch.tensor([ms_e], device="cuda", dtype=torch.float64)
        if ws > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_e = float(t.item())
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
    cpu = None
    gap = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        stage("oracle sample on the host cores")
        import oracle
        Sn = S.double().cpu().numpy()
        idx = list(range(0, count, max(1, count // args.cpu_sample)))[:args.cpu_sample]
        mats = [te[i].double().cpu().numpy() for i in idx]
        t0 = time.perf_counter()
        ref = [oracle.scw(A, Sn, spec.r, dense=False)["err"] for A in mats]
        dt = time.perf_counter() - t0
        cpu = {"value": len(mats) / dt, "unit": "matrices/s", "cores": cpu_threads(),
               "kind": "oracle",
               "sample": f"{len(mats)} of the {count} test matrices, FP64 numpy SCW"}
        plan.execute()
        torch.cuda.synchronize()
        g = err.cpu().numpy()[idx]
        gap = {"bf16": float(np.max(np.abs(g - ref) / np.asarray(ref)))}
        if fp32 is not None:
            plan32.execute()
            torch.cuda.synchronize()
            g32 = err32.cpu().numpy()[idx]
            gap["fp32"] = float(np.max(np.abs(g32 - ref) / np.asarray(ref)))
        gap["checked"] = len(mats)
        stage(f"oracle: {cpu}; gap {gap}")

    if rank == 0:
        line = {
            "metric": "stream matrices/s, rank-r SCW (BF16 vs FP32 path) at rel-err gap <=1e-3",
            "value": value, "unit": "matrices/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"C3 test pass: {count} stream matrices 2048x2048 BF16 "
                                   "per GPU, k=40, r=20, sketch trained on "
                                   f"{args.train} matrices of the stream",
                       "m": spec.m, "n": spec.n, "k": spec.k, "r": spec.r,
                       "matrices_per_step_per_gpu": count,
                       "l2": f"inputs ({alg_bytes / 1e9:.2f} GB per step) larger than "
                             "L2 (129 MB); no flush",
                       "sketch_kernel": plan_kind},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": f"hbm_gbs of {peak_src}",
                         "kernel": "sketch pass (X = A^T S^T, Y = A X)",
                         "kernel_ms": stage_avg,
                         "algorithmic_bytes": alg_bytes,
                         "traffic": (SKETCH_TRAFFIC_PER_MATRIX * count
                                     if plan_kind == "tcgen05" else None),
                         "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum "
                                            "of one 64-matrix launch, scaled to this launch "
                                            "by the number of matrices"
                                            if plan_kind == "tcgen05" else None)},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": info["launches"] * args.steps,
            "fp32_path": fp32,
            "rel_err_gap": gap,
            "train_s": train_s,
            "train": train_info,
            "train_status": st,
        }
        print(json.dumps(line), flush=True)
    if fp32 is not None:
        plan32.close()
        h32.close()
    plan.close()
    h.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    faulthandler.enable()
    faulthandler.dump_traceback_later(600, repeat=True)
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
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
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_tsk(args)


if __name__ == "__main__":
    sys.exit(main())
