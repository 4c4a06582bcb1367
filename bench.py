"""Benchmark of the genome scan: SNP-phenotype tests/s at N = 23,000 samples, P = 20,480 phenotypes.

One step = the whole scan path (decode with mean imputation, projection on the covariate
basis, marker norms, the contraction with the standardised panel and the fused statistics
epilogue with hit collection and per-phenotype best) over one block of 65,536 8-bit-dosage
markers, the streaming unit of the 8.9M-marker workload. Inputs are seeded synthetic data of
the paper's shape (the paper's cohort is not available). The blocks (1.5 GB each) and the
panel (1.9 GB of bf16 operands) are far larger than the 129 MB L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line. Its "e2e" entry streams --e2e-steps blocks from pinned host memory
through one tg_scan_host call (hits and best markers read back), after one untimed call that
measures the copy / scan ratio the block sizes grow by. --impl reference times the FP64 CPU
oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SNP-phenotype tests/s at N=23k,P=20,480: split-precision vs FP32, % roofline"
UNIT = "SNP-phenotype tests/s"
WORKLOAD = "n23000_m8900000_p20480_c20_u8"
THR = 7.30103  # -log10(5e-8)
RESIDENT = 4   # distinct genotype blocks kept in HBM and cycled
# ncu summary of the contraction kernel's DRAM traffic and tensor-pipe activity (profiles/)
PROFILE_TRAFFIC = "tc2_scan_traffic_n23000_p4864_m19456_u8.md"


def _args():
    a = argparse.ArgumentParser()
    a.add_argument("--gpus", type=int, default=1)
    a.add_argument("--steps", type=int, default=20)
    a.add_argument("--warmup", type=int, default=3)
    a.add_argument("--impl", default="ours", choices=["ours", "reference"])
    a.add_argument("--fp32-steps", type=int, default=2)
    a.add_argument("--e2e-steps", type=int, default=8)
    a.add_argument("--cpu-seconds", type=float, default=15.0)
    a.add_argument("--no-cpu-baseline", action="store_true")
    a.add_argument("--no-extra", action="store_true",
                   help="leave out the other workloads (2-bit P=2,048, N=2,000 P=16, batched, "
                        "P sweep) that the default line carries under other_configs")
    # smaller cases of the same kernels (profiling captures); the default is the full size
    a.add_argument("--workload", default=WORKLOAD,
                   help="n23000_m8900000_p20480_c20_u8 (default, 8-bit dosages, P=20,480), "
                        "n23000_m1000000_p2048_c10_2bit (PLINK 2-bit calls, 0.5%% missing, P=2,048) "
                        "or n23000_m500000_12panels_p8192_2bit (batched form)")
    a.add_argument("--phenotypes", type=int, default=None)
    a.add_argument("--block-markers", type=int, default=None)
    a.add_argument("--sweep-p", action="store_true",
                   help="instead of the bench line: time one block of the workload against panels "
                        "of growing P (the paper's Section 3.2 scaling in the number of phenotypes) "
                        "and print one JSON line with every point")
    a.add_argument("--points", default=None,
                   help="with --sweep-p: comma-separated panel sizes (default 16,40,64,100,200,256,"
                        "1024,2048,4096,8192,20480)")
    a.add_argument("--reps", type=int, default=None,
                   help="with --sweep-p: timed scans per point (default from P)")
    a.add_argument("--precision", default="split", choices=["split", "fp4"],
                   help="with --sweep-p: split BF16 (default) or FP4 pieces (2-bit workloads; "
                        "the block is drawn without missing calls, which the FP4 form does not test)")
    return a.parse_args()


def _workload(args):
    import dataclasses

    import synth
    w = synth.WORKLOADS[args.workload]
    if args.phenotypes or args.block_markers:
        w = dataclasses.replace(w, P=args.phenotypes or w.P, block=args.block_markers or w.block,
                                name=w.name + "_reduced")
    return w


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        return dist, dist.get_rank(), ws
    return None, 0, 1


def _max_over_ranks(dist, x: float) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_blocks(rank: int, ws: int, count: int):
    """Blocks of the marker stream scanned by `rank` of `ws` replicas: rank, rank + ws, ..."""
    return [rank + ws * i for i in range(count)]


def _barrier(dist):
    if dist is not None:
        dist.barrier()


# ------------------------------------------------------------------------- CPU oracle timing

def _oracle_sample(Yt, cov_t, G, seconds: float, encoding: str = "u8"):
    """Time the FP64 oracle (projected form, with p-values) on groups of 16 markers of the
    benchmark block against the full phenotype panel until `seconds` have passed."""
    import numpy as np

    import oracle

    ref_panel = oracle.prepare_panel(Yt.numpy().T.astype(np.float64), cov_t.numpy().T)
    G = G.numpy()
    done, t_total = 0, 0.0
    while t_total < seconds and done + 16 <= G.shape[0]:
        t0 = time.perf_counter()
        oracle.scan(G[done:done + 16], encoding, ref_panel, mode="projected")
        t_total += time.perf_counter() - t0
        done += 16
    return done, t_total, Yt.shape[0]


def _oracle_one_core(w, seconds: float):
    """The same oracle timing on one core: a child process with the BLAS and OpenMP pools at one
    thread and no GPU, on a slice of the workload (at most 2,048 phenotypes and 4,096 markers of
    block 0; the oracle's cost per test does not depend on P at these sizes). Returns
    (tests/s, sample description) or None if the child fails."""
    import subprocess
    import sys
    Pp = min(w.P, 2048)
    code = (
        "import dataclasses, sys, time\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import bench, synth\n"
        f"w = dataclasses.replace(synth.WORKLOADS[{w.name.replace('_reduced', '')!r}], P={Pp}, "
        f"N={w.N}, block=4096)\n"
        "pan = synth.make_panel(w)\n"
        "G = synth.make_block(w, 0)['G']\n"
        f"done, secs, P = bench._oracle_sample(pan['Yt'], pan['cov_t'], G, {seconds}, w.encoding)\n"
        "print(done, secs, P)\n")
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=max(120.0, 10 * seconds))
        done, secs, P = r.stdout.strip().splitlines()[-1].split()
        done, secs, P = int(done), float(secs), int(P)
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        return None
    return done * P / secs, f"{done} markers x {P} phenotypes on 1 thread, {secs:.1f} s"


def _reference(args, dist, rank, ws):
    """--impl reference: the FP64 CPU oracle, rank 0 only."""
    if rank != 0:
        return
    import numpy as np

    import oracle
    import synth

    w = _workload(args)
    pan = synth.make_panel(w, device="cpu", planted_blocks=1)
    ref_panel = oracle.prepare_panel(pan["Yt"].numpy().T.astype(np.float64), pan["cov_t"].numpy().T)
    per_step = 8
    f = synth.maf(w.seed, 0, per_step * (args.steps + args.warmup))
    if w.encoding == "u8":
        G = synth.dosage_bytes(w.seed, 0, f, w.N).numpy()
    else:
        counts, miss = synth.hard_calls(w.seed, 0, f, w.N, w.missing)
        G = synth.pack_2bit(counts, miss).numpy()
    for s in range(args.warmup):
        oracle.scan(G[s * per_step:(s + 1) * per_step], w.encoding, ref_panel, mode="projected")
    t0 = time.perf_counter()
    for s in range(args.warmup, args.warmup + args.steps):
        oracle.scan(G[s * per_step:(s + 1) * per_step], w.encoding, ref_panel, mode="projected")
    dt = time.perf_counter() - t0
    tests = per_step * w.P * args.steps
    value = tests / dt
    cores = os.cpu_count()
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(w),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} markers x {w.P} phenotypes per step, FP64 projected "
                                   "OLS with p-values (NumPy; BLAS threads on all cores)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def _paper_rate(w):
    """The paper's own throughput for this metric and panel size, as tests/s: Section 3.1 reports
    8.9 million markers and about 23,000 samples on one A100, 2,048 phenotypes in about 940 s and
    20,480 in about 1,108 s (another machine and real data: context for `vs_baseline`). None for
    panel sizes or sample counts the paper did not time."""
    secs = {2048: 940.0, 20480: 1108.0}.get(w.P)
    if secs is None or abs(w.N - 23_000) > 1_000:
        return None
    return 8.9e6 * w.P / secs


def _config(w):
    enc = "8-bit dosages" if w.encoding == "u8" else f"PLINK 2-bit calls ({100 * w.missing:g}% missing)"
    return {"workload": f"{w.name}: N={w.N} samples, {w.block}-marker blocks of {enc} "
                        f"(M={w.M} in the whole scan), P={w.P} phenotypes, C={w.n_cov + 1} covariate columns "
                        f"(intercept + {w.n_cov}), hits at -log10 p >= 7.30103",
            "N": w.N, "P": w.P, "C": w.n_cov + 1, "block_markers": w.block,
            "encoding": "u8 dosage" if w.encoding == "u8" else "2-bit PLINK",
            "precision": "split-bf16 (A exact bf16, panel bf16 hi+lo, fp32 accumulate)",
            "l2": f"inputs larger than L2: {RESIDENT} resident genotype blocks of "
                  f"{w.block * (w.N if w.encoding == 'u8' else (w.N + 3) // 4) / 1e9:.2f} GB cycled, "
                  f"{2 * 2 * w.P * w.N / 1e9:.2f} GB bf16 panel; the decoded operand alone is "
                  f"{2 * w.block * w.N / 1e9:.2f} GB per block"}


def sgemm_rate_tflops(dev, K: int) -> float:
    """The FP32 rate of cuBLAS SGEMM on this GPU (TF32 off): 8,192 x 8,192 outputs over K, the
    best of 3 timed calls after 2 warm-up calls (CUDA events). A library GEMM used only as the
    FP32 scan's yardstick."""
    import torch
    prev = torch.get_float32_matmul_precision()
    torch.set_float32_matmul_precision("highest")
    try:
        g = torch.Generator(device=dev).manual_seed(7)
        a = torch.randn(8192, K, device=dev, generator=g)
        b = torch.randn(K, 8192, device=dev, generator=g)
        for _ in range(2):
            torch.matmul(a, b)
        best = float("inf")
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        del a, b
        return 2.0 * 8192 * 8192 * K / (best / 1000.0) / 1e12
    finally:
        torch.set_float32_matmul_precision(prev)


def fp32_simt_peak_tflops(peaks) -> float:
    """FP32 FFMA peak of the SIMT cores: 152 SMs x 128 lanes x 2 flop per cycle at the maximum
    SM clock (80.5 TFLOP/s at 2,070 MHz)."""
    return 152 * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12


# ------------------------------------------------------------------------- ours

def _ours(args, dist, rank, ws):
    import numpy as np
    import torch

    import paper_2604_21095_gb300 as tg
    import synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    tg.build()
    w = _workload(args)
    enc = tg.TG_ENC_U8_DOSAGE if w.encoding == "u8" else tg.TG_ENC_2BIT
    ctx = tg.tg_create(local)
    stream = torch.cuda.current_stream(dev)

    # panel (prepared once, timed separately)
    pan = synth.make_panel(w, device=dev, planted_blocks=RESIDENT)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    panel = tg.tg_prepare_panel(ctx, pan["Yt"], w.N, w.P, pan["cov_t"], stream=stream)
    prepare_ms = 1000 * (time.perf_counter() - t0)
    want_cpu = rank == 0 and ws == 1 and not args.no_cpu_baseline
    cpu_inputs = (pan["Yt"].cpu(), pan["cov_t"].cpu()) if want_cpu else None
    del pan

    # resident blocks: rank r scans blocks r, r + ws, ... of the workload
    mine = rank_blocks(rank, ws, RESIDENT)
    blocks = [synth.make_block(w, b, device=dev)["G"] for b in mine]
    M = blocks[0].shape[0]
    cap = 1 << 20
    hits = torch.zeros(cap * 24, dtype=torch.uint8, device=dev)
    n_hits = torch.zeros(1, dtype=torch.int64, device=dev)
    best = torch.zeros(w.P, dtype=torch.int64, device=dev)
    out = tg.make_outputs(hits=hits, n_hits=n_hits, best=best)

    def step(i, prec):
        opts = tg.tg_scan_opts(prec, 0, THR)
        b = i % RESIDENT
        tg.tg_scan_block(ctx, panel, blocks[b], w.N, M, enc, opts, out,
                         marker_offset=mine[b] * w.block, stream=stream)

    # split-BF16, the headline
    for i in range(args.warmup):
        step(i, tg.TG_PREC_SPLIT_BF16)
    torch.cuda.synchronize()
    n_hits.zero_()
    best.zero_()
    tg.tg_stage_times(ctx, reset=True)
    tg.tg_set_profiling(ctx, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    _barrier(dist)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        ev0.record(stream)
        for i in range(args.steps):
            step(i, tg.TG_PREC_SPLIT_BF16)
        ev1.record(stream)
        torch.cuda.synchronize()
    _barrier(dist)
    ms = ev0.elapsed_time(ev1)
    tg.tg_set_profiling(ctx, False)
    stages = tg.tg_stage_times(ctx, reset=True)
    status = tg.tg_status_poll(ctx, stream)
    if status != tg.TG_OK:
        raise SystemExit(f"device status {status}: {tg.tg_last_error()}")
    ms_max = _max_over_ranks(dist, ms)
    tests_step = M * w.P
    value = tests_step * args.steps * ws / (ms_max / 1000.0)
    launches = sum(n for _, n in stages.values())
    nh = int(n_hits.item())

    # FP32 SIMT scan on the same GPU, same blocks
    fp32 = None
    if args.fp32_steps > 0:
        step(0, tg.TG_PREC_FP32)
        torch.cuda.synchronize()
        tg.tg_stage_times(ctx, reset=True)
        tg.tg_set_profiling(ctx, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(args.fp32_steps):
            step(i, tg.TG_PREC_FP32)
        e1.record(stream)
        torch.cuda.synchronize()
        tg.tg_set_profiling(ctx, False)
        st32 = tg.tg_stage_times(ctx, reset=True)
        ms32 = _max_over_ranks(dist, e0.elapsed_time(e1))
        k32 = st32["scan"][0] / max(1, st32["scan"][1])
        a32 = 2.0 * w.N * M * w.P / (k32 / 1000.0) / 1e12
        nominal32 = fp32_simt_peak_tflops(_peaks()[0])
        sgemm = sgemm_rate_tflops(dev, (w.N + 63) // 64 * 64)
        fp32 = {"value": tests_step * args.fp32_steps * ws / (ms32 / 1000.0), "unit": UNIT,
                "ms_per_step": ms32 / args.fp32_steps,
                "scan_kernel_ms": k32,
                "roofline": {"bound": "alu", "achieved": a32, "peak": sgemm, "unit": "TFLOP/s",
                             "frac": a32 / sgemm,
                             "peak_source": "measured: cuBLAS SGEMM (TF32 off), 8192 x 8192 x "
                                            "Npad on this GPU, best of 3",
                             "nominal_peak": nominal32, "nominal_frac": a32 / nominal32,
                             "nominal_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop (FFMA) "
                                               "x the maximum SM clock"},
                "stage_ms_per_step": {k: v[0] / args.fp32_steps for k, v in st32.items()}}

    # end to end through the host-buffer entry point: pinned host blocks in, hits and best out
    e2e = None
    if args.e2e_steps > 0:
        # one call streams all e2e steps' blocks (the resident blocks cycled), as a scan of a
        # genome chunk would: 1.5 GB of pinned host memory per step
        per_call = args.e2e_steps
        calls = 1
        host = torch.empty((per_call * M, blocks[0].shape[1]), dtype=torch.uint8, pin_memory=True)
        for i in range(per_call):
            host[i * M:(i + 1) * M].copy_(blocks[i % len(blocks)])
        hits_h = torch.zeros(cap * 24, dtype=torch.uint8, pin_memory=True)
        best_h = torch.zeros(w.P, dtype=torch.int64, pin_memory=True)
        opts = tg.tg_scan_opts(tg.TG_PREC_SPLIT_BF16, 0, THR)
        tg.tg_scan_host(ctx, panel, host, w.N, per_call * M, enc, M, opts, hits_h,
                        best_h, stream=stream)
        torch.cuda.synchronize()
        tg.tg_stage_times(ctx, reset=True)
        tg.tg_set_profiling(ctx, True)
        _barrier(dist)
        t0 = time.perf_counter()
        nh_e2e = 0
        for _ in range(calls):
            nh_e2e = tg.tg_scan_host(ctx, panel, host, w.N, per_call * M, enc, M,
                                     opts, hits_h, best_h, stream=stream)
        dt = _max_over_ranks(dist, time.perf_counter() - t0)
        tg.tg_set_profiling(ctx, False)
        ste = tg.tg_stage_times(ctx, reset=True)
        steps_e2e = calls * per_call
        growth, ratio = tg.tg_host_ramp(ctx)
        # the host link's rate: one block's pinned copy with the GPU otherwise idle (after the
        # timed region), against the copies' average while the scans ran
        blk_bytes = int(M * blocks[0].shape[1])
        dst = torch.empty(blk_bytes, dtype=torch.uint8, device=dev)
        side = torch.cuda.Stream(dev)
        idle_ms = []
        with torch.cuda.stream(side):
            for _ in range(2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(side)
                dst.copy_(host[:M].reshape(-1), non_blocking=True)
                e1.record(side)
                e1.synchronize()
                idle_ms.append(e0.elapsed_time(e1))
        del dst
        h2d_ms = ste["h2d"][0] / steps_e2e if "h2d" in ste else 0.0
        e2e = {"value": tests_step * steps_e2e * ws / dt, "unit": UNIT,
               "block_growth": {"factor": growth, "scan_over_copy": ratio},
               "copy_rate_gbs": {"idle": blk_bytes / min(idle_ms) / 1e6,
                                 "during_scans": blk_bytes / h2d_ms / 1e6 if h2d_ms else None},
               "h2d_bytes_per_step": int(M * blocks[0].shape[1]),
               "d2h_bytes_per_step": int((8 + 24 * min(nh_e2e, cap) + 8 * w.P) / per_call),
               "ms_per_step": 1000 * dt / steps_e2e, "api": "tg_scan_host (C ABI, host buffers)",
               "stage_ms_per_step": {k: v[0] / steps_e2e for k, v in ste.items()}}

    peaks, peak_src = _peaks()
    gemm_ms = stages["scan"][0] / max(1, stages["scan"][1])
    flops = 2.0 * w.N * M * w.P                      # Eq. 2, algorithmic
    achieved = flops / (gemm_ms / 1000.0) / 1e12
    peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
    prof = _kernel_profile()
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": prof.get("dram_bytes_per_launch"),
                "kernel": "k_tc2_scan (tcgen05 cta_group::2 split-BF16 + fused epilogue)",
                "issued_tflops": 2 * achieved, "issued_frac": 2 * achieved / peak,
                "tensor_pipe_active": prof.get("tensor_pipe_active"),
                "peak_source": f"{peak_src} bf16 sustained",
                "kernel_ms": gemm_ms,
                "stage_ms_per_step": {k: v[0] / max(1, args.steps) for k, v in stages.items()}}

    cpu = None
    if want_cpu:
        done, secs, P = _oracle_sample(cpu_inputs[0], cpu_inputs[1], blocks[0][:4096].cpu(),
                                       args.cpu_seconds, w.encoding)
        cpu = {"value": done * P / secs, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{done} markers x {P} phenotypes of block 0, FP64 projected OLS with "
                         f"p-values, {secs:.1f} s (panel preparation excluded, as on the GPU)"}
        one = _oracle_one_core(w, args.cpu_seconds / 3)
        if one:
            cpu["one_core"] = {"value": one[0], "unit": UNIT, "sample": one[1]}

    rec = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": (value / _paper_rate(w)) if _paper_rate(w) else None,
        "dtype": "bf16", "data": "synthetic",
        "config": _config(w), "clocks": clk.summary(), "gpu_launches": launches,
        "e2e": e2e, "roofline": roofline, "cpu_baseline": cpu, "fp32": fp32,
        "split_vs_fp32": (value / fp32["value"]) if fp32 else None,
        "prepare_panel_ms": prepare_ms, "hits_in_timed_steps": nh,
    }
    tg.tg_panel_free(panel)
    tg.tg_destroy(ctx)
    return rec


def _ours_batched(args, dist, rank, ws, workload=None, steps=None, warmup=None, e2e_steps=None,
                  cpu_seconds=None):
    """The batched form: 12 panels of uneven P (8,192 columns) concatenated into one panel,
    500,000 markers in ragged blocks (1k-64k), every block's scan captured in one CUDA graph
    and replayed once per step, with the tensor-core kernel autotuned per block-size bucket.
    Returns the bench record (rank 0) or None."""
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    e2e_steps = args.e2e_steps if e2e_steps is None else e2e_steps
    cpu_seconds = (0.0 if args.no_cpu_baseline else args.cpu_seconds) if cpu_seconds is None else cpu_seconds
    import numpy as np
    import torch

    import paper_2604_21095_gb300 as tg
    import synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    tg.build()
    w = synth.WORKLOADS[workload or args.workload]
    ctx = tg.tg_create(local)
    stream = torch.cuda.current_stream(dev)
    pan = synth.make_panel(w, device=dev, planted_blocks=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    parts, o = [], 0
    for k in synth.BATCHED_PANELS:
        parts.append(tg.tg_prepare_panel(ctx, pan["Yt"][o:o + k].contiguous(), w.N, k, pan["cov_t"],
                                         stream=stream))
        o += k
    panel = tg.tg_panel_concat(ctx, parts, stream=stream)
    prepare_ms = 1000 * (time.perf_counter() - t0)
    for p in parts:
        tg.tg_panel_free(p)
    sizes = synth.ragged_blocks(w.seed, w.M)
    # rank r takes every ws-th block (replicas over disjoint marker ranges)
    mine = list(range(rank, len(sizes), ws))
    offs = np.cumsum([0] + sizes[:-1])
    blocks = [synth.make_ragged_block(w, i, sizes[i], device=dev) for i in mine]
    enc = tg.TG_ENC_2BIT if w.encoding == "2bit" else tg.TG_ENC_U8_DOSAGE
    tuned = {}
    for i in mine:
        b = int(sizes[i]).bit_length() - 1
        if b not in tuned:
            tg.tg_autotune(ctx, panel, enc, int(sizes[i]), stream=stream)
            tuned[b] = dict(tg.tg_tuning(ctx, int(sizes[i])),
                            splits=tg.tg_tuning_split(ctx, int(sizes[i])))
    cap = 1 << 20
    hits = torch.zeros(cap * 24, dtype=torch.uint8, device=dev)
    n_hits = torch.zeros(1, dtype=torch.int64, device=dev)
    best = torch.zeros(w.P, dtype=torch.int64, device=dev)
    out = tg.make_outputs(hits=hits, n_hits=n_hits, best=best)
    opts = tg.tg_scan_opts(tg.TG_PREC_SPLIT_BF16, 0, THR)
    graph = tg.tg_scan_graph_create(ctx, panel, blocks, w.N, enc, opts, out,
                                    [int(offs[i]) for i in mine])
    markers = sum(sizes[i] for i in mine)
    for _ in range(warmup):
        tg.tg_scan_graph_launch(graph, stream=stream)
    torch.cuda.synchronize()
    n_hits.zero_()
    best.zero_()
    tg.tg_stage_times(ctx, reset=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    _barrier(dist)
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        ev0.record(stream)
        for _ in range(steps):
            tg.tg_scan_graph_launch(graph, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    _barrier(dist)
    ms = _max_over_ranks(dist, ev0.elapsed_time(ev1))
    status = tg.tg_status_poll(ctx, stream)
    if status != tg.TG_OK:
        raise SystemExit(f"device status {status}: {tg.tg_last_error()}")
    launches = sum(n for _, n in tg.tg_stage_times(ctx, reset=True).values())
    total_markers = sum(sizes)
    value = total_markers * w.P * steps / (ms / 1000.0)
    nh = int(n_hits.item())
    tg.tg_scan_graph_free(graph)

    # end to end: the same ragged blocks from pinned host memory, through one graph whose
    # replay copies them to the device on a forked stream while the previous block is scanned;
    # each step reads the hit count, the best keys and the hits back to the host
    e2e = None
    if e2e_steps > 0 and ws == 1:
        ldg = blocks[0].shape[1]
        host = [b.cpu().pin_memory() for b in blocks]
        hg = tg.tg_scan_graph_create_host(ctx, panel, host, w.N, enc, opts, out,
                                          [int(offs[i]) for i in mine])
        nh_h = torch.zeros(1, dtype=torch.int64, pin_memory=True)
        best_h = torch.zeros(w.P, dtype=torch.int64, pin_memory=True)
        hits_h = torch.zeros(cap * 24, dtype=torch.uint8, pin_memory=True)
        tg.tg_scan_graph_launch(hg, stream=stream)  # warm-up
        torch.cuda.synchronize()
        reps = max(1, e2e_steps // 2)
        d2h = 0
        t0 = time.perf_counter()
        for _ in range(reps):
            n_hits.zero_()
            best.zero_()
            tg.tg_scan_graph_launch(hg, stream=stream)
            nh_h.copy_(n_hits, non_blocking=True)
            best_h.copy_(best, non_blocking=True)
            stream.synchronize()
            k = 24 * min(int(nh_h.item()), cap)
            hits_h[:k].copy_(hits[:k], non_blocking=True)
            stream.synchronize()
            d2h = 8 + 8 * w.P + k
        dt = time.perf_counter() - t0
        if tg.tg_status_poll(ctx, stream) != tg.TG_OK:
            raise SystemExit(f"device status: {tg.tg_last_error()}")
        tg.tg_scan_graph_free(hg)
        e2e = {"value": markers * w.P * reps / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(markers * ldg), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": 1000 * dt / reps,
               "api": "tg_scan_graph_create_host + tg_scan_graph_launch (C ABI, pinned host "
                      "blocks copied inside the graph on a forked stream)"}

    peaks, peak_src = _peaks()
    flops = 2.0 * w.N * total_markers * w.P
    achieved = flops / (ms / steps / 1000.0) / 1e12
    peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
    cpu = None
    if rank == 0 and ws == 1 and cpu_seconds > 0:
        done, secs, P = _oracle_sample(pan["Yt"].cpu(), pan["cov_t"].cpu(), blocks[0][:4096].cpu(),
                                       cpu_seconds, w.encoding)
        cpu = {"value": done * P / secs, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{done} markers x {P} phenotypes, FP64 projected OLS with p-values, "
                         f"{secs:.1f} s (panel preparation excluded)"}
    rec = None
    if rank == 0:
        rec = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": steps,
            "warmup": warmup, "ms_per_step": ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"{w.name}: N={w.N} samples, 12 panels of P = "
                                   f"{list(synth.BATCHED_PANELS)} (8,192 columns) sharing the "
                                   f"covariates (intercept + {w.n_cov}), {total_markers} markers in "
                                   f"{len(sizes)} ragged 2-bit blocks ({min(sizes)}-{max(sizes)}), "
                                   "one captured CUDA graph per step",
                       "N": w.N, "P": w.P, "panels": len(synth.BATCHED_PANELS),
                       "blocks": len(sizes), "encoding": "2-bit PLINK",
                       "tuning": {str(1 << b): v for b, v in sorted(tuned.items())},
                       "l2": "inputs larger than L2: 2.9 GB of resident genotype blocks"},
            "clocks": clk.summary(), "gpu_launches": launches, "e2e": e2e,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "whole step (decode + projection + contraction + statistics of "
                                   "every block, replayed from one graph)",
                         "peak_source": f"{peak_src} bf16 sustained"},
            "cpu_baseline": cpu, "fp32": None, "prepare_panel_ms": prepare_ms,
            "hits_in_timed_steps": nh,
        }
    tg.tg_panel_free(panel)
    tg.tg_destroy(ctx)
    return rec


def _kernel_profile():
    """DRAM bytes per launch (a small case of the same wave shape, scaled to one bench launch by
    the tests it processes) and the tensor pipe's active fraction of the elapsed cycles of the
    contraction kernel, from the committed ncu summary, if it was taken on the current kernel
    sources (else an empty dict)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", PROFILE_TRAFFIC)
    csrc = os.path.join(ROOT, "paper_2604_21095_gb300", "csrc")
    try:
        h = hashlib.sha256(b"".join(open(os.path.join(csrc, f), "rb").read()
                                    for f in ("k_tc2.cu", "tc_common.cuh"))).hexdigest()
        rec = {}
        for line in open(path):
            if ":" in line and not line.startswith(("|", "#", " ")):
                k, v = line.split(":", 1)
                rec[k.strip()] = v.strip()
        if rec.get("source_sha256") != h:
            return {}
        return {"dram_bytes_per_launch": int(rec["dram_bytes_per_launch"]),
                "tensor_pipe_active": float(rec["tensor_pipe_active_pct"]) / 100.0}
    except (OSError, KeyError, ValueError):
        return {}


def fused_joint(M: int, P: int, q: int, sm_count: int) -> bool:
    """Whether the library scans a block with the decode fused into the small panel's joint
    projection pass (its documented default: projected form, no mask, P + q - 1 <= 128 and at
    least one 128-marker tile per SM)."""
    return q > 1 and P + q - 1 <= 128 and (M + 127) // 128 >= sm_count


def fused_projection(N: int, M: int, encoding: str, P: int, q: int, sm_count: int) -> bool:
    """Whether the library runs a larger panel's projection as the pass over the packed rows
    that also writes the block's operand (its default for P + q - 1 > 128 in the projected form,
    no mask, at least one 128-marker tile per SM; a panel with a 256-row joint operand,
    P + q - 1 <= 256, only where that pass also writes the marker statistics)."""
    return (q > 1 and P + q - 1 > 128 and (M + 127) // 128 >= sm_count and
            (P + q - 1 > 256 or one_pass_joint(N, M, encoding, sm_count)))


def one_pass_joint(N: int, M: int, encoding: str, sm_count: int) -> bool:
    """Whether the fused joint pass also writes the marker statistics, so that no counting pass
    reads the block first: dosage rows (no mask) on 256-marker tiles (at least one per SM), and
    N <= 66,051 (the rows' sums of squared bytes fit 32 bits)."""
    return encoding == "u8" and N <= 66051 and (M + 255) // 256 >= sm_count


def _hbm_bytes_per_block(N: int, M: int, encoding: str, P: int, q: int, fused: bool = False,
                         one_pass: bool = False, fused_proj: bool = False) -> float:
    """Algorithmic DRAM bytes of one block's scan. With the decoded operand in HBM: read the
    packed rows, write the 2-byte operand, read it once more for each pass over it (one joint
    pass when the panel and the q - 1 projection columns fit a 256-column tile, else the
    projection and the contraction), and read the bf16 hi + lo panel once. With the decode fused
    into the joint pass: read the packed rows twice (the counting pass, then the joint pass), or
    once where the joint pass writes the statistics itself (one_pass), and the joint operand (64
    or 128 rows of hi + lo) once. With the projection pass that writes the operand (fused_proj):
    the packed rows once or twice as before, the projection columns (64 rows of hi + lo) once,
    the operand written once and read once (the contraction), and the panel once."""
    npad = (N + 63) // 64 * 64
    packed = M * (N if encoding == "u8" else (N + 3) // 4)
    if fused:
        jc = 64 if P + q - 1 <= 64 else 128
        return (1 if one_pass else 2) * packed + 2 * 2 * jc * npad
    operand = 2 * M * npad
    if fused_proj:
        return ((1 if one_pass else 2) * packed + 2 * 2 * 64 * npad + 2 * operand
                + 2 * 2 * P * npad)
    passes = 1 if P + q - 1 <= 256 else 2
    return packed + operand + passes * operand + 2 * 2 * P * npad


FP4_PIECES = 6  # E2M1 pieces of the panel in the FP4 form (one kind::mxf4 product each)


def _scan_points(w, Ps, dev, reps_for, flush_bytes=0, prec="split"):
    """Per-block time of the whole scan path (one tg_scan_block of block 0 of workload w) for
    panels of each size in Ps (the first P phenotypes of the workload's panel), with the stage
    times and the binding roofline of each point. With flush_bytes > 0 a buffer that large is
    written before every timed scan and each scan is timed alone (for inputs that fit L2).
    prec is "split" (split BF16) or "fp4" (block-scaled FP4 pieces, complete 2-bit blocks)."""
    import torch

    import paper_2604_21095_gb300 as tg
    import synth

    enc = tg.TG_ENC_U8_DOSAGE if w.encoding == "u8" else tg.TG_ENC_2BIT
    peaks, src = _peaks()
    ctx = tg.tg_create(dev.index or 0)
    stream = torch.cuda.current_stream(dev)
    pan = synth.make_panel(w, device=dev, planted_blocks=1)
    G = synth.make_block(w, 0, device=dev)["G"]
    M = G.shape[0]
    hits = torch.zeros((1 << 20) * 24, dtype=torch.uint8, device=dev)
    n_hits = torch.zeros(1, dtype=torch.int64, device=dev)
    flush = torch.empty(flush_bytes, dtype=torch.uint8, device=dev) if flush_bytes else None
    points = []
    for P in Ps:
        if P > w.P:
            break
        Yt = pan["Yt"][:P].contiguous()
        panel = tg.tg_prepare_panel(ctx, Yt, w.N, P, pan["cov_t"], stream=stream)
        q = tg.tg_panel_info(panel)[2]
        best = torch.zeros(P, dtype=torch.int64, device=dev)
        out = tg.make_outputs(hits=hits, n_hits=n_hits, best=best)
        opts = tg.tg_scan_opts(tg.TG_PREC_FP4_PIECES if prec == "fp4" else tg.TG_PREC_SPLIT_BF16,
                               0, THR)
        reps = reps_for(P)
        for _ in range(3):
            tg.tg_scan_block(ctx, panel, G, w.N, M, enc, opts, out, stream=stream)
        torch.cuda.synchronize()
        tg.tg_stage_times(ctx, reset=True)
        tg.tg_set_profiling(ctx, True)
        ms = 0.0
        if flush is None:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                tg.tg_scan_block(ctx, panel, G, w.N, M, enc, opts, out, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
        else:
            evs = []
            for _ in range(reps):
                flush.fill_(1)  # evicts the block, the operand and the panel from L2
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                tg.tg_scan_block(ctx, panel, G, w.N, M, enc, opts, out, stream=stream)
                e1.record(stream)
                evs.append((e0, e1))
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in evs) / reps
        tg.tg_set_profiling(ctx, False)
        st = tg.tg_stage_times(ctx, reset=True)
        if tg.tg_status_poll(ctx, stream) != tg.TG_OK:
            raise RuntimeError(tg.tg_last_error())
        flops = 2.0 * w.N * M * P
        if prec == "fp4":
            # one kind::mxf4 product per piece; FP4 peak = measured bf16 burst x the nominal
            # dense FP4 / BF16 ratio (13.5 / 2.25 PFLOP/s)
            issued = FP4_PIECES * flops / (ms / 1000.0) / 1e12
            peak4 = float(peaks["bf16_tflops"]) * 13.5 / 2.25
            points.append({
                "P": P, "ms_per_block": ms, "tests_per_s": M * P / (ms / 1000.0),
                "precision": f"FP4 pieces ({FP4_PIECES} block-scaled E2M1 pieces, kind::mxf4)",
                "roofline": {"bound": "tensor", "achieved": issued, "peak": peak4,
                             "unit": "TFLOP/s", "frac": issued / peak4,
                             "basis": f"{FP4_PIECES} x Eq. 2 flops (2 N M P) per block, issued in "
                                      f"FP4, against the {src} burst bf16 rate x 6 (nominal "
                                      "FP4/BF16 ratio)"},
                "stage_ms": {k: v[0] / reps for k, v in st.items() if v[1]}})
            n_hits.zero_()
            tg.tg_panel_free(panel)
            continue
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        fz = fused_joint(M, P, q, sms)
        fp = fused_projection(w.N, M, w.encoding, P, q, sms)
        op = (fz or fp) and one_pass_joint(w.N, M, w.encoding, sms)
        byts = _hbm_bytes_per_block(w.N, M, w.encoding, P, q, fz, op, fp)
        hbm_frac = byts / (ms / 1000.0) / 1e9 / float(peaks["hbm_gbs"])
        tflops = flops / (ms / 1000.0) / 1e12
        tens_frac = tflops / float(peaks["bf16_tflops"])
        hbm_bound = hbm_frac >= tens_frac
        points.append({
            "P": P, "ms_per_block": ms, "tests_per_s": M * P / (ms / 1000.0),
            "decode": ("fused into the joint pass, which also writes the marker statistics"
                       if op and fz else "fused into the joint pass, after a counting pass" if fz
                       else "in the projection pass, which writes the operand and the marker "
                       "statistics" if op else "in the projection pass, which writes the "
                       "operand, after a counting pass" if fp else "decoded operand in HBM"),
            "roofline": {"bound": "hbm" if hbm_bound else "tensor",
                         "achieved": byts / (ms / 1000.0) / 1e9 if hbm_bound else tflops,
                         "peak": float(peaks["hbm_gbs"]) if hbm_bound else float(peaks["bf16_tflops"]),
                         "unit": "GB/s" if hbm_bound else "TFLOP/s",
                         "frac": hbm_frac if hbm_bound else tens_frac,
                         "basis": "whole step: algorithmic DRAM bytes (packed rows read once or "
                                  "twice with the fused decode; else packed rows, operand written and read per "
                                  "pass; panel) or Eq. 2 flops (2 N M P) per block, against the "
                                  f"{src} HBM copy rate / burst bf16 rate"},
            "stage_ms": {k: v[0] / reps for k, v in st.items() if v[1]}})
        n_hits.zero_()
        tg.tg_panel_free(panel)
    tg.tg_destroy(ctx)
    return M, points


def _sweep_p(args):
    """Per-block time of the whole scan path against the panel size P, on one GPU."""
    import torch

    import dataclasses

    w = _workload(args)
    if args.precision == "fp4":
        w = dataclasses.replace(w, missing=0.0)
    Ps = tuple(int(x) for x in args.points.split(",")) if args.points else (
        16, 40, 64, 100, 200, 256, 1024, 2048, 4096, 8192, 20480)
    M, points = _scan_points(w, Ps, torch.device("cuda", 0),
                             (lambda P: args.reps) if args.reps else
                             (lambda P: max(3, min(50, int(20480 * 5 / P)))),
                             prec=args.precision)
    print(json.dumps({"metric": "per-block scan time vs number of phenotypes", "unit": "ms",
                      "precision": args.precision,
                      "workload": f"{w.name}: one {M}-marker block, N={w.N}, C={w.n_cov + 1}"
                                  + (", no missing calls" if args.precision == "fp4" else ""),
                      "points": points}))


def _other_configs(args):
    """The benchmark set's other workloads on the same GPU after the headline, each with its
    binding roofline: the 2-bit P = 2,048 workload (one 65,536-marker block), the same block
    without missing calls in split BF16 and in FP4 pieces, the N = 2,000, P = 16 workload (its whole 10,000 markers per step; they fit L2, so L2 is flushed before
    every timed scan), the batched form (12 panels, ragged blocks, one graph per step) and a
    few points of the scaling in the number of phenotypes (Section 3.2) on the dosage workload."""
    import dataclasses

    import torch

    import synth
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    out = {}

    def run(name, fn):
        try:
            out[name] = fn()
        except Exception as e:  # a failed extra is reported on the line, not hidden
            out[name] = {"error": f"{type(e).__name__}: {e}"}

    def cfg_block(name, reps, flush):
        w = synth.WORKLOADS[name]
        M, pts = _scan_points(w, (w.P,), dev, lambda P: reps, flush)
        pt = pts[0]
        pt.update(workload=f"{name}: one {M}-marker block, N={w.N}, P={w.P}, C={w.n_cov + 1}, "
                           f"{'8-bit dosages' if w.encoding == 'u8' else '2-bit calls'}"
                           + (f", L2 flushed ({flush >> 20} MiB written) before each scan" if flush else ""))
        return pt

    run("n23000_m1000000_p2048_c10_2bit", lambda: cfg_block("n23000_m1000000_p2048_c10_2bit", 10, 0))
    run("n2000_m10000_p16_c5_2bit", lambda: cfg_block("n2000_m10000_p16_c5_2bit", 20, 256 << 20))

    def fp4_vs_split():
        # the FP4 form tests complete markers only: the same workload without missing calls
        w = dataclasses.replace(synth.WORKLOADS["n23000_m1000000_p2048_c10_2bit"], missing=0.0)
        res = {}
        for prec in ("split", "fp4"):
            M, pts = _scan_points(w, (w.P,), dev, lambda P: 10, 0, prec=prec)
            res[prec] = pts[0]
        res["workload"] = (f"{w.name} without missing calls: one {M}-marker block, N={w.N}, "
                           f"P={w.P}, C={w.n_cov + 1}, 2-bit calls, both forms on the same block")
        res["split_ms_over_fp4_ms"] = res["split"]["ms_per_block"] / res["fp4"]["ms_per_block"]
        return res

    run("fp4_vs_split_2bit_p2048", fp4_vs_split)

    def batched():
        r = _ours_batched(args, None, 0, 1, workload="n23000_m500000_12panels_p8192_2bit",
                          steps=5, warmup=2, e2e_steps=0, cpu_seconds=0.0)
        keep = ("value", "unit", "ms_per_step", "steps", "clocks", "gpu_launches", "roofline")
        d = {k: r[k] for k in keep}
        d["workload"] = r["config"]["workload"]
        d["tuning"] = r["config"]["tuning"]
        return d

    run("n23000_m500000_12panels_p8192_2bit", batched)

    def sweep():
        w = dataclasses.replace(synth.WORKLOADS[WORKLOAD], P=4096)
        M, pts = _scan_points(w, (16, 100, 256, 1024, 4096), dev,
                              lambda P: max(3, min(30, int(20480 * 3 / P))))
        return {"workload": f"{WORKLOAD}: one {M}-marker block, N={w.N}, C={w.n_cov + 1}, "
                            "panels of the first P phenotypes", "points": pts}

    run("sweep_p_n23000_u8", sweep)
    return out


def main():
    args = _args()
    if args.sweep_p:
        _sweep_p(args)
        return
    dist, rank, ws = _dist()
    if args.impl == "reference":
        _reference(args, dist, rank, ws)
    elif "panels" in args.workload:
        rec = _ours_batched(args, dist, rank, ws)
        if rank == 0:
            print(json.dumps(rec))
    else:
        rec = _ours(args, dist, rank, ws)
        if rank == 0:
            if ws == 1 and not args.no_extra and args.workload == WORKLOAD and not (
                    args.phenotypes or args.block_markers):
                t0 = time.perf_counter()
                rec["other_configs"] = _other_configs(args)
                rec["other_configs"]["seconds"] = time.perf_counter() - t0
            print(json.dumps(rec))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
