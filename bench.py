"""Throughput benchmark: frames/s of the fused Gerchberg + Wiener reconstruction
for 40x40 lenslets on a 128^2 grid (1000 seeded frames per step, k = 10).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gpu,reference}]

One step = one pass of the whole path (embed, periodic fill, k Gerchberg
iterations, final Wiener reconstruction) over a batch of 1000 frames that is
already resident in HBM; one kernel launch per step. Between timed steps the
L2 cache is flushed by writing a 256 MiB buffer (outside the timed region).
The end-to-end figure (`e2e`) times the C-ABI host entry point, which copies
the slopes in and the phase out inside the timed region.

--impl reference times the FP64 CPU oracle (the plain implementation the GPU
path is checked against) on the host cores, on a bounded sample of the same
workload. Under torchrun only rank 0 runs it.

With N > 1 (torchrun, one rank per GPU) each rank reconstructs its own batch
(weak scaling, no collective on the data path); the reported time is the
maximum over ranks.
"""

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# workload: 40x40 SPHERE-like lenslet array, D = 8 m, padded to 128^2
N_LENSLETS = 40
PAD = 3.2
FRAMES = 1000
ITERS = 10
SIGMA = 0.1
R0, L0 = 0.15, 25.0
SEED0 = 1000
METRIC = "frames/s at 40x40 lenslets (128² grid), ≤1e-5 rel err vs FP64; learned vs plain"

# Roofline of the FFT-bound path: FP32 FMA peak from the unit counts and the
# maximum SM clock (152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz).
SMS, FP32_LANES, MAX_SM_MHZ = 152, 128, 2070.0


# Side outputs of a run (the clocks sampled during the timed region, the
# autotuner's cache): FWR_BENCH_OUT, else bench_out/ beside this file.
OUT_DIR = os.environ.get("FWR_BENCH_OUT", os.path.join(ROOT, "bench_out"))


def fp32_peak_tflops():
    return SMS * FP32_LANES * 2 * MAX_SM_MHZ * 1e6 / 1e12


def flops_per_frame(N, k):
    """Algorithmic FFT flops: (2k + 1.5) complex N^2 transforms of 5 N^2 log2(N^2)
    flops each (k forward + k inverse packed transforms in the loop, one forward
    and half an inverse for the final real phase)."""
    return (2 * k + 1.5) * 5.0 * N * N * math.log2(N * N)


# DRAM bytes per launch of the fused kernel from an ncu capture, keyed by the
# SHA-256 of the kernel source it was taken on (stale entries are ignored).
TRAFFIC = {
    # ncu --set full, one k = 10 launch of 1000 frames: 12.985 MB read + 5.513 MB written
    "c4cdd161e6b0c782": 18497792,
    # same capture after the P2 twiddles and the P3-input y fill: 12.994 MB + 5.890 MB
    "97a3eb880aeb3f5d": 18883840,
    # compile-time spectral selects, slope prefetch, unrolled set-up: 12.982 MB + 5.505 MB
    "b7a334ff342cde75": 18486784,
    # + the Hudgin-extension instantiation (ncu --metrics dram__bytes_read.sum,
    # dram__bytes_write.sum, one k = 10 launch of 1000 frames): 12.98 MB + 4.83 MB
    "da16ea3515ab57b7": 17810000,
    # LSQ coefficients in tensor memory (ncu --set full, one k = 10 launch of 1000
    # frames, bench.py --workload fused128): 12.988 MB read + 5.487 MB written
    "28460c3873c63f98": 18475008,
    # the same kernel after the slab plans' L2-window fields joined the launch
    # parameters (ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum, one
    # k = 10 launch of 1000 frames, bench.py --workload fused128): 12.988 MB + 5.089 MB
    "6b8bd851c4600f15": 18076928,
    # the final filter's bins in a loop of their own (ncu --set full, one k = 10
    # launch of 1000 frames, bench.py --workload fused128): 13.629 MB + 7.559 MB
    "c13607d075322aea": 21188608,
    # the same kernel with a griddepcontrol.wait after its set-up (ncu --metrics
    # dram__bytes_read.sum,dram__bytes_write.sum, bench.py --workload fused128): 13.648 MB + 6.718 MB
    "eb5006958f98e602": 20365824,
    # unchanged kernel, internal header comments edited (ncu --metrics dram__bytes_read.sum,
    # dram__bytes_write.sum, bench.py --workload fused128): 13.637 MB + 6.909 MB
    "c42445c2dd37e6f3": 20546560,
    # the launcher caches its occupancy queries (kernel unchanged; ncu --metrics
    # dram__bytes_read.sum,dram__bytes_write.sum, bench.py --workload fused128): 13.636 MB + 6.874 MB
    "87a73a622d7087ed": 20509952,
}


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("fwr_fused.cu", "fwr_fused.cuh", "fwr_fft.cuh", "fwr_w32t.inc", "fwr_internal.h"):
        with open(os.path.join(ROOT, "paper_1705_04298_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            os.makedirs(OUT_DIR, exist_ok=True)
            self.path = os.path.join(OUT_DIR, "clocks_gpu%d.csv" % self.gpu)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- oracle -----

def _oracle_worker(args):
    slopes, mask, r0p, L0p = args
    import oracle
    t0 = time.perf_counter()
    oracle.reconstruct(slopes, mask, PAD, ITERS, oracle.FILTER_WIENER, SIGMA ** 2, r0p, L0p)
    return time.perf_counter() - t0


class OraclePool:
    """The FP64 oracle on all host cores: a spawn-started process pool, one
    frame per process at a time, BLAS single-threaded in the workers."""

    def __init__(self):
        from paper_1705_04298_gb300 import synth
        self.cores = os.cpu_count() or 1
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"
        self.r0p, self.L0p = synth.pitch_units(N_LENSLETS, R0, L0)
        self.sl, _, self.mask = synth.batch(N_LENSLETS, self.cores * 8, SEED0, SIGMA, R0, L0)
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.pool.map(_oracle_worker, [(self.sl[0], self.mask, self.r0p, self.L0p)] * self.cores)

    def step(self, frames_per_core):
        n = self.cores * frames_per_core
        work = [(self.sl[i % len(self.sl)], self.mask, self.r0p, self.L0p) for i in range(n)]
        t0 = time.perf_counter()
        self.pool.map(_oracle_worker, work, chunksize=1)
        return n, time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_oracle_run(frames_per_core=6):
    """Bounded sample (about 10 s of CPU work) of the workload on the oracle,
    and beside it the CPU FFT baseline (cpu_baseline/: the same loop with a
    radix-2 FFT, FP64 and FP32, one frame per host thread)."""
    pool = OraclePool()
    try:
        n, wall = pool.step(frames_per_core)
    finally:
        pool.close()
    res = {"value": n / wall, "unit": "frames/s", "cores": pool.cores, "kind": "oracle",
           "sample": "%d frames (%d per core) of the 40x40 -> 128^2 k=%d Wiener workload, FP64 "
                     "direct-DFT oracle, one process per core" % (n, frames_per_core, ITERS)}
    res["fft_baseline"] = cpu_fft_run()
    return res


def cpu_fft_run(frames_per_thread=16):
    """The CPU FFT baseline on all host threads, FP64 and FP32, on the
    benchmark workload's frames (a bounded sample: frames_per_thread each)."""
    try:
        import cpu_baseline
        from paper_1705_04298_gb300 import synth
        threads = cpu_baseline.threads()
        F = threads * frames_per_thread
        r0p, L0p = synth.pitch_units(N_LENSLETS, R0, L0)
        sl, _, mask = synth.batch(N_LENSLETS, 64, SEED0, SIGMA, R0, L0)
        sl = np.concatenate([sl] * ((F + 63) // 64))[:F]
        out = {"kind": "cpu_fft", "unit": "frames/s", "cores": threads,
               "sample": "%d frames of the 40x40 -> 128^2 k=%d Wiener workload, project-written radix-2 FFT "
                         "(cpu_baseline/fft_gerchberg.cpp), one frame per thread" % (F, ITERS)}
        for prec in (64, 32):
            cpu_baseline.reconstruct(sl[:threads], mask, PAD, ITERS, 1, SIGMA ** 2, r0p, L0p, 0, precision=prec)
            t0 = time.perf_counter()
            cpu_baseline.reconstruct(sl, mask, PAD, ITERS, 1, SIGMA ** 2, r0p, L0p, 0, precision=prec)
            out["fp%d" % prec] = F / (time.perf_counter() - t0)
        out["value"] = out["fp32"]
        return out
    except Exception as e:  # the baseline is context; its absence must not stop the benchmark
        return {"kind": "cpu_fft", "unavailable": str(e)}


# ------------------------------------------------------------------ main ----

def _time_launches(fn, flush, reps, torch):
    """Median CUDA-event time (ms) of fn() over reps launches, L2 flushed before each."""
    stream = torch.cuda.current_stream()
    out = []
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return statistics.median(out)


def extra_measurements(fwr, synth, torch, flush):
    """The other workloads of the path, timed the same way (device time, L2
    flushed): 40x40 at each iteration count, the 16x16 single-frame latency
    (FP32 and FP64), a ragged 4096-frame batch of 40/64/80/128-lenslet pupils
    (one graph-captured launch, autotuned schedule) and 128x128 lenslets on a
    256^2 grid with 10 iterations, with the FFT and with the split-BF16
    DFT-as-GEMM transform. The warm starts are measured by
    learned_measurements."""
    peak, _ = fwr.fp32_fma_peak()
    res = {"fp32_peak_tflops_measured": peak}
    # 40x40 on 128^2, k in {0, 1, 2, 5}
    sl, _, mask = synth.batch(N_LENSLETS, FRAMES, SEED0, SIGMA, R0, L0)
    r0p, L0p = synth.pitch_units(N_LENSLETS, R0, L0)
    plan = fwr.Plan(mask, PAD, fwr.WIENER, SIGMA ** 2, r0p, L0p)
    s = torch.tensor(sl, dtype=torch.float32, device="cuda")
    ph = torch.empty((FRAMES, 128, 128), device="cuda")
    per_k = {}
    for k in (0, 1, 2, 5):
        for _ in range(3):
            plan.reconstruct(s, k, ph)
        ms = _time_launches(lambda: plan.reconstruct(s, k, ph), flush, 20, torch)
        tf = flops_per_frame(128, k) * FRAMES / (ms / 1e3) / 1e12
        per_k[str(k)] = {"frames_per_s": FRAMES / (ms / 1e3), "ms": ms, "tflops": tf, "frac": tf / peak}
    res["40x40_128grid_per_k"] = per_k
    # 16x16 on 32^2, one frame, k = 10, LSQ: latency
    fr = synth.frame(16, 0, 0.05)
    p16 = fwr.Plan(fr["mask"], 2.0, fwr.LSQ)
    lat = {}
    for name, dt, call in (("fp32", torch.float32, p16.reconstruct), ("fp64", torch.float64, p16.reconstruct_f64)):
        x = torch.tensor(fr["slopes"][None], dtype=dt, device="cuda")
        y = torch.empty((1, 32, 32), dtype=dt, device="cuda")
        for _ in range(10):
            call(x, 10, y)
        torch.cuda.synchronize()
        ts = []
        for _ in range(200):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            call(x, 10, y)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3)
        lat[name] = {"us_median": statistics.median(ts), "us_min": min(ts)}
    res["16x16_32grid_k10_1frame_latency"] = lat
    # ragged: 1024 frames each of 40, 64, 80, 128 lenslets (128^2, 128^2, 256^2, 256^2), k = 5
    sizes = [(40, 3.2), (64, 2.0), (80, 3.2), (128, 2.0)]
    plans = [fwr.Plan(synth.pupil_mask(n), pad, fwr.LSQ) for n, pad in sizes]
    rng = np.random.default_rng(2)
    fp = rng.permutation(np.repeat(np.arange(4), 1024))
    base = []
    for pl, (n, _) in enumerate(sizes):
        b, _, _ = synth.batch(n, 64, 30000 + 100 * pl, 0.05)
        base.append(torch.tensor(b, dtype=torch.float32, device="cuda"))
    slopes = [base[pl][i % 64] for i, pl in enumerate(fp)]
    phases = [torch.empty((plans[pl].N,) * 2, device="cuda") for pl in fp]
    sp, pp = fwr.Batch.pointer_table(slopes), fwr.Batch.pointer_table(phases)
    batch = fwr.Batch(plans, fp, 5)
    tune_path = os.path.join(OUT_DIR, "fwr_tune.jsonl")
    os.makedirs(os.path.dirname(tune_path), exist_ok=True)
    ctas, ratio = batch.autotune(sp, pp, tune_path)
    g = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream()
    cs.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g, stream=cs):
        batch.run(sp, pp, stream=cs)
    torch.cuda.synchronize()
    g.replay()
    ms = _time_launches(g.replay, flush, 10, torch)
    fl = sum(flops_per_frame(plans[pl].N, 5) for pl in fp)
    # each size class alone (its 1024 frames through the same kernel, one launch)
    per_class = {}
    for pl, (n, _) in enumerate(sizes):
        idx = [i for i, q in enumerate(fp) if q == pl]
        spc = fwr.Batch.pointer_table([slopes[i] for i in idx])
        ppc = fwr.Batch.pointer_table([phases[i] for i in idx])
        bc = fwr.Batch(plans, [pl] * len(idx), 5)
        bc.set_shape(batch.shape)
        bc.run(spc, ppc)
        msc = _time_launches(lambda: bc.run(spc, ppc), flush, 5, torch)
        flc = flops_per_frame(plans[pl].N, 5) * len(idx)
        per_class["%dx%d_on_%d" % (n, n, plans[pl].N)] = {
            "frames": len(idx), "ms": msc, "frames_per_s": len(idx) / (msc / 1e3),
            "frac": flc / (msc / 1e3) / 1e12 / peak}
    res["ragged_4096_40-64-80-128_k5"] = {"frames_per_s": 4096 / (ms / 1e3), "ms": ms,
                                          "tflops": fl / (ms / 1e3) / 1e12, "frac": fl / (ms / 1e3) / 1e12 / peak,
                                          "launches": 1, "graph": True, "ctas": ctas, "cost_ratio": ratio,
                                          "shape": batch.shape, "size_classes_alone": per_class}
    # 128x128 lenslets on 256^2, k = 10, frozen-flow frames
    sl4, _, m4 = synth.frozen_flow(128, 32, 7, 0.05, r0=0.12, L0=25.0)
    p4 = fwr.Plan(m4, 2.0, fwr.LSQ)
    s4 = torch.tensor(sl4, dtype=torch.float32, device="cuda").repeat(32, 1, 1, 1)[:1000].contiguous()
    ph4 = torch.empty((1000, 256, 256), device="cuda")
    launch4 = p4.autotune(s4, 10, ph4, os.path.join(OUT_DIR, "fwr_plan_tune.jsonl"))
    p4.reconstruct(s4, 10, ph4)
    ms = _time_launches(lambda: p4.reconstruct(s4, 10, ph4), flush, 5, torch)
    tf = flops_per_frame(256, 10) * 1000 / (ms / 1e3) / 1e12
    res["128x128_256grid_k10_frozen_flow"] = {"frames_per_s": 1000 / (ms / 1e3), "ms": ms, "tflops": tf,
                                              "frac": tf / peak, "launch": {"shape": launch4[0], "ctas": launch4[1],
                                                                            "l2_persist": p4.l2_persist}}
    # ELT scale: 200x200 lenslets on 512^2 (slab kernel, grid in HBM), k = 10
    sl5, _, m5 = synth.batch(200, 16, 7000, 0.05)
    p5 = fwr.Plan(m5, 2.56, fwr.LSQ)
    F5 = 2 * torch.cuda.get_device_properties(0).multi_processor_count
    s5 = torch.tensor(sl5, dtype=torch.float32, device="cuda").repeat(F5 // 16 + 1, 1, 1, 1)[:F5].contiguous()
    ph5 = torch.empty((F5, 512, 512), device="cuda")
    launch5 = p5.autotune(s5, 10, ph5, os.path.join(OUT_DIR, "fwr_plan_tune.jsonl"))
    ms = _time_launches(lambda: p5.reconstruct(s5, 10, ph5), flush, 3, torch)
    tf = flops_per_frame(512, 10) * F5 / (ms / 1e3) / 1e12
    res["200x200_512grid_k10"] = {"frames": F5, "frames_per_s": F5 / (ms / 1e3), "ms": ms, "tflops": tf,
                                  "frac": tf / peak, "launch": {"shape": launch5[0], "ctas": launch5[1],
                                                                "l2_persist": p5.l2_persist}}
    del s5, ph5
    # the same frames through the split-BF16 DFT-as-GEMM transform (batched
    # tcgen05 GEMMs): 2 GEMMs per 2-D transform, 2 (k + 1) transforms, each
    # GEMM 2 x (2N) x (6N) x N flop per frame
    p4.set_transform(fwr.TRANSFORM_DFT_BF16X3)
    p4.reconstruct(s4, 10, ph4)
    ms = _time_launches(lambda: p4.reconstruct(s4, 10, ph4), flush, 3, torch)
    bpeak, bsrc = measured_bf16_peak()
    gfl = 2 * (10 + 1) * 2 * (2.0 * 512 * 1536 * 256) * 1000
    res["128x128_256grid_k10_frozen_flow_dft_bf16x3"] = {
        "frames_per_s": 1000 / (ms / 1e3), "ms": ms,
        "roofline": {"bound": "tensor", "achieved": gfl / (ms / 1e3) / 1e12, "peak": bpeak, "peak_source": bsrc,
                     "unit": "TFLOP/s", "frac": gfl / (ms / 1e3) / 1e12 / bpeak, "flops_per_launch": gfl,
                     "note": "GEMM flops only; element-wise kernels between the GEMMs are not counted"}}
    # the same with the three-way split, six products (K = 12N)
    p4.set_transform(fwr.TRANSFORM_DFT_BF16X6)
    p4.reconstruct(s4, 10, ph4)
    ms6 = _time_launches(lambda: p4.reconstruct(s4, 10, ph4), flush, 3, torch)
    gfl6 = 2 * gfl
    res["128x128_256grid_k10_frozen_flow_dft_bf16x6"] = {
        "frames_per_s": 1000 / (ms6 / 1e3), "ms": ms6,
        "roofline": {"bound": "tensor", "achieved": gfl6 / (ms6 / 1e3) / 1e12, "peak": bpeak, "peak_source": bsrc,
                     "unit": "TFLOP/s", "frac": gfl6 / (ms6 / 1e3) / 1e12 / bpeak, "flops_per_launch": gfl6,
                     "note": "GEMM flops only (K = 12N); element-wise kernels between the GEMMs are not counted"}}
    p4.set_transform(fwr.TRANSFORM_FFT)
    return res


def measured_bf16_peak():
    """Dense BF16 tensor peak (TFLOP/s): the measured cuBLAS burst figure of
    MEASURED_PEAKS.json when present, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"]), "measured"
    except (OSError, ValueError, KeyError):
        return 1900.0, "fallback"


def l2_window_measurement(fwr, synth, torch, flush):
    """The 256^2 frozen-flow workload of the extras (128x128 lenslets, LSQ,
    k = 10, 1000 frames, L2 flushed) with FWR_OPT_L2_PERSIST: the slab kernel's
    working memory held in a persisting L2 window; the set-aside is given back
    afterwards (fwr_l2_persist_reset)."""
    peak, _ = fwr.fp32_fma_peak()
    sl4, _, m4 = synth.frozen_flow(128, 32, 7, 0.05, r0=0.12, L0=25.0)
    p4 = fwr.Plan(m4, 2.0, fwr.LSQ)
    s4 = torch.tensor(sl4, dtype=torch.float32, device="cuda").repeat(32, 1, 1, 1)[:1000].contiguous()
    ph4 = torch.empty((1000, 256, 256), device="cuda")
    launch = p4.autotune(s4, 10, ph4, os.path.join(OUT_DIR, "fwr_plan_tune.jsonl"))
    p4.set_l2_persist(1)
    p4.reconstruct(s4, 10, ph4)
    ms = _time_launches(lambda: p4.reconstruct(s4, 10, ph4), flush, 5, torch)
    fwr.l2_persist_reset(torch.cuda.current_device())
    tf = flops_per_frame(256, 10) * 1000 / (ms / 1e3) / 1e12
    return {"frames_per_s": 1000 / (ms / 1e3), "ms": ms, "tflops": tf, "frac": tf / peak,
            "launch": {"shape": launch[0], "ctas": launch[1], "l2_persist": 1}}


def learned_measurements(fwr, torch, flush):
    """Warm starts against the plain loop on the held-out frames of the
    warm-start workload (40x40 on 128^2, sigma 0.05 rad, Wiener, 1000
    frames, seeds 2e6 + i): residual phase rms against the true screens and
    frames/s (device time, L2 flushed) of the plain loop at k = 1..10, of the
    U-Net (committed weights) followed by k = 1, 2, and of the linear warm
    start (rank linws.DEFAULT_RANK) followed by k = 1, 2 through
    fwr_linws_reconstruct, called directly and replayed from a CUDA graph
    (its four kernels are short: the graph removes the host launch gaps); the
    equal-residual comparison; the warm start's tensor roofline."""
    from paper_1705_04298_gb300 import learned, linws, synth
    F = 1000
    rank = linws.DEFAULT_RANK
    mask = synth.pupil_mask(learned.N_LENSLETS)
    plan = learned.make_plan(fwr, fwr.WIENER, learned.EVAL_SIGMA)
    slopes, truth = learned.frames(F, learned.EVAL_SEED0, learned.EVAL_SIGMA)
    phase = torch.empty((F, 128, 128), device="cuda")
    warm = torch.empty((F, 2, 128, 128), device="cuda")

    def entry(fn, reps=20):
        for _ in range(3):
            fn()
        ms = _time_launches(fn, flush, reps, torch)
        return {"residual_rad": learned.residual_rms(fwr, phase, truth, mask), "ms": ms,
                "frames_per_s": F / (ms / 1e3)}

    lin = "linear_r%d" % rank
    res = {"plain": {}, "unet": {}, lin: {}}
    for k in (1, 2, 3, 4, 5, 6, 8, 10):
        res["plain"]["k%d" % k] = entry(lambda: plan.reconstruct(slopes, k, phase))
    net = learned.load_net(fwr, learned.WEIGHTS, max_batch=F)
    for k in (1, 2):
        res["unet"]["k%d" % k] = entry(lambda: (net.forward(plan, slopes, warm),
                                                plan.reconstruct(slopes, k, phase, ext_init=warm)))
    ws, _ = linws.build(fwr, plan, mask, rank, max_batch=F)
    for k in (1, 2):
        v = entry(lambda: ws.reconstruct(slopes, k, phase))
        stream = torch.cuda.Stream()
        stream.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            ws.reconstruct(slopes, k, phase, stream=stream)
        torch.cuda.synchronize()
        g = entry(graph.replay)
        v["graph_ms"] = g["ms"]
        v["graph_frames_per_s"] = g["frames_per_s"]
        res[lin]["k%d" % k] = v
    ws.status()
    p10 = res["plain"]["k10"]
    for fam in ("unet", lin):
        for k, v in res[fam].items():
            # the cheapest plain loop reaching this residual, and the target
            # comparison: against ten plain iterations
            match = [kk for kk, pv in res["plain"].items() if pv["residual_rad"] <= v["residual_rad"]]
            v["plain_k_same_residual"] = match[0] if match else None
            v["speedup_same_residual"] = (res["plain"][match[0]]["ms"] / v["ms"]) if match else None
            v["residual_vs_plain_k10"] = v["residual_rad"] / p10["residual_rad"]
            v["speedup_vs_plain_k10"] = p10["ms"] / v["ms"]
            if "graph_ms" in v:
                v["graph_speedup_vs_plain_k10"] = p10["ms"] / v["graph_ms"]
    # the warm start alone (gather + two tcgen05 GEMMs), FP32 output
    ms_ws = _time_launches(lambda: ws.forward(slopes, warm), flush, 20, torch)
    ws.status()
    K = 2 * plan.valid_count
    fl = 2.0 * F * rank * (K + 2 * 128 * 128)
    peak, src = measured_bf16_peak()
    res[lin]["warm_start_roofline"] = {
        "bound": "tensor", "achieved": fl / (ms_ws / 1e3) / 1e12, "peak": peak, "peak_source": src,
        "unit": "TFLOP/s", "frac": fl / (ms_ws / 1e3) / 1e12 / peak, "ms": ms_ws, "flops_per_launch": fl,
        "kernels": "k_gather + umma::gemm_kernel (X A, then (X A) V^T)"}
    return res


def learned_summary(extras):
    """The warm start that meets the residual of ten plain iterations (within
    1 %) with one iteration, against those ten plain iterations."""
    if not extras or "learned_warm_start_40x40_128grid" not in extras:
        return None
    L = extras["learned_warm_start_40x40_128grid"]
    lin = [k for k in L if k.startswith("linear_r")][0]
    v, p10 = L[lin]["k1"], L["plain"]["k10"]
    return {"path": "%s warm start + 1 Gerchberg iteration (fwr_linws_reconstruct, CUDA graph)" % lin,
            "residual_rad": v["residual_rad"], "plain_k10_residual_rad": p10["residual_rad"],
            "residual_vs_plain_k10": v["residual_vs_plain_k10"],
            "frames_per_s": v["graph_frames_per_s"], "plain_k10_frames_per_s": p10["frames_per_s"],
            "speedup_vs_plain_k10": v["graph_speedup_vs_plain_k10"],
            "speedup_direct_call": v["speedup_vs_plain_k10"],
            "unet_k1_residual_rad": L["unet"]["k1"]["residual_rad"],
            "unet_k1_speedup_vs_plain_k10": L["unet"]["k1"]["speedup_vs_plain_k10"]}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed0(rank):
    """First frame seed of a rank: ranks reconstruct disjoint seeded batches
    (weak scaling, no collective on the data path)."""
    return SEED0 + rank * FRAMES


def max_over_ranks(x, dist, device):
    """The largest value of x over the ranks (the slowest rank sets the job's
    time); x itself without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def whole_job_frames_per_s(frames_per_rank, world, ms_per_step):
    return frames_per_rank * world / (ms_per_step / 1000.0)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    pool = OraclePool()
    fpc = 2
    try:
        for _ in range(args.warmup):
            pool.step(1)
        walls, frames = [], 0
        for _ in range(args.steps):
            n, w = pool.step(fpc)
            walls.append(w)
            frames = n
    finally:
        pool.close()
    ms_per_step = 1000.0 * statistics.median(walls)
    value = frames / (ms_per_step / 1000.0)
    cpu = {"value": value, "unit": "frames/s", "cores": pool.cores, "kind": "oracle",
           "sample": "%d frames per step (%d per core) of the 40x40 -> 128^2 k=%d Wiener workload, "
                     "FP64 direct-DFT oracle, one process per core" % (frames, fpc, ITERS)}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "40x40 lenslets (D=8 m) padded to 128^2, seeded von Karman frames, "
                                   "k=%d Gerchberg iterations, Wiener sigma=%g rad" % (ITERS, SIGMA),
                       "frames_per_step": frames},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


WORKLOADS = ("fused128", "slab256", "slab512", "dftgemm256", "unet", "linws")


def run_workload(args):
    """One of the path's workloads, run --reps times after one warm-up call
    and timed with CUDA events (mean; no L2 flush): the command that the
    profile summaries capture under ncu. Each is a plain sequence of library
    calls on seeded synthetic frames (--frames, 1000 by default):
      fused128    40x40 lenslets on 128^2, Wiener, --iters iterations
      slab256     128x128 lenslets on 256^2 (frozen-flow frames), LSQ, --iters
      slab512     200x200 lenslets on 512^2 (ELT scale, seeded frames), LSQ, --iters
                  (both with the persisting L2 window under --l2-persist 1)
      dftgemm256  the same through the split-BF16 DFT-as-GEMM transform
      unet        the warm-start U-Net forward on 40x40 slopes (committed weights)
      linws       the linear warm start (--rank) alone, then with --iters
                  iterations (fwr_linws_forward, fwr_linws_reconstruct)
    """
    import torch
    from paper_1705_04298_gb300 import fwr, learned, synth
    fwr.load()
    F, k = args.frames, args.iters
    runs = []
    if args.workload == "fused128":
        sl, _, mask = synth.batch(40, min(F, 64), SEED0, SIGMA)
        r0p, L0p = synth.pitch_units(40, R0, L0)
        plan = fwr.Plan(mask, PAD, fwr.WIENER, SIGMA ** 2, r0p, L0p)
        s = torch.tensor(sl, dtype=torch.float32, device="cuda").repeat((F + 63) // 64, 1, 1, 1)[:F].contiguous()
        out = torch.empty((F, plan.N, plan.N), device="cuda")
        runs.append(("fused128_k%d" % k, lambda: plan.reconstruct(s, k, out)))
    elif args.workload in ("slab256", "dftgemm256"):
        sl, _, mask = synth.frozen_flow(128, 32, 7, 0.05, r0=0.12, L0=25.0)
        plan = fwr.Plan(mask, 2.0, fwr.LSQ)
        if args.workload == "dftgemm256":
            plan.set_transform(fwr.TRANSFORM_DFT_BF16X3)
        elif args.l2_persist:
            plan.set_l2_persist(1)
        s = torch.tensor(sl, dtype=torch.float32, device="cuda").repeat((F + 31) // 32, 1, 1, 1)[:F].contiguous()
        out = torch.empty((F, plan.N, plan.N), device="cuda")
        runs.append(("%s_k%d" % (args.workload, k), lambda: plan.reconstruct(s, k, out)))
    elif args.workload == "slab512":
        sl, _, mask = synth.batch(200, 16, 7000, 0.05)
        plan = fwr.Plan(mask, 2.56, fwr.LSQ)
        if args.l2_persist:
            plan.set_l2_persist(1)
        s = torch.tensor(sl, dtype=torch.float32, device="cuda").repeat((F + 15) // 16, 1, 1, 1)[:F].contiguous()
        out = torch.empty((F, plan.N, plan.N), device="cuda")
        runs.append(("slab512_k%d" % k, lambda: plan.reconstruct(s, k, out)))
    elif args.workload == "unet":
        net = learned.load_net(fwr, learned.WEIGHTS, max_batch=F)
        plan = learned.make_plan(fwr, fwr.WIENER, learned.EVAL_SIGMA)
        s, _ = learned.frames(F, learned.EVAL_SEED0, learned.EVAL_SIGMA)
        out = torch.empty((F, 2, 128, 128), device="cuda")
        runs.append(("unet_forward", lambda: net.forward(plan, s, out)))
    else:
        from paper_1705_04298_gb300 import linws
        mask = synth.pupil_mask(learned.N_LENSLETS)
        plan = learned.make_plan(fwr, fwr.WIENER, learned.EVAL_SIGMA)
        ws, _ = linws.build(fwr, plan, mask, args.rank, max_batch=F, frames=1024, log=None)
        s, _ = learned.frames(F, learned.EVAL_SEED0, learned.EVAL_SIGMA)
        warm = torch.empty((F, 2, 128, 128), device="cuda")
        out = torch.empty((F, 128, 128), device="cuda")
        runs.append(("linws_r%d_forward" % args.rank, lambda: ws.forward(s, warm)))
        runs.append(("linws_r%d_reconstruct_k%d" % (args.rank, k), lambda: ws.reconstruct(s, k, out)))
    res = {}
    for name, run in runs:
        run()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.reps):
            run()
        e1.record()
        torch.cuda.synchronize()
        res[name + "_ms"] = e0.elapsed_time(e1) / args.reps
    res["frames"] = F
    print(json.dumps(res), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--iters", type=int, default=ITERS)
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--workload", choices=WORKLOADS, default=None,
                    help="run one workload --reps times (for profiling) instead of the benchmark")
    ap.add_argument("--frames", type=int, default=FRAMES)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--rank", type=int, default=256, help="rank of the linws workload")
    ap.add_argument("--l2-persist", type=int, default=0, choices=[0, 1],
                    help="slab256/slab512: FWR_OPT_L2_PERSIST on the plan")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload:
        return run_workload(args)

    rank, world, local = dist_env()
    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # before the first GPU call: the oracle's process pool is spawned
        cpu_base = cpu_oracle_run()

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.distributed.is_nccl_available() else "gloo")

    from paper_1705_04298_gb300 import fwr, synth
    k = args.iters
    sl, _, mask = synth.batch(N_LENSLETS, FRAMES, rank_seed0(rank), SIGMA, R0, L0)
    r0p, L0p = synth.pitch_units(N_LENSLETS, R0, L0)
    plan = fwr.Plan(mask, PAD, fwr.WIENER, SIGMA ** 2, r0p, L0p)
    N = plan.N
    slopes = torch.tensor(sl, dtype=torch.float32, device="cuda")
    phase = torch.empty((FRAMES, N, N), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    # launch shape picked by timing on this workload (cached per device, driver, problem)
    os.makedirs(OUT_DIR, exist_ok=True)
    launch = plan.autotune(slopes, k, phase, os.path.join(OUT_DIR, "fwr_plan_tune.jsonl"))
    for _ in range(args.warmup):
        plan.reconstruct(slopes, k, phase)
    torch.cuda.synchronize()
    # the roofline's denominator: measured FP32 FMA throughput of this GPU
    peak_meas, _ = fwr.fp32_fma_peak()

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.reconstruct(slopes, k, phase)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    barrier()
    clk = clocks.stop()
    gpu_launches = args.steps  # one fused kernel launch per step
    total_ms = max_over_ranks(sum(times), dist, "cuda")
    ms_per_step = total_ms / args.steps
    value = whole_job_frames_per_s(FRAMES, world, ms_per_step)

    # end to end through the host entry point: H2D slopes, kernel, D2H phase
    sh = torch.tensor(sl, dtype=torch.float32).pin_memory()
    ph_host = torch.empty((FRAMES, N, N), dtype=torch.float32).pin_memory()
    plan.reserve(FRAMES)
    for _ in range(2):
        plan.reconstruct_host(sh, k, ph_host)
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        plan.reconstruct_host(sh, k, ph_host)
        torch.cuda.synchronize()
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
    e2e_step = max_over_ranks(statistics.median(e2e_ms), dist, "cuda")

    extras = None
    if rank == 0 and not args.no_extras:
        extras = extra_measurements(fwr, synth, torch, flush)
        extras["learned_warm_start_40x40_128grid"] = learned_measurements(fwr, torch, flush)
        # last, since its L2 set-aside would slow what runs after it
        extras["128x128_256grid_k10_frozen_flow_l2_window"] = l2_window_measurement(fwr, synth, torch, flush)

    if rank == 0:
        fl = flops_per_frame(N, k) * FRAMES
        achieved = fl / (ms_per_step / 1000.0) / 1e12
        peak = peak_meas
        src = kernel_source_hash()
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "40x40 lenslets (D=8 m) padded to 128^2, %d seeded von Karman frames "
                                   "per GPU, k=%d Gerchberg iterations, Wiener sigma=%g rad" % (FRAMES, k, SIGMA),
                       "n_lenslets": N_LENSLETS, "grid": N, "frames_per_gpu": FRAMES, "iters": k,
                       "filter": "wiener", "periodic": "before_each_fft", "l2": "flushed between steps",
                       "valid_lenslets": plan.valid_count, "parallelism": "replicas (frames sharded)",
                       "launch": {"shape": launch[0], "ctas": launch[1], "chosen_by": "fwr_plan_autotune"}},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": TRAFFIC.get(src),
                         "kernel": "fused_kernel<float,128>", "flops_per_launch": fl,
                         "peak_source": "measured: fwr_fp32_fma_peak (FP32 FMA throughput, burst, this GPU)",
                         "peak_derived": fp32_peak_tflops(), "frac_of_derived": achieved / fp32_peak_tflops(),
                         "peak_derived_note": "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (max SM clock)",
                         "source_hash": src},
            "e2e": {"value": FRAMES * world / (e2e_step / 1000.0), "unit": "frames/s",
                    "h2d_bytes_per_step": int(sh.numel() * 4), "d2h_bytes_per_step": int(ph_host.numel() * 4)},
            "learned_vs_plain": learned_summary(extras),
            "gpu_launches": gpu_launches,
            "clocks": clk,
            "cpu_baseline": cpu_base,
            "extras": extras,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
