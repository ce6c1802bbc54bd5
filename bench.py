#!/usr/bin/env python
"""Throughput of AO accelerated stochastic nonnegative tensor completion on one
GB300: observed entries per second per AO epoch, and the fraction of the HBM
roofline that the algorithmic-bytes model of the sampled visits reaches.

Workload (default): a 10^4 x 10^4 x 10^4 tensor, rank 32, 100M observation
draws whose indices follow Zipf(1.1) over a seeded row permutation in every
mode, planted U[0, 1] factors, sigma = 0.01 Gaussian noise, 2% held out (98M
train entries), minibatch fraction c = 0.1, MAX_INNER = 1, float32 factors.
One step is one epoch: ceil(1/c) = 10 AO iterations over the 3 modes (Sec. IV
epoch).  --workload uniform4way: 10^5 x 5*10^4 x 2*10^4 x 10^3, R = 16, 200M
uniform draws, Gamma(2, 0.5) factors, sigma = 0.05; --workload rating:
10^6 x 5*10^5 x 200 user x item x time, R = 64, 500M draws (Zipf(1.2) users
and items), values rounded to 1..5; each with --storage-bf16 for bfloat16
factor storage, and --rmse-epochs E for the held-out RMSE of both storage
forms after E epochs.

--impl reference times the FP64 CPU oracle (OpenMP over rows, the paper's
Algorithm 3 design) on the host cores instead: one whole epoch.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "observed entries/s per AO epoch"
UNIT = "entries/s"
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ntc", choices=["ntc", "reference"])
    ap.add_argument("--nnz", type=int, default=0,
                    help="observation draws (default: the workload's: 100M zipf, 200M uniform4way, 500M rating)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--storage-bf16", action="store_true")
    ap.add_argument("--workload", default="zipf", choices=["zipf", "uniform4way", "rating", "uber"],
                    help="zipf: Zipf(1.1) 10^4-cube, R=32, 100M; uniform4way: 4-way R=16 200M uniform; rating: "
                         "user x item x time R=64 500M; uber: the Uber-shaped 4-way timing twin")
    ap.add_argument("--rmse-epochs", type=int, default=0,
                    help="E > 0: held-out RMSE after E epochs from the initial factors with FP32 and with BF16 "
                         "factor storage (same seeds), reported beside the throughput")
    ap.add_argument("--cpu-sample", default="epoch", choices=["epoch", "iteration"],
                    help="CPU baseline sample: one whole epoch (default) or one AO iteration (all modes once)")
    ap.add_argument("--ref-epochs", type=int, default=1,
                    help="--impl reference: whole epochs timed (the requested --steps are not all run: an "
                         "epoch of the FP64 oracle takes minutes; the line says so)")
    ap.add_argument("--rank", type=int, default=0, help="fitted rank (default: the workload's)")
    ap.add_argument("--overlap", type=int, default=2, choices=[0, 1, 2],
                    help="light rows on a second stream: 2 beside the split-row Gram (default), 1 beside the "
                         "sampler, 0 stream order")
    ap.add_argument("--gram-tc", type=int, default=1, choices=[0, 1, 2, 3],
                    help="split-row Gram where the shape has a tensor-core kernel (R_pad = 32, orders 2-4): "
                         "1 tensor cores, rows gathered into registers (default); 2 tensor cores, rows gathered "
                         "by TMA gather4 in a warp-specialised pipeline; 0: FP32 FMA")
    ap.add_argument("--sampler", default="independent", choices=["independent", "perm"],
                    help="perm: epoch-permutation minibatches (labelled variant)")
    ap.add_argument("--power-warm", type=int, default=0,
                    help="N > 0: warm-started power method with N iterations (labelled variant)")
    # serving stream (continuous-batching completion server)
    ap.add_argument("--serve", action="store_true", help="run the serving stream instead of the epoch bench")
    ap.add_argument("--serve-full", action="store_true",
                    help="full stream: 256 jobs, mode sizes 1e3..2e5, 1M..50M observations")
    ap.add_argument("--serve-jobs", type=int, default=32)
    ap.add_argument("--serve-rate", type=float, default=4.0, help="mean job arrivals per second")
    ap.add_argument("--serve-dims", default="1000,20000", help="log-uniform mode-size range")
    ap.add_argument("--serve-nnz", default="1000000,5000000", help="log-uniform observation range")
    ap.add_argument("--serve-budget", type=float, default=150e9, help="HBM budget, bytes")
    ap.add_argument("--serve-max-epochs", type=int, default=40)
    ap.add_argument("--serve-gen", default="host", choices=["host", "device"],
                    help="draw the jobs' data on the host up front, or on the GPU one by one as they arrive "
                         "(always device with --serve-full)")
    ap.add_argument("--serve-qps", type=float, default=10000.0, help="prediction queries per second")
    # convergence study (synthetic twin of the MovieLens experiments)
    ap.add_argument("--study", default="", choices=["", "convergence", "packing"])
    ap.add_argument("--study-trials", type=int, default=5)
    ap.add_argument("--study-epochs", type=int, default=100)
    ap.add_argument("--study-nnz", type=int, default=10_000_000)
    return ap.parse_args()


DEFAULT_NNZ = {"zipf": 100_000_000, "uniform4way": 200_000_000, "rating": 500_000_000, "uber": 3_309_490}


def workload(args):
    from paper_2109_09534_gb300 import synth
    n = args.nnz or DEFAULT_NNZ[args.workload]
    args.nnz = n
    if args.workload == "uber":
        p = synth.uber_twin()
    elif args.workload == "uniform4way":
        p = synth.uniform_4way(nnz_total=n)
    elif args.workload == "rating":
        p = synth.rating_3way(nnz_total=n)
    else:
        p = synth.zipf_1e4cube(nnz_total=n)
    if args.rank:
        p.rank = args.rank
    return p


def config(p, args):
    import math
    T = int(math.ceil(1.0 / p.c - 1e-12))
    N = len(p.dims)
    storage = "bf16" if args.storage_bf16 else "fp32"
    if args.workload == "uber":
        text = (f"uber-shaped 183x24x1140x1717 tensor, 3,309,490 uniform draws of a planted rank-10 "
                f"noiseless tensor ({p.nnz} train), fitted R={p.rank}, c=0.5, MAX_INNER=1, {storage} factor storage")
        l2 = "inputs larger than L2: 4 per-mode buckets of 16 B/entry (0.21 GB) re-read every epoch"
    elif args.workload == "uniform4way":
        text = (f"uniform 4-way 100000x50000x20000x1000 tensor, R={p.rank}, {args.nnz // 1_000_000}M uniform draws "
                f"({p.nnz} train), planted Gamma(2, 0.5) factors, sigma=0.05, c=0.1, MAX_INNER=1, "
                f"{storage} factor storage")
        l2 = "inputs larger than L2: 4 per-mode buckets of 16 B/entry (~12.5 GB) re-read every epoch"
    elif args.workload == "rating":
        text = (f"rating-shaped user x item x time 1000000x500000x200 tensor, R={p.rank}, "
                f"{args.nnz // 1_000_000}M draws ({p.nnz} train; Zipf(1.2) users and items, uniform time), "
                f"planted U[0, 2a] factors, values rounded and clamped to 1..5, c=0.1, MAX_INNER=1, "
                f"{storage} factor storage")
        l2 = "inputs larger than L2: 3 per-mode buckets of 16 B/entry (~23.8 GB) re-read every epoch"
    else:
        text = (f"zipf1.1 10000^3 tensor, R={p.rank}, {args.nnz // 1_000_000}M draws ({p.nnz} train), c=0.1, "
                f"MAX_INNER=1, {storage} factor storage")
        l2 = "inputs larger than L2: 3 per-mode buckets of 16 B/entry (~4.7 GB) re-read every epoch"
    if getattr(args, "power_warm", 0):
        text += f", variant: warm-started power method, {args.power_warm} iterations"
    if getattr(args, "overlap", 2) == 0:
        text += ", light rows in stream order"
    if getattr(args, "gram_tc", 1) == 0:
        text += ", split-row Gram on FP32 FMA"
    elif getattr(args, "gram_tc", 1) == 2:
        text += ", split-row Gram on the tensor cores with TMA gather4 row loads"
    if getattr(args, "sampler", "independent") == "perm":
        text += ", variant: epoch-permutation minibatches (disjoint stretches of one permutation per row and epoch)"
    return {"workload": text, "dims": p.dims, "rank": p.rank, "nnz_train": p.nnz, "c": p.c, "lambda": p.lam,
            "step": f"one epoch = {T} AO iterations x {N} modes", "l2": l2,
            "parallelism": "replicas" if args.gpus > 1 else "single GPU"}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


# nominal dense TF32 / BF16 tensor rates of the part (1.1 and 2.25 PFLOP/s)
TF32_PER_BF16 = 1.1 / 2.25


def tf32_peak():
    """TF32 dense peak in TFLOP/s: the measured bf16 GEMM burst times the nominal ratio."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path))["bf16_tflops"]) * TF32_PER_BF16, "measured bf16 burst x 1.1/2.25"
    return FALLBACK_BF16_TFLOPS * TF32_PER_BF16, "fallback bf16 x 1.1/2.25"


# sources of the epoch kernels (the serving runtime and the host API are not
# part of what the DRAM counters measured)
KERNEL_SOURCES = ("ntc_internal.cuh", "nmc_kernels.cuh", "gram_tc.cuh", "gram_tc64.cuh", "gram_tma.cuh",
                  "tiny_rows.cuh", "launch_rp.cuh",
                  "nmc_rp8.cu", "nmc_rp16.cu", "nmc_rp32.cu", "nmc_rp64.cu")


def csrc_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2109_09534_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """dram bytes per launch of `kernel` from the committed ncu summary, if the
    kernel sources are unchanged since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except ValueError:
        return None
    if d.get("csrc_sha256_16") != csrc_hash():
        return None
    k = d.get("kernels", {}).get(kernel)
    if not k:
        return None
    return k.get("dram_bytes_per_launch_full_size")


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id):
        self.device_id = device_id
        self.proc = None
        self.path = os.path.join("/tmp", f"ntc_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device_id), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as td
        td.init_process_group("gloo")
    return ws, rank, local


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as td
    t = torch.tensor([x], dtype=torch.float64)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as td
        td.barrier()


def replica_value(units_per_rank, ws, ms_local):
    """Whole-job throughput of ws independent replicas (weak scaling): the
    units all ranks processed over the slowest rank's time.  Returns (value
    per second, max ms)."""
    ms = max_over_ranks(ms_local, ws)
    return ws * units_per_rank / (ms * 1e-3), ms


def cpu_baseline(p, epochs=1, warmup=0, sample="epoch"):
    """The FP64 oracle as it stands, OpenMP over rows (the paper's Algorithm 3),
    on the host cores.  sample="epoch": `epochs` whole epochs (ceil(1/c) AO
    iterations over every mode) are timed, after `warmup` single Algorithm-1
    calls; sample="iteration": one AO iteration (every mode once) is timed and
    the epoch is that times ceil(1/c) (each AO iteration does the same work).
    Returns (the cpu_baseline object, the timed seconds per epoch)."""
    import numpy as np

    import oracle
    o = oracle.Oracle(p.dims, p.rank, p.lam, omp=True)
    o.set_observed(p.idx_train, p.val_train.astype(np.float64))
    o.init_factors(3)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    cores = int(os.environ.get("OMP_NUM_THREADS", cores))
    T = int(np.ceil(1.0 / p.c - 1e-12))
    N = len(p.dims)
    for w in range(warmup):
        o.ao_iter = 1000 + w
        o.snmc(w % N, p.c, seed=3)
    o.ao_iter = 0
    if sample == "iteration":
        t0 = time.perf_counter()
        for m in range(N):
            o.snmc(m, p.c, seed=4)
        t_iter = time.perf_counter() - t0
        t_epoch = t_iter * T
        text = (f"one AO iteration (Algorithm 1 on each of the {N} modes) of the full {p.nnz}-entry workload, "
                f"{t_iter:.2f} s; epoch = {T} such iterations")
        return {"value": p.nnz / t_epoch, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": text}, [t_epoch]
    times = []
    for s in range(epochs):
        t0 = time.perf_counter()
        o.epoch(p.c, seed=4 + s)
        times.append(time.perf_counter() - t0)
    t_epoch = statistics.median(times)
    text = (f"whole epoch{'s' if epochs > 1 else ''} ({T} AO iterations x {N} modes) of the full {p.nnz}-entry "
            f"workload, {t_epoch:.2f} s{' median of %d' % epochs if epochs > 1 else ''}"
            + (f"; warm-up: {warmup} single Algorithm-1 calls" if warmup else ""))
    return {"value": p.nnz / t_epoch, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": text}, times


def run_reference(args):
    """The reference arm: the paper ships no code, so the FP64 oracle (the
    paper's OpenMP design) is timed on the host cores, on the same workload.
    Its epochs take minutes, so it times --ref-epochs whole epochs after
    --warmup single Algorithm-1 calls, and the line reports what was timed."""
    ws, rank, _ = dist()
    if rank != 0:
        return
    p = workload(args)
    cb, times = cpu_baseline(p, epochs=args.ref_epochs, warmup=args.warmup, sample=args.cpu_sample)
    v = cb["value"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": len(times), "steps_requested": args.steps, "warmup": args.warmup,
            "warmup_unit": "one Algorithm-1 call (one mode update)", "ms_per_step": p.nnz / v * 1e3,
            "timed_s": sum(times),
            "steps_note": (f"one step = one whole epoch of the FP64 oracle ({len(times)} timed; the "
                           f"{args.steps} requested would take about {args.steps * p.nnz / v / 60:.0f} min)"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(p, args), "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ntc(args):
    import numpy as np
    import torch

    from paper_2109_09534_gb300 import ntc

    ws, rank, local = dist()
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    p = workload(args)
    params = dict(profile=1, overlap=args.overlap, gram_tc=args.gram_tc)
    if args.storage_bf16:
        params["storage_bf16"] = 1
    if args.power_warm:
        params.update(power_warm=1, power_iters=args.power_warm)
    if args.sampler == "perm":
        params["sampler"] = 1
    g = ntc.NTC(p.dims, p.rank, p.lam, stream=stream.cuda_stream, **params)
    g.set_observed(p.idx_train, p.val_train)
    fp32_peak = ntc.measure_fp32_peak(stream.cuda_stream)

    for w in range(args.warmup):
        g.epoch(p.c, seed=1000 + w)
    g.sync()
    g.profile()   # clear the warm-up launches

    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        dev_id = uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"
    except Exception:
        dev_id = local
    clocks = Clocks(dev_id)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    launches = 0
    alg_bytes = 0
    visits = 0
    for s in range(args.steps):
        g.epoch(p.c, seed=4 + s)
        st = g.stats()
        launches += st["kernel_launches"]
        alg_bytes += st["alg_bytes"]
        visits += st["visits"]
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(ws)
    value, ms = replica_value(p.nnz * args.steps, ws, ev0.elapsed_time(ev1))
    prof = g.profile()

    ms_step = ms / args.steps
    hbm, hbm_kind = peaks()
    # dominant kernel and its roofline
    # (kernels that carry algorithmic bytes: the sampler and resolver touch
    # positions only, whose keys are computed, not read; with light rows on a
    # second stream their event time and the finish's include concurrent work)
    concurrent = ("light", "finish") if args.overlap else ()
    dom = max((k for k in prof if prof[k]["alg_bytes"] > 0 and k not in concurrent), key=lambda k: prof[k]["ms"])
    d = prof[dom]
    per_launch_ms = d["ms"] / max(d["launches"], 1)
    bytes_per_launch = d["alg_bytes"] / max(d["launches"], 1)
    achieved = bytes_per_launch / (per_launch_ms * 1e-3) / 1e9 if per_launch_ms > 0 else 0.0
    R, N = p.rank, p.order
    # the tensor-core Gram runs at padded ranks 32 (16 < R <= 32) and 64 (R > 32), orders 2-4
    rp = 8 if R <= 8 else 16 if R <= 16 else 32 if R <= 32 else 64
    tensor_gram = bool(args.gram_tc) and rp >= 32 and N <= 4
    if not tensor_gram:
        gram_name = "k_heavy_gram"
    elif rp == 64:
        gram_name = "k_heavy_gram_tc64"
    else:
        gram_name = "k_heavy_gram_tma" if args.gram_tc in (2, 3) else "k_heavy_gram_tc"
    kname = {"light": "k_light", "heavy_sample": "k_heavy_sample", "heavy_resolve": "k_heavy_resolve",
             "heavy_gram": gram_name, "finish": "k_rows_finish"}[dom]
    total_k = sum(v["ms"] for v in prof.values())
    flops_per_visit = (N - 2) * R + 2 * R + R * (R + 1)
    s_bytes = 2 if args.storage_bf16 else 4
    gram_visits = prof["heavy_gram"]["alg_bytes"] // ((N - 1) * 4 + 4 + (N - 1) * R * s_bytes)
    gram_s = prof["heavy_gram"]["ms"] * 1e-3
    gram_tf = gram_visits * flops_per_visit / gram_s / 1e12 if gram_s > 0 else 0.0
    # the split-row Gram's algorithmic flops against the FP32 FMA peak (the
    # ALU roofline of the method's arithmetic, whichever unit runs it) and,
    # on the tensor cores, its issued TF32 work against the tensor peak
    compute_roof = {"roofline_alu": {
        "kernel": gram_name, "achieved": gram_tf, "peak": fp32_peak, "unit": "TFLOP/s",
        "frac": gram_tf / fp32_peak if fp32_peak else None,
        "peak_kind": "measured FP32 FMA microbenchmark, same run", "flops_per_visit": flops_per_visit}}
    if tensor_gram:
        # issued tensor work: one M x N=R_pad x K=8 TF32 MMA per 8 visits, M = 2 R_pad
        # (the S = [big; small] rows) in the register-gather kernels, M = 128 in the
        # TMA-gather form
        m_rows = 128 if args.gram_tc in (2, 3) else 2 * rp
        tc_flops_per_visit = 2 * m_rows * rp
        tc_tf = gram_visits * tc_flops_per_visit / gram_s / 1e12 if gram_s > 0 else 0.0
        tpk, tpk_kind = tf32_peak()
        compute_roof["roofline_tensor"] = {
            "kernel": gram_name, "achieved": tc_tf, "peak": tpk, "unit": "TFLOP/s", "frac": tc_tf / tpk,
            "peak_kind": tpk_kind, "dtype": "tf32 (3xTF32 split of FP32)",
            "flops_per_visit_issued": tc_flops_per_visit, "alg_flops_per_visit": flops_per_visit,
            "alg_tflops": gram_tf}

    # split-row sampler: a Philox4x32-10 key for every position of every split row
    # (more than 4096 observations, the handle's default threshold) in each mode
    # update, four keys per block; each block takes 16 32x32->64-bit multiplies
    # (two rounds start from per-thread precomputed values, the rest two per
    # round), reported against a nominal integer multiply rate of 64 per clock
    # per SM at the sampled SM clock
    import math as _m
    keyed = 0
    for m in range(N):
        cnt = np.bincount(p.idx_train[:, m].astype(np.int64), minlength=p.dims[m])
        keyed += int(cnt[cnt > 4096].sum())
    keyed_epoch = keyed * _m.ceil(1.0 / p.c - 1e-12)
    samp_s = prof["heavy_sample"]["ms"] * 1e-3 / max(args.steps, 1)
    if keyed_epoch and samp_s > 0:
        mul_s = keyed_epoch / 4 * 16 / samp_s
        sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        mul_peak = 64.0 * nsm * sm_mhz * 1e6
        compute_roof["sampler"] = {
            "kernel": "k_heavy_sample", "keys_per_epoch": keyed_epoch, "ms_per_epoch": samp_s * 1e3,
            "keys_per_s": keyed_epoch / samp_s, "mul64_per_key": 4.0, "int_mul_per_s": mul_s,
            "int_mul_peak_nominal": mul_peak, "int_mul_frac": mul_s / mul_peak,
            "note": "event time inside the overlapped epoch; the ncu capture gives the pipe shares"}

    # end to end through the C ABI with pinned host buffers
    idx_pin = torch.from_numpy(np.ascontiguousarray(p.idx_train)).pin_memory()
    val_pin = torch.from_numpy(np.ascontiguousarray(p.val_train)).pin_memory()
    h2d = idx_pin.numel() * 4 + val_pin.numel() * 4
    d2h = sum(d_ * R * 4 for d_ in p.dims)
    e2e_times = []
    g.set_param("profile", 0)
    for s in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.set_observed_ptr(p.nnz, idx_pin.data_ptr(), val_pin.data_ptr(), device=False)
        g.epoch(p.c, seed=77 + s)
        _ = g.factors()
        torch.cuda.synchronize()
        if s > 0:
            e2e_times.append(time.perf_counter() - t0)
    e2e_t = max_over_ranks(statistics.median(e2e_times), ws) if e2e_times else None

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16-storage/f32" if args.storage_bf16 else "f32",
            "data": "synthetic", "config": config(p, args), "clocks": clk,
            "e2e": {"value": ws * p.nnz / e2e_t if e2e_t else None, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "step": "ntc_set_observed (pinned host COO, device bucketing) + ntc_epoch + "
                            "ntc_get_factor x3"},
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm,
                         "peak_kind": hbm_kind, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": ncu_traffic(kname),
                         "alg_bytes_per_launch": bytes_per_launch, "ms_per_launch": per_launch_ms},
            "roofline_epoch": {"alg_bytes_per_epoch": alg_bytes / args.steps,
                               "achieved_gbs": alg_bytes / (ms * 1e-3) / 1e9 * ws,
                               "frac_of_hbm": alg_bytes / (ms * 1e-3) / 1e9 / hbm, "peak_kind": hbm_kind},
            **compute_roof,
            "kernels": {k: {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] / args.steps,
                            "share": v["ms"] / total_k if total_k else None} for k, v in prof.items()},
            "kernels_note": ("CUDA-event times per kernel class; light rows run on a second stream beside the "
                             "split-row Gram and the next update's split-row sampling on a third, so these "
                             "times include concurrent execution (the serialised shares are in the committed "
                             "ncu launch list)") if args.overlap else
                            "CUDA-event times per kernel class; split-row sampling runs beside the Gram",
            "visits_per_s": ws * visits / (ms * 1e-3)}
    if args.rmse_epochs > 0:
        line["heldout_rmse"] = storage_rmse(p, args, stream.cuda_stream)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        del g
        torch.cuda.empty_cache()
        line["cpu_baseline"], _ = cpu_baseline(p, epochs=1, sample=args.cpu_sample)
    if rank == 0:
        print(json.dumps(line), flush=True)


def storage_rmse(p, args, stream):
    """Held-out RMSE after args.rmse_epochs epochs from the initial factors,
    FP32 and BF16 factor storage on the same seeds (the precision contract:
    BF16 storage within 1% of FP32)."""
    from paper_2109_09534_gb300 import ntc
    out = {}
    for bf in (0, 1):
        g = ntc.NTC(p.dims, p.rank, p.lam, stream=stream, storage_bf16=bf, gram_tc=args.gram_tc)
        g.set_observed(p.idx_train, p.val_train)
        r0 = g.rmse(p.idx_test, p.val_test)
        for e in range(args.rmse_epochs):
            g.epoch(p.c, seed=500 + e)
        out["bf16" if bf else "fp32"] = g.rmse(p.idx_test, p.val_test)
        out["initial"] = r0
        g.close()
    out["epochs"] = args.rmse_epochs
    out["bf16_vs_fp32"] = out["bf16"] / out["fp32"] - 1.0
    return out


def run_serve(args):
    """Serving stream: Poisson job arrivals admitted under the HBM budget, each
    job run epoch by epoch until its held-out RMSE reaches 1.1 sigma (or the
    epoch limit), with Poisson prediction queries against running jobs
    batched into one multi-job launch per tick."""
    import numpy as np
    import torch

    from paper_2109_09534_gb300 import ntc, synth

    torch.cuda.set_device(0)
    if args.serve_full:
        args.serve_jobs, args.serve_dims, args.serve_nnz = 256, "1000,200000", "1000000,50000000"
    dlo, dhi = (float(x) for x in args.serve_dims.split(","))
    nlo, nhi = (float(x) for x in args.serve_nnz.split(","))
    specs = synth.serving_stream(args.serve_jobs, rate=args.serve_rate, dim_range=(dlo, dhi),
                                 nnz_range=(nlo, nhi))
    sigma = 0.01
    target = 1.1 * sigma
    device_gen = args.serve_full or args.serve_gen == "device"
    t_gen = time.perf_counter()
    probs = None
    jobq = None
    if device_gen:
        # jobs drawn on the GPU one by one, in arrival order and a few ahead of
        # the submission loop; a job's host arrays are released once admitted
        import queue
        import threading
        jobq = queue.Queue(maxsize=6)

        def produce():
            torch.cuda.set_device(0)
            for s in specs:
                jobq.put((s, synth.serving_job_device(s, sigma=sigma, test_frac=0.01)))
        gen_thread = threading.Thread(target=produce, daemon=True)
        gen_thread.start()
    else:
        probs = [synth.serving_job(s, sigma=sigma, test_frac=0.01) for s in specs]
    t_gen = time.perf_counter() - t_gen
    srv = ntc.Server(args.serve_budget, 64)
    srv.set_param("max_enqueue_per_step", 2)
    clocks = Clocks(0)
    clocks.start()
    t0 = srv.now()
    ids = []
    dims_of = {}           # job id -> mode sizes (queries)
    obs_ratio = []         # observations per factor entry, per job

    def submit_job(k, s, p):
        jid = srv.submit(p.dims, p.rank, p.lam, p.c, p.idx_train, p.val_train, p.idx_test, p.val_test,
                         target, args.serve_max_epochs, arrival=t0 + s.arrival, seed=1000 + 97 * k,
                         init_seed=3, storage_bf16=s.storage_bf16)
        ids.append(jid)
        dims_of[jid] = list(p.dims)
        obs_ratio.append(p.nnz / float(p.rank * sum(p.dims)))

    if not device_gen:
        for k, (s, p) in enumerate(zip(specs, probs)):
            submit_job(k, s, p)
    rng = np.random.default_rng(7)
    lat = []
    t_q = srv.now()
    pending = []          # arrival times of queries not yet served
    while True:
        while device_gen and len(ids) < len(specs) and not jobq.empty():
            s, p = jobq.get()
            submit_job(len(ids), s, p)
            del p
        srv.step()
        now = srv.now()
        # queries that arrived since the last tick (Poisson), against running
        # jobs: while none is running there is nothing to query
        running = [(j, dims_of[j]) for j in ids if srv.job_info(j)["state"] == ntc.JOB_RUNNING]
        if running:
            nq = rng.poisson(args.serve_qps * (now - t_q))
            pending += list(np.sort(rng.uniform(t_q, now, nq)))
        t_q = now
        if pending and running:
            pick = rng.integers(0, len(running), len(pending))
            q_job = np.array([j for j, _ in running], dtype=np.int64)[pick]
            dmat = np.ones((len(running), 8))
            for r, (_, dm) in enumerate(running):
                dmat[r, :len(dm)] = dm
            q_idx = (rng.random((len(pending), 8)) * dmat[pick]).astype(np.int32)   # padding columns stay 0
            srv.predict(q_job, q_idx)
            t_ret = srv.now()
            lat += [t_ret - a for a in pending]
            pending = []
        if len(ids) == len(specs) and all(srv.job_info(j)["state"] >= ntc.JOB_DONE for j in ids):
            break
        time.sleep(0.0002)
    wall = srv.now() - t0
    clk = clocks.stop()
    infos = [srv.job_info(j) for j in ids]
    st = srv.stats()
    reached = [i for i in infos if i["reached"]]
    ttt = np.array([i["t_done"] - i["t_arrival"] for i in reached]) if reached else np.array([np.nan])
    lat_ms = np.array(lat) * 1e3 if lat else np.array([np.nan])
    line = {"metric": "serving p50/p99 time-to-target-RMSE", "unit": "s", "mode": "serve",
            "value": float(np.percentile(ttt, 50)), "p50_time_to_target_s": float(np.percentile(ttt, 50)),
            "p99_time_to_target_s": float(np.percentile(ttt, 99)), "higher_is_better": False,
            "jobs": len(ids), "reached": len(reached), "failed": st["failed"],
            "censored_at_max_epochs": sum(1 for i in infos if i["state"] == ntc.JOB_DONE and not i["reached"]),
            "query_latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99)),
                                 "queries": st["predict_queries"], "launches": st["predict_launches"]},
            "entries_per_s": st["entries"] / wall, "epochs": st["epochs"], "wall_s": wall,
            "peak_running": st["peak_running"], "peak_bytes": st["peak_bytes"], "budget_bytes": args.serve_budget,
            "job_results": [{"order": len(s.dims), "rank": s.rank, "nnz": s.nnz, "bf16": s.storage_bf16,
                             "obs_per_param": round(r, 2),
                             "epochs": i["epochs"], "rmse0": round(i["rmse0"], 5), "rmse": round(i["rmse"], 5),
                             "reached": i["reached"], "queue_s": round(i["t_admit"] - i["t_arrival"], 4),
                             "run_s": round(i["t_done"] - i["t_admit"], 4)}
                            for s, i, r in zip(specs, infos, obs_ratio)],
            "rmse_over_sigma": {q: float(np.percentile([i["rmse"] / sigma for i in infos], q))
                                for q in (10, 50, 90)},
            "generation": "device (torch, per job, a few ahead of submission)" if device_gen else "host (numpy)",
            "n_gpus": 1, "data": "synthetic", "dtype": "f32 / bf16-storage (half the jobs each)", "clocks": clk,
            "config": {"workload": f"{args.serve_jobs} jobs, Poisson {args.serve_rate}/s, order 3-4, mode sizes "
                                   f"log-uniform {args.serve_dims}, R in 8/16/32/64, observations log-uniform "
                                   f"{args.serve_nnz}, uniform indices, planted U[0,1], sigma 0.01, target "
                                   f"RMSE 1.1 sigma, max {args.serve_max_epochs} epochs, "
                                   f"{args.serve_qps:.0f} queries/s",
                       "generation_s": t_gen}}
    srv.close()
    print(json.dumps(line), flush=True)


def run_study(args):
    """Convergence study: RRE of the held-out entries against the planted
    (noise-free) values after each epoch, for minibatch fractions c and two
    noise levels, over several seeded trials (Sec. IV-B experiments, on a
    planted tensor of MovieLens-10M's shape instead of the dataset)."""
    import numpy as np
    import torch

    from paper_2109_09534_gb300 import ntc, synth

    dims, R = [71567, 65133, 730], 10
    snrs_db = [40.0, 20.0]
    cs = [0.05, 0.2, 0.5]
    marks = [e for e in (1, 2, 5, 10, 20, 50, 100, 200) if e <= args.study_epochs]
    stream = torch.cuda.current_stream().cuda_stream
    res = {}
    t0 = time.perf_counter()
    for snr in snrs_db:
        for trial in range(args.study_trials):
            p0 = synth.make_problem(dims, R, args.study_nnz, lam=1e-3, c=0.1, index_dist="uniform", sigma=0.0,
                                    test_frac=0.01, seed=100 + trial, name="ml10m-twin")
            # noise for the requested SNR: sigma^2 = E[x^2] / 10^(snr/10)
            power = float(np.mean(p0.val_train.astype(np.float64) ** 2))
            sigma = float(np.sqrt(power / 10 ** (snr / 10)))
            rng = np.random.default_rng(7000 + trial)
            vals = (p0.val_train + sigma * rng.standard_normal(p0.val_train.shape)).astype(np.float32)
            clean = p0.val_test_clean
            for c in cs:
                g = ntc.NTC(dims, R, p0.lam, stream=stream, init_seed=3 + trial,
                            sampler=1 if args.sampler == "perm" else 0)
                g.set_observed(p0.idx_train, vals)
                curve = {}
                for e in range(1, args.study_epochs + 1):
                    g.epoch(c, seed=10_000 * trial + e)
                    if e in marks:
                        x = g.predict(p0.idx_test).astype(np.float64)
                        curve[e] = float(np.linalg.norm(x - clean) / np.linalg.norm(clean))
                g.close()
                res.setdefault((snr, c), []).append(curve)
    table = {}
    for (snr, c), curves in res.items():
        key = f"snr{snr:g}dB_c{c:g}"
        table[key] = {str(e): {"mean": float(np.mean([cv[e] for cv in curves])),
                               "std": float(np.std([cv[e] for cv in curves]))} for e in marks}
    line = {"metric": "held-out RRE vs epoch", "mode": "study", "unit": "relative", "data": "synthetic",
            "config": {"workload": f"planted rank-{R} U[0,1] tensor of MovieLens-10M shape {dims}, "
                                   f"{args.study_nnz} uniform draws (1% held out), lambda 1e-3, fitted R = {R}, "
                                   f"SNR {snrs_db} dB, c {cs}, {args.study_trials} trials, "
                                   f"{args.study_epochs} epochs, {args.sampler} minibatches"},
            "rre": table, "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


def run_packing_study(args):
    """Does the server leave throughput on the table by running each job's
    epochs as its own launches on its own stream instead of packing several
    jobs' updates into shared launches?  The same work three ways: J jobs of n
    observations at once through the server, the same J jobs one at a time,
    and one handle holding all J n observations (the throughput a perfectly
    packed launch sequence could approach).  Each job runs E epochs."""
    import numpy as np
    import torch

    from paper_2109_09534_gb300 import ntc, synth

    torch.cuda.set_device(0)
    J, n, E, R, dims = 16, 2_000_000, 10, 16, [20_000, 20_000, 20_000]
    specs = [synth.JobSpec(0.0, dims, R, n, 0, 900 + k) for k in range(J)]
    probs = [synth.serving_job_device(s, sigma=0.01, test_frac=0.01) for s in specs]
    res = {}
    for mode, max_running in (("concurrent", J), ("one_at_a_time", 1)):
        srv = ntc.Server(150e9, max_running)
        srv.set_param("max_enqueue_per_step", 4)
        ids = [srv.submit(p.dims, p.rank, p.lam, p.c, p.idx_train, p.val_train, p.idx_test, p.val_test, 0.0, E,
                          arrival=0.0, seed=10 * k, init_seed=3) for k, p in enumerate(probs)]
        # admission (upload and bucketing) is not part of the comparison: time
        # from the first epoch enqueued to the last collected
        while any(srv.job_info(j)["state"] == ntc.JOB_QUEUED for j in ids[:max_running]):
            srv.step()
            time.sleep(0.0005)
        t0 = time.perf_counter()
        while not all(srv.job_info(j)["state"] >= ntc.JOB_DONE for j in ids):
            srv.step()
            time.sleep(0.0002)
        wall = time.perf_counter() - t0
        st = srv.stats()
        res[mode] = {"wall_s": wall, "entries_per_s": st["entries"] / wall, "epochs": st["epochs"],
                     "peak_running": st["peak_running"]}
        srv.close()
    # one handle with all J n observations and J times the rows per mode, so that
    # its rows hold as many observations as each job's: the same kernels on a
    # J-times larger grid, which is what packed launches of the J jobs would run
    big = synth.serving_job_device(synth.JobSpec(0.0, [J * d for d in dims], R, J * n, 0, 950), sigma=0.01,
                                   test_frac=0.01)
    s = torch.cuda.current_stream()
    g = ntc.NTC(big.dims, big.rank, big.lam, stream=s.cuda_stream)
    g.set_observed(big.idx_train, big.val_train)
    g.epoch(big.c, seed=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for e in range(E):
        g.epoch(big.c, seed=2 + e)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    res["one_handle_all_observations"] = {"wall_s": wall, "entries_per_s": big.nnz * E / wall,
                                          "dims": big.dims, "launches_per_epoch": g.stats()["kernel_launches"]}
    # one job alone
    g1 = ntc.NTC(probs[0].dims, R, probs[0].lam, stream=s.cuda_stream)
    g1.set_observed(probs[0].idx_train, probs[0].val_train)
    g1.epoch(0.1, seed=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for e in range(E):
        g1.epoch(0.1, seed=2 + e)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    res["one_job_alone"] = {"wall_s": wall, "entries_per_s": probs[0].nnz * E / wall,
                            "launches_per_epoch": g1.stats()["kernel_launches"]}
    line = {"metric": "serving packing study: aggregate observed entries/s", "mode": "study", "unit": "entries/s",
            "data": "synthetic", "config": {"workload": f"{J} jobs of {n} uniform observations, dims {dims}, "
                                                         f"R={R}, FP32, c=0.1, {E} epochs each"},
            "results": res,
            "concurrent_over_one_handle": res["concurrent"]["entries_per_s"] /
            res["one_handle_all_observations"]["entries_per_s"]}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.study == "packing":
        run_packing_study(args)
        return
    if args.study:
        run_study(args)
        return
    if args.serve:
        run_serve(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ntc(args)


if __name__ == "__main__":
    main()
