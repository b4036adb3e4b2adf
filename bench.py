"""Benchmark of the FBST hot path on GB300.

Default workload (ULA1024): 1024-element linear array, fb = 0.5, N = 512 snapshots per block,
B = 1024 beams, L = 1024, 64 contiguous blocks of one record per step, complex64 in and out. This
is the array size (M = B = 1024) at which the transform's roofline is stated. Stage 1 (the fan
chirp-z) runs in FP32 on the CUDA cores; stage 2 by default is the precomputed-inverse apply on the
tensor cores in split FP16 (hi + lo halves with exact power-of-two scales) with split FP32
accumulation (FP32-class: its error against the FP64 oracle is measured and reported on every run);
--stage2 dense_tf32x3 selects the split-TF32 form, gs_ir1 the Gohberg-Semencul path, dense_fp32 the
CUDA-core apply. One step = fbst_execute over the 64 blocks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fbst|reference] [--stage2 VARIANT]
                  [--workload ULA1024|NU1024|C2|C3|NUC3|C4|C5|C2N|C2NT|OG|STREAM|GEN] [--contraction tf32x3|fp32]

With N > 1 (torchrun) every rank runs its own replica of the plan on its own share of the
stream's blocks (rank r takes blocks [r*nblk, (r+1)*nblk) of one continuous record: weak scaling;
the method has no cross-block exchange, so there is no collective on the data path). Rank 0 prints
one JSON line. `value` is device time measured with CUDA events on the launching stream, L2
flushed (256 MiB write) before every timed step; `e2e` goes through the C-ABI host-buffer entry
point with pinned host memory, copies included; `roofline` times each kernel live with events
around its own C-ABI stage call; the FP32 ALU peak is measured live (an FMA-chain kernel of the
library, with the SM clock sampled meanwhile); `cpu_baseline` times the FP64 oracle on the host
cores on a bounded sample. `--impl reference` times the oracle alone (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "beam-samples/s at rel err ≤1e-5 vs FP64 oracle, %HBM roofline; p50/p99 latency"
UNIT = "beam-samples/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}
FP32_LANES = 128   # FP32 lanes per SM (4 sub-partitions x 32)


def load_peaks() -> tuple[dict, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return dict(PEAKS_FALLBACK), "fallback"


def fft_flops(P: int) -> float:
    """Nominal complex FFT cost, 5 P log2 P."""
    return 5.0 * P * math.log2(P)


def flop_model(info) -> dict:
    """Nominal FLOPs per launch unit of each kernel (5 P log2 P per transform, 6 per complex multiply,
    2 per complex add), counted for the transforms the kernels perform."""
    M, N, B, L = info.M, info.N, info.B, info.L
    S, Pt = info.S_time, info.P_time
    time_per_sensor = (1 + S) * fft_flops(Pt) + 6.0 * (N + S * Pt + L)
    Ps = info.P_space_x
    space_per_freq = 2 * fft_flops(Ps) + 6.0 * (M + Ps + B)
    Pg, Pr, Sr = info.P_gs, info.P_rec, info.S_rec
    gs = 6 * fft_flops(Pg) + 6.0 * 4 * Pg + 2.0 * Pg
    rec = (Sr + 1) * fft_flops(Pr) + 6.0 * (L + Sr * Pr + N) + 2.0 * (Sr - 1) * Pr
    # Stage 2: GS + F_u for the FFT variants (the refinement step's transforms are not counted);
    # 8 N L flops per beam-block (complex multiply-add) for the dense apply.
    dense = info.stage2 >= 3
    stage2 = 8.0 * N * L * B if dense else (gs + rec) * B
    return {"czt_time": time_per_sensor * M, "czt_space": space_per_freq * L, "stage2": stage2}


# Tensor-core variants: (planes of G, bytes per element, products per complex term, peak dtype,
# passes over w: prepared planes = read + write + read; the fused TF32x3 kernel reads w once; the
# FP16x3 stage-2 call reads it once more for the block scales, which the whole transform takes from
# stage 1b instead). FP16 MMAs run at the BF16 rate.
TC_VARIANTS = {4: (4, 2, 3, "bf16", 3), 5: (2, 4, 1, "tf32", 3), 6: (2, 4, 3, "tf32", 1), 7: (2, 4, 3, "f16", 2)}


def tc_peak_of(peaks: dict, dt: str) -> tuple:
    """Tensor peak for a variant's MMA type: the measured BF16 figure, halved for TF32 (nominal ratio)."""
    if dt == "tf32":
        return float(peaks["bf16_tflops"]) * 0.5, "bf16_tflops x 0.5 (tf32 nominal ratio)"
    return float(peaks["bf16_tflops"]), "bf16_tflops x 1" + (" (f16 = bf16 nominal rate)" if dt == "f16" else "")


def nominal_fp32_peak(sms: int, sm_mhz: float) -> dict:
    """FP32 FMA peak from unit counts and clock: SMs x 128 lanes x 2 flops x clock."""
    return {"tflops": sms * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12,
            "source": f"nominal: {sms} SMs x {FP32_LANES} lanes x 2 x {sm_mhz:.0f} MHz"}


def path_bytes(info, nblk: int) -> float:
    """Compulsory HBM bytes of the whole transform over nblk blocks: y in, bhat out and one
    generator per beam per block, 8 (M N + B N + B L) bytes per block (32 B per beam-sample at
    M = B and L = 2N)."""
    M, N, B, L = info.M, info.N, info.B, info.L
    return 8.0 * nblk * (M * N + B * N + B * L)


def roofline(kernel: str, info, nblk: int, ms: float, peaks: dict, peak_kind: str, fp32: dict,
             w_scales_from_stage1: bool = False) -> dict:
    """Roofline entry of one kernel launch (nblk blocks) that took `ms` milliseconds. `fp32` is the
    FP32 ALU peak ({"tflops", "source"}), measured where possible. w_scales_from_stage1: the FP16
    split's per-block scales of w come from the spatial chirp-z (inside fbst_execute on a linear
    grid array), so stage 2 reads w once instead of twice."""
    fp32_peak = float(fp32["tflops"])
    flops = flop_model(info)[kernel] * nblk
    M, N, B, L = info.M, info.N, info.B, info.L
    if kernel == "stage2" and info.stage2 in TC_VARIANTS:
        npl, esz, terms, dt, wpass = TC_VARIANTS[info.stage2]
        if w_scales_from_stage1 and dt == "f16":
            wpass = 1
        nbytes = float(B) * npl * N * L * esz + wpass * B * L * nblk * 8.0 + B * N * nblk * 8.0
        hbm = float(peaks["hbm_gbs"])
        tc_peak, tc_src = tc_peak_of(peaks, dt)
        if nbytes / (hbm * 1e9) >= terms * flops / (tc_peak * 1e12):
            ach = nbytes / (ms / 1e3) / 1e9
            return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                    "peak_source": f"{peak_kind} hbm_gbs; bytes = G planes + w passes + bhat"}
        ach = terms * flops / (ms / 1e3) / 1e12
        return {"bound": "tensor", "achieved": ach, "peak": tc_peak, "unit": "TFLOP/s", "frac": ach / tc_peak,
                "peak_source": f"{peak_kind} {tc_src}"}
    ach = flops / (ms / 1e3) / 1e12
    return {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
            "peak_source": fp32["source"]}


def path_roofline(info, nblk: int, ms: float, peaks: dict, fp32: dict) -> dict:
    """Fraction of the binding roof of the whole step: t_roof = max(compulsory bytes / HBM peak,
    FP32 flops / FP32 peak + tensor-core flops / TF32 peak) against the measured step time."""
    fm = flop_model(info)
    alu = (fm["czt_time"] + fm["czt_space"]) * nblk
    tc = 0.0
    if info.stage2 in TC_VARIANTS:
        _, _, terms, dt, _ = TC_VARIANTS[info.stage2]
        tc_peak, _ = tc_peak_of(peaks, dt)
        tc = terms * fm["stage2"] * nblk / (tc_peak * 1e12)
    else:
        alu += fm["stage2"] * nblk
    t_bytes = path_bytes(info, nblk) / (float(peaks["hbm_gbs"]) * 1e9)
    t_flops = alu / (float(fp32["tflops"]) * 1e12) + tc
    t_roof = max(t_bytes, t_flops)
    return {"bound": "hbm" if t_bytes >= t_flops else "compute", "t_roof_ms": t_roof * 1e3, "t_step_ms": ms,
            "frac": t_roof / (ms / 1e3), "t_hbm_ms": t_bytes * 1e3, "t_compute_ms": t_flops * 1e3,
            "bytes_per_beam_sample": path_bytes(info, nblk) / (nblk * info.B * info.N)}


def measure_fp32_peak(fb, gpu_index: int, budget_ms: float = 600.0) -> dict:
    """FP32 FMA throughput of this GPU measured with the library's FMA-chain kernel, the SM clock
    sampled by nvidia-smi while it runs. Best of three timed launches of about budget_ms each."""
    tf, ms = fb.fp32_fma_peak(1024)
    iters = max(1024, int(1024 * budget_ms / max(ms, 1e-3)))
    sampler = ClockSampler(gpu_index)
    time.sleep(0.25)
    best = 0.0
    for _ in range(3):
        tf, ms = fb.fp32_fma_peak(iters)
        best = max(best, tf)
    clocks = sampler.stop()
    src = f"measured: FMA-chain kernel, {iters} x 128 FMAs per thread on every resident CTA, best of 3"
    if clocks.get("sm_mhz"):
        src += f", SM clock median {clocks['sm_mhz']:.0f} MHz during the run"
    return {"tflops": best, "source": src, "sm_mhz": clocks.get("sm_mhz"), "reasons": clocks.get("reasons")}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def w_is_stream(args) -> bool:
    """Workloads whose blocks are cut from one continuous record (replicas take later segments)."""
    return args.workload in ("C2", "ULA1024", "NU1024")


def workload(args, first_block: int = 0):
    """The workload's geometry and a generator of its input; a replica's record starts at block
    `first_block` of the stream (linear arrays)."""
    from synth import configs
    if args.workload in ("C2", "ULA1024", "NU1024"):
        c = configs.CONFIGS[args.workload]
        nb = args.nblk or c["nblk"]
        return dict(kind="ula", mx=c["mx"], my=1, bx=c["bx"], by=1, N=c["N"], frac_bw=c["frac_bw"], nblk=nb,
                    name=args.workload, offsets=configs.config_geometry(args.workload).offsets), \
            lambda: configs.config_data(args.workload, nblk=nb, first_block=first_block)["y"]
    if args.workload in ("C3", "NUC3"):
        nb = args.nblk or configs.CONFIGS[args.workload]["nblk"]
        return dict(kind="ura", mx=32, my=32, bx=32, by=32, N=512, frac_bw=0.3, nblk=nb, name=args.workload,
                    offsets=configs.config_geometry(args.workload).offsets), \
            lambda: configs.config_data(args.workload, nblk=nb, Q=64)["y"]
    raise SystemExit(f"unknown workload {args.workload}")


def oracle_sample(w: dict, y: np.ndarray, beams, nblk: int, budget_s: float):
    """Time the FP64 oracle (execute part, per-plan LU excluded) on a bounded sample."""
    import oracle as O
    pb = O.make_problem(w["kind"], w["mx"], w["my"], w["bx"], w["by"], w["N"], frac_bw=w["frac_bw"],
                        epsilon=1.01, delta_rel=1e-3, offsets=w.get("offsets"))
    t0 = time.perf_counter()
    fac = O.Stage2Factors(pb, beams)
    t_plan = time.perf_counter() - t0
    done, t_exec = 0, 0.0
    out = None
    while t_exec < budget_s or done == 0:
        t0 = time.perf_counter()
        out = O.fbst(pb, y[:nblk], factors=fac)
        t_exec += time.perf_counter() - t0
        done += 1
    samples = done * nblk * len(beams) * w["N"]
    return samples / t_exec, t_plan, done, out, pb


def run_c4(args) -> None:
    """C4: 64 independent linear arrays (M = 2^U{5..10}, N from {128..1024}, B = M, fb ~ U[0.2,0.6]),
    one block each: the batch (grouped launches, CUDA-graph replay, autotuned shapes) against the
    plain per-array fbst_execute loop on the same GPU, same outputs."""
    import torch
    import paper_2512_08887_gb300 as fb
    from paper_2512_08887_gb300 import autotune
    from paper_2512_08887_gb300.build import build
    from synth import configs
    build()
    torch.cuda.set_device(0)
    insts = configs.c4_instances(count=64)
    plans = [fb.Plan(fb.make_geometry("ula", d["M"]), d["N"], fb.make_band(d["frac_bw"], max_blocks=1))
             for d in insts]
    if not args.no_tune:
        for p in plans:
            autotune.tune(p, 1)
    ys = [torch.from_numpy(d["y"]).cuda() for d in insts]
    outs = [torch.empty((1, d["B"], d["N"]), dtype=torch.complex64, device="cuda") for d in insts]
    ref = [torch.empty_like(o) for o in outs]
    batch = fb.Batch(plans)
    ones = [1] * len(plans)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for p, y, r in zip(plans, ys, ref):
        p.execute(y, r, 1)
    batch.execute(ys, outs, ones)
    torch.cuda.synchronize()
    identical = all(torch.equal(o, r) for o, r in zip(outs, ref))
    units = float(sum(d["B"] * d["N"] for d in insts))

    def timed(fn):
        for _ in range(args.warmup):
            flush.zero_()
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    sampler = ClockSampler(torch.cuda.current_device())
    t_batch = timed(lambda: batch.execute(ys, outs, ones))
    clocks = sampler.stop()
    t_plain = timed(lambda: [p.execute(y, o, 1) for p, y, o in zip(plans, ys, outs)])
    import oracle as O
    errs = []
    for k in (0, 21, 63):
        d, i = insts[k], plans[k].info
        pb = O.make_problem("ula", d["M"], 1, d["M"], 1, d["N"], frac_bw=i.fb_num / i.fb_den,
                            epsilon=i.eps_num / i.eps_den, delta=i.delta, L=i.L)
        beams = np.array([0, d["M"] // 2, d["M"] - 1])
        errs.append(O.rel_l2(outs[k].cpu().numpy()[:, beams], O.fbst(pb, d["y"], beams=beams)))
    value = units / (statistics.mean(t_batch) / 1e3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(t_batch), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "C4: 64 uneven ULAs (M=2^U{5..10}, N in {128..1024}, B=M, fb~U[0.2,0.6]), "
                                   "1 block each, batched + CUDA graph, autotuned stage-1 shapes",
                       "l2": "flushed before every timed step (256 MiB write, untimed)"},
            "plain_value": units / (statistics.mean(t_plain) / 1e3),
            "speedup_vs_plain": statistics.mean(t_plain) / statistics.mean(t_batch),
            "latency_ms": {"p50": float(np.percentile(t_batch, 50)), "p99": float(np.percentile(t_batch, 99))},
            "plain_latency_ms": {"p50": float(np.percentile(t_plain, 50)), "p99": float(np.percentile(t_plain, 99))},
            "batch_equals_plain_bitwise": identical, "rel_err_vs_oracle_max": max(errs),
            "gpu_launches": batch.launch_count() * args.steps, "plain_launches_per_step": 3 * len(plans),
            "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_c5(args) -> None:
    """C5: Poisson request streams at rates 1e2..1e5 /s over the 64 C4 arrays (one block per
    request, two seeded data blocks per array), served by the continuous-batching server and by the
    plain one-request-at-a-time server on the same GPU; p50/p99 latency and throughput per rate."""
    import torch
    import paper_2512_08887_gb300 as fb
    from paper_2512_08887_gb300 import autotune, serve
    from paper_2512_08887_gb300.build import build
    from synth import configs
    build()
    torch.cuda.set_device(0)
    insts = configs.c4_instances(count=64)
    plans = [fb.Plan(fb.make_geometry("ula", d["M"]), d["N"], fb.make_band(d["frac_bw"], max_blocks=32))
             for d in insts]
    if not args.no_tune:
        for p in plans:
            autotune.tune(p, 1)
    rng = np.random.default_rng(55)
    pools = []
    for d in insts:
        blocks = [torch.from_numpy(d["y"]).pin_memory()]
        noise = 0.1 * (rng.standard_normal(d["y"].shape) + 1j * rng.standard_normal(d["y"].shape))
        blocks.append(torch.from_numpy((d["y"] + noise).astype(np.complex64)).pin_memory())
        pools.append(blocks)
    req_work = [p.B * p.N for p in plans]
    # Resident per-stream arenas sized from the device's free memory; admission against them.
    ex = serve.GPUExecutor(plans, n_streams=args.streams)
    req_bytes = [ex.request_bytes(a) for a in range(len(plans))]
    budget = min(args.mem_budget, ex.device_budget)
    sched = lambda: serve.Scheduler(req_bytes, budget, 32, req_work, args.batch_work, max_batch_bytes=ex.arena_bytes)
    rates = [float(r) for r in args.rates.split(",")]
    # Warm both paths (one-time kernel set-up).
    warm = serve.poisson_requests(1e5, 128, pools, seed=1)
    serve.run_loop(warm, sched(), ex)
    serve.serve_plain(serve.poisson_requests(1e5, 64, pools, seed=2), plans)
    results = []
    for k, rate in enumerate(rates):
        reqs = serve.poisson_requests(rate, args.requests, pools, seed=100 + k)
        st_b = serve.run_loop(reqs, sched(), ex)
        reqs_p = serve.poisson_requests(rate, args.requests, pools, seed=100 + k)
        st_p = serve.serve_plain(reqs_p, plans)
        results.append({"rate_per_s": rate, "batched": st_b, "plain": st_p})
        print(json.dumps({"rate": rate, "batched": st_b, "plain": st_p}), file=sys.stderr, flush=True)
    ex.close()
    top = results[-1]
    line = {"metric": METRIC, "value": top["batched"]["beam_samples_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.requests, "warmup": 128, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"C5: Poisson requests over the 64 C4 arrays, {args.requests} per rate, "
                                   f"{args.streams} streams, memory budget {budget >> 20} MiB "
                                   f"(resident arenas of {ex.arena_bytes >> 20} MiB per stream)"},
            "latency_ms": {"p50": top["batched"]["p50_ms"], "p99": top["batched"]["p99_ms"]},
            "per_rate": results}
    print(json.dumps(line), flush=True)


def null_roofline(B: int, L: int, P: int, nblk: int, ms: float, contraction: str, peaks: dict,
                  peak_kind: str, fp32: dict) -> dict:
    """Roofline of the bracket of Eq. (14) over nblk blocks (its three launches together): the
    compulsory bytes are the cross Gram operator (FP32 re/im planes, read once), w read and the
    nulled w written; the contraction does 8 B L P L flops per block (x3 products when split-TF32)."""
    nbytes = 8.0 * B * L * P * L + 2 * 8.0 * nblk * B * L
    flops = 8.0 * B * L * P * L * nblk
    hbm = float(peaks["hbm_gbs"])
    if contraction == "tf32x3":
        tc_peak = float(peaks["bf16_tflops"]) * 0.5
        if nbytes / (hbm * 1e9) >= 3 * flops / (tc_peak * 1e12):
            ach = nbytes / (ms / 1e3) / 1e9
            return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                    "peak_source": f"{peak_kind} hbm_gbs; bytes = cross Gram planes + w in + nulled w out"}
        ach = 3 * flops / (ms / 1e3) / 1e12
        return {"bound": "tensor", "achieved": ach, "peak": tc_peak, "unit": "TFLOP/s", "frac": ach / tc_peak,
                "peak_source": f"{peak_kind} bf16_tflops x 0.5 (tf32 nominal ratio); 3 split-TF32 products"}
    fp32_peak = float(fp32["tflops"])
    ach = flops / (ms / 1e3) / 1e12
    return {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
            "peak_source": fp32["source"]}


def run_null(args) -> None:
    """C2N: the transform of the C2 array with beamspace nulling (Eq. (14)) of grid beams 64 and 96,
    64 blocks per step; one step = fbst_null_execute (stage 1, the bracket of Eq. (14), stage 2).
    C2NT: the same scene with the time-domain form (Eq. (15)); one step = fbst_null_execute of a
    time-domain object (stage 1, the plain stage 2, the interferers' beams over the broader interval,
    the time-domain subtraction)."""
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        raise SystemExit("--workload C2N/C2NT runs on one GPU (replicas of it scale like C2)")
    time_form = args.workload == "C2NT"
    import torch
    import paper_2512_08887_gb300 as fb
    from paper_2512_08887_gb300.build import build
    from synth import configs
    import oracle as O
    build()
    torch.cuda.set_device(0)
    c = configs.NULLING["C2N"]
    nblk = args.nblk or c["nblk"]
    d = configs.nulling_data("C2N", nblk=nblk)
    M, B, N, ints = c["mx"], c["bx"], c["N"], c["interferers"]
    P = len(ints)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    plan = fb.Plan(fb.make_geometry("ula", M), N, fb.make_band(c["frac_bw"], stage2=args.stage2, max_blocks=nblk))
    info = plan.info
    L = info.L
    t0 = time.perf_counter()
    nl = fb.Nulling(plan, ints, args.contraction, time_domain=time_form)
    t_create = time.perf_counter() - t0
    y = torch.from_numpy(d["y"]).to(dev)
    out = torch.empty((nblk, B, N), dtype=torch.complex64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    nl.execute(y, out, nblk)
    if plan.sync_status() != 0:
        raise SystemExit("device status word set after the nulled transform")
    beams = [63, 64, 65, 96, 160, 255]
    pb = O.make_problem("ula", M, 1, B, 1, N, frac_bw=info.fb_num / info.fb_den, epsilon=info.eps_num / info.eps_den,
                        delta=info.delta, L=L)
    got = out[:2].cpu().numpy()[:, beams]
    ref = (O.fbst_nulled_time if time_form else O.fbst_nulled)(pb, d["y"][:2], ints, beams=beams)
    rel_err = O.rel_l2(got, ref)
    # Nulling subtracts large corrections: FP32 errors follow the input scale, so the error is also
    # given relative to the plain transform's output of the same blocks and beams.
    err_plain = float(np.linalg.norm(got - ref) / np.linalg.norm(O.fbst(pb, d["y"][:2], beams=beams)))

    for _ in range(args.warmup):
        flush.zero_()
        nl.execute(y, out, nblk)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(0)
    time.sleep(0.3)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        nl.execute(y, out, nblk)
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    value = float(nblk) * B * N * args.steps / (sum(step_ms) / 1e3)

    # Per-stage live timing through the C-ABI stage calls, events on the launching stream.
    kin = min(args.steps, 200)
    yhat = torch.empty((nblk, L, M), dtype=torch.complex64, device=dev)
    wbuf = torch.empty((nblk, B, L), dtype=torch.complex64, device=dev)
    wt = torch.empty_like(wbuf)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(kin)]
    if time_form:
        # The time-domain subtraction alone needs the interferers' beams over the broader interval:
        # the oracle's, rounded to complex64 (untimed set-up).
        tf = O.TimeNullingFactors(pb, ints, beams=[])
        y_int = torch.from_numpy(tf.interferer_beams(O.fan_coefficients(pb, d["y"], ints)).astype(np.complex64)).to(dev)
        plain = torch.empty_like(out)
    for i in range(kin):
        flush.zero_()
        ev[i][0].record(stream)
        plan.czt_time(y, yhat, nblk)
        ev[i][1].record(stream)
        plan.czt_space(yhat, wbuf, nblk)
        ev[i][2].record(stream)
        if time_form:
            plan.toeplitz_apply(wbuf, plain, nblk)
            ev[i][3].record(stream)
            nl.apply_time(plain, y_int, out, nblk)
        else:
            nl.apply(wbuf, wt, nblk)
            ev[i][3].record(stream)
            plan.toeplitz_apply(wt, out, nblk)
        ev[i][4].record(stream)
    torch.cuda.synchronize()
    names = ["czt_time", "czt_space", "stage2", "null_time_apply"] if time_form else \
        ["czt_time", "czt_space", "null_bracket", "stage2"]
    kern_ms = {n: statistics.mean(ev[i][j].elapsed_time(ev[i][j + 1]) for i in range(kin)) for j, n in enumerate(names)}

    # End to end through the public API: pinned host input copied in, the nulled transform, the
    # result copied back to pinned host memory, all on the stream and inside the timed region.
    y_host = torch.from_numpy(d["y"]).pin_memory()
    out_host = torch.empty((nblk, B, N), dtype=torch.complex64).pin_memory()
    e2e_t = []
    for i in range(min(args.steps, 200) + 3):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        y.copy_(y_host, non_blocking=True)
        nl.execute(y, out, nblk)
        out_host.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        if i >= 3:
            e2e_t.append(time.perf_counter() - t0)

    peaks, peak_kind = load_peaks()
    fp32 = measure_fp32_peak(fb, 0)
    roofs = {k: roofline(k, info, nblk, v, peaks, peak_kind, fp32) for k, v in kern_ms.items()
             if k not in ("null_bracket", "null_time_apply")}
    if time_form:
        # F_x^{-1} per interferer, the cross Gram contraction (the bracket's shape), the plan's
        # stage 2 of the correction and the subtraction: reported against the contraction's roof,
        # as the bracket of Eq. (14) is.
        roofs["null_time_apply"] = null_roofline(B, L, P, nblk, kern_ms["null_time_apply"], args.contraction, peaks,
                                                 peak_kind, fp32)
    else:
        roofs["null_bracket"] = null_roofline(B, L, P, nblk, kern_ms["null_bracket"], args.contraction, peaks,
                                              peak_kind, fp32)
    dom = max(kern_ms, key=kern_ms.get)

    cpu = None
    if not args.no_cpu_baseline:
        sb = [int(b) for b in np.linspace(0, B - 1, 32).astype(int)]
        t0 = time.perf_counter()
        fac = (O.TimeNullingFactors if time_form else O.NullingFactors)(pb, ints, sb)
        t_fac = time.perf_counter() - t0
        done, t_exec = 0, 0.0
        while t_exec < 10.0 or done == 0:
            t0 = time.perf_counter()
            (O.fbst_nulled_time if time_form else O.fbst_nulled)(pb, d["y"][:4], ints, factors=fac)
            t_exec += time.perf_counter() - t0
            done += 1
        cpu = {"value": done * 4 * len(sb) * N / t_exec, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{done} x (4 blocks x 32 of {B} beams) of {args.workload}, FP64 numpy oracle of "
                         f"Eq. ({15 if time_form else 14}), "
                         f"per-plan factors and cross Gram matrices ({t_fac:.1f} s) excluded"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(step_ms), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": f"f32 stage 1, {args.contraction} nulling contraction with FP64 interferer solves, "
                 f"{fb.STAGE2_NAMES[info.stage2]} stage 2",
        "data": "synthetic",
        "config": {"workload": (f"C2NT: ULA M={M} B={B} N={N} L={L} fb={c['frac_bw']}, time-domain nulling "
                                f"(Eq. (15)) of grid beams {ints}, {nblk} blocks/step, complex64") if time_form else
                               (f"C2N: ULA M={M} B={B} N={N} L={L} fb={c['frac_bw']}, beamspace nulling (Eq. (14)) "
                                f"of grid beams {ints}, {nblk} blocks/step, complex64"),
                   "M": M, "B": B, "N": N, "L": L, "interferers": ints, "nblk_per_gpu": nblk,
                   "stage2": fb.STAGE2_NAMES[info.stage2], "contraction": args.contraction,
                   "l2": "flushed before every timed step (256 MiB write, untimed)", "parallelism": "replicas x1"},
        "rel_err_vs_oracle": rel_err,
        "err_vs_oracle_rel_to_plain_output": err_plain,
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "roofline": dict(roofs[dom], kernel=dom, traffic=None),
        "kernels_ms": kern_ms,
        "kernels_roofline": roofs,
        "e2e": {"value": float(nblk) * B * N * len(e2e_t) / sum(e2e_t), "unit": UNIT,
                "h2d_bytes_per_step": int(8 * nblk * M * N), "d2h_bytes_per_step": int(8 * nblk * B * N)},
        "gpu_launches": nl.launch_count(nblk) * args.steps,
        "clocks": clocks,
        "fp32_peak": fp32,
        "wall_s_timed_region": wall,
        "nulling_create_s": t_create,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    nl.close()
    print(json.dumps(line), flush=True)


def run_gen(args) -> None:
    """GEN: the solve for the stage-2 generators x_b = A_b^{-1} e_0 (Sec. V) of every beam of a
    1024-element ULA plan (1024 Hermitian positive definite Toeplitz systems, L = 2N), in FP64 on
    the GPU: the superfast solver (doubling Schur algorithm with FFT polynomial products,
    O(L log^2 L)) against the Levinson recursion (O(L^2)). One step = fbst_solve_generators (the
    generators a_b in FP64 and the solve). --gen-n sets N (512: L = 1024, the ULA1024 plan;
    1024: L = 2048, the largest L)."""
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        raise SystemExit("--workload GEN runs on one GPU")
    import torch
    import paper_2512_08887_gb300 as fb
    from paper_2512_08887_gb300.build import build
    import oracle as O
    build()
    torch.cuda.set_device(0)
    M, N = 1024, args.gen_n
    plan = fb.Plan(fb.make_geometry("ula", M), N, fb.make_band(0.5, stage2="gs", max_blocks=1))
    B, L = plan.B, plan.L
    x = {m: torch.empty((B, L), dtype=torch.complex128, device="cuda") for m in ("superfast", "levinson")}
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(method):
        for _ in range(args.warmup):
            plan.solve_generators(method, x[method])
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            plan.solve_generators(method, x[method])
            b.record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    sampler = ClockSampler(torch.cuda.current_device())
    t_sf = timed("superfast")
    clocks = sampler.stop()
    t_lev = timed("levinson")
    if plan.sync_status() != 0:
        raise SystemExit("a generator solve reported an error")
    xs, xl = x["superfast"].cpu().numpy(), x["levinson"].cpu().numpy()
    i = plan.info
    pb = O.make_problem("ula", M, 1, M, 1, N, frac_bw=i.fb_num / i.fb_den, epsilon=i.eps_num / i.eps_den,
                        delta=i.delta, L=L)
    beams = [0, B // 2 + 1]
    errs = {"superfast": 0.0, "levinson": 0.0}
    for b in beams:
        ref = np.linalg.solve(O.gram(pb, b), np.eye(L)[:, 0])
        for m, xv in (("superfast", xs), ("levinson", xl)):
            errs[m] = max(errs[m], O.rel_l2(xv[b], ref))
    ms = statistics.mean(t_sf)
    line = {"metric": "Toeplitz generator systems solved/s (FP64, rel err vs dense solve)", "value": B / (ms / 1e3),
            "unit": "systems/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"GEN: generators of the ULA M={M} B={B} N={N} L={L} plan, {B} systems per step, "
                                   "superfast (doubling Schur) vs Levinson",
                       "l2": "flushed before every timed step (256 MiB write, untimed)"},
            "levinson_value": B / (statistics.mean(t_lev) / 1e3), "levinson_ms_per_step": statistics.mean(t_lev),
            "speedup_vs_levinson": statistics.mean(t_lev) / ms,
            "rel_err_vs_dense_solve": errs, "superfast_vs_levinson": O.rel_l2(xs, xl),
            "gpu_launches": 2 * args.steps, "clocks": clocks,
            "roofline": None, "roofline_note": "FP64 latency-bound recursion (sequential Schur steps and FFT passes "
                                               "per system); no measured FP64 peak to set a roof"}
    print(json.dumps(line), flush=True)


def run_offgrid(args) -> None:
    """OG: off-grid beams (Sec. VIII-A) on a 2x oversampled grid, the paper's setting: 256-element
    ULA, 512 grid beams, N = 256, 64 blocks per step, 64 off-grid directions, each interpolated from
    8 grid beam vectors; one step = fbst_offgrid_execute (stage 1, interpolation, stage 2 of the
    off-grid directions)."""
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        raise SystemExit("--workload OG runs on one GPU (replicas of it scale like the plain transform)")
    import torch
    import paper_2512_08887_gb300 as fb
    from paper_2512_08887_gb300.build import build
    from synth import configs
    import oracle as O
    build()
    torch.cuda.set_device(0)
    M, B, N, nblk, ndir = 256, 512, 256, args.nblk or 64, 64
    d = configs.config_data("C2", nblk=nblk)                  # the 256-element record of C2
    dirs = np.stack([np.random.default_rng(2026).uniform(-0.98, 0.98, ndir), np.zeros(ndir)], axis=1)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    # The grid plan provides stage 1 and the workspace; its own stage 2 is not used here.
    plan = fb.Plan(fb.make_geometry("ula", M, 1, B, 1), N, fb.make_band(0.5, stage2="gs", max_blocks=nblk))
    info = plan.info
    L = info.L
    t0 = time.perf_counter()
    og = fb.OffGrid(plan, dirs)
    t_create = time.perf_counter() - t0
    y = torch.from_numpy(d["y"]).to(dev)
    out = torch.empty((nblk, ndir, N), dtype=torch.complex64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    og.execute(y, out, nblk)
    if plan.sync_status() != 0:
        raise SystemExit("device status word set after the off-grid transform")
    pb = O.make_problem("ula", M, 1, B, 1, N, frac_bw=info.fb_num / info.fb_den, epsilon=info.eps_num / info.eps_den,
                        delta=info.delta, L=L)
    sel = [0, 17, 40, 63]
    fac = O.OffGridFactors(pb, dirs[sel])
    ref = fac.apply(fac.interpolate(O.fan_coefficients(pb, d["y"][:2])))
    rel_err = O.rel_l2(out[:2].cpu().numpy()[:, sel], ref)
    exact = fac.apply(O.fan_coefficients(pb, d["y"][:2], directions=dirs[sel]))
    interp_vs_exact = O.rel_l2(ref, exact)

    for _ in range(args.warmup):
        flush.zero_()
        og.execute(y, out, nblk)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(0)
    time.sleep(0.3)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        og.execute(y, out, nblk)
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    value = float(nblk) * ndir * N * args.steps / (sum(step_ms) / 1e3)

    # Per-stage live timing: stage 1 (two C-ABI calls), the interpolation, the interpolation + the
    # off-grid stage 2 (fbst_offgrid_apply), each with events on the launching stream.
    kin = min(args.steps, 200)
    yhat = torch.empty((nblk, L, M), dtype=torch.complex64, device=dev)
    wbuf = torch.empty((nblk, B, L), dtype=torch.complex64, device=dev)
    wstar = torch.empty((nblk, ndir, L), dtype=torch.complex64, device=dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(kin)]
    for i in range(kin):
        flush.zero_()
        ev[i][0].record(stream)
        plan.czt_time(y, yhat, nblk)
        ev[i][1].record(stream)
        plan.czt_space(yhat, wbuf, nblk)
        ev[i][2].record(stream)
        og.interpolate(wbuf, wstar, nblk)
        ev[i][3].record(stream)
        og.apply(wbuf, out, nblk)
        ev[i][4].record(stream)
    torch.cuda.synchronize()
    names = ["czt_time", "czt_space", "interp", "interp_and_stage2"]
    kern_ms = {n: statistics.mean(ev[i][j].elapsed_time(ev[i][j + 1]) for i in range(kin)) for j, n in enumerate(names)}
    kern_ms["offgrid_stage2"] = kern_ms["interp_and_stage2"] - kern_ms["interp"]

    y_host = torch.from_numpy(d["y"]).pin_memory()
    out_host = torch.empty((nblk, ndir, N), dtype=torch.complex64).pin_memory()
    e2e_t = []
    for i in range(min(args.steps, 200) + 3):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        y.copy_(y_host, non_blocking=True)
        og.execute(y, out, nblk)
        out_host.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        if i >= 3:
            e2e_t.append(time.perf_counter() - t0)

    peaks, peak_kind = load_peaks()
    fp32 = measure_fp32_peak(fb, 0)
    # The interpolation reads K = 8 beam vectors per direction and writes one: HBM-bound, with the
    # compulsory bytes w* out + the grid vectors it reads (once each, at most the whole w).
    rows_read = min(B, ndir * 8)
    interp_bytes = 8.0 * nblk * L * (rows_read + ndir)
    ach = interp_bytes / (kern_ms["interp"] / 1e3) / 1e9
    roofs = {k: roofline(k, info, nblk, kern_ms[k], peaks, peak_kind, fp32) for k in ("czt_time", "czt_space")}
    roofs["interp"] = {"bound": "hbm", "achieved": ach, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                       "frac": ach / float(peaks["hbm_gbs"]),
                       "peak_source": f"{peak_kind} hbm_gbs; bytes = grid beam vectors read once + w* written"}
    sinfo = type("S", (), dict(M=M, N=N, B=ndir, L=L, S_time=info.S_time, P_time=info.P_time, P_space_x=info.P_space_x,
                               P_gs=info.P_gs, P_rec=info.P_rec, S_rec=info.S_rec, stage2=2))
    roofs["offgrid_stage2"] = roofline("stage2", sinfo, nblk, kern_ms["offgrid_stage2"], peaks, peak_kind, fp32)
    dom = max(("czt_time", "czt_space", "interp", "offgrid_stage2"), key=lambda k: kern_ms[k])

    cpu = None
    if not args.no_cpu_baseline:
        t0 = time.perf_counter()
        facs = O.OffGridFactors(pb, dirs[:16])
        t_fac = time.perf_counter() - t0
        done, t_exec = 0, 0.0
        while t_exec < 10.0 or done == 0:
            t0 = time.perf_counter()
            O.fbst_offgrid(pb, d["y"][:4], dirs[:16], factors=facs)
            t_exec += time.perf_counter() - t0
            done += 1
        cpu = {"value": done * 4 * 16 * N / t_exec, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{done} x (4 blocks x 16 of {ndir} off-grid directions), FP64 numpy oracle of Sec. VIII-A, "
                         f"per-plan factors ({t_fac:.1f} s) excluded"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(step_ms), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"OG: off-grid beams (Sec. VIII-A), ULA M={M} with {B} grid beams (2x oversampled), "
                               f"N={N} L={L} fb=0.5, {ndir} off-grid directions from 8 grid beams each, "
                               f"{nblk} blocks/step, complex64; value counts off-grid beam-samples",
                   "M": M, "B_grid": B, "N": N, "L": L, "directions": ndir, "nblk_per_gpu": nblk,
                   "l2": "flushed before every timed step (256 MiB write, untimed)", "parallelism": "replicas x1"},
        "rel_err_vs_oracle": rel_err,
        "interpolated_vs_exact_offgrid_beam": interp_vs_exact,
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "roofline": dict(roofs[dom], kernel=dom, traffic=None),
        "kernels_ms": kern_ms,
        "kernels_roofline": roofs,
        "e2e": {"value": float(nblk) * ndir * N * len(e2e_t) / sum(e2e_t), "unit": UNIT,
                "h2d_bytes_per_step": int(8 * nblk * M * N), "d2h_bytes_per_step": int(8 * nblk * ndir * N)},
        "gpu_launches": 4 * ((nblk + plan.band.max_blocks - 1) // plan.band.max_blocks) * args.steps,
        "clocks": clocks,
        "fp32_peak": fp32,
        "wall_s_timed_region": wall,
        "offgrid_create_s": t_create,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    og.close()
    print(json.dumps(line), flush=True)


def run_stream(args) -> None:
    """STREAM: the ULA1024 record (1024 elements, 64 x 512 = 32768 samples) as one continuous stream,
    cut into blocks of N = 512 every hop = 384 samples (25% overlap, 85 blocks); each block
    contributes its central 384 output samples; one step = fbst_execute_stream over the record;
    `value` counts output beam-samples."""
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        raise SystemExit("--workload STREAM runs on one GPU (replicas take later records)")
    import torch
    import paper_2512_08887_gb300 as fb
    from paper_2512_08887_gb300 import autotune
    from paper_2512_08887_gb300.build import build
    from synth import configs
    import oracle as O
    build()
    torch.cuda.set_device(0)
    c = configs.CONFIGS["ULA1024"]
    M, B, N, hop = c["mx"], c["bx"], c["N"], args.hop
    y = configs.config_data("ULA1024")["y"]                    # [64][M][N] blocks of one record
    rec_np = np.ascontiguousarray(y.transpose(1, 0, 2).reshape(M, -1))
    T = rec_np.shape[1]
    nblk = (T - N) // hop + 1
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    plan = fb.Plan(fb.make_geometry("ula", M), N, fb.make_band(c["frac_bw"], stage2=args.stage2, max_blocks=64))
    info = plan.info
    if not args.no_tune:
        autotune.tune(plan, 64)
    rec = torch.from_numpy(rec_np).to(dev)
    out = torch.empty((B, nblk * hop), dtype=torch.complex64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    plan.execute_stream(rec, T, hop, out, nblk)
    if plan.sync_status() != 0:
        raise SystemExit("device status word set after the streamed transform")
    pb = O.make_problem("ula", M, 1, B, 1, N, frac_bw=info.fb_num / info.fb_den, epsilon=info.eps_num / info.eps_den,
                        delta=info.delta, L=info.L)
    beams = [0, 300, 511, 1023]
    k0 = 40                                                    # 3 blocks in the middle of the record
    ref = O.fbst_stream(pb, rec_np[:, k0 * hop:], hop, 3, beams=beams)
    got = out.cpu().numpy()[beams][:, k0 * hop:(k0 + 3) * hop]
    rel_err = O.rel_l2(got, ref)

    for _ in range(args.warmup):
        flush.zero_()
        plan.execute_stream(rec, T, hop, out, nblk)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(0)
    time.sleep(0.3)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        plan.execute_stream(rec, T, hop, out, nblk)
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    units = float(B) * nblk * hop
    value = units * args.steps / (sum(step_ms) / 1e3)

    rec_host = torch.from_numpy(rec_np).pin_memory()
    out_host = torch.empty((B, nblk * hop), dtype=torch.complex64).pin_memory()
    e2e_t = []
    for i in range(min(args.steps, 50) + 3):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rec.copy_(rec_host, non_blocking=True)
        plan.execute_stream(rec, T, hop, out, nblk)
        out_host.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        if i >= 3:
            e2e_t.append(time.perf_counter() - t0)
    peaks, peak_kind = load_peaks()
    fp32 = measure_fp32_peak(fb, 0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(step_ms), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 stage 1 + " + fb.STAGE2_NAMES[info.stage2] + " stage 2", "data": "synthetic",
        "config": {"workload": f"STREAM: ULA M={M} B={B} N={N} L={info.L}, one record of {T} samples in {nblk} "
                               f"blocks every {hop} samples (overlap {N - hop}), central {hop} samples of each; "
                               "value counts output beam-samples",
                   "M": M, "B": B, "N": N, "hop": hop, "T": T, "blocks": nblk,
                   "l2": "flushed before every timed step (256 MiB write, untimed)", "parallelism": "replicas x1"},
        "rel_err_vs_oracle": rel_err,
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "path_roofline": path_roofline(info, nblk, statistics.mean(step_ms), peaks, fp32),
        "e2e": {"value": units * len(e2e_t) / sum(e2e_t), "unit": UNIT,
                "h2d_bytes_per_step": int(8 * M * T), "d2h_bytes_per_step": int(8 * B * nblk * hop)},
        "gpu_launches": 4 * ((nblk + 63) // 64) * args.steps,
        "clocks": clocks,
        "fp32_peak": fp32,
        "wall_s_timed_region": wall,
    }
    print(json.dumps(line), flush=True)


def run_reference_null(args) -> None:
    """Reference arm of C2N (C2NT): the FP64 oracle of Eq. (14) (Eq. (15)) on one block x 16 beams per
    step."""
    import oracle as O
    from synth import configs
    c = configs.NULLING["C2N"]
    y = configs.nulling_data("C2N", nblk=1)["y"]
    beams = [int(b) for b in np.linspace(0, c["bx"] - 1, 16).astype(int)]
    pb = O.make_problem("ula", c["mx"], 1, c["bx"], 1, c["N"], frac_bw=c["frac_bw"], epsilon=1.01, delta_rel=1e-3)
    tform = args.workload == "C2NT"
    fac = (O.TimeNullingFactors if tform else O.NullingFactors)(pb, c["interferers"], beams)
    run = O.fbst_nulled_time if tform else O.fbst_nulled
    for _ in range(args.warmup):
        run(pb, y, c["interferers"], factors=fac)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        run(pb, y, c["interferers"], factors=fac)
        times.append(time.perf_counter() - t0)
    value = len(beams) * c["N"] * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload} oracle sample", "M": c["mx"], "N": c["N"], "B": c["bx"],
                       "interferers": c["interferers"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"per step: 1 block x 16 beams of {args.workload} (FP64 numpy oracle of "
                                       f"Eq. ({15 if tform else 14}), "
                                       "per-plan factors and cross Gram matrices excluded)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_offgrid(args) -> None:
    """Reference arm of OG: the FP64 oracle of Sec. VIII-A on one block x 16 off-grid directions per step."""
    import oracle as O
    from synth import configs
    y = configs.config_data("C2", nblk=1)["y"]
    dirs = np.stack([np.random.default_rng(2026).uniform(-0.98, 0.98, 64), np.zeros(64)], axis=1)[:16]
    pb = O.make_problem("ula", 256, 1, 512, 1, 256, frac_bw=0.5, epsilon=1.01, delta_rel=1e-3)
    fac = O.OffGridFactors(pb, dirs)
    for _ in range(args.warmup):
        O.fbst_offgrid(pb, y, dirs, factors=fac)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.fbst_offgrid(pb, y, dirs, factors=fac)
        times.append(time.perf_counter() - t0)
    value = len(dirs) * 256 * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "OG oracle sample", "M": 256, "B_grid": 512, "N": 256, "directions": 16},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "per step: 1 block x 16 off-grid directions of OG (FP64 numpy oracle of "
                                       "Sec. VIII-A, per-plan factors excluded)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_gen(args) -> None:
    """Reference arm of GEN: the oracle's generators, a dense FP64 solve of each beam's Gram matrix
    built by direct sums (Eq. (5)), for 2 beams per step of the same 1024-element ULA plan."""
    import oracle as O
    M, N = 1024, args.gen_n
    pb = O.make_problem("ula", M, 1, M, 1, N, frac_bw=0.5, epsilon=1.01, delta_rel=1e-3)
    L = pb.L
    beams = [0, M // 2 + 1]
    e0 = np.eye(L)[:, 0]
    for _ in range(args.warmup):
        np.linalg.solve(O.gram(pb, beams[0]), e0)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for b in beams:
            np.linalg.solve(O.gram(pb, b), e0)
        times.append(time.perf_counter() - t0)
    value = len(beams) * len(times) / sum(times)
    unit = "systems/s"
    line = {"impl": "reference", "metric": "Toeplitz generator systems solved/s (FP64, rel err vs dense solve)",
            "value": value, "unit": unit, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"GEN oracle sample: ULA M={M} N={N} L={L}, {len(beams)} systems per step"},
            "cpu_baseline": {"value": value, "unit": unit, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"per step: the Gram matrices of {len(beams)} beams by direct sums and their "
                                       "dense FP64 solves (numpy)"},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload in ("C2N", "C2NT"):
        run_reference_null(args)
        return
    if args.workload == "OG":
        run_reference_offgrid(args)
        return
    if args.workload == "GEN":
        run_reference_gen(args)
        return
    if args.workload == "STREAM":
        # The streamed transform is the per-block transform of the same array on overlapping blocks;
        # its oracle sample is the block oracle of ULA1024 (one block x 16 beams per step).
        args.workload = "ULA1024"
    args.nblk = 1                     # the oracle runs one block per step: generate only that one
    w, gen = workload(args)
    y = gen()
    beams = np.linspace(0, w["bx"] * w["by"] - 1, 16).astype(int)
    import oracle as O
    pb = O.make_problem(w["kind"], w["mx"], w["my"], w["bx"], w["by"], w["N"], frac_bw=w["frac_bw"],
                        epsilon=1.01, delta_rel=1e-3, offsets=w.get("offsets"))
    fac = O.Stage2Factors(pb, beams)
    for _ in range(args.warmup):
        O.fbst(pb, y[:1], factors=fac)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.fbst(pb, y[:1], factors=fac)
        times.append(time.perf_counter() - t0)
    per_step = len(beams) * w["N"]
    value = per_step * len(times) / sum(times)
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"{w['name']} oracle sample", "M": w["mx"] * w["my"],
                                            "N": w["N"], "B": w["bx"] * w["by"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"per step: 1 block x {len(beams)} beams of {w['name']} (FP64 numpy oracle, "
                                       "per-plan LU excluded)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="fbst", choices=["fbst", "reference"])
    ap.add_argument("--workload", default="ULA1024")
    ap.add_argument("--nblk", type=int, default=None)
    ap.add_argument("--stage2", default="dense_f16x3")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--contraction", default="fp32", choices=["tf32x3", "fp32"])
    ap.add_argument("--rates", default="1e2,3e2,1e3,3e3,1e4,3e4,1e5")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--streams", type=int, default=3)
    ap.add_argument("--mem-budget", type=int, default=8 << 30)
    ap.add_argument("--batch-work", type=float, default=4e6)
    ap.add_argument("--hop", type=int, default=384)
    ap.add_argument("--gen-n", type=int, default=512)
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "C4":
        run_c4(args)
        return
    if args.workload == "C5":
        run_c5(args)
        return
    if args.workload in ("C2N", "C2NT"):
        run_null(args)
        return
    if args.workload == "OG":
        run_offgrid(args)
        return
    if args.workload == "STREAM":
        run_stream(args)
        return
    if args.workload == "GEN":
        run_gen(args)
        return

    import torch
    import paper_2512_08887_gb300 as fb
    from paper_2512_08887_gb300.build import build
    from paper_2512_08887_gb300.dist import max_over_ranks, rank_blocks, whole_job_rate

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        build()
    if dist is not None:
        dist.barrier()
    build()

    # Weak scaling: every rank takes its own nblk blocks of one continuous stream of world x nblk.
    nblk0, _ = workload(args)
    first, last = rank_blocks(world * nblk0["nblk"], rank, world)
    w, gen = workload(args, first_block=first if w_is_stream(args) else 0)
    y_np = gen()
    nblk = last - first
    M, B, N = w["mx"] * w["my"], w["bx"] * w["by"], w["N"]
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    positions = None
    if w.get("offsets") is not None:
        from synth.planewave import ArrayGeometry, array_positions
        positions = array_positions(ArrayGeometry(w["kind"], w["mx"], w["my"], w["offsets"]))
    plan = fb.Plan(fb.make_geometry(w["kind"], w["mx"], w["my"], w["bx"], w["by"]), N,
                   fb.make_band(w["frac_bw"], stage2=args.stage2, max_blocks=nblk), positions=positions)
    info = plan.info
    y = torch.from_numpy(y_np).to(dev)
    out = torch.empty((nblk, B, N), dtype=torch.complex64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    # Stage-1 launch shapes from the library's autotuner (untimed set-up; cached per shape key).
    shapes = None
    if not args.no_tune:
        from paper_2512_08887_gb300 import autotune
        shapes = autotune.tune(plan, nblk)

    # Accuracy on a sample of beams (rank 0; untimed).
    plan.execute(y, out, nblk)
    torch.cuda.synchronize()
    rel_err = None
    if rank == 0:
        import oracle as O
        beams = np.unique(np.array([0, 1, 77, B // 4, B // 2, 3 * B // 4, B - 2, B - 1]))
        pb = O.make_problem(w["kind"], w["mx"], w["my"], w["bx"], w["by"], N, frac_bw=info.fb_num / info.fb_den,
                            epsilon=info.eps_num / info.eps_den, delta=info.delta, L=info.L, offsets=w.get("offsets"))
        ref = O.fbst(pb, y_np[:2], beams=beams)
        rel_err = O.rel_l2(out[:2].cpu().numpy()[:, beams], ref)

    for _ in range(args.warmup):
        flush.zero_()
        plan.execute(y, out, nblk)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    # The library's stage trace: events on the launching stream around each stage of every timed
    # fbst_execute call, so the kernel times are those of the timed steps themselves.
    plan.trace_stages(args.steps)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        plan.execute(y, out, nblk)
        ends[i].record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop() if sampler else None
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = max_over_ranks(sum(step_ms))
    units = float(nblk) * B * N * world
    value = whole_job_rate(float(nblk) * B * N * args.steps, world, total_ms / 1e3)
    trace = plan.trace_read(args.steps)
    plan.trace_stages(0)
    names = ["czt_time", "czt_space", "stage2"]
    kern_ms = {n: statistics.mean(t[j] for t in trace) for j, n in enumerate(names)}

    # The same kernels through their own C-ABI stage calls (stage 2 of the FP16 split then runs
    # its own pass for the scales of w): reported beside the in-step times.
    kin = min(args.steps, 200)
    yhat = torch.empty((nblk, info.L, M), dtype=torch.complex64, device=dev)
    wbuf = torch.empty((nblk, B, info.L), dtype=torch.complex64, device=dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(kin)]
    for i in range(kin):
        flush.zero_()
        ev[i][0].record(stream)
        plan.czt_time(y, yhat, nblk)
        ev[i][1].record(stream)
        plan.czt_space(yhat, wbuf, nblk)
        ev[i][2].record(stream)
        plan.toeplitz_apply(wbuf, out, nblk)
        ev[i][3].record(stream)
    torch.cuda.synchronize()
    kern_ms_calls = {n: statistics.mean(ev[i][j].elapsed_time(ev[i][j + 1]) for i in range(kin))
                     for j, n in enumerate(names)}

    # End to end through the host-buffer entry point, pinned host memory, copies included.
    e2e_steps = min(args.steps, 200)
    y_host = torch.from_numpy(y_np).pin_memory()
    out_host = torch.empty((nblk, B, N), dtype=torch.complex64).pin_memory()
    plan.execute_host(y_host, out_host, nblk)
    e2e_t = []
    for _ in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.execute_host(y_host, out_host, nblk)
        e2e_t.append(time.perf_counter() - t0)
    e2e_total = max_over_ranks(sum(e2e_t))

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peaks, peak_kind = load_peaks()
    fp32 = measure_fp32_peak(fb, torch.cuda.current_device())
    dom = max(kern_ms, key=kern_ms.get)
    # Inside fbst_execute the spatial chirp-z of a linear grid array supplies the FP16 split's
    # scales of w; the stand-alone stage-2 call makes its own pass for them.
    scales_in_step = w["kind"] == "ula" and w.get("offsets") is None
    roof = roofline(dom, info, nblk, kern_ms[dom], peaks, peak_kind, fp32, scales_in_step)
    s2name = fb.STAGE2_NAMES[info.stage2]
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        import hashlib
        with open(tfile) as f:
            tr = json.load(f)
        rec = tr.get(f"{w['name']}:{dom}:{s2name}" if dom == "stage2" else f"{w['name']}:{dom}")
        if rec and nblk == 64:
            blob = b"".join(open(os.path.join(ROOT, s), "rb").read() for s in rec["sources"])
            if hashlib.sha256(blob).hexdigest()[:16] == rec["sha256_16"]:
                traffic = rec["bytes_per_launch"]  # else: the kernel changed since the capture
    # Whole-path HBM fraction on the compulsory bytes: y in, bhat out, one generator per beam.
    hbm_frac = (path_bytes(info, nblk) / (statistics.mean(step_ms) / 1e3)) / (float(peaks["hbm_gbs"]) * 1e9)

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        beams = np.linspace(0, B - 1, 32).astype(int)
        val, t_plan, reps, _, _ = oracle_sample(w, y_np, beams, 4, budget_s=10.0)
        cpu = {"value": val, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{reps} x (4 blocks x 32 of {B} beams) of {w['name']}, FP64 numpy oracle, per-plan LU "
                         f"of the 32 beams ({t_plan:.1f} s) excluded"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if info.stage2 <= 3 else f"f32 stage 1 + {fb.STAGE2_NAMES[info.stage2][6:]} tensor-core stage 2",
        "data": "synthetic",
        "config": {"workload": f"{w['name']}: {w['kind'].upper()} M={M} B={B} N={N} L={info.L} fb={w['frac_bw']}, "
                               f"{nblk} blocks/step per GPU, complex64",
                   "blocks_of_rank0": [first, last],
                   "stage1_shapes": None if shapes is None else {"time": list(shapes[:2]), "space": list(shapes[2:])},
                   "element_positions": ("grid" if w.get("offsets") is None else
                                         "non-uniform: grid moved by N(0, 0.2^2) half wavelengths (Sec. IX); "
                                         "stage 1b by type-1 NUFFT"),
                   "M": M, "B": B, "N": N, "L": info.L, "nblk_per_gpu": nblk, "stage2": fb.STAGE2_NAMES[info.stage2],
                   "l2": "flushed before every timed step (256 MiB write, untimed)",
                   "parallelism": f"replicas x{world}"},
        "rel_err_vs_oracle": rel_err,
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "hbm_roofline_frac": hbm_frac,
        "hbm_roofline_bytes_per_beam_sample": path_bytes(info, nblk) / (nblk * B * N),
        "path_roofline": path_roofline(info, nblk, statistics.mean(step_ms), peaks, fp32),
        "roofline": dict(roof, kernel=dom, traffic=traffic),
        "kernels_ms": kern_ms,
        "kernels_timing": "device time of each stage inside the timed fbst_execute steps (the library's stage "
                          "trace: CUDA events on the launching stream between the stages)",
        "kernels_roofline": {k: roofline(k, info, nblk, v, peaks, peak_kind, fp32, scales_in_step)
                             for k, v in kern_ms.items()},
        "kernels_ms_separate_calls": kern_ms_calls,
        "fp32_peak": fp32,
        "e2e": {"value": units * e2e_steps / e2e_total, "unit": UNIT,
                "h2d_bytes_per_step": int(8 * nblk * M * N), "d2h_bytes_per_step": int(8 * nblk * B * N)},
        "gpu_launches": plan.launch_count(nblk) * args.steps,
        "clocks": clocks,
        "wall_s_timed_region": wall,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
