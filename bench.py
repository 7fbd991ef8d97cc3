"""Benchmark of the rank-structured Coulomb convolution hot path on GB300.

One step = one pass of the hot path over the density600_n8192 workload (a
molecule-like density of 600 Gaussians on an 8192^3 grid of [-20,20]^3, Newton
kernel with R_N = 61 terms): grid sampling of the factors, the 3 x 36600
batched 1D convolutions giving the Hartree potential factors, the convolution
matrices and the Hartree energy E_H.  The kernel tables (nodes, weights, cell
integrals, spectra) are built once before timing.

Prints one JSON line (see the metric/config keys).  `--impl reference` times
the float64 CPU oracle on a bounded sample of the same workload instead.
Under torchrun every rank runs its own density (weak scaling, no collective
on the data path); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

WORKLOAD = "density600_n8192"
# kernels timed by the library's events in the density step
CHEB = ("cheb_moments_kernel", "cheb_coef_kernel", "cheb_eval_kernel")
TIMED = ("spectra_kernel", "conv_kernel", "band_conv_kernel", *CHEB, "slice_rows_kernel", "gemm3_tc_kernel",
         "cheb_gram_kernel", "lag_slice32_kernel", "lag_gram_kernel")
METRIC = "1D factor convolutions/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# GB300 unit counts for ALU roofs: 152 SMs, 128 FP32 lanes per SM (FMA = 2 flop)
SMS = 152
FP32_LANES = 128
# nominal GB300 float64 CUDA-core rate (GFLOP/s): a context figure, not measured here
FP64_PEAK_GFLOPS = 1250.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "split", "fp64", "fp64tc"])
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="steps of the float64 and split forms timed for comparison (0: skip)")
    ap.add_argument("--seed", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rf", type=int, default=None,
                    help="override the rank R_f (profiling a smaller case of the same kernels)")
    ap.add_argument("--cpu-sample", type=float, default=None, help=argparse.SUPPRESS)
    ap.add_argument("--conv-paths", default="all", choices=["all", "band", "fft"],
                    help="convolution paths: all (banded, Chebyshev and FFT terms), band (banded and FFT) "
                         "or fft (every term through the FFT), for comparison")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "basis80_n4096", "density200_n4096", "lattice32_n16384",
                             "lattice_energy256_n16384", "nuclear80_n4096", "tei80_n4096"],
                    help="the default is the headline workload; the others time their own rows")
    return ap.parse_args()


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws, device=None):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def recorded_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu record, or None
    when there is none or the kernel's source changed since it was taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(kernel)
        if not rec:
            return None
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest()[:16] != rec["sha"]:
                return None
        return rec["dram_read_bytes"] + rec["dram_write_bytes"]
    except (OSError, ValueError, KeyError):
        return None


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_conv_sample(cfg, seed, budget_s):
    """The oracle, as it stands, on a bounded sample of the workload: direct
    O(n^2) convolutions (Toeplitz products) of 16 factor columns with 4 kernel
    terms, on all three axes, repeated until `budget_s` or 4 repetitions.
    Returns (convolutions, seconds, repetitions)."""
    from oracle import cp as ocp
    from oracle import kernel_vectors as okv
    from oracle import sinc as osinc
    n, b, M = cfg["n"], cfg["b"], cfg["M"]
    g = workloads.mixture_for(WORKLOAD, seed)
    t, a = osinc.conv_nodes(n, b, M)
    k_sub, q_sub = 16, 4
    qs = np.linspace(0, 2 * M, q_sub).round().astype(int)
    P = okv.conv_kernel_vectors(n, b, t[qs], a[qs])
    U = ocp.sample_gaussians(n, b, g["a"][:k_sub], g["X"][:k_sub])
    done, reps = 0, 0
    t0 = time.perf_counter()
    while True:
        ocp.convolve_factors(U, P)
        done += 3 * k_sub * q_sub
        reps += 1
        if time.perf_counter() - t0 > budget_s or reps >= 4:
            break
    return done, time.perf_counter() - t0, reps


def _cpu_sample_child(threads, seed, budget_s):
    """Run the oracle sample in a fresh interpreter whose BLAS uses `threads`
    threads (the thread count of a BLAS pool is fixed when it starts)."""
    env = dict(os.environ)
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[var] = str(threads)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", str(budget_s), "--seed", str(seed)],
                       env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return None
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(cfg, seed, budget_s=10.0):
    """The oracle timed on the host cores twice: one thread, and one BLAS
    thread per core (the Toeplitz products are the only parallel part)."""
    cores = os.cpu_count()
    runs = {}
    for label, threads in (("single_thread", 1), ("all_cores", cores)):
        rec = _cpu_sample_child(threads, seed, budget_s)
        if rec:
            runs[label] = {"value": rec["done"] / rec["seconds"], "threads": threads,
                           "convolutions": rec["done"], "seconds": rec["seconds"]}
    head = runs.get("all_cores") or runs.get("single_thread")
    if head is None:
        return None
    n = cfg["n"]
    return {"value": head["value"], "unit": "convolutions/s", "cores": head["threads"], "kind": "oracle",
            "sample": f"(16 Gaussians x 4 kernel terms x 3 axes) direct length-{n} convolutions of {WORKLOAD}, "
                      f"repeated up to 4 times or {budget_s:.0f} s, in a fresh process per thread count",
            **runs}


def run_reference(args, ws, rank):
    cfg = workloads.CONFIGS[WORKLOAD]
    if rank != 0:
        return
    from oracle import cp as ocp
    from oracle import kernel_vectors as okv
    from oracle import sinc as osinc
    n, b, M = cfg["n"], cfg["b"], cfg["M"]
    g = workloads.mixture_for(WORKLOAD, args.seed)
    t, a = osinc.conv_nodes(n, b, M)
    # the same sample as the CPU baseline of the default run: 16 Gaussians x
    # 4 kernel terms x 3 axes per step
    qs = np.linspace(0, 2 * M, 4).round().astype(int)
    P = okv.conv_kernel_vectors(n, b, t[qs], a[qs])
    U = ocp.sample_gaussians(n, b, g["a"][:16], g["X"][:16])
    per_step = 3 * 16 * len(qs)
    for _ in range(args.warmup):
        ocp.convolve_factors(U, P)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ocp.convolve_factors(U, P)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "convolutions/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if not args.rf else f"{WORKLOAD} (R_f={args.rf} profiling case)", "n": n,
                   "R_f": cfg["R_f"], "R_N": 2 * M + 1,
                   "sample_per_step": "16 Gaussians x 4 kernel terms x 3 axes (192 direct convolutions)"},
        "cpu_baseline": {"value": value, "unit": "convolutions/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "192 direct length-8192 convolutions per step"},
        "e2e": {"value": value, "unit": "convolutions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ours(args, ws, rank, local):
    import torch
    import paper_1504_06289_gb300 as cpc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = workloads.CONFIGS[WORKLOAD]
    n, b, M, R_f = cfg["n"], cfg["b"], cfg["M"], cfg["R_f"]
    P = cpc.make_newton_kernel(n, b, M, "conv", device=dev)
    R_N = P.R_N
    if args.conv_paths != "all":
        P.set_conv_paths(*({"band": (20, 24, -1, -1), "fft": (-1, -1, -1, -1)}[args.conv_paths]))
    # the energy paths' lag plan (host only): per W type the lag count and the banded terms it covers
    eh_plan = cpc.make_newton_kernel_eh_plan(
        n, b, M, *({"all": (20, 24, 16, 16), "band": (20, 24, -1, -1), "fft": (-1, -1, -1, -1)}[args.conv_paths]))
    g = workloads.mixture_for(WORKLOAD, args.seed + rank)
    if args.rf:
        R_f = args.rf
        g = {k: v[:R_f] for k, v in g.items()}
    a_h = torch.tensor(g["a"]).pin_memory()
    X_h = torch.tensor(g["X"]).pin_memory()
    c_h = torch.tensor(g["c"]).pin_memory()
    a, X, c = a_h.to(dev), X_h.to(dev), c_h.to(dev)
    stream = torch.cuda.current_stream(dev)
    lib = cpc.load()

    def buffers(prec):
        dt = torch.float32 if prec == "fp32" else torch.float64
        W = torch.empty((3, R_f * R_N, n), dtype=dt, device=dev)
        U = torch.empty((3, R_f, n), dtype=torch.float64, device=dev)
        E = torch.empty((), dtype=torch.float64, device=dev)
        nb = lib.cp_hartree_energy_workspace(P.handle, R_f, cpc._prec(prec))
        ws_g = torch.empty(max(256, nb), dtype=torch.uint8, device=dev)
        return W, U, E, ws_g

    def step(prec, bufs, ev=None):
        """sample -> cp_hartree_energy (spectra, convolutions = V_H factors W, contraction = E_H):
        two ABI calls; per-kernel times come from the library's event timing."""
        W, U, E, ws_g = bufs
        pr = cpc._prec(prec)
        sp = cpc._stream(stream)
        cpc.check(lib.cp_sample_gaussians(n, b, R_f, cpc._ptr(a), cpc._ptr(X), cpc._ptr(U), sp), "sample")
        if ev is not None:
            ev[0].record(stream)
        cpc.check(lib.cp_hartree_energy(P.handle, R_f, cpc._ptr(U), cpc._ptr(c), cpc._ptr(W), None, cpc._ptr(E),
                                        pr, cpc._ptr(ws_g), ws_g.numel(), sp), "cp_hartree_energy")
        if ev is not None:
            ev[1].record(stream)
        return E

    prec = args.precision
    bufs = buffers(prec)
    for _ in range(args.warmup):
        step(prec, bufs)
    torch.cuda.synchronize(dev)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        barrier(ws)
        torch.cuda.synchronize(dev)
        cpc.kernel_timing(True)  # events around the library's main kernels, on their stream
        start.record(stream)
        for k in range(args.steps):
            step(prec, bufs, evs[k])
        stop.record(stream)
        torch.cuda.synchronize(dev)
        cpc.kernel_timing(False)
        barrier(ws)
    ms_total = start.elapsed_time(stop)
    kt = {k: cpc.kernel_timing_read(k) for k in TIMED}
    ms_total = max_over_ranks(ms_total, ws, dev)
    E_fast = bufs[2].item()
    energy_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))  # the cp_hartree_energy call
    spec_ms = kt["spectra_kernel"][0] / max(1, kt["spectra_kernel"][1])
    # the convolutions: FFT terms (conv_kernel), banded terms (band_conv_kernel)
    # and smooth terms (the three Chebyshev kernels)
    conv_ms = (kt["conv_kernel"][0] + kt["band_conv_kernel"][0] + sum(kt[k][0] for k in CHEB)) / args.steps
    gram_ms = energy_ms - spec_ms - conv_ms  # slicing of U, contraction, final sum
    ms_step = ms_total / args.steps
    convs_per_step = 3 * R_f * R_N
    value = ws * convs_per_step * args.steps / (ms_total * 1e-3)

    # end to end through the public API: pinned host inputs -> device, step, E_H -> host
    e2e_steps = max(1, min(args.steps, 5))
    E_host = torch.empty((), dtype=torch.float64).pin_memory()
    barrier(ws)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        a.copy_(a_h, non_blocking=True)
        X.copy_(X_h, non_blocking=True)
        c.copy_(c_h, non_blocking=True)
        E = step(prec, bufs)
        E_host.copy_(E, non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws, dev)
    h2d = a_h.numel() * 8 + X_h.numel() * 8 + c_h.numel() * 8

    # the other precision forms on the same GPU and inputs: plain float64 (the
    # baseline) and split (float64 convolutions, float32-product contractions)
    others = {}
    if args.fp64_steps > 0:
        del bufs
        torch.cuda.empty_cache()
        for form in ("fp64", "split", "fp64tc"):
            if form == prec:
                continue
            bf = buffers(form)
            step(form, bf)
            torch.cuda.synchronize(dev)
            eo = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.fp64_steps)]
            so, to = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            cpc.kernel_timing(True)
            so.record(stream)
            for k in range(args.fp64_steps):
                step(form, bf, eo[k])
            to.record(stream)
            torch.cuda.synchronize(dev)
            cpc.kernel_timing(False)
            mso = so.elapsed_time(to) / args.fp64_steps
            kto = {k: cpc.kernel_timing_read(k) for k in TIMED}
            sp_o = kto["spectra_kernel"][0] / max(1, kto["spectra_kernel"][1])
            cv_o = (kto["conv_kernel"][0] + kto["band_conv_kernel"][0] + sum(kto[k][0] for k in CHEB)) / args.fp64_steps
            en_o = float(np.mean([e[0].elapsed_time(e[1]) for e in eo]))
            others[form] = {"ms_per_step": mso, "value": convs_per_step / (mso * 1e-3),
                            "spectra_ms": sp_o, "conv_ms": cv_o, "contraction_ms": en_o - sp_o - cv_o,
                            "conv_fft_ms": kto["conv_kernel"][0] / args.fp64_steps,
                            "conv_band_ms": kto["band_conv_kernel"][0] / args.fp64_steps,
                            "conv_cheb_ms": sum(kto[k][0] for k in CHEB) / args.fp64_steps,
                            "E_H": bf[2].item()}
            if form == "fp64tc" and kto["gemm3_tc_kernel"][1]:
                # the float64-accurate tensor-core contraction: 15 bf16 slice products
                # per multiply-add of the method's symmetric Gram
                tc_ms64 = kto["gemm3_tc_kernel"][0] / kto["gemm3_tc_kernel"][1]
                _, rk64 = P.conv_paths("fp64tc")  # the smooth terms' Gram matrices come from their moments
                gf = 3 * (R_N - int((rk64 > 0).sum())) * (R_f * (R_f + 1) // 2) * n * 2
                bf16_peak = float(load_peaks()[0].get("bf16_tflops", 1900.0))
                others[form]["gemm3_tc_kernel"] = {
                    "ms": tc_ms64, "achieved_TFLOPs": gf / (tc_ms64 * 1e-3) / 1e12,
                    "frac_of_bf16_peak": gf / (tc_ms64 * 1e-3) / 1e12 / bf16_peak,
                    "slice_products_TFLOPs": 15 * gf / (tc_ms64 * 1e-3) / 1e12}
                others[form]["slice_ms_per_step"] = kto["slice_rows_kernel"][0] / args.fp64_steps
            del bf
            torch.cuda.empty_cache()
        E64 = others.get("fp64", {}).get("E_H", E_fast if prec == "fp64" else None)
        if E64 is not None:
            for form, o in others.items():
                o["rel_err_E_H_vs_fp64_gpu"] = abs(o["E_H"] / E64 - 1)
        if "fp64" in others:
            for form, o in others.items():
                o["speedup_vs_fp64_gpu"] = others["fp64"]["ms_per_step"] / o["ms_per_step"]
    fp64 = others.get("fp64")

    if rank != 0:
        return
    peaks, peak_kind = load_peaks()
    hbm_peak = float(peaks["hbm_gbs"])
    clk = clocks.summary()
    elem = 4 if prec == "fp32" else 8
    sm_mhz = clk["sm_mhz"] or float(peaks.get("sm_max_mhz", 2070.0))
    alu32_peak_tf = SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12

    def per_launch(name, fallback_ms):
        tot, cnt = kt.get(name, (0.0, 0))
        return (tot / cnt, cnt) if cnt else (fallback_ms, 0)

    # convolution, the method's work: per convolution an n-point complex inverse
    # FFT (5 n log2 n flop) and the spectral product (6 n flop); bytes: the V_H
    # factors written once plus the operand spectra and kernel pairs read once.
    # conv_kernel takes the n_fft FFT terms; the banded terms are direct sums
    # (band_conv_kernel) and the smooth terms Chebyshev sums (cheb_conv_kernels):
    # for both, W written once and each factor column read once.
    hw, rk = P.conv_paths(prec)
    n_band = int((hw >= 0).sum())
    n_smooth = int((rk > 0).sum())
    n_fft = R_N - n_band - n_smooth
    conv_k_ms, _ = per_launch("conv_kernel", conv_ms)
    conv_flops = 3 * R_f * n_fft * (5 * n * math.log2(n) + 6 * n)
    # (operands: 16 bytes per bin of each factor column, float4 (X1, X2) or double2;
    # kernel terms: 8 bytes per bin, float2 pairs or float64)
    conv_bytes = 3 * R_f * n_fft * n * elem + 3 * R_f * n * 16 + n_fft * n * 8
    conv_tf = conv_flops / (conv_k_ms * 1e-3) / 1e12
    conv_gbs = conv_bytes / (conv_k_ms * 1e-3) / 1e9
    kernels = {
        "conv_kernel": {
            "ms": conv_k_ms, "bound": "alu", "achieved": conv_tf, "unit": "TFLOP/s",
            "peak": alu32_peak_tf if prec == "fp32" else FP64_PEAK_GFLOPS / 1e3,
            "frac": conv_tf / (alu32_peak_tf if prec == "fp32" else FP64_PEAK_GFLOPS / 1e3),
            "algorithmic_flops": conv_flops, "terms": n_fft,
            "peak_note": ("float32 CUDA-core peak: 152 SMs x 128 lanes x 2 flop x median SM clock"
                          if prec == "fp32" else "nominal GB300 float64 rate"),
            "hbm": {"algorithmic_bytes": conv_bytes, "achieved_GBps": conv_gbs, "peak_GBps": hbm_peak,
                    "frac": conv_gbs / hbm_peak},
        },
    }
    if n_band:
        bd_ms, _ = per_launch("band_conv_kernel", 0.0)
        # bytes: W of the banded terms written once, each factor column read once
        bd_bytes = 3 * R_f * n_band * n * elem + 3 * R_f * n * 8
        bd_taps = 3 * R_f * n * int(np.sum(2 * hw[hw >= 0] + 1))
        kernels["band_conv_kernel"] = {
            "ms": bd_ms, "bound": "hbm", "achieved": bd_bytes / (bd_ms * 1e-3) / 1e9, "unit": "GB/s",
            "peak": hbm_peak, "frac": bd_bytes / (bd_ms * 1e-3) / 1e9 / hbm_peak, "algorithmic_bytes": bd_bytes,
            "terms": n_band, "half_widths": [int(x) for x in hw[hw >= 0]],
            "taps_multiply_adds": bd_taps,
            "note": "direct sums over the band of the narrow kernel terms; the energy path's bf16 slices "
                    "(6 B per output for float32 W, 10 B for float64) are written too and not counted"}
    if n_smooth:
        ch_parts = {k: per_launch(k, 0.0)[0] for k in CHEB}
        ch_ms = sum(ch_parts.values())
        # bytes: W of the smooth terms written once, each factor column read once (moments)
        ch_bytes = 3 * R_f * n_smooth * n * elem + 3 * R_f * n * 8
        kernels["cheb_conv_kernels"] = {
            "ms": ch_ms, "bound": "hbm", "achieved": ch_bytes / (ch_ms * 1e-3) / 1e9, "unit": "GB/s",
            "peak": hbm_peak, "frac": ch_bytes / (ch_ms * 1e-3) / 1e9 / hbm_peak, "algorithmic_bytes": ch_bytes,
            "terms": n_smooth, "ranks": [int(x) for x in rk[rk > 0]], "parts_ms": ch_parts,
            "note": "separable Chebyshev form of the smooth kernel terms (moments, coefficients, evaluation)"}
    # contraction, the method's work: the unique entries of the symmetric convolution
    # matrices (Sec. 3.2), 3 axes x R_N terms x R_f (R_f + 1) / 2 entries x n cells, 2 flop
    # per multiply-add; the fused product over axes and weighted sum are not counted.
    # The tensor-core forms take the smooth terms' matrices from their Chebyshev moments
    # (K-term sums, cheb_gram_kernel) and contract only the banded and FFT terms over
    # the n cells (gemm3_tc_kernel).
    gram_flops = 3 * R_N * (R_f * (R_f + 1) // 2) * n * 2
    cg_ms = 0.0
    if prec in ("fp32", "fp64tc", "split"):
        n_dense = R_N - n_smooth
        if prec in ("fp32", "fp64tc"):
            # lag rows replace the covered banded terms in the cell contraction
            n_lag, n_cov = (int(x) for x in eh_plan[0 if prec == "fp32" else 1][:2])
            n_dense += n_lag - n_cov
            if n_lag:
                ls_ms, _ = per_launch("lag_slice32_kernel", 0.0)
                lg_ms, _ = per_launch("lag_gram_kernel", 0.0)
                # U read, lag-row slices written (3 bf16 digits per cell, 5 in the float64 form)
                lag_bytes = 3 * R_f * n * 8 + 3 * R_f * n_lag * n * (6 if prec == "fp32" else 10)
                kernels["lag_kernels"] = {
                    "ms": ls_ms + lg_ms, "bound": "hbm", "achieved": lag_bytes / ((ls_ms + lg_ms) * 1e-3) / 1e9,
                    "unit": "GB/s", "peak": hbm_peak,
                    "frac": lag_bytes / ((ls_ms + lg_ms) * 1e-3) / 1e9 / hbm_peak, "algorithmic_bytes": lag_bytes,
                    "parts_ms": {"lag_slice32_kernel": ls_ms, "lag_gram_kernel": lg_ms},
                    "lags": n_lag, "terms": n_cov,
                    "note": "the covered banded terms' Gram matrices as sums of the lag Gram matrices "
                            "(lag rows sliced for the cell contraction, then G_q = sum_m p_q[m] S_m)"}
        gram_flops = 3 * n_dense * (R_f * (R_f + 1) // 2) * n * 2
        if n_smooth:
            cg_ms, _ = per_launch("cheb_gram_kernel", 0.0)
            cg_flops = 3 * (R_f * (R_f + 1) // 2) * int(np.sum(rk[rk > 0])) * 2
            kernels["cheb_gram_kernel"] = {
                "ms": cg_ms, "bound": "alu", "achieved": cg_flops / (cg_ms * 1e-3) / 1e12, "unit": "TFLOP/s",
                "peak": alu32_peak_tf, "frac": cg_flops / (cg_ms * 1e-3) / 1e12 / alu32_peak_tf,
                "algorithmic_flops": cg_flops, "terms": n_smooth,
                "note": "convolution matrices of the smooth terms from their Chebyshev moments, "
                        "G_q = M^T (C_q M), K-term sums in double-float arithmetic (about 16 float32 "
                        "operations per multiply-add, not counted)"}
    if prec in ("fp32", "fp64tc"):
        n_slice_products = 6 if prec == "fp32" else 15
        tc_ms, _ = per_launch("gemm3_tc_kernel", gram_ms)
        bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
        tc_tf = gram_flops / (tc_ms * 1e-3) / 1e12
        kernels["gemm3_tc_kernel"] = {
            "ms": tc_ms, "bound": "tensor", "achieved": tc_tf, "peak": bf16_peak, "unit": "TFLOP/s",
            "frac": tc_tf / bf16_peak, "algorithmic_flops": gram_flops, "terms": n_dense,
            "peak_note": "bf16 dense burst (cuBLAS), " + peak_kind,
            # the implementation's work, kept apart from the method's: every multiply-add
            # is 6 (float32 form) or 15 (float64 form) bf16 slice products (exact slicing)
            "slice_products": {"flops": n_slice_products * gram_flops, "TFLOP/s": n_slice_products * tc_tf,
                               "frac_of_peak": n_slice_products * tc_tf / bf16_peak},
        }
        # slicing (read the float64 rows, write the bf16 slices): bookkeeping of the
        # tensor-core form; U only in the float32 form (the convolution slices W)
        sl_tot, sl_cnt = kt.get("slice_rows_kernel", (0.0, 0))
        sl_ms = sl_tot / max(1, sl_cnt)
        sl_bytes = 3 * R_f * n * (8 + (6 if prec == "fp32" else 10))  # U only (the convolution slices W)
        kernels["slice_rows_kernel"] = {"ms": sl_ms, "bound": "hbm", "achieved": sl_bytes / (sl_ms * 1e-3) / 1e9,
                                        "peak": hbm_peak, "unit": "GB/s",
                                        "frac": sl_bytes / (sl_ms * 1e-3) / 1e9 / hbm_peak,
                                        "algorithmic_bytes": sl_bytes}
    else:
        # (split: the cell contraction of the banded and FFT terms is the rest of the
        # contraction phase once the smooth terms' Gram kernel is taken out)
        g_ms = gram_ms - cg_ms
        gram_tf = gram_flops / (g_ms * 1e-3) / 1e12
        peak = alu32_peak_tf if prec == "split" else FP64_PEAK_GFLOPS / 1e3
        kernels[{"split": "gemm3_kernel", "fp64": "tri_gram_kernel"}[prec]] = {
            "ms": g_ms, "bound": "alu", "achieved": gram_tf, "unit": "TFLOP/s", "terms": R_N - (
                n_smooth if prec == "split" else 0),
            "peak": peak, "frac": gram_tf / peak, "algorithmic_flops": gram_flops,
            "peak_note": ("float32 CUDA-core peak: 152 SMs x 128 lanes x 2 flop x median SM clock"
                          if prec == "split" else "nominal GB300 float64 rate")}
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    d = kernels[dom]
    if args.rf is None:
        for kname, kd in kernels.items():
            kd["traffic"] = recorded_traffic(kname)
    roofline = {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"],
                "unit": d["unit"], "frac": d["frac"], "traffic": d.get("traffic"),
                "peak_source": peak_kind if d["bound"] in ("hbm", "tensor") else "derived (unit counts x clock)"}
    out = {
        "metric": METRIC, "value": value, "unit": "convolutions/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if not args.rf else f"{WORKLOAD} (R_f={R_f} profiling case)", "n": n, "box": [-b, b], "R_f": R_f, "R_N": R_N,
                   "convolutions_per_step": convs_per_step, "precision_form": prec,
                   "terms_fft": n_fft, "terms_banded": n_band, "terms_chebyshev": n_smooth,
                   "l2": "each step writes the V_H factors (%.2f GB), far larger than L2" % (
                       3 * R_f * R_N * n * elem / 1e9)},
        "E_H": E_fast, "E_H_evals_per_s": ws * args.steps / (ms_total * 1e-3),
        "phases_ms": {"spectra": spec_ms, "convolve": conv_ms, "contraction": gram_ms},
        "kernels": kernels, "roofline": roofline,
        "other_forms": others,
        "rel_err_E_H_vs_fp64_gpu": (abs(E_fast / fp64["E_H"] - 1) if fp64 else 0.0),
        "speedup_vs_fp64_gpu": (fp64["ms_per_step"] / ms_step) if fp64 else None,
        "e2e": {"value": ws * convs_per_step * e2e_steps / e2e_s, "unit": "convolutions/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8},
        # sample, spectra, FFT conv (+ W slices), [slice U (fp64tc: exponents, digits),] contraction,
        # [fp64tc: E_H from G,] final sum; banded conv; Chebyshev moments, coefficients,
        # evaluation [and the smooth terms' Gram matrices]
        "gpu_launches": ({"fp32": 6, "fp64tc": 8}.get(prec, 5) + (1 if n_band else 0)
                         + (2 if prec in ("fp32", "fp64tc") and eh_plan[0 if prec == "fp32" else 1][0] else 0)
                         + ((4 if prec in ("fp32", "fp64tc", "split") else 3) if n_smooth else 0)
                         - (0 if n_fft else 1)) * args.steps,
        "clocks": clk,
    }
    if ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(cfg, args.seed)
    print(json.dumps(out), flush=True)


def _timed(stream, fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def _line(args, ws, metric, value, unit, ms, dtype, config, **extra):
    out = {"metric": metric, "value": value, "unit": unit, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
           "data": "synthetic", "config": config}
    out.update(extra)
    print(json.dumps(out), flush=True)


def run_coulomb(args, ws, rank, local):
    """a8: all 3240 Coulomb-matrix entries of basis80_n4096 per step: density and
    item factors by Hadamard products, V_H factors of rho, persistent contraction
    (schedule from the autotuner), captured in one CUDA graph and replayed."""
    import torch
    import paper_1504_06289_gb300 as cpc
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    name = "basis80_n4096"
    cfg = workloads.CONFIGS[name]
    n, b, M = cfg["n"], cfg["b"], cfg["M"]
    basis = workloads.basis_for(name, 3 + rank)
    nb = cfg["n_basis"]
    P = cpc.make_newton_kernel(n, b, M, device=dev)
    first = basis["fn_first"]
    centre = np.repeat(basis["fn_centre"], np.diff(first), axis=0)
    t = lambda x, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device=dev)
    alpha, cen, d = t(basis["prim_alpha"]), t(centre), t(basis["prim_d"])
    pa, pb, sc = workloads.basis_density_pairs(basis)  # index bookkeeping only
    items, ia, ib, off = workloads.basis_item_pairs(basis)
    pa_t, pb_t, sc_t = t(pa, torch.int32), t(pb, torch.int32), t(sc)
    ia_t, ib_t, off_t = t(ia, torch.int32), t(ib, torch.int32), t(off, torch.int32)
    n_factors, R_rho = len(ia), len(pa)
    stream = torch.cuda.Stream(dev)  # graphs are captured on a non-default stream
    torch.cuda.set_stream(stream)
    res = {}
    for prec in (["fp32", "split"] if args.precision != "fp64" else ["fp64"]):
        F = cpc.cp_sample_gaussians(n, b, alpha, cen)
        U_rho, c_rho = cpc.cp_hadamard_pairs(F, pa_t, pb_t, d, sc_t)
        U_it, c_it = cpc.cp_hadamard_pairs(F, ia_t, ib_t, d)
        J, W_rho = cpc.coulomb_matrix(P, off_t, U_it, c_it, U_rho, c_rho, prec, tiles_per_cta="tune")
        key = cpc._tune_key(P, n_factors, R_rho, prec, dev)
        tiles = cpc._tune_lookup(key)["tiles_per_cta"]
        wsb = torch.empty(cpc.load().coulomb_matrix_workspace(P.handle, len(items), n_factors, R_rho, cpc._prec(prec)),
                          dtype=torch.uint8, device=dev)
        def body():
            cpc.load().cp_sample_gaussians(n, b, len(basis["prim_alpha"]), cpc._ptr(alpha), cpc._ptr(cen),
                                           cpc._ptr(F), cpc._stream(stream))
            cpc.load().cp_hadamard_pairs(n, F.shape[1], R_rho, cpc._ptr(pa_t), cpc._ptr(pb_t), cpc._ptr(F),
                                         cpc._ptr(d), cpc._ptr(sc_t), cpc._ptr(U_rho), cpc._ptr(c_rho),
                                         cpc._stream(stream))
            cpc.load().cp_hadamard_pairs(n, F.shape[1], n_factors, cpc._ptr(ia_t), cpc._ptr(ib_t), cpc._ptr(F),
                                         cpc._ptr(d), None, cpc._ptr(U_it), cpc._ptr(c_it), cpc._stream(stream))
            cpc.check(cpc.load().coulomb_matrix(P.handle, len(items), cpc._ptr(off_t), n_factors, cpc._ptr(U_it),
                                                cpc._ptr(c_it), R_rho, cpc._ptr(U_rho), cpc._ptr(c_rho),
                                                cpc._ptr(W_rho), cpc._ptr(J), cpc._prec(prec), int(tiles),
                                                cpc._ptr(wsb), wsb.numel(), cpc._stream(stream)), "coulomb_matrix")
        body()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            body()
        ms = _timed(stream, g.replay, args.steps, max(1, args.warmup))
        # per-kernel device times: one more (uncaptured) step with the library's event timing on
        torch.cuda.synchronize()
        cpc.kernel_timing(True)
        body()
        torch.cuda.synchronize()
        cpc.kernel_timing(False)
        kms = {k: cpc.kernel_timing_read(k)[0] for k in ("spectra_kernel", "conv_kernel", "slice_rows_kernel",
                                                           "gemm3_tc_kernel")}
        res[prec] = {"ms_per_step": ms, "tiles_per_cta": tiles, "kernel_ms": kms, "J_diag_sum_w": float(np.dot(
            basis["w"], J.cpu().numpy()[[items.index((m, m)) for m in range(nb)]]))}
        del U_it, W_rho, wsb
        torch.cuda.empty_cache()
    if args.precision != "fp64" and args.fp64_steps > 0:
        # the plain float64 form on the same GPU and inputs (CUDA-core contraction,
        # default schedule, not tuned: one step takes tens of seconds), the
        # baseline of the speedup and of the energy error
        F = cpc.cp_sample_gaussians(n, b, alpha, cen)
        U_rho, c_rho = cpc.cp_hadamard_pairs(F, pa_t, pb_t, d, sc_t)
        U_it, c_it = cpc.cp_hadamard_pairs(F, ia_t, ib_t, d)
        J64 = None
        def fp64_step():
            nonlocal J64
            J64, _ = cpc.coulomb_matrix(P, off_t, U_it, c_it, U_rho, c_rho, "fp64", tiles_per_cta=0)
        ms64 = _timed(stream, fp64_step, 1, 0)
        res["fp64"] = {"ms_per_step": ms64, "steps": 1, "J_diag_sum_w": float(np.dot(
            basis["w"], J64.cpu().numpy()[[items.index((m, m)) for m in range(nb)]]))}
        del U_it, J64
        torch.cuda.empty_cache()
    if rank != 0:
        return
    head = "fp32" if "fp32" in res else "fp64"
    ms = res[head]["ms_per_step"]
    flops = 2.0 * 3 * n_factors * R_rho * P.R_N * n  # contraction multiply-adds x 2
    peaks, peak_kind = load_peaks()
    if "split" in res:
        res["split"]["rel_diff_E_vs_fp32"] = abs(res["split"]["J_diag_sum_w"] / res["fp32"]["J_diag_sum_w"] - 1)
    extra = {}
    if "fp64" in res and head != "fp64":
        # E_H = sum_mu w_mu J_mu,mu of each reduced-precision form against the float64 form
        for form in ("fp32", "split"):
            if form in res:
                res[form]["rel_err_E_H_vs_fp64_gpu"] = abs(res[form]["J_diag_sum_w"] / res["fp64"]["J_diag_sum_w"] - 1)
        extra = {"speedup_vs_fp64_gpu": res["fp64"]["ms_per_step"] / res[head]["ms_per_step"],
                 "rel_err_E_H_vs_fp64_gpu": res[head]["rel_err_E_H_vs_fp64_gpu"]}
    tc_ms = res[head]["kernel_ms"].get("gemm3_tc_kernel", 0.0)
    if head == "fp32" and tc_ms > 0:
        # the method's work (2 flop per multiply-add of the 3 axes' scalar products
        # of item factors with the V_H factors of rho) against the bf16 peak: the
        # banded and FFT terms over the n cells, the smooth terms over their K
        # Chebyshev moments (the second rows contraction, padded to 128 "cells":
        # the padding and the 6 bf16 slice products per multiply-add are the
        # implementation's, reported apart)
        hw, rk = P.conv_paths("fp32")
        n_band, n_smooth = int((hw >= 0).sum()), int((rk > 0).sum())
        n_dense = P.R_N - n_smooth
        flops = 2.0 * 3 * n_factors * R_rho * (n_dense * n + int(np.sum(rk[rk > 0])))
        impl = 2.0 * 3 * n_factors * R_rho * (n_dense * n + n_smooth * 128) * 6
        achieved = flops / (tc_ms * 1e-3) / 1e12
        peak = float(peaks.get("bf16_tflops", 1900.0))
        roof = {"kernel": "gemm3_tc_kernel", "bound": "tensor", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None, "peak_source": peak_kind,
                "kernel_ms": tc_ms, "terms_over_cells": n_dense, "terms_from_moments": n_smooth,
                "slice_products": {"flops": impl, "TFLOP/s": impl / (tc_ms * 1e-3) / 1e12,
                                   "frac_of_peak": impl / (tc_ms * 1e-3) / 1e12 / peak},
                "note": "method flops 2*3*factors*R_rho*(n_dense*n + sum_smooth K_q) over both launches / event time"}
        # sample, 2 Hadamard; forward transforms, FFT conv, [banded], [Chebyshev x3]; dense columns:
        # coefficients, slice items, slice W, contraction; [smooth: moments, moment rows, coefficient
        # rows, coefficients, slice, slice, contraction]; item sums
        launches = 3 + 2 + (1 if n_band else 0) + (3 if n_smooth else 0) + 4 + (7 if n_smooth else 0) + 1
    else:
        clk = 2070.0
        peak = SMS * FP32_LANES * 2 * clk * 1e6 / 1e12
        achieved = flops / (ms * 1e-3) / 1e12
        roof = {"kernel": "gemm3_kernel(ROWS)+conv", "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "note": "whole step; contraction flops 2*3*factors*R_rho*R_N*n"}
        launches = None
    _line(args, ws, "Coulomb-matrix entries/s", ws * len(items) / (ms * 1e-3), "entries/s", ms,
          "f32" if head == "fp32" else "f64",
          {"workload": name, "n": n, "items": len(items), "item_factors": n_factors, "R_rho": R_rho, "R_N": P.R_N,
           "graph": "sample + 2 Hadamard + coulomb_matrix captured in one CUDA graph"},
          forms=res, roofline=roof, gpu_launches=launches * args.steps if launches else None, **extra)


def run_adjoint(args, ws, rank, local):
    """a7: forward E_H and its gradients in exponents, centres and coefficients
    through CPHartreeEnergy (sampling, convolutions, contraction with G, adjoint
    GEMM, chain rule) for density200_n4096."""
    import torch
    import paper_1504_06289_gb300 as cpc
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    name = "density200_n4096"
    cfg = workloads.CONFIGS[name]
    n, b, M, R_f = cfg["n"], cfg["b"], cfg["M"], cfg["R_f"]
    g = workloads.mixture_for(name, 5 + rank)
    P = cpc.make_newton_kernel(n, b, M, device=dev)
    stream = torch.cuda.current_stream(dev)
    res = {}
    for prec in ("fp32", "split", "fp64"):
        a = torch.tensor(g["a"], device=dev).requires_grad_()
        X = torch.tensor(g["X"], device=dev).requires_grad_()
        c = torch.tensor(g["c"], device=dev).requires_grad_()
        def body():
            E = cpc.CPHartreeEnergy.apply(a, X, c, P, prec)
            E.backward()
            return E
        ms = _timed(stream, body, args.steps, args.warmup)
        torch.cuda.synchronize()
        cpc.kernel_timing(True)
        E_last = body().item()
        torch.cuda.synchronize()
        cpc.kernel_timing(False)
        kms = {k: cpc.kernel_timing_read(k)[0] for k in ("spectra_kernel", "conv_kernel", "slice_rows_kernel",
                                                           "gemm3_tc_kernel", "adjoint_gemm_kernel")}
        res[prec] = {"ms_per_step": ms, "E_H": E_last, "grad_a_norm": float(a.grad.norm()), "kernel_ms": kms}
    for prec in ("fp32", "split"):
        res[prec]["rel_err_E_H_vs_fp64"] = abs(res[prec]["E_H"] / res["fp64"]["E_H"] - 1)
    if rank != 0:
        return
    head = args.precision if args.precision in res else "fp32"
    ms = res[head]["ms_per_step"]
    # dominant kernel of the backward pass: dU^l = B^l W^l, 2 flop per multiply-add,
    # 3 axes x R_f rows x (R_f R_N) x n; float32 CUDA-core peak from unit counts
    adj_ms = res[head]["kernel_ms"].get("adjoint_gemm_kernel", 0.0)
    adj_flops = 2.0 * 3 * R_f * R_f * P.R_N * n
    peak = SMS * FP32_LANES * 2 * 2070.0 * 1e6 / 1e12
    roof = ({"kernel": "adjoint_gemm_kernel", "bound": "alu", "kernel_ms": adj_ms,
             "achieved": adj_flops / (adj_ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
             "frac": adj_flops / (adj_ms * 1e-3) / 1e12 / peak, "traffic": None,
             "peak_note": "FP32 CUDA-core peak: 152 SMs x 128 lanes x 2 flop x 2070 MHz"}
            if head == "fp32" and adj_ms > 0 else None)
    _line(args, ws, "E_H + gradient evaluations/s", ws / (ms * 1e-3), "evaluations/s", ms,
          {"fp32": "f32", "split": "f64/f32", "fp64": "f64"}[head],
          {"workload": name, "n": n, "R_f": R_f, "R_N": P.R_N,
           "parameters": "200 exponents, 600 centre coordinates, 200 coefficients"},
          forms=res, speedup_vs_fp64_gpu=res["fp64"]["ms_per_step"] / ms, roofline=roof)


def run_lattice(args, ws, rank, local):
    """a9/a10: assembled lattice vectors of a 32^3 lattice of unit charges and
    the potential on the 512^3 sub-grid (lattice32_n16384)."""
    import torch
    import paper_1504_06289_gb300 as cpc
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    name = "lattice32_n16384"
    cfg = workloads.CONFIGS[name]
    n, b, M, L, sub_n = cfg["n"], cfg["b"], cfg["M"], cfg["L"], cfg["sub"]
    geo = workloads.lattice_geometry(n, L, sub_n)
    P = cpc.make_newton_kernel(n, b, M, "master", device=dev)
    sub = torch.as_tensor(np.stack([geo["sub_idx"]] * 3), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    res = {}
    for prec in ("fp64", "fp32"):
        ms = _timed(stream, lambda: cpc.lattice_potential_sum(P, [geo["edges"]] * 3, sub, prec), args.steps,
                    args.warmup)
        res[prec] = {"ms_per_step": ms}
    # the float32 sub-grid kernel's own device time (library event timing, one more call)
    torch.cuda.synchronize()
    cpc.kernel_timing(True)
    cpc.lattice_potential_sum(P, [geo["edges"]] * 3, sub, "fp32")
    torch.cuda.synchronize()
    cpc.kernel_timing(False)
    sg_ms, sg_n = cpc.kernel_timing_read("subgrid_tc_kernel")
    if rank != 0:
        return
    points = sub_n ** 3
    head = "fp32" if args.precision == "fp32" else "fp64"
    ms = res[head]["ms_per_step"]
    fma = points * P.R_N
    clk = 2070.0
    out_bytes = points * (4 if head == "fp32" else 8)
    # float64 ALU peak from the measured float64 contraction rate is not a unit count; report HBM and ALU both
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        from oracle import kernel_vectors as okv
        from oracle import lattice as olat
        from oracle import sinc as osinc
        t, w = osinc.master_nodes(n, b, M)
        Pm = okv.master_kernel_vectors(n, b, t, w)
        t0 = time.perf_counter()
        S0 = olat.assembled_vectors(Pm, geo["edges"], n)
        pts = workloads.check_points(sub_n, 20000, seed=1)
        olat.potential_on_points([S0] * 3, 2 * b / n, geo["sub_idx"][pts])
        dt = time.perf_counter() - t0
        cpu = {"value": 20000 / dt, "unit": "points/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "assembled vectors + 20000 sub-grid points"}
    _line(args, ws, "lattice potential points/s", ws * points / (ms * 1e-3), "points/s", ms,
          "f32" if head == "fp32" else "f64",
          {"workload": name, "n": n, "L": L, "sub_grid": sub_n, "R_N": P.R_N}, forms=res,
          roofline=({"kernel": "subgrid_tc_kernel", "bound": "hbm", "kernel_ms": sg_ms,
                     "achieved": out_bytes / (sg_ms * 1e-3) / 1e9, "peak": load_peaks()[0]["hbm_gbs"],
                     "unit": "GB/s", "frac": out_bytes / (sg_ms * 1e-3) / 1e9 / load_peaks()[0]["hbm_gbs"],
                     "traffic": None, "note": "float32 sub-grid values written per launch / event time"}
                    if head == "fp32" and sg_n else
                    {"kernel": "subgrid_kernel", "bound": "hbm", "achieved": out_bytes / (ms * 1e-3) / 1e9,
                     "peak": load_peaks()[0]["hbm_gbs"], "unit": "GB/s",
                     "frac": out_bytes / (ms * 1e-3) / 1e9 / load_peaks()[0]["hbm_gbs"], "traffic": None,
                     "alu_fma_per_s": fma / (ms * 1e-3)}),
          gpu_launches=(2 * args.steps if head == "fp32" else None),
          cpu_baseline=cpu)


def run_nuclear(args, ws, rank, local):
    """f3: the nuclear-attraction matrix (3240 entries) of the 80-function basis:
    master kernel windowed onto 10 nuclei (Sec. 3.3) and contracted with the
    item factors; the item factors are built once (the Coulomb workload's)."""
    import torch
    import paper_1504_06289_gb300 as cpc
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    name = "nuclear80_n4096"
    cfg = workloads.CONFIGS[name]
    n, b, M = cfg["n"], cfg["b"], cfg["M"]
    basis = workloads.basis_for(name, 3 + rank)
    nb = cfg["n_basis"]
    nuc, Z = workloads.nuclei_for(basis, n, b, 5 + rank)
    P = cpc.make_newton_kernel(n, b, M, "master", device=dev)
    first = basis["fn_first"]
    centre = np.repeat(basis["fn_centre"], np.diff(first), axis=0)
    t = lambda x, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device=dev)
    items, ia, ib, off = workloads.basis_item_pairs(basis)
    G = cpc.cp_sample_gaussians(n, b, t(basis["prim_alpha"]), t(centre))
    U_it, c_it = cpc.cp_hadamard_pairs(G, t(ia, torch.int32), t(ib, torch.int32), t(basis["prim_d"]))
    off_t, Z_t = t(off, torch.int32), t(Z)
    n_factors, n_nuc = U_it.shape[1], nuc.shape[1]
    stream = torch.cuda.current_stream(dev)
    res = {}
    for prec, steps in (("fp32", args.steps), ("fp64", max(1, min(args.steps, 3)))):
        V, F = cpc.nuclear_matrix(P, off_t, U_it, c_it, nuc, Z_t, prec)
        wsb = torch.empty(max(256, cpc.load().nuclear_matrix_workspace(P.handle, len(items), n_factors, n_nuc,
                                                                        cpc._prec(prec))), dtype=torch.uint8,
                          device=dev)
        ms = _timed(stream, lambda: cpc.nuclear_matrix(P, off_t, U_it, c_it, nuc, Z_t, prec, F=F, ws=wsb), steps,
                    max(1, min(args.warmup, 3)))
        torch.cuda.synchronize()
        cpc.kernel_timing(True)
        V, _ = cpc.nuclear_matrix(P, off_t, U_it, c_it, nuc, Z_t, prec, F=F, ws=wsb)
        torch.cuda.synchronize()
        cpc.kernel_timing(False)
        res[prec] = {"ms_per_step": ms, "kernel_ms": {k: cpc.kernel_timing_read(k)[0]
                                                      for k in ("slice_rows_kernel", "gemm3_tc_kernel")},
                     "V_trace": float(V.cpu().numpy()[[items.index((m, m)) for m in range(nb)]].sum())}
        del F, wsb
        torch.cuda.empty_cache()
    if rank != 0:
        return
    res["fp32"]["rel_diff_trace_vs_fp64"] = abs(res["fp32"]["V_trace"] / res["fp64"]["V_trace"] - 1)
    ms = res["fp32"]["ms_per_step"]
    flops = 2.0 * 3 * n_factors * n_nuc * P.R_N * n
    peaks, peak_kind = load_peaks()
    tc_ms = res["fp32"]["kernel_ms"]["gemm3_tc_kernel"]
    achieved = flops / (tc_ms * 1e-3) / 1e12 if tc_ms > 0 else None
    peak = float(peaks.get("bf16_tflops", 1900.0))
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        from oracle import kernel_vectors as okv
        from oracle import nuclear as onuc
        from oracle import sinc as osinc
        tq, wq = osinc.master_nodes(n, b, M)
        Pm = okv.master_kernel_vectors(n, b, tq, wq)
        sample = items[:40]
        t0 = time.perf_counter()
        onuc.nuclear_items(n, b, basis, Pm, sample, nuc, Z)
        dt = time.perf_counter() - t0
        cpu = {"value": len(sample) / dt, "unit": "entries/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "the first 40 items (factors, windows and products formed per call)"}
    _line(args, ws, "nuclear-attraction matrix entries/s", ws * len(items) / (ms * 1e-3), "entries/s", ms, "f32",
          {"workload": name, "n": n, "items": len(items), "item_factors": n_factors, "nuclei": n_nuc, "R_N": P.R_N},
          forms=res,
          roofline={"kernel": "gemm3_tc_kernel", "bound": "tensor", "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak if achieved else None, "traffic": None,
                    "peak_source": peak_kind, "kernel_ms": tc_ms,
                    "slice_products": ({"flops": 6 * flops, "TFLOP/s": 6 * achieved, "frac_of_peak": 6 * achieved / peak}
                                       if achieved else None),
                    "note": "method flops 2*3*factors*nuclei*R_N*n per launch / event time"},
          gpu_launches=6 * args.steps, cpu_baseline=cpu)


def run_tei(args, ws, rank, local):
    """f2/f4: two-electron integrals of 80 s primitives (3240 pairs): 1D density
    fitting, convolution matrices, truncated Cholesky of the TEI matrix, and
    J(D) and K(D) for one density matrix per step (Secs. 3.1, 3.2); float64."""
    import torch
    import paper_1504_06289_gb300 as cpc
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    name = "tei80_n4096"
    cfg = workloads.CONFIGS[name]
    n, b, M, nb = cfg["n"], cfg["b"], cfg["M"], cfg["n_prims"]
    g = workloads.gaussian_mixture(nb, cfg["a_lo"], cfg["a_hi"], 11 + rank, centres=cfg["centres"],
                                   cluster_radius=cfg["cluster_radius"])
    P = cpc.make_newton_kernel(n, b, M, device=dev)
    t = lambda x, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device=dev)
    U = cpc.cp_sample_gaussians(n, b, t(g["a"]), t(g["X"]))
    pa0, pb0 = workloads.upper_pairs(nb)
    pa, pb = t(pa0, torch.int32), t(pb0, torch.int32)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((nb, nb))
    D = t(X + X.T)
    w = rng.uniform(0.0, 2.0, nb)
    stream = torch.cuda.current_stream(dev)
    def step():
        L, ranks = cpc.tei_cholesky(P, U, pa, pb, cfg["tol_df"], cfg["tol_b"], 128, cfg["max_rank_b"])
        cpc.tei_exchange(L, ranks, pa, pb, D)
        return cpc.tei_coulomb(L, ranks, pa, pb, D), L, ranks
    ms = _timed(stream, step, args.steps, max(1, min(args.warmup, 3)))
    torch.cuda.synchronize()
    cpc.kernel_timing(True)
    J, L, ranks = step()
    torch.cuda.synchronize()
    cpc.kernel_timing(False)
    phases = {k: cpc.kernel_timing_read(k)[0] for k in ("tei_fit", "tei_conv_matrices", "tei_factor", "conv_kernel")}
    rk = [int(x) for x in ranks.cpu().numpy()]
    # the diagonal-density J against the Coulomb-matrix path (no fitting, no Cholesky)
    d1, idx = t(np.ones(nb)), t(np.arange(nb), torch.int32)
    U_rho, c_rho = cpc.cp_hadamard_pairs(U, idx, idx, d1, t(w))
    U_it, c_it = cpc.cp_hadamard_pairs(U, pa, pb, d1)
    Jc, _ = cpc.coulomb_matrix(P, t(np.arange(len(pa0) + 1), torch.int32), U_it, c_it, U_rho, c_rho, "fp64",
                               tiles_per_cta=0)
    Jd = cpc.tei_coulomb(L, ranks, pa, pb, t(np.diag(w)))
    rel_vs_coulomb = float((Jd - Jc).abs().max() / Jc.abs().max())
    if rank != 0:
        return
    # float64 work of the factor phase: the TEI diagonal (3 R_N sum_l R_l^2 per pair)
    # and per pivot column 3 R_N (R_l^2 + n_pairs R_l) multiply-adds, plus the rank-s updates
    R_N, npair = P.R_N, len(pa0)
    RB = rk[3]
    fl = 2.0 * (R_N * npair * sum(r * r for r in rk[:3]) + RB * R_N * sum(r * r + npair * r for r in rk[:3])
                + npair * RB * RB / 2.0)
    fp64_peak = FP64_PEAK_GFLOPS
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        from oracle import cp as ocp
        from oracle import tei as otei
        U0 = ocp.sample_gaussians(n, b, g["a"], g["X"])
        t0 = time.perf_counter()
        otei.density_fit(otei.side_matrix(U0[0], pa0, pb0), cfg["tol_df"], 128)
        dt = time.perf_counter() - t0
        cpu = {"value": 1.0 / (3 * dt), "unit": "factorisations/s (fitting stage of one axis x 3, lower bound)",
               "cores": os.cpu_count(), "kind": "oracle",
               "sample": "the 1D density fitting of one axis (A = G G^T and its truncated Cholesky), times 3"}
    _line(args, ws, "TEI factorisations + J(D) + K(D)/s", ws / (ms * 1e-3), "factorisations/s", ms, "f64",
          {"workload": name, "n": n, "primitives": nb, "pairs": npair, "R_N": R_N, "tol_df": cfg["tol_df"],
           "tol_b": cfg["tol_b"]},
          ranks={"fit": rk[:3], "tei": RB}, phases_ms=phases, rel_diff_J_vs_coulomb_path=rel_vs_coulomb,
          roofline={"kernel": "tei_factor (pick, pivot-column and update kernels)", "bound": "alu",
                    "kernel_ms": phases["tei_factor"],
                    "achieved": fl / (phases["tei_factor"] * 1e-3) / 1e9 if phases["tei_factor"] else None,
                    "peak": fp64_peak, "unit": "GFLOP/s",
                    "frac": fl / (phases["tei_factor"] * 1e-3) / 1e9 / fp64_peak if phases["tei_factor"] else None,
                    "traffic": None,
                    "note": "float64 multiply-adds x 2 of the TEI diagonal, pivot columns and updates / phase time; "
                            "peak: nominal GB300 float64 rate"},
          gpu_launches=None, cpu_baseline=cpu)


def run_lattice_energy(args, ws, rank, local):
    """f1: interaction energy of a 256^3 hydrogen lattice (charges 2 bohr apart,
    64 cells) by the traced tensor lattice sum with the singular-point
    correction (Sec. 5.3, Eq. EnergyLattice); float64, one E_L per step."""
    import torch
    import paper_1504_06289_gb300 as cpc
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    name = "lattice_energy256_n16384"
    cfg = workloads.CONFIGS[name]
    n, b, M, L, cells = cfg["n"], cfg["b"], cfg["M"], cfg["L"], cfg["cells"]
    h = 2 * b / n
    edges = [workloads.lattice_energy_edges(n, L, cells)] * 3
    P = cpc.make_newton_kernel(n, b, M, "master", device=dev)
    stream = torch.cuda.current_stream(dev)
    ms = _timed(stream, lambda: cpc.lattice_interaction_energy(P, edges), args.steps, args.warmup)
    torch.cuda.synchronize()
    cpc.kernel_timing(True)
    E = cpc.lattice_interaction_energy(P, edges)
    torch.cuda.synchronize()
    cpc.kernel_timing(False)
    k_ms, k_n = cpc.kernel_timing_read("lattice_energy_kernel")
    p_ms, _ = cpc.kernel_timing_read("lattice_pairs_kernel")
    # end to end: host edge lists in, E_L read back, every step
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_val = cpc.lattice_interaction_energy(P, edges).item()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    if rank != 0:
        return
    # per axis, q and distinct difference d: p~[d-1] + p~[d] and one multiply-add
    n_diff = sum(len(np.unique(np.subtract.outer(e.astype(np.int64), e))) for e in edges)
    flops = 3 * P.R_N * n_diff
    fp64_peak = FP64_PEAK_GFLOPS
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        from oracle import kernel_vectors as okv
        from oracle import lattice as olat
        from oracle import sinc as osinc
        t, w = osinc.master_nodes(n, b, M)
        Pm = okv.master_kernel_vectors(n, b, t, w)
        t0 = time.perf_counter()
        E0 = olat.interaction_energy_tensor(Pm, edges, n, h)
        dt = time.perf_counter() - t0
        cpu = {"value": 1.0 / dt, "unit": "evaluations/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "one E_L of the same lattice (traced tensor sum, master vectors given)",
               "rel_diff": abs(E.item() / E0 - 1),
               "E_L_direct": olat.interaction_energy_direct(edges, h)}
    _line(args, ws, "lattice interaction energy evaluations/s", ws / (ms * 1e-3), "evaluations/s", ms, "f64",
          {"workload": name, "n": n, "L": L, "cells_per_spacing": cells, "R_N": P.R_N},
          E_L=E.item(),
          kernel_ms={"lattice_pairs_kernel": p_ms, "lattice_energy_kernel": k_ms},
          e2e={"value": 1e3 / e2e_ms, "unit": "evaluations/s", "h2d_bytes_per_step": 4 * 3 * L,
               "d2h_bytes_per_step": 8},
          roofline={"kernel": "lattice_energy_kernel", "bound": "alu", "kernel_ms": k_ms,
                    "achieved": flops / (k_ms * 1e-3) / 1e9 if k_n else None, "peak": fp64_peak,
                    "unit": "GFLOP/s", "frac": flops / (k_ms * 1e-3) / 1e9 / fp64_peak if k_n else None,
                    "traffic": None, "note": "float64 flops of the traced sums over the distinct differences "
                                             "per launch / event time (a microsecond launch: latency-bound); "
                                             "peak: nominal GB300 float64 rate"},
          gpu_launches=2 * args.steps, cpu_baseline=cpu)


def main():
    args = parse()
    if args.cpu_sample is not None:  # child of cpu_baseline: the oracle sample alone, no GPU
        done, dt, reps = _oracle_conv_sample(workloads.CONFIGS[WORKLOAD], args.seed, args.cpu_sample)
        print(json.dumps({"done": done, "seconds": dt, "reps": reps}), flush=True)
        return
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "basis80_n4096":
        run_coulomb(args, ws, rank, local)
    elif args.workload == "density200_n4096":
        run_adjoint(args, ws, rank, local)
    elif args.workload == "lattice32_n16384":
        run_lattice(args, ws, rank, local)
    elif args.workload == "lattice_energy256_n16384":
        run_lattice_energy(args, ws, rank, local)
    elif args.workload == "nuclear80_n4096":
        run_nuclear(args, ws, rank, local)
    elif args.workload == "tei80_n4096":
        run_tei(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
