#!/usr/bin/env python3
"""Throughput of the GB300 FX correlator + beamformer on the GMRT-scale workload.

Workload (one step = one integration through every hot-path stage): 32 antennas
x 2 polarisations of real int8 samples (66.67 MS/s, 33.33 MHz band), integer +
fractional delays 0-2000 samples, fringe rates 0-0.1 rad/spectrum, 2048-point
real FFT -> 1024 channels, 8192 spectra (~0.25 s of sky data, 1.07 GB of
samples), incoherent beam over 32 antennas and coherent beam over antennas
0-29, 528 baselines x 4 products accumulated in FP32.  Inputs are seeded
synthetic streams resident in HBM; at 1.07 GB per step they are larger than L2.
The timed step's X-engine is the FP32 form on the tcgen05 tensor cores
(CORR_FP32TC: FP32 spectra as exact fp16 hi + lo pairs, error within the FP32
bound); --xmode fp32 times the plain CUDA-core FP32 form instead, and both are
reported.

value   antenna-samples/s over all ranks (device-resident input)
e2e     the same through corr_push_samples from pinned host memory plus the
        read-back of visibilities and beams, copies inside the timed region
The JSON line also carries the real-time factor, the per-stage times, the
roofline of the dominant kernel, every form of the X-engine (plain FP32 on CUDA
cores, FP32 / int8 / FP16 on tensor cores, same data) with its speedup over the
plain FP32 form, clocks seen during the timed
region and the FP64 oracle timed on a bounded sample of the same workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank correlates its own time slice (no data-path
collective): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "antenna-samples/s, real-time factor at 32 ant/33 MHz/2 pol; X-engine % of peak"
UNIT = "antenna-samples/s"
SAMPLE_RATE = 66.67e6                      # per stream, 33.33 MHz Nyquist
N_ANT, N_POL, N_FFT, N_INT = 32, 2, 2048, 8192
N_IN, N_CHAN = N_ANT * N_POL, N_FFT // 2
N_BL = N_ANT * (N_ANT + 1) // 2
COH_ANTENNAS = 30                          # the "30-antenna phased" coherent beam
CONFIG = {
    "workload": "GMRT-scale FP32 FX correlator + beamformer: 32 ant x 2 pol int8 at 66.67 MS/s, "
                "2048-pt FFT -> 1024 ch, 8192 spectra/integration, 528 baselines x 4 products, "
                "incoherent (32 ant) + coherent (30 ant) beams",
    "n_ant": N_ANT, "n_pol": N_POL, "n_fft": N_FFT, "n_int": N_INT, "xmode": "fp32tc",
    "l2": "inputs larger than L2 (1.07 GB of samples per step)",
    "parallelism": "time slices across ranks (replicas), no data-path collective",
}
FORMS = {
    "fp32": "plain FP32: FP32 spectra, X-engine FP32 multiply-adds on the CUDA cores",
    "fp32tc": "FP32 spectra held as fp16 hi + lo planes (v = hi + lo to 2^-22 |v|), X-engine on tcgen05: "
              "H H^T in 128-frame FP32 chunks, H L^T + L H^T in a separate accumulator; FP32 accuracy bound",
    "i8": "per-channel scaled int8 requantisation, exact integer X-engine on tcgen05",
    "f16": "per-channel scaled FP16 requantisation, X-engine on tcgen05 with FP32 accumulation",
    "fp32_self": "self-polar (total-intensity) mode of the plain FP32 form: products RR*, LL* only "
                 "(528 baselines x 2 products), half the CUDA-core multiply-adds",
}
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def set_n_int(n):
    """Scale the integration length (profiling runs); the headline workload is 8192."""
    global N_INT
    N_INT = n
    CONFIG["n_int"] = n
    CONFIG["workload"] += f" [scaled to {n} spectra per integration]"


def peaks():
    p = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0,
         "source": "fallback"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained", "sm_max_mhz"):
            if k in m:
                p[k] = float(m[k])
        p["source"] = "measured"
    except (OSError, ValueError):
        pass
    return p


# ------------------------------------------------------ ranks (one per GPU)

def world_env():
    """(world size, rank, local rank) as torchrun exports them; (1, 0, 0) when run directly."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def slice_seed(rank):
    """Seed of this rank's time slice of the synthetic sky: every rank correlates its own data."""
    return 1002 + rank


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (a whole-job time is its slowest rank's); x without ranks."""
    if not dist:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, seconds):
    """Whole-job throughput: each of `world` ranks processed units_per_rank within `seconds`."""
    return world * units_per_rank / seconds


def emit(line, rank):
    """The one JSON line of a run, printed by rank 0 only."""
    if rank == 0:
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_id):
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "100", "-i", str(dev_id)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        rows = []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in out.splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                rows.append((float(f[0]), float(f[1]), float(f[2]), f[4:8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        pmax = max(r[2] for r in rows)
        load = [r for r in rows if r[2] >= 0.5 * pmax]          # samples taken under load
        reasons = set()
        for r in load:
            for n, v in zip(names, r[3]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(load), "power_w_max": pmax}


# ------------------------------------------------------------ work accounting

def step_samples():
    return N_IN * N_INT * N_FFT


# Algorithmic work per input sample (the GMRT-scale workload: 64 inputs, 2048-point FFT):
#   F-engine: 2.5 log2 N (real FFT) + 3 (Eq. 2 phasor) + 6 (beams) = 36.5 flop, and 1 B of int8
#   samples read + 0.0625 B of beams written (2 x 4 B per channel-frame of 1024 channels, over
#   2048 x 64 samples); its FP32 spectra hand-off is not algorithmic.  At ~34 flop/B the F-engine
#   sits above the FP32 ridge (80.5 TFLOP/s / 6.7 TB/s ~ 12 flop/B): it is graded on the FP32 ALU,
#   with its fraction of HBM on the algorithmic bytes reported beside it.
#   X-engine, tensor-core forms: the operand read -- 1 B (int8), 2 B (FP16) or 4 B (the FP32 form:
#   FP32 spectra, split on chip) per sample -- plus the visibilities, against HBM.
#   X-engine, CUDA-core FP32 form: n_in (n_in + 1) / 2 useful complex MACs per channel-frame.
FE_FLOP_PER_SAMPLE = 2.5 * math.log2(N_FFT) + 3 + 6
FE_BYTES_PER_SAMPLE = 1.0 + 2 * 4 / (2 * N_IN)
X_OPERAND_BYTES = {"i8": 1, "f16": 2, "fp32tc": 4}


def stage_roofline(stage, mode, ms, pk):
    """(bound, achieved, peak, unit, algorithmic amount per launch) of one kernel."""
    if stage == "fengine":
        alg = FE_FLOP_PER_SAMPLE * step_samples()
        return "alu", alg / (ms * 1e-3) / 1e12, fp32_peak_tflops(pk), "TFLOP/s", alg
    if stage == "xengine" and mode == "fp32":
        # useful FP32 work: n_in(n_in+1)/2 complex MACs (8 flop) per channel and frame
        alg = 8.0 * N_CHAN * N_INT * N_IN * (N_IN + 1) / 2
        peak = fp32_peak_tflops(pk)
        return "alu", alg / (ms * 1e-3) / 1e12, peak, "TFLOP/s", alg
    alg = step_samples() * X_OPERAND_BYTES[mode] + N_CHAN * N_BL * 4 * 8
    return "hbm", alg / (ms * 1e-3) / 1e9, pk["hbm_gbs"], "GB/s", alg


def fp32_peak_tflops(pk):
    """FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x the maximum SM clock."""
    return SM_COUNT * FP32_LANES_PER_SM * 2 * pk["sm_max_mhz"] * 1e6 / 1e12


def fengine_hbm(ms, pk, mode):
    """The F-engine against HBM: on its algorithmic bytes (samples in, beams out), and on the bytes
    it actually moves (plus the spectra hand-off: 4 B per sample in the FP32 forms, 2 B as fp16)."""
    alg = FE_BYTES_PER_SAMPLE * step_samples()
    moved = alg + step_samples() * (4 if mode in ("fp32", "fp32tc") else 2)
    return {"bound": "hbm", "algorithmic_bytes": alg, "achieved": alg / (ms * 1e-3) / 1e9, "peak": pk["hbm_gbs"],
            "unit": "GB/s", "frac": alg / (ms * 1e-3) / 1e9 / pk["hbm_gbs"], "moved_bytes": moved,
            "moved_frac": moved / (ms * 1e-3) / 1e9 / pk["hbm_gbs"]}


def useful_tflops(ms):
    """Useful X-engine work: n_in (n_in + 1) / 2 complex MACs (8 flop) per channel and frame."""
    return 8.0 * N_CHAN * N_INT * N_IN * (N_IN + 1) / 2 / (ms * 1e-3) / 1e12


def tensor_fraction(ms, pk, mmas=1):
    """Executed tcgen05 flops (full 128x128 Gram per channel, `mmas` products) vs the dense fp16 peak."""
    executed = 2.0 * mmas * N_CHAN * N_INT * (2 * N_IN) ** 2
    return executed / (ms * 1e-3) / 1e12 / pk["bf16_tflops_sustained"]


def source_sha(files):
    """First 16 hex digits of the SHA-256 over a kernel's source files (a name or a list), in order."""
    h = hashlib.sha256()
    for f in [files] if isinstance(files, str) else files:
        h.update(open(os.path.join(ROOT, "paper_0910_1517_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(kernel):
    """DRAM bytes per launch from the committed ncu summary, if the kernel is unchanged since."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        e = t[kernel]
        if source_sha(e["source"]) != e["source_sha"]:
            return None
        return float(e["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


# ------------------------------------------------------------------ oracle

def oracle_sample(x, s, n_frames):
    """FP64 oracle (F-engine, beams, X-engine) on n_frames of the workload; seconds."""
    import oracle
    t0 = time.perf_counter()
    Y = oracle.fengine(x, s.n_ant, s.n_pol, s.n_fft, n_frames, s.delay, s.phi0, s.rate)
    oracle.beams(Y, s.n_ant, s.n_pol, s.n_fft, coh_mask=(np.arange(s.n_ant) < COH_ANTENNAS).astype(np.uint8))
    oracle.xengine(Y, s.n_ant, s.n_pol)
    return time.perf_counter() - t0


def fft_sample(x, s, n_frames):
    """CPU FFT baseline (FP32 radix-2 FFT F-engine, FP64 oracle beams and X-stage) on n_frames; seconds."""
    import oracle
    t0 = time.perf_counter()
    Y = oracle.fft_fengine(x, s.n_ant, s.n_pol, s.n_fft, n_frames, s.delay, s.phi0, s.rate)
    oracle.beams(Y, s.n_ant, s.n_pol, s.n_fft, coh_mask=(np.arange(s.n_ant) < COH_ANTENNAS).astype(np.uint8))
    oracle.xengine(Y, s.n_ant, s.n_pol)
    return time.perf_counter() - t0


def cpu_fft_baseline_auto(x, s, target_s=8.0):
    import oracle
    t1 = fft_sample(x, s, 16)
    n_frames = int(max(16, min(s.n_int, round(16 * target_s / max(t1, 1e-3)))))
    n_frames -= n_frames % 16
    dt = fft_sample(x, s, n_frames)
    return {"value": N_IN * n_frames * N_FFT / dt, "unit": UNIT, "cores": oracle.threads(),
            "kind": "cpu FFT baseline",
            "sample": f"FP32 radix-2 FFT F-engine (own C, OpenMP) + FP64 oracle beams and X-stage on {n_frames} "
                      f"of the 8192 spectra of all 64 inputs, all 1024 channels ({dt:.1f} s)"}


def cpu_baseline_auto(x, s, target_s=15.0):
    import oracle
    t1 = oracle_sample(x, s, 2)
    n_frames = int(max(2, min(s.n_int, round(2 * target_s / max(t1, 1e-3)))))
    n_frames -= n_frames % 2
    dt = oracle_sample(x, s, n_frames)
    v = N_IN * n_frames * N_FFT / dt
    return {"value": v, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"FP64 direct-DFT oracle (F-engine, beams, X-engine) on {n_frames} of the 8192 spectra of "
                      f"all 64 inputs, all 1024 channels ({dt:.1f} s)"}


def run_reference(args, world, rank):
    """The FP64 oracle timed on bounded samples of the same workload (rank 0 only)."""
    if rank != 0:
        return 0
    import oracle
    from synth import make_config
    oracle.build()
    s = make_config(2, n_int=64)
    t_one = oracle_sample(s.x, s, 1)
    budget = 150.0
    nf = int(max(1, min(64, budget / max(t_one, 1e-3) / max(1, args.steps + args.warmup))))
    for _ in range(args.warmup):
        oracle_sample(s.x, s, nf)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_sample(s.x, s, nf)
    dt = time.perf_counter() - t0
    v = args.steps * N_IN * nf * N_FFT / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": CONFIG,
        "rtf": v / (N_IN * SAMPLE_RATE),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                         "sample": f"each step: FP64 direct-DFT oracle on {nf} spectra x 64 inputs x 1024 channels"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    emit(line, rank)
    return 0


# -------------------------------------------------------------------- ours

def pack4(x):
    """4-bit ADC card rows (4 inputs x 4 bits per 2 bytes) of the int8 stream x scaled by 1/5."""
    n_cards, n = x.shape[0] // 4, x.shape[1]
    out = np.empty((n_cards, 2 * n), np.uint8)
    for c in range(n_cards):                   # one card (4 rows) at a time
        nib = (np.clip(np.rint(x[4 * c:4 * c + 4].astype(np.float32) / 5.0), -8, 7).astype(np.int8)
               .view(np.uint8) & 0xF)
        out[c, 0::2] = nib[0] | (nib[1] << 4)
        out[c, 1::2] = nib[2] | (nib[3] << 4)
    return out


def run_e2e(args, corr, torch, dist, s, coh, world, xmode, four_bit=False):
    """The public streaming path: samples pushed from pinned host memory (corr_push_samples,
    two sample rings so the copy of integration j + 1 overlaps the correlation of j) and every
    integration's visibilities and beams copied back into a ring of pinned host slots
    (corr_set_output_ring / corr_wait_output).  Timed from the first push to the last result
    in host memory."""
    K = args.steps
    body = N_INT * N_FFT
    if four_bit:   # the paper's 33 MHz mode: 4-bit samples, 4 inputs per ADC card
        p4 = pack4(s.x)
        hx0 = torch.from_numpy(np.ascontiguousarray(p4[:, :2 * (body + 2048)])).pin_memory()
        hx = torch.from_numpy(np.ascontiguousarray(p4[:, 2 * 2048:2 * (2048 + body)])).pin_memory()
        push = lambda buf, n, q: corr.corr_push_samples_4bit(he, buf.numpy(), n, q)
    else:
        hx0 = torch.from_numpy(np.ascontiguousarray(s.x[:, :body + 2048])).pin_memory()
        hx = torch.from_numpy(np.ascontiguousarray(s.x[:, 2048:2048 + body])).pin_memory()
        push = lambda buf, n, q: corr.corr_push_samples(he, buf.numpy(), q)
    n_slots = 2
    hv = torch.empty((n_slots, N_CHAN, N_BL, 4, 2), dtype=torch.float32).pin_memory()
    hb = torch.empty((n_slots, 2, N_INT, N_CHAN), dtype=torch.float32).pin_memory()
    he = corr.corr_create(N_ANT, N_POL, N_FFT, N_INT)
    corr.corr_set_delays(he, s.delay, s.phi0, s.rate)
    corr.corr_set_beam_weights(he, None, None, None, coh)
    corr.corr_set_mode(he, xmode, 0, 1)
    corr.corr_set_output_ring(he, hv.numpy(), hb.numpy(), n_slots)
    seq = 0
    push(hx0, body + 2048, seq)                            # first integration + the delay overlap
    seq += body + 2048
    corr.corr_wait_output(he, 0)
    j = 1
    for _ in range(2):                                     # warm the path
        push(hx, body, seq)
        seq += body
        corr.corr_wait_output(he, j)
        j += 1
    k3 = max(5, min(K, 40))
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for q in range(k3):
        push(hx, body, seq)                                # launches integration j + q
        seq += body
        if q > 0:
            corr.corr_wait_output(he, j + q - 1)          # the previous one's results, in host memory
    corr.corr_wait_output(he, j + k3 - 1)
    dt = time.perf_counter() - t0
    dt = max_over_ranks(dt, dist, "cuda")
    # the host link itself: one step's samples, pinned host to device, one copy, CUDA events
    dev = torch.empty(hx.shape, dtype=hx.dtype, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        dev.copy_(hx, non_blocking=True)
    e0.record()
    for _ in range(5):
        dev.copy_(hx, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    link_gbs = 5 * hx.numel() * hx.element_size() / (e0.elapsed_time(e1) * 1e-3) / 1e9
    del dev
    e2e = {"value": job_rate(world, k3 * step_samples(), dt), "unit": UNIT,
           "h2d_bytes_per_step": N_IN * body // (2 if four_bit else 1),
           "d2h_bytes_per_step": (hv.numel() + hb.numel()) * 4 // n_slots, "steps": k3,
           "ms_per_step": 1e3 * dt / k3,
           "host_link_h2d_gbs": link_gbs,
           "host_link_floor_ms_per_step": N_IN * body / (2 if four_bit else 1) / (link_gbs * 1e9) * 1e3,
           "path": ("corr_push_samples_4bit (pinned host ADC card rows, 4 bits per sample)" if four_bit else
                    "corr_push_samples (pinned host, two sample rings)") +
                   " + corr_wait_output (visibilities and beams of every integration in a ring of pinned host slots)"}
    corr.corr_destroy(he)
    return e2e


def run_multibeam_leg(corr, torch, s, xt, ld, coh, xmode, k, st_plain, pk, n_beams=16, avg=32):
    """Multiple phased beams (Sec. 2.2, 5) on the GMRT-scale step: n_beams (16, or 64) beams with
    per-antenna phase gradients across the band (different pointings), full-polar products in
    32-frame (~1 ms) windows, read from the FP32 spectra after the X-engine.  Reports the beam
    kernel's time (the last stage of the step) against its rooflines: the FP32 spectra read once
    from HBM, and either the useful FP32 work n_beams x n_in complex MACs per channel-frame
    against the FP32 CUDA-core peak (up to 24 beams: the CUDA-core kernel) or the executed fp16
    tensor work against the measured tensor peak (beyond 24 beams: the tcgen05 kernel)."""
    rng = np.random.default_rng(31)
    delays = rng.uniform(-20, 20, (n_beams, N_ANT, 1))          # samples of geometric delay per beam
    W = np.exp(2j * np.pi * delays * np.arange(N_CHAN)[None, None, :] / N_FFT)
    h2 = corr.corr_create(N_ANT, N_POL, N_FFT, N_INT)
    try:
        corr.corr_set_delays(h2, s.delay, s.phi0, s.rate)
        corr.corr_set_beam_weights(h2, None, None, None, coh)
        corr.corr_set_mode(h2, xmode, 0, 1)
        corr.corr_set_multibeam(h2, W, 0, avg)
        stream = torch.cuda.current_stream()
        for j in range(3):
            corr.corr_integrate_device(h2, xt, n_avail=ld, g0=j * N_INT, stream=stream)
        torch.cuda.synchronize()
        corr.corr_set_timing(h2, 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for j in range(k):
            corr.corr_integrate_device(h2, xt, n_avail=ld, g0=(3 + j) * N_INT, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        st, cnt = corr.corr_stage_times(h2)
        corr.corr_set_timing(h2, 0)
        ms = e0.elapsed_time(e1) / k
        mb_ms = float(st[3] / max(cnt, 1))
        flop = 8.0 * n_beams * N_IN * N_CHAN * N_INT
        k_pad = ((2 * N_ANT + 15) // 16) * 16
        tc_flop = 3 * 2.0 * 128 * (N_POL * 64) * k_pad * N_CHAN * (N_INT // 64)
        bytes_ = N_CHAN * N_INT * 2 * N_IN * 4 + n_beams * (N_INT // avg) * N_CHAN * 16
        return {"workload": f"GMRT-scale step + {n_beams} phased beams, full-polar products in {avg}-frame windows",
                "form": "tcgen05 (fp16 hi/lo split)" if n_beams > 24 else "CUDA cores (FP32)",
                "ms_per_step": ms, "value": step_samples() / (ms * 1e-3), "unit": UNIT,
                "beam_kernel_ms": mb_ms,
                "roofline_hbm": {"achieved": bytes_ / (mb_ms * 1e-3) / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                 "frac": bytes_ / (mb_ms * 1e-3) / 1e9 / pk["hbm_gbs"]},
                **({"roofline_tensor": {"executed_tflops": tc_flop / (mb_ms * 1e-3) / 1e12,
                                        "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s",
                                        "frac": tc_flop / (mb_ms * 1e-3) / 1e12 / pk["bf16_tflops_sustained"],
                                        "executed": "3 fp16 MMAs (hi/lo split) of 128 x (n_pol x 64) x K per "
                                                    "64-frame stage and channel, K = 2 n_ant padded to 16"}}
                   if n_beams > 24 else
                   {"roofline_alu": {"achieved": flop / (mb_ms * 1e-3) / 1e12, "peak": fp32_peak_tflops(pk),
                                     "unit": "TFLOP/s", "frac": flop / (mb_ms * 1e-3) / 1e12 / fp32_peak_tflops(pk)}})}
    finally:
        corr.corr_destroy(h2)


def run_dedisp_leg(corr, torch, pk, k=20, dm=30.0, f_lo=1780.0 / 3.0, bw=100.0 / 3.0):
    """Coherent dedispersion of the phased-array voltage beam (Sec. 5) at GMRT scale: one beam's
    voltage spectra (1024 channels over 33.3 MHz at 610 MHz, both polarisations), one
    integration (8192 frames) per push, DM 30 pc/cc (1.22 M samples = 1192 frames of smear),
    blocks of 4096 frames overlapping by 1200 (just above the smear: 2896 new frames per
    block, 2.83 blocks per push on average), one total-power sample per frame.  Input
    spectra (seeded Gaussian) are resident in HBM; each push copies them into the frame ring.
    Reports the push time, per-stage times and each pass's HBM traffic of the design (A: read the
    frames, write the work block; B: read it and the chirp, write it back; C: read it, write the
    column sums) against the measured HBM peak, and the real-time factor."""
    F, O, n_push = 4096, 1200, N_INT
    d = corr.corr_dd_create(N_CHAN, F, O, n_push, dm, f_lo, bw, N_CHAN)
    try:
        g = torch.Generator(device="cuda").manual_seed(555)
        v = torch.randn((n_push, N_CHAN, 4), generator=g, device="cuda") * 100.0
        keep = F - O
        out = torch.empty((n_push // keep + 1) * keep, dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream()
        for _ in range(4):                                  # fill the ring, reach the steady state
            corr.corr_dd_push_device(d, v, out, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        n_out = 0
        for _ in range(k):
            n_out += corr.corr_dd_push_device(d, v, out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        corr.corr_dd_set_timing(d, True)
        for _ in range(k):
            corr.corr_dd_push_device(d, v, out, stream=stream)
        st, cnt = corr.corr_dd_stage_times(d)
        corr.corr_dd_set_timing(d, False)
        st = [float(x) / max(cnt, 1) for x in st]
        nb = n_out / k / keep                               # blocks per push, averaged (one output per frame)
        M = F * N_CHAN
        traffic = {"ring_copy": 2 * n_push * N_CHAN * 16, "A": nb * 2 * M * 16, "B": nb * (2 * M * 16 + M * 8),
                   "C": nb * (M * 16 + keep * (N_CHAN // 2) * 4), "D": nb * keep * (N_CHAN // 2) * 4}
        traffic = {q: int(b) for q, b in traffic.items()}
        names = ["ring_copy", "A", "B", "C", "D"]
        stages = {}
        for nme, t in zip(names, st):
            gbs = traffic[nme] / (t * 1e-3) / 1e9
            stages[nme] = {"ms": round(t, 4), "bytes": traffic[nme], "achieved_gbs": gbs,
                           "frac_of_measured_hbm": gbs / pk["hbm_gbs"]}
        dom = max(("A", "B", "C"), key=lambda q: stages[q]["ms"])
        samples = n_push * N_CHAN
        return {"workload": f"coherent dedispersion of one voltage beam: {N_CHAN} ch x 33.3 MHz at 610 MHz, DM {dm}, "
                            f"{F}-frame blocks overlapping {O}, {n_push} frames per push, 1 output per frame",
                "ms_per_push": ms, "outputs_per_push": n_out / k, "value": samples / (ms * 1e-3),
                "unit": "beam samples/s (complex, both polarisations)",
                "rtf": samples / (ms * 1e-3) / (bw * 1e6), "stages": stages,
                "roofline": {"bound": "hbm", "kernel": f"pass {dom}", "achieved": stages[dom]["achieved_gbs"],
                             "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": stages[dom]["frac_of_measured_hbm"]}}
    finally:
        corr.corr_dd_destroy(d)


def run_blank_leg(corr, torch, s, xt, ld, coh, xmode, k, st_plain):
    """The time-domain MAD voltage blanker (Sec. 5, Eq. 3-4) on the GMRT-scale step: broadband
    bursts (+-90 counts, 100 samples each, independent signs per input) cover ~2.5 % of a copy of
    the samples; M = 3, 16384-sample blocks, a 65536-entry noise table per input.  Reports the
    F-engine stage (blanker kernel: statistics and the blanked copy, then the F-engine) against
    the plain one and the fraction of samples replaced (the paper: 2-3 %)."""
    g = torch.Generator(device="cuda").manual_seed(4321)
    n = s.n_int * N_FFT + 2048
    x2 = xt.clone()
    n_burst, blen = int(0.025 * n / 100), 100
    starts = torch.randint(0, n - blen, (n_burst,), generator=g, device="cuda")
    idx = (starts[:, None] + torch.arange(blen, device="cuda")[None, :]).reshape(-1)
    sign = torch.randint(0, 2, (N_IN, idx.numel()), generator=g, device="cuda", dtype=torch.int16) * 2 - 1
    x2[:, idx] = (x2[:, idx].to(torch.int16) + 90 * sign).clamp(-127, 127).to(torch.int8)
    noise = np.random.default_rng(77).standard_normal((N_IN, 1 << 16)).astype(np.float32)
    h2 = corr.corr_create(N_ANT, N_POL, N_FFT, N_INT)
    try:
        corr.corr_set_delays(h2, s.delay, s.phi0, s.rate)
        corr.corr_set_beam_weights(h2, None, None, None, coh)
        corr.corr_set_mode(h2, xmode, 0, 1)
        corr.corr_set_blanker(h2, 3.0, 16384, noise)
        stream = torch.cuda.current_stream()
        for j in range(3):
            corr.corr_integrate_device(h2, x2, n_avail=ld, g0=j * N_INT, stream=stream)
        torch.cuda.synchronize()
        corr.corr_set_timing(h2, 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for j in range(k):
            corr.corr_integrate_device(h2, x2, n_avail=ld, g0=(3 + j) * N_INT, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        st, cnt = corr.corr_stage_times(h2)
        corr.corr_set_timing(h2, 0)
        stats, covered = corr.corr_read_blank_stats(h2)
        ms = e0.elapsed_time(e1) / k
        return {"workload": "GMRT-scale step with broadband bursts on ~2.5 % of the samples; M = 3, 16384-sample blocks",
                "ms_per_step": ms, "value": step_samples() / (ms * 1e-3), "unit": UNIT,
                "fengine_stage_ms": float(st[1] / max(cnt, 1)), "fengine_stage_ms_without": float(st_plain[1]),
                "replaced_fraction": float(stats[..., 3].sum()) / (N_IN * covered)}
    finally:
        corr.corr_destroy(h2)
        del x2


BATCH_SUBS = ((8, 2, 512), (16, 2, 1024), (32, 2, 2048), (64, 2, 4096))
BATCH_N_INT = 4096


def run_batch_leg(args, corr, torch, rank):
    """Four uneven sub-arrays in one graph launch per step, int8 tensor-core X-engine,
    X-engine stage sizes chosen by the autotuner."""
    from synth import uniform_params
    from synth.device import make_streams_device
    stream = torch.cuda.current_stream()
    hs, xs, na, samples = [], [], [], 0
    for q, (n_ant, n_pol, n_fft) in enumerate(BATCH_SUBS):
        d, w, f = uniform_params(n_ant, 4000 + q + 10 * rank, (0.0, 2000.0), (0.0, 0.1), (-math.pi, math.pi))
        d = np.floor(d + 0.5)                       # integer sky delays for the device generator
        n_samp = BATCH_N_INT * n_fft + 2048
        x = make_streams_device(n_ant, n_pol, n_samp, delays=d, seed=4000 + q + 10 * rank)
        h = corr.corr_create(n_ant, n_pol, n_fft, BATCH_N_INT)
        corr.corr_set_delays(h, d, f, w)
        corr.corr_integrate_device(h, x, n_avail=x.shape[1], stream=stream)
        corr.corr_set_scales(h, None)                # calibration integration (FP32)
        corr.corr_set_mode(h, corr.CORR_I8, 0, 1)
        hs.append(h)
        xs.append(x)
        na.append(x.shape[1])
        samples += n_ant * n_pol * BATCH_N_INT * n_fft
    b = corr.corr_batch_create(hs)
    try:
        corr.corr_batch_integrate_device(b, xs, n_avail=na, stream=stream)
        ks, ms_x = corr.corr_batch_tune(b, len(hs))
        for _ in range(3):
            corr.corr_batch_integrate_device(b, xs, n_avail=na, stream=stream)
        torch.cuda.synchronize()
        k = max(10, min(args.steps, 100))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for j in range(k):
            corr.corr_batch_integrate_device(b, xs, n_avail=na, g0=[(j + 4) * BATCH_N_INT] * len(hs), stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
    finally:
        corr.corr_batch_destroy(b)
        for h in hs:
            corr.corr_destroy(h)
    return {"workload": "4 sub-arrays (ant, pol, FFT) = " + ", ".join(str(t) for t in BATCH_SUBS) +
                        f", {BATCH_N_INT} spectra each, int8 tensor-core X-engine, one CUDA graph per step",
            "value": samples / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": k,
            "tuned_frames_per_stage": [int(v) for v in ks], "tuned_xengine_ms": [float(v) for v in ms_x],
            "launches_per_step": f"1 graph of {len(hs)} concurrent branches (phasor set-up, F-engine, X-engine): "
                                 f"{3 * len(hs)} kernels"}


def run_rfi_leg(corr, torch, n_train_int=25, n_test_int=3):
    """Learned RFI flagger on the GMRT-shaped correlator's own 1 ms power dumps with injected
    RFI: 4096 patches per integration; one training epoch; held-out comparison with the MAD
    flagger."""
    from synth.rfi import patch_masks, rfi_streams
    stream = torch.cuda.current_stream()
    n_in, n_fft, n_int = N_IN, N_FFT, N_INT
    n_dump = n_int // 32
    h = corr.corr_create(N_ANT, N_POL, n_fft, n_int)
    corr.corr_set_power_dump(h, 32)
    B = n_in * (n_dump // 64) * (N_CHAN // 64)

    def data(n, seed):
        xs, fs, ms = [], [], []
        for j in range(n):
            x, mask = rfi_streams(n_in, n_fft, n_int, seed=seed + j)
            corr.corr_integrate_device(h, x, n_avail=n_int * n_fft, stream=stream)
            xp = torch.empty((B, 64, 64), dtype=torch.float16, device="cuda")
            fl = torch.empty((B, 64, 64), dtype=torch.uint8, device="cuda")
            corr.rfi_patches(corr.corr_power_device(h), n_in, n_dump, N_CHAN, 5.0, xp, fl, None, stream=stream)
            xs.append(xp)
            fs.append(fl)
            ms.append(patch_masks(mask))
            del x
        torch.cuda.synchronize()
        return torch.cat(xs), torch.cat(fs), torch.cat(ms)

    try:
        t0 = time.perf_counter()
        xtr, _, mtr = data(n_train_int, 20000)
        xte, fte, mte = data(n_test_int, 90000)
        t_data = time.perf_counter() - t0
    finally:
        corr.corr_destroy(h)
    rng = np.random.default_rng(1)
    p = np.zeros(corr.rfi_n_params())
    offs = ((0, 144, 9), (160, 4608, 144), (4800, 4608, 288), (9424, 16, 16))
    for o, n, fan in offs:
        p[o:o + n] = rng.normal(scale=math.sqrt(2.0 / fan), size=n)
    for o, n in ((144, 16), (4768, 32), (9408, 16)):
        p[o:o + n] = 0.05
    net = corr.rfi_create(256)
    try:
        corr.rfi_set_params(net, p)
        g = torch.Generator(device="cuda").manual_seed(0)
        perm = torch.randperm(xtr.shape[0], generator=g, device="cuda")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        steps = 0
        for b0 in range(0, xtr.shape[0] - 255, 256):
            idx = perm[b0:b0 + 256]
            corr.rfi_train_step(net, xtr[idx].contiguous(), mtr[idx].contiguous(), 256, 2e-3, stream=stream)
            steps += 1
        e1.record(stream)
        torch.cuda.synchronize()
        train_ms = e0.elapsed_time(e1)
        prob = torch.empty(xte.shape, dtype=torch.float32, device="cuda")
        e0.record(stream)
        for b0 in range(0, xte.shape[0], 256):
            nb = min(256, xte.shape[0] - b0)
            corr.rfi_infer(net, xte[b0:b0 + nb].contiguous(), nb, prob[b0:b0 + nb], stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        infer_ms = e0.elapsed_time(e1)
    finally:
        corr.rfi_destroy(net)

    def rates(flags, mask):
        f, m = flags.bool(), mask.bool()
        return (float((m & ~f).sum()) / max(1, int(m.sum())), float((f & ~m).sum()) / max(1, int((~m).sum())))

    cnn, mad = rates(prob > 0.5, mte), rates(fte, mte)
    return {"workload": "32 ant x 2 pol, 1024 ch, 32-frame (0.98 ms) power dumps, 64x64 FP16 patches, "
                        "injected tones 5-50 sigma and 0.1-5 ms bursts",
            "train_patches": int(xtr.shape[0]), "test_patches": int(xte.shape[0]),
            "occupancy": float(mte.float().mean()), "epochs": 1, "train_steps": steps,
            "train_patches_per_s": steps * 256 / (train_ms * 1e-3),
            "infer_patches_per_s": xte.shape[0] / (infer_ms * 1e-3),
            "cnn": {"miss": cnn[0], "false_flag": cnn[1]}, "mad_5sigma": {"miss": mad[0], "false_flag": mad[1]},
            "data_generation_s": t_data}


def run_ours(args, world, rank, local_rank):
    import torch
    from paper_0910_1517_gb300 import build as libbuild
    from paper_0910_1517_gb300 import corr
    from synth import make_config

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if rank == 0:
        libbuild.build()
    if dist:
        dist.barrier()
    corr.load()
    pk = peaks()
    if args.leg != "all":                                 # one extra leg alone (profiling runs)
        if args.leg == "e2e4bit":                        # the 4-bit ADC streaming path alone
            s4 = make_config(2, seed=slice_seed(rank), n_int=N_INT)
            res = {"e2e_4bit_adc": run_e2e(args, corr, torch, dist, s4, (np.arange(N_ANT) < COH_ANTENNAS).astype(np.uint8),
                                           world, corr.CORR_FP32TC, four_bit=True)}
        elif args.leg == "multibeam":                    # the phased-beam kernels alone (16 and 64 beams)
            sm = make_config(2, seed=slice_seed(rank), n_int=N_INT)
            ldm = ((sm.x.shape[1] + 15) // 16) * 16 + 16
            xm = torch.zeros((N_IN, ldm), dtype=torch.int8, device="cuda")
            xm[:, :sm.x.shape[1]] = torch.from_numpy(sm.x).cuda()
            cm = (np.arange(N_ANT) < COH_ANTENNAS).astype(np.uint8)
            res = {f"beams_{nb}": run_multibeam_leg(corr, torch, sm, xm, ldm, cm, corr.CORR_FP32TC, 10, None,
                                                    peaks(), n_beams=nb) for nb in (16, 64)}
        elif args.leg == "blank":                        # the voltage blanker alone, on the GMRT-scale step
            sb = make_config(2, seed=slice_seed(rank), n_int=N_INT)
            ldb = ((sb.x.shape[1] + 15) // 16) * 16 + 16
            xb = torch.zeros((N_IN, ldb), dtype=torch.int8, device="cuda")
            xb[:, :sb.x.shape[1]] = torch.from_numpy(sb.x).cuda()
            cb = (np.arange(N_ANT) < COH_ANTENNAS).astype(np.uint8)
            hp = corr.corr_create(N_ANT, N_POL, N_FFT, N_INT)   # the same step unblanked, for its F-engine stage
            try:
                corr.corr_set_delays(hp, sb.delay, sb.phi0, sb.rate)
                corr.corr_set_beam_weights(hp, None, None, None, cb)
                corr.corr_set_mode(hp, corr.CORR_FP32TC, 0, 1)
                st = torch.cuda.current_stream()
                for j in range(3):
                    corr.corr_integrate_device(hp, xb, n_avail=ldb, g0=j * N_INT, stream=st)
                torch.cuda.synchronize()
                corr.corr_set_timing(hp, 1)
                for j in range(max(args.steps, 1)):
                    corr.corr_integrate_device(hp, xb, n_avail=ldb, g0=(3 + j) * N_INT, stream=st)
                torch.cuda.synchronize()
                t_plain, n_plain = corr.corr_stage_times(hp)
            finally:
                corr.corr_destroy(hp)
            res = {"voltage_blanker": run_blank_leg(corr, torch, sb, xb, ldb, cb, corr.CORR_FP32TC, max(args.steps, 1),
                                                    t_plain / max(n_plain, 1))}
        if args.leg in ("e2e4bit", "multibeam", "blank"):
            pass
        else:
            res = run_batch_leg(args, corr, torch, rank) if args.leg == "batched" else \
                run_dedisp_leg(corr, torch, peaks()) if args.leg == "dedisp" else run_rfi_leg(corr, torch)
        emit({"leg": args.leg, **res}, rank)
        if dist:
            dist.destroy_process_group()
        return 0

    s = make_config(2, seed=slice_seed(rank), n_int=N_INT)    # this rank's time slice
    n_avail = s.x.shape[1]
    ld = ((n_avail + 15) // 16) * 16 + 16
    xt = torch.zeros((N_IN, ld), dtype=torch.int8, device="cuda")
    xt[:, :n_avail] = torch.from_numpy(s.x).cuda()
    stream = torch.cuda.current_stream()
    coh = (np.arange(N_ANT) < COH_ANTENNAS).astype(np.uint8)

    h = corr.corr_create(N_ANT, N_POL, N_FFT, N_INT)
    corr.corr_set_delays(h, s.delay, s.phi0, s.rate)
    corr.corr_set_beam_weights(h, None, None, None, coh)

    def steps(n, mode, g_start):
        for j in range(n):
            corr.corr_integrate_device(h, xt, n_avail=ld, g0=(g_start + j) * N_INT, stream=stream)

    def timed(mode, k, w, sample_clocks=False, polmode=0):
        corr.corr_set_mode(h, mode, polmode, 1)
        steps(w, mode, 0)
        torch.cuda.synchronize()
        corr.corr_set_timing(h, 1)
        sampler = None
        if sample_clocks:
            bus = getattr(torch.cuda.get_device_properties(local_rank), "pci_bus_id", None)
            sampler = ClockSampler(bus if bus else local_rank)
            time.sleep(0.3)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        steps(k, mode, w)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clocks = sampler.stop() if sampler else None
        ms = e0.elapsed_time(e1)
        st, n = corr.corr_stage_times(h)
        corr.corr_set_timing(h, 0)
        ms = max_over_ranks(ms, dist, "cuda")
        return ms, st / max(n, 1), clocks

    K, W = args.steps, args.warmup
    all_forms = {"fp32": corr.CORR_FP32, "fp32tc": corr.CORR_FP32TC, "i8": corr.CORR_I8, "f16": corr.CORR_F16,
                 "fp32_self": corr.CORR_FP32}
    ms, st, clocks = timed(all_forms[args.xmode], K, W, sample_clocks=True)
    value = job_rate(world, K * step_samples(), ms * 1e-3)
    stage_names = ["phasor_setup", "fengine", "xengine", "beam_average"]

    # the other forms of the X-engine on the same data (scales for i8 / f16 from the last
    # integration's autos); speedups are against the plain CUDA-core FP32 form
    corr.corr_set_scales(h, None)
    runs = {args.xmode: (ms / K, st)}
    for name, m in (() if args.no_extras else all_forms.items()):
        if name in runs:
            continue
        k2 = max(10, min(K, 100))
        ms2, st2, _ = timed(m, k2, 3, polmode=corr.CORR_POL_SELF if name.endswith("_self") else 0)
        runs[name] = (ms2 / k2, st2)
    modes = {}
    for name, (step_ms, st2) in runs.items():
        d = {"value": job_rate(world, step_samples(), step_ms * 1e-3), "ms_per_step": step_ms,
             "stage_ms": dict(zip(stage_names, [round(v, 4) for v in st2]))}
        if "fp32" in runs and name != "fp32":
            d["xengine_speedup_vs_fp32"] = runs["fp32"][1][2] / st2[2]
            d["step_speedup_vs_fp32"] = runs["fp32"][0] / step_ms
        if name not in ("fp32", "fp32_self"):
            d["xengine_tensor_frac_of_sustained_peak"] = tensor_fraction(st2[2], pk, 3 if name == "fp32tc" else 1)
        if name == "fp32_self":
            # useful self-polar work: n_ant (n_ant + 1) / 2 baselines x 2 products, complex MAC (8 flop)
            alg = 8.0 * N_CHAN * N_INT * N_BL * N_POL
            d["xengine_useful_tflops"] = alg / (st2[2] * 1e-3) / 1e12
            d["xengine_roofline"] = {"bound": "alu", "achieved": d["xengine_useful_tflops"],
                                     "peak": fp32_peak_tflops(pk), "unit": "TFLOP/s",
                                     "frac": d["xengine_useful_tflops"] / fp32_peak_tflops(pk)}
            d["form"] = FORMS[name]
            modes[name] = d
            continue
        d["xengine_useful_tflops"] = useful_tflops(st2[2])
        bound, ach, peak, unit, _ = stage_roofline("xengine", name, st2[2], pk)
        d["xengine_roofline"] = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak}
        d["form"] = FORMS[name]
        modes[name] = d
    corr.corr_set_mode(h, all_forms[args.xmode], 0, 1)
    if "fp32_self" in modes and "fp32" in runs:
        modes["fp32_self"]["xengine_speedup_vs_full_polar_fp32"] = runs["fp32"][1][2] / runs["fp32_self"][1][2]

    # the time-domain voltage blanker on an RFI-hit copy of the same samples
    blank = None if args.no_extras else run_blank_leg(corr, torch, s, xt, ld, coh, all_forms[args.xmode],
                                                      max(10, min(K, 50)), st)

    # multiple phased beams (16 beams, full polar, 32-frame windows) on the same samples
    multibeam = None if args.no_extras else run_multibeam_leg(corr, torch, s, xt, ld, coh, all_forms[args.xmode],
                                                              max(10, min(K, 50)), st, pk)
    # 64 beams: the tensor-core form (more than 24 beams)
    multibeam64 = None if args.no_extras else run_multibeam_leg(corr, torch, s, xt, ld, coh, all_forms[args.xmode],
                                                                max(10, min(K, 50)), st, pk, n_beams=64)

    # coherent dedispersion of one phased-array voltage beam (one integration per push)
    dedisp = None if args.no_extras else run_dedisp_leg(corr, torch, pk)
    torch.cuda.empty_cache()

    # end to end through the public API: pinned host samples in, visibilities + beams out
    e2e = None if args.no_extras else run_e2e(args, corr, torch, dist, s, coh, world, all_forms[args.xmode])
    e2e_4bit = None if args.no_extras else run_e2e(args, corr, torch, dist, s, coh, world, all_forms[args.xmode],
                                                   four_bit=True)

    # roofline of the dominant kernel of the timed step
    dom = 1 if st[1] >= st[2] else 2
    kname = {1: "fengine", 2: "xengine"}[dom]
    bound, ach, peak, unit, alg = stage_roofline(kname, args.xmode, st[dom], pk)
    kern_id = "fengine_w_kernel" if kname == "fengine" else \
        ("xengine_fp32_kernel" if args.xmode == "fp32" else "xengine_tc_kernel")
    roofline = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                "traffic": traffic_for(kern_id), "kernel": kern_id,
                "algorithmic_per_launch": alg, "avg_launch_ms": st[dom],
                "peak_source": ("derived from the FP32 lane count and the measured maximum SM clock "
                                "(152 SMs x 128 lanes x 2 flop x sm_max_mhz)") if bound == "alu" else
                               f"{pk['source']} (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic": (f"{FE_FLOP_PER_SAMPLE} flop per input sample" if kname == "fengine" else
                                "operand bytes per input sample + visibilities")}
    stages = {}
    for i, nme in ((1, "fengine"), (2, "xengine")):
        b, a, p, u, _ = stage_roofline(nme, args.xmode, st[i], pk)
        stages[nme] = {"ms": st[i], "bound": b, "achieved": a, "peak": p, "unit": u, "frac": a / p}
    stages["fengine"]["hbm_roofline"] = fengine_hbm(st[1], pk, args.xmode)
    stages["xengine"]["useful_tflops"] = useful_tflops(st[2])
    stages["phasor_setup"] = {"ms": st[0]}

    cpu = cpu_fft = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline_auto(s.x, s)
        cpu_fft = cpu_fft_baseline_auto(s.x, s)

    corr.corr_destroy(h)
    del xt
    torch.cuda.empty_cache()
    batch = rfi = None
    if not args.no_extras:
        batch = run_batch_leg(args, corr, torch, rank)
        torch.cuda.empty_cache()
        if rank == 0:
            rfi = run_rfi_leg(corr, torch)
    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (seeded Gaussian sky + noise + tones, GMRT shapes)",
            "config": {**CONFIG, "xmode": args.xmode},
            "rtf": value / (world * N_IN * SAMPLE_RATE),
            "xengine_frac_of_fp32_peak": modes["fp32"]["xengine_roofline"]["frac"] if "fp32" in modes else None,
            "roofline": roofline, "stages": stages, "precision_forms": modes,
            "batched_subarrays": batch, "learned_rfi": rfi,
            "e2e": e2e, "gpu_launches": 3 * K, "clocks": clocks, "cpu_baseline": cpu,
            "cpu_fft_baseline": cpu_fft, "voltage_blanker": blank, "multibeam": multibeam, "multibeam_64": multibeam64,
            "e2e_4bit_adc": e2e_4bit, "coherent_dedispersion": dedisp,
        }
    emit(line, rank)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle cpu_baseline leg")
    ap.add_argument("--no-extras", action="store_true",
                    help="time only the FP32 step (no precision forms, no end-to-end leg); for profiling runs")
    ap.add_argument("--leg", choices=("all", "batched", "rfi", "dedisp", "multibeam", "e2e4bit", "blank"), default="all",
                    help="run one extra leg alone: batched sub-arrays, learned RFI, dedispersion, phased beams, the "
                         "4-bit ADC streaming path or the voltage blanker (profiling runs)")
    ap.add_argument("--xmode", choices=("fp32tc", "fp32"), default="fp32tc",
                    help="form of the timed step: FP32 on the tensor cores (default) or the plain CUDA-core FP32 form")
    ap.add_argument("--n-int", type=int, default=N_INT,
                    help="spectra per integration (default 8192, the GMRT-scale workload; smaller for profiling)")
    args = ap.parse_args()
    if args.n_int != N_INT:
        set_n_int(args.n_int)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local_rank = world_env()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local_rank)


if __name__ == "__main__":
    sys.exit(main())
