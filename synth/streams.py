"""Seeded int8 baseband streams for the FX correlator workloads.

Each stream (antenna a, polarisation p) is

    x_{a,p}[n] = clip(rint( sqrt(1-rho) * sigma * w_{a,p}[n]
                            + sqrt(rho) * sigma * s_p[n - tau_a]
                            + sum_tones A cos(2 pi k n / N) ), -127, 127)

with w independent unit Gaussian noise, s_p a unit Gaussian "sky" signal
common to all antennas (independent between polarisations) that reaches
antenna a tau_a samples late, and bin-centred tones that are identical in
every stream (terrestrial interference is not geometrically delayed).  A
fractional tau is applied by exact frequency-domain interpolation (Nyquist
bin zeroed); an integer tau by an index shift.

The configurations mirror the paper's workloads: 32 dual-polarisation
antennas, 33 MHz band sampled at 66.67 MS/s, 8-bit samples, 2048-point FFT.
Seeds: ``1000 + config`` by default, one SeedSequence child per stream.
"""
from __future__ import annotations

import dataclasses
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import scipy.fft

SAMPLE_RATE_HZ = 66.67e6  # 33.33 MHz Nyquist-sampled band

CONFIGS = {
    # tiny FX correlator: 4 ant x 2 pol, 512-pt FFT, 64 spectra, integer delays
    1: dict(n_ant=4, n_pol=2, n_fft=512, n_int=64, sigma=20.0, rho=0.3,
            tones=((37, 8.0),), delays=(0.0, 1.0, 2.0, 3.0),
            rates=(0.0, 0.01, 0.02, 0.03), phi0=(0.0, 0.0, 0.0, 0.0), tail=3),
    # GMRT scale: 32 ant x 2 pol, 2048-pt FFT, 8192 spectra (~0.25 s), delays 0-2000 samples
    2: dict(n_ant=32, n_pol=2, n_fft=2048, n_int=8192, sigma=20.0, rho=0.05,
            tones=((100, 8.0), (333, 8.0), (777, 8.0)), delay_range=(0.0, 2000.0),
            rate_range=(0.0, 0.1), phi0_range=(-math.pi, math.pi), tail=2048),
}

# uneven sub-arrays run together in one batched launch: (n_ant, n_pol, n_fft), 4096 spectra each
BATCH_SUBARRAYS = ((8, 2, 512), (16, 2, 1024), (32, 2, 2048), (64, 2, 4096))


@dataclasses.dataclass
class StreamSet:
    x: np.ndarray          # int8 [n_in][n_samp], input i = a * n_pol + p
    n_ant: int
    n_pol: int
    n_fft: int
    n_int: int
    delay: np.ndarray      # [n_ant] samples: the sky delay injected, to be corrected
    phi0: np.ndarray       # [n_ant] fringe phase at frame 0 (rad)
    rate: np.ndarray       # [n_ant] fringe rate (rad / frame)
    recipe: dict

    @property
    def n_in(self) -> int:
        return self.n_ant * self.n_pol


def _fast_len(n: int) -> int:
    return scipy.fft.next_fast_len(n, real=True)


def _common_delayed(rng, n_samp, delays, dtype):
    """Copies of one unit-variance white Gaussian signal, each delayed by delays[a]."""
    delays = np.asarray(delays, dtype=np.float64)
    n_ant = delays.size
    out = np.empty((n_ant, n_samp), dtype=dtype)
    if np.all(delays == np.round(delays)):
        dmax = int(delays.max()) if n_ant else 0
        dmin = int(delays.min()) if n_ant else 0
        s = rng.standard_normal(n_samp + dmax - dmin).astype(dtype)
        for a in range(n_ant):
            off = dmax - int(delays[a])       # s(n - tau_a) with s indexed from -dmax+dmin
            out[a] = s[off: off + n_samp]
        return out
    L = _fast_len(n_samp + int(math.ceil(delays.max())) + 64)
    s = rng.standard_normal(L)
    S = scipy.fft.rfft(s)
    if L % 2 == 0:
        S[-1] = 0.0                       # Nyquist bin has no well-defined delay
    S = S.astype(np.complex64)
    nf = S.size
    # exp(-2 pi i m tau / L) for m = mh*B + ml, from two short FP64 tables
    B = int(math.ceil(math.sqrt(nf)))
    mh = np.arange(-(-nf // B), dtype=np.float64) * B
    ml = np.arange(B, dtype=np.float64)
    batch = 4
    workers = max(1, min(batch, os.cpu_count() or 1))
    for a0 in range(0, n_ant, batch):
        a1 = min(n_ant, a0 + batch)
        spec = np.empty((a1 - a0, nf), dtype=np.complex64)
        for j, a in enumerate(range(a0, a1)):
            th = np.exp(-2j * np.pi * np.outer(mh, delays[a] / L)).astype(np.complex64)
            tl = np.exp(-2j * np.pi * ml * delays[a] / L).astype(np.complex64)
            spec[j] = (th * tl[None, :]).ravel()[:nf] * S
        blk = scipy.fft.irfft(spec, n=L, axis=-1, workers=workers)
        out[a0:a1] = blk[:, :n_samp]
    return out


def make_streams(n_ant, n_pol, n_samp, *, n_fft, sigma=20.0, rho=0.3, tones=(),
                 sky_delay=None, seed=0, dtype=np.float32):
    """int8 [n_ant*n_pol][n_samp] streams per the module recipe."""
    n_in = n_ant * n_pol
    ss = np.random.SeedSequence(seed)
    child = ss.spawn(n_in + n_pol)
    sky_delay = np.zeros(n_ant) if sky_delay is None else np.asarray(sky_delay, np.float64)
    x = np.empty((n_in, n_samp), dtype=np.int8)
    tone = None
    if tones:
        n = np.arange(n_fft)
        per = np.zeros(n_fft)
        for k, A in tones:
            per += A * np.cos(2 * np.pi * k * n / n_fft)
        reps = -(-n_samp // n_fft)
        tone = np.tile(per, reps)[:n_samp].astype(dtype)
    a_w = np.float32(math.sqrt(1.0 - rho) * sigma)
    a_s = np.float32(math.sqrt(rho) * sigma)
    for p in range(n_pol):
        common = None
        if rho > 0:
            common = _common_delayed(np.random.default_rng(child[n_in + p]), n_samp, sky_delay, dtype)

        def one(a):
            i = a * n_pol + p
            v = np.random.default_rng(child[i]).standard_normal(n_samp, dtype=np.float32)
            v *= a_w
            if common is not None:
                v += a_s * common[a]
            if tone is not None:
                v += tone
            np.rint(v, out=v)
            np.clip(v, -127, 127, out=v)
            x[i] = v.astype(np.int8)

        with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
            list(ex.map(one, range(n_ant)))
        del common
    return x


def uniform_params(n_ant, seed, delay_range, rate_range, phi0_range):
    """Per-antenna delay, fringe rate and phase drawn uniformly (seeded)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 7]))
    d = rng.uniform(*delay_range, size=n_ant)
    w = rng.uniform(*rate_range, size=n_ant)
    f = rng.uniform(*phi0_range, size=n_ant)
    return d, w, f


def make_config(cfg: int, *, n_int=None, n_ant=None, n_fft=None, seed=None, tail=None,
                n_pol=None) -> StreamSet:
    """Streams for configuration ``cfg`` (1 or 2), optionally scaled down.

    The sample count is n_int * n_fft + tail, the tail covering the largest delay.
    """
    c = dict(CONFIGS[cfg])
    if n_int is not None:
        c["n_int"] = n_int
    if n_ant is not None:
        c["n_ant"] = n_ant
    if n_fft is not None:
        c["n_fft"] = n_fft
    if n_pol is not None:
        c["n_pol"] = n_pol
    if tail is not None:
        c["tail"] = tail
    seed = 1000 + cfg if seed is None else seed
    na, N = c["n_ant"], c["n_fft"]
    if "delays" in c and na == len(c["delays"]):
        d = np.asarray(c["delays"], np.float64)
        w = np.asarray(c["rates"], np.float64)
        f = np.asarray(c["phi0"], np.float64)
    else:
        dr = c.get("delay_range", (0.0, 2000.0))
        d, w, f = uniform_params(na, seed, dr, c.get("rate_range", (0.0, 0.1)),
                                 c.get("phi0_range", (-math.pi, math.pi)))
    tail = max(int(c["tail"]), int(math.floor(d.max() + 0.5)) if na else 0)
    n_samp = c["n_int"] * N + tail
    tones = tuple((k, A) for k, A in c["tones"] if k < N // 2)
    x = make_streams(na, c["n_pol"], n_samp, n_fft=N, sigma=c["sigma"], rho=c["rho"],
                     tones=tones, sky_delay=d, seed=seed)
    recipe = dict(cfg=cfg, seed=seed, sigma=c["sigma"], rho=c["rho"], tones=tones, tail=tail)
    return StreamSet(x=x, n_ant=na, n_pol=c["n_pol"], n_fft=N, n_int=c["n_int"],
                     delay=d, phi0=f, rate=w, recipe=recipe)
