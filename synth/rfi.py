"""Seeded int8 streams with injected radio-frequency interference and its mask.

Generation runs on the GPU with torch (the training set for the learned flagger is
tens of GB of raw samples); it holds none of the correlator's arithmetic.  Each
stream is Gaussian noise of standard deviation sigma, plus:

- persistent narrowband tones: bin-centred (channel k of an n_fft-point FFT),
  random phase, lasting 8-64 power dumps, with an amplitude chosen so that one
  dump's excess power is kappa standard deviations of the dump's noise power,
  kappa log-uniform in [5, 50]: per frame the noise power of a channel is
  n_fft sigma^2 with standard deviation equal to its mean, a dump sums `dump`
  frames, so A = 2 sigma sqrt(kappa / (sqrt(dump) n_fft));
- broadband impulses: Gaussian noise bursts of 0.1-5 ms (log-uniform at 66.67
  MS/s) with standard deviation sigma_b set for kappa in [5, 50] over a whole
  dump (capped at 60 to limit clipping).

The mask marks (dump, channel) pixels with injected interference: a tone's
channel over its dumps, and every channel of a dump in which a burst's expected
excess is at least 3 standard deviations.  Rates give about 5% occupancy.
"""
from __future__ import annotations

import math

import numpy as np

SAMPLE_RATE_HZ = 66.67e6


def rfi_streams(n_in, n_fft, n_int, *, dump=32, seed=0, sigma=20.0, tones_per_256_dumps=150.0,
                bursts_per_256_dumps=3.0, pad=16, device="cuda"):
    """(x int8 [n_in][n_int*n_fft + pad] on `device`, mask uint8 [n_in][n_int/dump][n_fft/2]).

    Rows are padded with zeros so that the row stride is a multiple of 16 bytes."""
    import torch

    assert n_int % dump == 0
    n_dump, n_chan, N = n_int // dump, n_fft // 2, n_fft
    rng = np.random.default_rng(np.random.SeedSequence([seed, 5]))
    g = torch.Generator(device=device)
    g.manual_seed(int(rng.integers(1 << 62)))
    n_body = n_int * N
    x = torch.randn((n_in, n_body), generator=g, device=device, dtype=torch.float32)
    x.mul_(sigma)
    mask = torch.zeros((n_in, n_dump, n_chan), dtype=torch.uint8, device=device)

    # tones: a complex amplitude map T[i][d][k]; each dump's periodic waveform is its real inverse DFT
    T = np.zeros((n_in, n_dump, n_chan + 1), dtype=np.complex64)
    n_tone = rng.poisson(tones_per_256_dumps * n_dump / 256.0, size=n_in)
    for i in range(n_in):
        for _ in range(n_tone[i]):
            k = int(rng.integers(1, n_chan))
            d0 = int(rng.integers(0, n_dump))
            d1 = min(n_dump, d0 + int(rng.integers(8, 65)))
            kappa = math.exp(rng.uniform(math.log(5.0), math.log(50.0)))
            A = 2.0 * sigma * math.sqrt(kappa / (math.sqrt(dump) * N))
            T[i, d0:d1, k] += A * np.exp(1j * rng.uniform(0, 2 * math.pi))
    Tt = torch.from_numpy(T).to(device)
    # sum_k A cos(2 pi k m / N + phi) = (N / 2) irfft(A e^{i phi})[m] for 0 < k < N/2
    wave = torch.fft.irfft(Tt, n=N, dim=-1) * (N / 2.0)
    x.view(n_in, n_dump, dump, N).add_(wave[:, :, None, :])
    mask |= (Tt[..., :n_chan].abs() > 0).to(torch.uint8)
    del Tt, wave

    # bursts
    n_burst = rng.poisson(bursts_per_256_dumps * n_dump / 256.0, size=n_in)
    for i in range(n_in):
        for _ in range(n_burst[i]):
            dur = int(math.exp(rng.uniform(math.log(0.1e-3), math.log(5e-3))) * SAMPLE_RATE_HZ)
            dur = max(N, min(dur, n_body))
            s0 = int(rng.integers(0, n_body - dur + 1))
            kappa = math.exp(rng.uniform(math.log(5.0), math.log(50.0)))
            sb = min(60.0, sigma * math.sqrt(kappa / math.sqrt(dump)))
            x[i, s0:s0 + dur] += sb * torch.randn(dur, generator=g, device=device)
            for d in range(s0 // (dump * N), min(n_dump, (s0 + dur - 1) // (dump * N) + 1)):
                lo, hi = max(s0, d * dump * N), min(s0 + dur, (d + 1) * dump * N)
                frames = (hi - lo) / N
                if frames * sb * sb / (math.sqrt(dump) * sigma * sigma) >= 3.0:
                    mask[i, d, :] = 1

    out = torch.zeros((n_in, n_body + pad), dtype=torch.int8, device=device)
    out[:, :n_body] = x.round_().clamp_(-127, 127).to(torch.int8)
    return out, mask


def patch_masks(mask, patch=64):
    """Cut a [n_in][n_dump][n_chan] mask into the patch order used by rfi_patches."""
    n_in, n_dump, n_chan = mask.shape
    m = mask.reshape(n_in, n_dump // patch, patch, n_chan // patch, patch)
    return m.permute(0, 1, 3, 2, 4).reshape(-1, patch, patch).contiguous()
