"""Seeded int8 streams generated on the GPU with torch, for workloads too large to
generate on the host in a benchmark (several GB of samples).

Same recipe as ``synth.streams`` without tones: per stream
``clip(rint(sqrt(1-rho) sigma w + sqrt(rho) sigma s(n - D_a)), -127, 127)`` with a
common sky signal s per polarisation delayed by an integer number of samples D_a
per antenna.  Holds none of the correlator's arithmetic.
"""
from __future__ import annotations

import math

import numpy as np


def make_streams_device(n_ant, n_pol, n_samp, *, sigma=20.0, rho=0.05, delays=None, seed=0, device="cuda"):
    """int8 [n_ant*n_pol][ld] on `device` (ld = n_samp rounded up to 16, plus 16 bytes of zeros)."""
    import torch

    n_in = n_ant * n_pol
    d = np.zeros(n_ant, dtype=np.int64) if delays is None else np.floor(np.asarray(delays) + 0.5).astype(np.int64)
    dmax = int(d.max()) if n_ant else 0
    g = torch.Generator(device=device)
    g.manual_seed(int(np.random.default_rng(np.random.SeedSequence([seed, 3])).integers(1 << 62)))
    ld = ((n_samp + 15) // 16) * 16 + 16
    out = torch.zeros((n_in, ld), dtype=torch.int8, device=device)
    a_w, a_s = math.sqrt(1.0 - rho) * sigma, math.sqrt(rho) * sigma
    for p in range(n_pol):
        sky = torch.randn(n_samp + dmax, generator=g, device=device)
        for a in range(n_ant):
            v = torch.randn(n_samp, generator=g, device=device).mul_(a_w)
            off = dmax - int(d[a])                         # s(n - D_a)
            v.add_(sky[off:off + n_samp], alpha=a_s)
            out[a * n_pol + p, :n_samp] = v.round_().clamp_(-127, 127).to(torch.int8)
    return out
