"""FP64 oracle of coherent dedispersion of the phased-array voltage beam (Sec. 5).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): tests, ``__graft_entry__.smoke()``
and the bench's CPU legs may call it; the product path never does.

What the paper's off-line pipeline computes, in its order:
  1. the beam's pre-detected voltage spectra (each frame: the n_chan channels of one real FFT,
     per polarisation) are turned back into a broadband voltage time series by an inverse FFT
     per frame -- here the complex baseband series z[t n_chan + m] = ifft(V[t])[m], sampled at
     the band's width (channel k of frame t lies at sky frequency f_lo + k bw / n_chan);
  2. the series is deconvolved from the interstellar dispersion by multiplying its Fourier
     transform with the inverse of the ISM transfer function (the cold-plasma chirp): blocks of
     M = fft_frames * n_chan samples, overlapping by overlap_frames * n_chan (overlap-save),
     y_block = ifft(fft(z_block) * C), C[j] = exp(-i Phi(nu_j)), nu_j = f_lo + j bw / M,
         Phi(nu) = 2 pi * 1e6 * D * DM * (nu - nu_ref)^2 / (nu_ref^2 * nu)   [nu in MHz],
     nu_ref = f_lo + bw (the top of the band: every frequency is advanced to its arrival time,
     so the first M - overlap samples of each block are free of wrap-around);
  3. both polarisations are detected and added, |y_X|^2 + |y_Y|^2, and the total power is
     integrated (averaged) over `avg` samples.
numpy's FFT serves as the library step of 1 and 2; the chirp is evaluated in FP64.
"""
from __future__ import annotations

import numpy as np

D_MHZ2_S = 4.148808e3      # dispersion constant: delay (s) = D * DM / nu^2, nu in MHz, DM in pc cm^-3


def dispersion_delay(dm: float, nu_mhz) -> np.ndarray:
    """Cold-plasma arrival delay (s) at sky frequency nu relative to infinite frequency."""
    return D_MHZ2_S * dm / np.asarray(nu_mhz, np.float64) ** 2


def smear_samples(dm: float, f_lo: float, bw: float) -> float:
    """Samples (at bw MHz complex rate) by which the band's bottom lags its top."""
    return (dispersion_delay(dm, f_lo) - dispersion_delay(dm, f_lo + bw)) * bw * 1e6


def chirp(M: int, dm: float, f_lo: float, bw: float) -> np.ndarray:
    """C[j] = exp(-i Phi(nu_j)) over the M bins of one block (step 2)."""
    nu = f_lo + np.arange(M, dtype=np.float64) * (bw / M)
    nu_ref = f_lo + bw
    cycles = 1e6 * D_MHZ2_S * dm * (nu - nu_ref) ** 2 / (nu_ref ** 2 * nu)
    return np.exp(-2j * np.pi * (cycles - np.floor(cycles)))


def coherent_dedisperse(VX, VY, fft_frames: int, overlap_frames: int, dm: float, f_lo: float, bw: float,
                        avg: int) -> np.ndarray:
    """Total-power time series (mean over `avg` samples) of the dedispersed beam.

    VX, VY: complex [n_frames][n_chan] voltage spectra of the two polarisations.  Block b covers
    samples [b S, b S + M) of the series, S = (fft_frames - overlap_frames) * n_chan, and gives
    its first S samples; every complete block is used, in order."""
    VX = np.asarray(VX, np.complex128)
    VY = np.asarray(VY, np.complex128)
    n_frames, n_chan = VX.shape
    F, O = fft_frames, overlap_frames
    if not (0 <= O < F) or bw <= 0:
        raise ValueError("need 0 <= overlap < fft_frames and bw > 0")
    M, S = F * n_chan, (F - O) * n_chan
    if S % avg:
        raise ValueError("avg must divide the block step")
    zX = np.fft.ifft(VX, axis=1).reshape(-1)          # step 1
    zY = np.fft.ifft(VY, axis=1).reshape(-1)
    C = chirp(M, dm, f_lo, bw)
    n_blocks = (n_frames - F) // (F - O) + 1 if n_frames >= F else 0
    out = []
    for b in range(n_blocks):                          # step 2, block by block
        sl = slice(b * S, b * S + M)
        yX = np.fft.ifft(np.fft.fft(zX[sl]) * C)[:S]
        yY = np.fft.ifft(np.fft.fft(zY[sl]) * C)[:S]
        p = np.abs(yX) ** 2 + np.abs(yY) ** 2          # step 3
        out.append(p.reshape(-1, avg).mean(axis=1))
    return np.concatenate(out) if out else np.zeros(0)
