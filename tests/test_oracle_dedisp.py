"""Pins of the coherent-dedispersion oracle (Sec. 5) against what physics and mathematics fix:
Parseval at zero DM, the cold-plasma arrival-time law for narrow-band bursts, the chirp's group
delay, and the independence of the result from the block geometry (overlap-save)."""
import numpy as np
import pytest

from oracle import dedisp

F_LO, BW = 1780.0 / 3.0, 100.0 / 3.0          # 593.33 .. 626.67 MHz, the 610 MHz band


def _rand_spectra(n_frames, n_chan, seed):
    g = np.random.default_rng(seed)
    c = lambda: g.standard_normal((n_frames, n_chan)) + 1j * g.standard_normal((n_frames, n_chan))
    return c(), c()


def test_zero_dm_is_parseval_per_frame():
    # DM = 0: the chirp is 1, the output is the series' own power; with avg = n_chan each output
    # is one frame, whose mean |z|^2 is sum_k |V_k|^2 / n_chan^2 (Parseval)
    n_chan, F, O = 32, 64, 16
    VX, VY = _rand_spectra(64 + 3 * 48 + 20, n_chan, 1)
    I = dedisp.coherent_dedisperse(VX, VY, F, O, 0.0, F_LO, BW, n_chan)
    n_blocks = (VX.shape[0] - F) // (F - O) + 1
    assert I.shape == (n_blocks * (F - O),)
    want = (np.abs(VX) ** 2 + np.abs(VY) ** 2).sum(axis=1)[:I.size] / n_chan ** 2
    assert np.allclose(I, want, rtol=1e-12, atol=0)


def test_avg_is_a_mean_over_consecutive_samples():
    n_chan, F, O = 16, 32, 8
    VX, VY = _rand_spectra(32 + 24, n_chan, 2)
    I1 = dedisp.coherent_dedisperse(VX, VY, F, O, 0.3, F_LO, BW, 1)
    I8 = dedisp.coherent_dedisperse(VX, VY, F, O, 0.3, F_LO, BW, 8)
    assert np.allclose(I8, I1.reshape(-1, 8).mean(axis=1), rtol=1e-13)


def test_chirp_group_delay_is_the_dispersion_delay_difference():
    # the phase step of C between neighbouring bins is 2 pi (t(nu) - t(nu_ref)) times the bin
    # width (the advance that brings frequency nu to the top of the band), t = D DM / nu^2
    M, dm = 1 << 16, 3.0
    C = dedisp.chirp(M, dm, F_LO, BW)
    step = np.angle(C[1:] * np.conj(C[:-1]))
    nu_mid = F_LO + (np.arange(M - 1) + 0.5) * BW / M
    t = dedisp.dispersion_delay(dm, nu_mid) - dedisp.dispersion_delay(dm, F_LO + BW)
    want = 2 * np.pi * t * (BW * 1e6 / M)
    assert np.max(np.abs(np.angle(np.exp(1j * (step - want))))) < 1e-6 * np.max(np.abs(want))
    assert abs(C[-1] * np.conj(C[-2]) - 1) < 1e-2       # the top of the band is hardly advanced


def _burst_spectra(n_chan, n_frames, frac, n_arrive, sigma):
    """One narrow-band burst at baseband frequency frac * bw, its envelope centred at sample
    n_arrive, channelised frame by frame (the inverse of the oracle's step 1)."""
    n = np.arange(n_frames * n_chan, dtype=np.float64)
    z = np.exp(-0.5 * ((n - n_arrive) / sigma) ** 2) * np.exp(2j * np.pi * frac * n)
    V = np.fft.fft(z.reshape(n_frames, n_chan), axis=1)
    return V, np.zeros_like(V)


@pytest.mark.parametrize("frac", [0.125, 0.5, 0.875])
def test_bursts_arrive_at_the_top_of_band_time(frac):
    # a burst at sky frequency nu arrives D DM (1/nu^2 - 1/nu_top^2) after the top of the band;
    # dedispersion brings it back to the top-of-band time, the zero-DM run leaves it where it is
    n_chan, F, O, dm, sigma = 256, 1024, 512, 2.0, 1024.0
    assert dedisp.smear_samples(dm, F_LO, BW) < O * n_chan
    n_frames = F + 2 * (F - O)
    n_top = 200000.0
    nu = F_LO + frac * BW
    lag = (dedisp.dispersion_delay(dm, nu) - dedisp.dispersion_delay(dm, F_LO + BW)) * BW * 1e6
    VX, VY = _burst_spectra(n_chan, n_frames, frac, n_top + lag, sigma)

    def centroid(I):
        c = np.arange(I.size) * n_chan + (n_chan - 1) / 2.0
        return float((I * c).sum() / I.sum())

    I = dedisp.coherent_dedisperse(VX, VY, F, O, dm, F_LO, BW, n_chan)
    I0 = dedisp.coherent_dedisperse(VX, VY, F, O, 0.0, F_LO, BW, n_chan)
    Iw = dedisp.coherent_dedisperse(VX, VY, F, O, -dm, F_LO, BW, n_chan)   # the wrong sign
    assert abs(centroid(I) - n_top) < 16
    assert abs(centroid(I0) - (n_top + lag)) < 16
    if lag > 1000:                                   # the wrong sign does not bring it back
        assert abs(centroid(Iw) - n_top) > 0.5 * lag
    # the energy is kept (the chirp is unitary; the burst lies inside the valid samples)
    assert I.sum() == pytest.approx(I0.sum(), rel=1e-6)


def test_block_geometry_does_not_change_the_result():
    # overlap-save: with the overlap above the smear, blocks of different lengths give the same
    # dedispersed series, up to the chirp response's tails beyond the smear, largest just after
    # each block start (a wrong block offset would differ by the whole signal)
    n_chan, O, dm = 64, 1024, 1.0
    assert dedisp.smear_samples(dm, F_LO, BW) < 0.7 * O * n_chan
    VX, VY = _rand_spectra(4096 + 3 * 1024, n_chan, 3)
    Ia = dedisp.coherent_dedisperse(VX, VY, 2048, O, dm, F_LO, BW, n_chan)
    Ib = dedisp.coherent_dedisperse(VX, VY, 4096, O, dm, F_LO, BW, n_chan)
    n = min(Ia.size, Ib.size)
    assert n >= 4096
    err = np.abs(Ia[:n] - Ib[:n]) / Ia[:n].mean()
    assert np.sqrt((err ** 2).mean()) < 1e-3 and err.max() < 3e-2


def test_channel_smear_of_the_papers_b1937_example():
    # the dispersion law the oracle uses reproduces the paper's printed worked example:
    # arrival-time difference across one 65.1 kHz channel at 325 MHz for DM 71.0398
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "dispersion_smear_b1937.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for dm, nu, dnu, want_ms, tol_ms in ((float(x) for x in r) for r in rows):
        got = (dedisp.dispersion_delay(dm, nu - dnu / 2) - dedisp.dispersion_delay(dm, nu + dnu / 2)) * 1e3
        assert abs(got - want_ms) <= tol_ms, got
        # and the per-channel smear in samples of that channel's complex rate, the quantity the
        # block overlap must cover when a single channel is dedispersed
        assert dedisp.smear_samples(dm, nu - dnu / 2, dnu) == pytest.approx(got * 1e-3 * dnu * 1e6, rel=1e-9)
