"""Coherent dedispersion of the phased-array voltage beam (Sec. 5) on the GPU against the FP64
oracle: uneven pushes through the frame ring, every window size regime, the bench's full-size
configuration, a dispersed burst brought back to the top-of-band time, and argument errors."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

F_LO, BW = 1780.0 / 3.0, 100.0 / 3.0          # 593.33 .. 626.67 MHz


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0910_1517_gb300 import build, corr
    build.build()
    corr.load()
    from oracle import dedisp
    return torch, corr, dedisp


def _spectra(n_frames, n_chan, seed, sigma=100.0):
    g = np.random.default_rng(seed)
    v = (g.standard_normal((n_frames, n_chan, 4)) * sigma).astype(np.float32)
    return v


def _run(torch, corr, v, cuts, n_chan, F, O, dm, avg, max_push):
    d = corr.corr_dd_create(n_chan, F, O, max_push, dm, F_LO, BW, avg)
    try:
        keep = F - O
        outs = []
        cap = (max_push // keep + 1) * keep * n_chan // avg
        buf = torch.empty(cap, dtype=torch.float32, device="cuda")
        vt = torch.from_numpy(v).cuda()
        for a, b in zip(cuts[:-1], cuts[1:]):
            n = corr.corr_dd_push_device(d, vt[a:b].contiguous(), buf, stream=torch.cuda.current_stream())
            outs.append(buf[:n].cpu().numpy().copy())
        torch.cuda.synchronize()
        return np.concatenate(outs)
    finally:
        corr.corr_dd_destroy(d)


def _oracle(dedisp, v, F, O, dm, avg):
    vx = v[..., 0].astype(np.float64) + 1j * v[..., 1]
    vy = v[..., 2].astype(np.float64) + 1j * v[..., 3]
    return dedisp.coherent_dedisperse(vx, vy, F, O, dm, F_LO, BW, avg)


@pytest.mark.parametrize("avg", [2, 64, 256, 4096])
def test_uneven_pushes_match_the_oracle(env, avg):
    torch, corr, dedisp = env
    n_chan, F, O, dm = 256, 1024, 512, 2.0
    v = _spectra(F + 3 * (F - O) + 100, n_chan, 11)
    cuts = [0, 700, 701, 1900, 1937, v.shape[0]]
    got = _run(torch, corr, v, cuts, n_chan, F, O, dm, avg, max_push=2048)
    want = _oracle(dedisp, v, F, O, dm, avg)
    assert got.shape == want.shape
    err = np.abs(got - want) / want.mean()
    assert err.max() < 2e-5, err.max()


@pytest.mark.parametrize("n_chan,F,O,dm", [(64, 4096, 2048, 0.5), (4096, 256, 64, 0.4), (512, 512, 300, 0.7),
                                           (128, 2048, 1024, 0.9)])
def test_geometries_match_the_oracle(env, n_chan, F, O, dm):
    torch, corr, dedisp = env
    assert corr.corr_dd_smear_samples(dm, F_LO, BW) < O * n_chan
    keep = F - O
    avg = 2 * n_chan if (keep * n_chan) % (2 * n_chan) == 0 else n_chan
    v = _spectra(F + 2 * keep, n_chan, 12)
    got = _run(torch, corr, v, [0, F + keep, v.shape[0]], n_chan, F, O, dm, avg, max_push=F + keep)
    want = _oracle(dedisp, v, F, O, dm, avg)
    assert got.shape == want.shape
    assert (np.abs(got - want) / want.mean()).max() < 2e-5


def test_bench_configuration_matches_the_oracle(env):
    # the bench's workload: 1024 channels over 33.3 MHz at 610 MHz, DM 30, blocks of 4096 frames
    # overlapping by 1200 (the smear is 1192 frames), one integration of 8192 frames per push,
    # one output per frame
    torch, corr, dedisp = env
    n_chan, F, O, dm, avg = 1024, 4096, 1200, 30.0, 1024
    assert corr.corr_dd_smear_samples(dm, F_LO, BW) < O * n_chan
    v = _spectra(2 * 8192, n_chan, 13)
    got = _run(torch, corr, v, [0, 8192, 16384], n_chan, F, O, dm, avg, max_push=8192)
    want = _oracle(dedisp, v, F, O, dm, avg)
    assert got.shape == want.shape == (((16384 - F) // (F - O) + 1) * (F - O),)
    assert (np.abs(got - want) / want.mean()).max() < 2e-5


def test_dispersed_burst_returns_to_the_top_of_band_time(env):
    torch, corr, dedisp = env
    n_chan, F, O, dm = 256, 1024, 512, 2.0
    n_frames = F + 2 * (F - O)
    nu = F_LO + 0.25 * BW
    lag = (dedisp.dispersion_delay(dm, nu) - dedisp.dispersion_delay(dm, F_LO + BW)) * BW * 1e6
    n = np.arange(n_frames * n_chan, dtype=np.float64)
    z = np.exp(-0.5 * ((n - (200000.0 + lag)) / 1024.0) ** 2) * np.exp(2j * np.pi * 0.25 * n)
    V = np.fft.fft(z.reshape(n_frames, n_chan), axis=1) * 50
    v = np.zeros((n_frames, n_chan, 4), np.float32)
    v[..., 0], v[..., 1] = V.real, V.imag
    I = _run(torch, corr, v, [0, n_frames], n_chan, F, O, dm, n_chan, max_push=n_frames)
    c = np.arange(I.size) * n_chan + (n_chan - 1) / 2.0
    assert abs((I * c).sum() / I.sum() - 200000.0) < 16


def test_arguments(env):
    torch, corr, dedisp = env
    with pytest.raises(corr.CorrError) as ei:          # overlap below the smear
        corr.corr_dd_create(256, 1024, 64, 1024, 2.0, F_LO, BW, 256)
    assert ei.value.code == -2
    for bad in [(100, 1024, 512, 1024, 2.0, F_LO, BW, 256),     # n_chan not a power of two
                (256, 1024, 1024, 1024, 2.0, F_LO, BW, 256),    # overlap = fft_frames
                (256, 1024, 512, 1024, 2.0, F_LO, -BW, 256),    # lower sideband
                (256, 1024, 512, 1024, 2.0, F_LO, BW, 3)]:      # avg not a power of two
        with pytest.raises(corr.CorrError) as ei:
            corr.corr_dd_create(*bad)
        assert ei.value.code == -1
    d = corr.corr_dd_create(256, 1024, 512, 1024, 2.0, F_LO, BW, 256)
    try:
        corr.corr_dd_set_timing(d, True)               # stage timing of a push that completes blocks
        v0 = torch.zeros((1024, 256, 4), dtype=torch.float32, device="cuda")
        out0 = torch.empty(512, dtype=torch.float32, device="cuda")
        assert corr.corr_dd_push_device(d, v0, out0) == 512
        ms, cnt = corr.corr_dd_stage_times(d)
        assert cnt == 1 and (ms >= 0).all() and ms[1:4].sum() > 0
        corr.corr_dd_set_timing(d, False)
        corr.corr_dd_reset(d)
        v = torch.zeros((1024, 256, 4), dtype=torch.float32, device="cuda")
        small = torch.empty(10, dtype=torch.float32, device="cuda")
        assert corr.corr_dd_push_device(d, v[:0], small) == 0          # nothing pushed
        with pytest.raises(corr.CorrError) as ei:                       # out too small
            corr.corr_dd_push_device(d, v, small)
        assert ei.value.code == -1
        big = torch.zeros((1025, 256, 4), dtype=torch.float32, device="cuda")
        with pytest.raises(corr.CorrError):                             # above max_push_frames
            corr.corr_dd_push_device(d, big, small)
    finally:
        corr.corr_dd_destroy(d)
