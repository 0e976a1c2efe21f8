"""Time-domain voltage blanker (Sec. 5, Eq. 3-4) on the GPU against the oracle: the per-block
statistics (2 med, 4 MAD, threshold, samples replaced) are bit-exact, the spectra and
visibilities of the blanked stream match the oracle run on the oracle's blanked samples, and
blanking brings the visibilities of an RFI-hit stream back towards the clean sky's."""
import numpy as np
import pytest

from fxhelp import vis_norm_error
from synth import make_config

pytestmark = pytest.mark.gpu

N_ANT, N_POL, N_FFT, N_INT = 8, 2, 1024, 64
BLOCK, M, L = 4096, 3.0, 4096


@pytest.fixture(scope="module")
def env(orc):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0910_1517_gb300 import build, corr
    build.build()
    corr.load()
    return torch, corr, orc


def _stream(seed=6100):
    s = make_config(2, n_ant=N_ANT, n_pol=N_POL, n_fft=N_FFT, n_int=N_INT, seed=seed)
    clean = s.x.copy()
    rng = np.random.default_rng(seed + 1)
    x = s.x.astype(np.int16)
    for _ in range(40):                               # broadband bursts of 20-200 samples in every input
        p0 = int(rng.integers(0, x.shape[1] - 200))
        ln = int(rng.integers(20, 200))
        x[:, p0:p0 + ln] += rng.choice([-1, 1], size=(x.shape[0], ln)) * 90
    s.x[:] = np.clip(x, -127, 127).astype(np.int8)
    noise = np.random.default_rng(seed + 2).standard_normal((s.n_in, L)).astype(np.float32)
    return s, clean, noise


def _run(env, s, x, mode=0, blank=True, noise=None, block=BLOCK):
    torch, corr, _ = env
    h = corr.corr_create(s.n_ant, s.n_pol, s.n_fft, s.n_int)
    corr.corr_set_delays(h, s.delay, s.phi0, s.rate)
    if blank:
        corr.corr_set_blanker(h, M, block, noise)
    n = x.shape[1]
    xt = torch.zeros((s.n_in, ((n + 15) // 16) * 16 + 16), dtype=torch.int8, device="cuda")
    xt[:, :n] = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    if mode:
        corr.corr_integrate_device(h, xt, n_avail=n, stream=torch.cuda.current_stream())
        corr.corr_set_scales(h, None)
        corr.corr_set_mode(h, mode, 0, 1)
    corr.corr_integrate_device(h, xt, n_avail=n, stream=torch.cuda.current_stream())
    out = {"V": corr.corr_read_visibilities(h).astype(np.complex128), "h": h}
    if blank:
        out["stats"], out["n"] = corr.corr_read_blank_stats(h)
    if mode == 0:
        out["Y"] = corr.corr_read_spectra(h, 0, s.n_fft // 2, s.n_int).astype(np.complex128)
    return out


# 4096: one 16-byte piece a thread, kept in registers; 16384: four, all kept; 32768: the pieces
# past the fourth read again for the copy; every size ends in a ragged block
@pytest.mark.parametrize("block", [4096, 16384, 32768])
def test_blank_statistics_bit_exact_and_spectra_match_oracle(env, block):
    torch, corr, orc = env
    s, _, noise = _stream()
    r = _run(env, s, s.x, noise=noise, block=block)
    n = r["n"]
    assert n == s.n_int * s.n_fft + int(np.floor(s.delay + 0.5).max())
    assert n % block
    xb, st = orc.mad_blank(s.x[:, :n], block, M, noise)
    assert r["stats"].shape == st.shape and np.array_equal(r["stats"], st)
    assert st[..., 3].sum() > 1000                   # the bursts are there and get replaced
    chans = [0, 1, 100, 255, 256, 333, 511]
    Y = orc.fengine(xb, s.n_ant, s.n_pol, s.n_fft, s.n_int, s.delay, s.phi0, s.rate, chans=chans)
    V = orc.xengine(Y, s.n_ant, s.n_pol)
    e_y = max(float(np.abs(r["Y"][i][:, chans] - Y[i]).max() / np.abs(Y[i]).max()) for i in range(s.n_in))
    e_v = vis_norm_error(r["V"][chans], V, s.n_ant, s.n_pol)
    print(f"blanker: {st[..., 3].sum()} of {s.n_in * n} samples replaced; spectra {e_y:.2e} vis {e_v:.2e}")
    assert e_y <= 1e-5 and e_v <= 1e-5
    corr.corr_destroy(r["h"])


def test_blanking_restores_the_clean_visibilities(env):
    torch, corr, orc = env
    s, clean, noise = _stream(6200)
    chans = [10, 100, 333, 500]
    Yc = orc.fengine(clean, s.n_ant, s.n_pol, s.n_fft, s.n_int, s.delay, s.phi0, s.rate, chans=chans)
    Vc = orc.xengine(Yc, s.n_ant, s.n_pol)
    hit = _run(env, s, s.x, blank=False)
    bl = _run(env, s, s.x, noise=noise)
    e_hit = vis_norm_error(hit["V"][chans], Vc, s.n_ant, s.n_pol)
    e_bl = vis_norm_error(bl["V"][chans], Vc, s.n_ant, s.n_pol)
    print(f"vs clean sky: RFI-hit {e_hit:.3f}, blanked {e_bl:.3f}")
    assert e_bl < 0.5 * e_hit
    for r in (hit, bl):
        corr.corr_destroy(r["h"])


@pytest.mark.parametrize("mode", [1, 2], ids=["i8", "f16"])
def test_blanker_in_the_tensor_core_forms(env, mode):
    torch, corr, orc = env
    s, _, noise = _stream(6300)
    r32 = _run(env, s, s.x, noise=noise)
    rq = _run(env, s, s.x, mode=mode, noise=noise)
    assert np.array_equal(rq["stats"], r32["stats"])   # same decisions whatever the X-engine form
    # per-channel error against the FP32 form, DC aside (its 4-sigma int8 scale clips); with 64
    # frames the int8 tail is wide (the clean stream's own: median 4e-3, max 5e-2), so the median
    # is checked for int8 -- unblanked, the bursts push it to ~5e-2 (they set the scales)
    errs = [vis_norm_error(rq["V"][c:c + 1], r32["V"][c:c + 1], s.n_ant, s.n_pol) for c in range(1, s.n_fft // 2)]
    print(f"blanker with xmode {mode}: vis vs the FP32 form, median {np.median(errs):.2e} max {max(errs):.2e}")
    if mode == 1:
        assert np.median(errs) < 1e-2
    else:
        assert max(errs) < 1e-2
    for r in (r32, rq):
        corr.corr_destroy(r["h"])


def test_blanker_arguments(env):
    torch, corr, orc = env
    h = corr.corr_create(4, 2, 1024, 16)
    g = np.zeros((8, 64), np.float32)
    try:
        for block, gg in ((512, g), (2048, g), (3000, g), (65536, g), (4096, np.zeros((8, 48), np.float32))):
            with pytest.raises(corr.CorrError) as ei:
                corr.corr_set_blanker(h, 3.0, block, gg)
            assert ei.value.code == -1
        with pytest.raises(corr.CorrError) as ei:
            corr.corr_read_blank_stats(h)
        assert ei.value.code == -7                     # off
        corr.corr_set_blanker(h, 3.0, 4096, g)
        with pytest.raises(corr.CorrError) as ei:
            corr.corr_read_blank_stats(h)
        assert ei.value.code == -7                     # not run yet
        with pytest.raises(corr.CorrError) as ei:
            corr.corr_batch_create([h])
        assert ei.value.code == -1
        corr.corr_set_blanker(h, 0.0)
        b = corr.corr_batch_create([h])
        try:
            with pytest.raises(corr.CorrError) as ei:
                corr.corr_set_blanker(h, 3.0, 4096, g)
            assert ei.value.code == -7
        finally:
            corr.corr_batch_destroy(b)
    finally:
        corr.corr_destroy(h)
