"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.

Tolerances (the arithmetic behind them is in the design notes):
  FP32 path    visibilities: max |V - V64| / sqrt(V64_aa V64_a'a') <= 1e-5
               beams: relative (incoherent) / Cauchy-Schwarz-normalised (coherent) <= 1e-5
               spectra: max |Y - Y64| <= 1e-5 * max |Y64| per input
  CORR_I8      integer visibilities equal the oracle's int64 MAC on the GPU's own
               requantised spectra, bit for bit
  CORR_F16     normalised error vs FP64 on raw samples <= 1e-3
  rail inputs  -128 and long runs of +-127 in the raw samples: the FP32 bound, and int8 bit-exactness
  CORR_FP32TC  the FP32 visibility bound above; spectra and beams bit-identical to
               CORR_FP32's (the same F-engine; only the X-engine differs)
"""
import math

import numpy as np
import pytest

from fxhelp import beam_errors, vis_norm_error
from synth import make_config

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def env(orc):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0910_1517_gb300 import build, corr
    build.build()
    corr.load()
    return torch, corr, orc


def to_device(torch, x):
    n_in, n = x.shape
    ld = ((n + 15) // 16) * 16 + 16
    xt = torch.zeros((n_in, ld), dtype=torch.int8, device="cuda")
    xt[:, :n] = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return xt, n


def run_gpu(env, s, mode=0, beam_avg=1, gain=None, theta=None, inc=None, coh=None, scales=None,
            g0=0, want_spec=None, handle=None):
    torch, corr, _ = env
    h = handle or corr.corr_create(s.n_ant, s.n_pol, s.n_fft, s.n_int)
    corr.corr_set_delays(h, s.delay, s.phi0, s.rate)
    corr.corr_set_beam_weights(h, gain, theta, inc, coh)
    if scales is not None:
        corr.corr_set_scales(h, scales)
    corr.corr_set_mode(h, mode, 0, beam_avg)
    xt, n = to_device(torch, s.x)
    corr.corr_integrate_device(h, xt, n_avail=n, g0=g0, stream=torch.cuda.current_stream())
    V = corr.corr_read_visibilities(h)
    B = corr.corr_read_beams(h)
    out = dict(V=V.astype(np.complex128), B=B.astype(np.float64), h=h)
    if want_spec is not None:
        k0, nk = want_spec
        out["Y"] = corr.corr_read_spectra(h, k0, nk, s.n_int).astype(np.complex128)
    return out


def oracle_all(orc, s, chans=None, g0=0):
    Y = orc.fengine(s.x, s.n_ant, s.n_pol, s.n_fft, s.n_int, s.delay, s.phi0, s.rate, g0=g0, chans=chans)
    V = orc.xengine(Y, s.n_ant, s.n_pol)
    return Y, V


def test_tiny_config_fp32_parity(env):
    torch, corr, orc = env
    s = make_config(1)
    r = run_gpu(env, s, want_spec=(0, s.n_fft // 2))
    Y, V = oracle_all(orc, s)
    Bi, Bc = orc.beams(Y, s.n_ant, s.n_pol, s.n_fft)
    e_v = vis_norm_error(r["V"], V, s.n_ant, s.n_pol)
    e_y = max(float(np.abs(r["Y"][i] - Y[i]).max() / np.abs(Y[i]).max()) for i in range(s.n_in))
    e_bi, e_bc = beam_errors(r["B"], Bi, Bc, Y, np.ones(s.n_ant), np.ones(s.n_ant), s.n_pol)
    print(f"tiny fp32: vis {e_v:.2e} spectra {e_y:.2e} beam_inc {e_bi:.2e} beam_coh {e_bc:.2e}")
    assert e_y <= FP32_TOL and e_v <= FP32_TOL and e_bi <= FP32_TOL and e_bc <= FP32_TOL
    corr.corr_destroy(r["h"])


def test_tiny_config_beams_weights_and_averaging(env):
    torch, corr, orc = env
    s = make_config(1)
    rng = np.random.default_rng(3)
    gain = rng.uniform(0.5, 1.5, s.n_ant)
    theta = rng.uniform(-np.pi, np.pi, (s.n_ant, s.n_fft // 2))
    inc = np.array([1, 1, 0, 1], np.uint8)
    coh = np.array([1, 0, 1, 1], np.uint8)
    for beam_avg in (1, 8, 64):
        r = run_gpu(env, s, beam_avg=beam_avg, gain=gain, theta=theta, inc=inc, coh=coh)
        Y, _ = oracle_all(orc, s)
        Bi, Bc = orc.beams(Y, s.n_ant, s.n_pol, s.n_fft, gain=gain.astype(np.float32).astype(np.float64),
                           theta=theta.astype(np.float32).astype(np.float64), inc_mask=inc, coh_mask=coh,
                           beam_avg=beam_avg)
        e_bi, e_bc = beam_errors(r["B"], Bi, Bc, Y, gain, coh, s.n_pol, beam_avg)
        print(f"beam_avg {beam_avg}: inc {e_bi:.2e} coh {e_bc:.2e}")
        assert e_bi <= FP32_TOL and e_bc <= FP32_TOL
        corr.corr_destroy(r["h"])


# channels sampled at GMRT scale: edges, tones, tile boundaries
C2_CHANS = [0, 1, 2, 31, 32, 100, 255, 256, 333, 511, 512, 513, 700, 777, 1000, 1022, 1023]


@pytest.mark.parametrize("n_ant,n_pol,n_fft,n_int", [
    (32, 2, 2048, 64),     # GMRT shape, 8 F-engine tiles, several X stages
    (3, 1, 64, 16),        # smallest FFT, ragged 4-input X tile, one polarisation
    (5, 2, 256, 48),       # ragged tile with two polarisations, 3 F-engine tiles
    (16, 2, 4096, 32),     # largest FFT
    (1, 2, 1024, 16),      # single antenna
    (8, 2, 1024, 256),     # 512 channels x 64 K-blocks: the CUDA-core X-engine splits frames in 4 parts
])
def test_scaled_configs_fp32_parity(env, n_ant, n_pol, n_fft, n_int):
    torch, corr, orc = env
    s = make_config(2, n_ant=n_ant, n_pol=n_pol, n_fft=n_fft, n_int=n_int, seed=2000 + n_fft + n_ant)
    chans = sorted({c for c in C2_CHANS if c < n_fft // 2} | {n_fft // 2 - 1, n_fft // 4})
    r = run_gpu(env, s, want_spec=(0, n_fft // 2))
    Y, V = oracle_all(orc, s, chans=chans)
    Vg = r["V"][chans]
    e_v = vis_norm_error(Vg, V, s.n_ant, s.n_pol)
    Yg = r["Y"][:, :, chans]
    e_y = max(float(np.abs(Yg[i] - Y[i]).max() / np.abs(Y[i]).max()) for i in range(s.n_in))
    Bi, Bc = orc.beams(Y, s.n_ant, s.n_pol, s.n_fft, chans=chans)
    Bg = r["B"][:, :, chans]
    e_bi, e_bc = beam_errors(Bg, Bi, Bc, Y, np.ones(s.n_ant), np.ones(s.n_ant), s.n_pol)
    print(f"{(n_ant, n_pol, n_fft, n_int)}: vis {e_v:.2e} spectra {e_y:.2e} inc {e_bi:.2e} coh {e_bc:.2e}")
    assert e_v <= FP32_TOL and e_y <= FP32_TOL and e_bi <= FP32_TOL and e_bc <= FP32_TOL
    corr.corr_destroy(r["h"])


def _calibrated_scales(env, s):
    torch, corr, _ = env
    r = run_gpu(env, s)
    corr.corr_set_scales(r["h"], None)
    return r["h"]


# GMRT shape, and the 4096-point FFT whose 4-frame CTAs trade channel halves in cluster pairs
# (channels 1023 / 1024 straddle the halves); the int8 form writes bytes in the channel-quad
# layout up to 1024 channels (the 64-point case: 32 channels, 8 quads; 6 inputs per frame)
TC_SHAPES = [dict(n_int=128), dict(n_ant=16, n_fft=4096, n_int=64)]
I8_SHAPES = TC_SHAPES + [dict(n_ant=3, n_fft=64, n_int=48)]
TC_CHANS = {2048: [0, 1, 100, 333, 512, 777, 1023], 4096: [0, 1, 100, 1023, 1024, 1500, 2047],
            64: [0, 1, 3, 4, 16, 30, 31]}


@pytest.mark.parametrize("shape", I8_SHAPES, ids=["gmrt", "fft4096", "fft64"])
def test_i8_bit_exact_on_requantised_spectra(env, shape):
    torch, corr, orc = env
    s = make_config(2, seed=3003, **shape)
    h = _calibrated_scales(env, s)
    r = run_gpu(env, s, mode=corr.CORR_I8, handle=h)
    Vi = corr.corr_read_vis_int(h)
    chans = TC_CHANS[s.n_fft]
    for c in chans:
        q, sc = corr.corr_read_requant(h, c, 1, s.n_int)
        Vo, Vd = orc.xint(q, sc[:, c:c + 1].astype(np.float64), s.n_ant, s.n_pol)
        assert np.array_equal(Vi[c], Vo[0].astype(np.int32)), c
        assert np.abs(r["V"][c] - Vd[0]).max() <= 1e-6 * np.abs(Vd[0]).max()
    # requantisation itself vs the FP64 reading, and accuracy vs FP64 on raw samples
    Y, V = oracle_all(orc, s, chans=chans)
    qg, sc = corr.corr_read_requant(h, 0, s.n_fft // 2, s.n_int)
    qo = orc.requant(Y, sc[:, chans].astype(np.float64))
    mism = np.abs(qg[:, :, chans].astype(int) - qo.astype(int))
    frac = float((mism > 0).mean())
    e_ch = [vis_norm_error(r["V"][c:c + 1], V[j:j + 1], s.n_ant, s.n_pol) for j, c in enumerate(chans)]
    print(f"i8: requant mismatch fraction {frac:.2e} (max {mism.max()}), vis error vs FP64 per channel "
          + " ".join(f"{c}:{e:.1e}" for c, e in zip(chans, e_ch)))
    assert mism.max() <= 1 and frac <= 1e-3
    # quantisation noise of a 4-sigma / 127 step (0.9 % of sigma per value): ~3e-3 normalised at
    # circular channels over these 128 frames; the DC scale takes the full power (its spectrum is
    # real before the fringe rotation): a sqrt(2) coarser step and no clipping, ~5e-3.  A channel
    # where a component beyond 4 sigma was clipped to +-127 (about one value in 16,000) carries
    # that clip in its input's autocorrelation: (x^2 - 16) sigma^2 / (256 sigma^2), 3.5e-2 at 5 sigma
    clipped = [bool((np.abs(qg[:, :, c]) == 127).any()) for c in chans]
    print("channels with a clipped value: " + " ".join(str(c) for c, k in zip(chans, clipped) if k))
    assert chans[0] == 0 and not clipped[0] and e_ch[0] <= 1e-2
    assert all(e <= (4e-2 if k else 1e-2) for e, k in zip(e_ch, clipped))
    corr.corr_destroy(h)


@pytest.mark.parametrize("shape", TC_SHAPES, ids=["gmrt", "fft4096"])
def test_f16_mode_accuracy(env, shape):
    torch, corr, orc = env
    s = make_config(2, seed=3004, **shape)
    h = _calibrated_scales(env, s)
    r = run_gpu(env, s, mode=corr.CORR_F16, handle=h)
    chans = TC_CHANS[s.n_fft]
    Y, V = oracle_all(orc, s, chans=chans)
    e_v = vis_norm_error(r["V"][chans], V, s.n_ant, s.n_pol)
    Bi, Bc = orc.beams(Y, s.n_ant, s.n_pol, s.n_fft, chans=chans)
    e_bi, e_bc = beam_errors(r["B"][:, :, chans], Bi, Bc, Y, np.ones(s.n_ant), np.ones(s.n_ant), s.n_pol)
    print(f"f16: vis error vs FP64 {e_v:.2e}; beams (FP32 spectra) {e_bi:.2e} {e_bc:.2e}")
    # fp16 keeps 11 significant bits of values scaled to ~32 sigma: relative rounding 2^-12 per value,
    # ~1e-4 normalised over 128 frames (measured 1.7e-4); 1e-3 leaves a factor 6
    assert e_v <= 1e-3
    assert e_bi <= FP32_TOL and e_bc <= FP32_TOL
    corr.corr_destroy(h)


@pytest.mark.parametrize("n_ant,n_pol,n_fft,n_int", [
    (32, 2, 2048, 512),    # GMRT shape (64 inputs: paired hi / lo rows), one 512-frame chunk
    (32, 2, 256, 144),     # paired rows, one partial chunk of 9 K-block pairs
    (32, 2, 512, 1040),    # paired rows, two 512-frame chunks and a 16-frame one
    (5, 2, 256, 48),       # ragged rows (R = 20), one short chunk, 3 F-engine tiles
    (3, 1, 64, 16),        # smallest FFT and integration, one polarisation
    (16, 2, 4096, 64),     # 4-frame F-engine CTAs: 8-byte half-row stores of both planes
    (64, 2, 512, 272),     # 256 Gram rows: two work items per channel; ragged last chunk
])
def test_fp32tc_split_tensor_core_parity(env, n_ant, n_pol, n_fft, n_int):
    torch, corr, orc = env
    s = make_config(2, n_ant=n_ant, n_pol=n_pol, n_fft=n_fft, n_int=n_int, seed=5000 + n_fft + n_ant)
    chans = sorted({c for c in C2_CHANS if c < n_fft // 2} | {n_fft // 2 - 1, n_fft // 4})
    r32 = run_gpu(env, s, want_spec=(0, n_fft // 2))
    rtc = run_gpu(env, s, mode=corr.CORR_FP32TC, want_spec=(0, n_fft // 2))
    Y, V = oracle_all(orc, s, chans=chans)
    e_v = vis_norm_error(rtc["V"][chans], V, s.n_ant, s.n_pol)
    e_v32 = vis_norm_error(r32["V"][chans], V, s.n_ant, s.n_pol)
    print(f"{(n_ant, n_pol, n_fft, n_int)}: fp32tc vis {e_v:.2e} (CUDA-core fp32 {e_v32:.2e})")
    assert np.array_equal(rtc["Y"], r32["Y"])       # one F-engine: the same FP32 spectra
    assert np.array_equal(rtc["B"], r32["B"])       # and the same beams
    assert e_v <= FP32_TOL
    for q in (rtc, r32):
        corr.corr_destroy(q["h"])


def test_fp32tc_batch_interplay_and_power_dumps(env):
    torch, corr, orc = env
    s = make_config(1, n_int=64)
    h = corr.corr_create(s.n_ant, s.n_pol, s.n_fft, s.n_int)
    try:
        with pytest.raises(corr.CorrError) as ei:      # a batch member cannot switch to it
            b = corr.corr_batch_create([h])
            try:
                corr.corr_set_mode(h, corr.CORR_FP32TC, 0, 1)
            finally:
                corr.corr_batch_destroy(b)
        assert ei.value.code == -7
        corr.corr_set_mode(h, corr.CORR_FP32TC, 0, 1)
        with pytest.raises(corr.CorrError) as ei:      # nor can an FP32TC handle join a batch
            corr.corr_batch_create([h])
        assert ei.value.code == -1
        # the RFI stage's power dumps come from the same FP32 spectra in both FP32 forms
        corr.corr_set_power_dump(h, 16)
        dumps = {}
        for mode in (corr.CORR_FP32TC, corr.CORR_FP32):
            run_gpu(env, s, mode=mode, handle=h)
            dumps[mode] = corr.corr_read_power_host(h, s.n_int // 16)
        assert np.array_equal(dumps[corr.CORR_FP32TC], dumps[corr.CORR_FP32])
        assert np.all(dumps[corr.CORR_FP32] > 0)
    finally:
        corr.corr_destroy(h)


def test_streaming_push_matches_oracle_across_integrations(env):
    """Two consecutive integrations pushed from host memory in uneven chunks: the
    delay overlap carries over and the fringe phase follows the global frame count."""
    torch, corr, orc = env
    base = make_config(1, n_int=128, tail=3)           # two integrations of 64 frames
    n_int = 64
    h = corr.corr_create(base.n_ant, base.n_pol, base.n_fft, n_int)
    corr.corr_set_max_delay(h, 3)
    corr.corr_set_delays(h, base.delay, base.phi0, base.rate)
    x = base.x
    cuts = [0, 1000, 17001, 33000, x.shape[1]]
    results = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        before = corr.corr_info(h)["completed"]
        corr.corr_push_samples(h, np.ascontiguousarray(x[:, a:b]), seq=a)
        del before
        if b >= n_int * 512 + 3 and len(results) == 0:
            results.append(corr.corr_read_visibilities(h).astype(np.complex128))
    results.append(corr.corr_read_visibilities(h).astype(np.complex128))
    for g, Vg in enumerate(results):
        sub = x[:, g * n_int * 512:]
        Y = orc.fengine(sub, base.n_ant, base.n_pol, base.n_fft, n_int, base.delay, base.phi0, base.rate, g0=g * n_int)
        V = orc.xengine(Y, base.n_ant, base.n_pol)
        e = vis_norm_error(Vg, V, base.n_ant, base.n_pol)
        print(f"streamed integration {g}: {e:.2e}")
        assert e <= FP32_TOL
    # a sequence gap drops the partial integration and reports data loss
    with pytest.raises(corr.CorrError) as ei:
        corr.corr_push_samples(h, np.ascontiguousarray(x[:, :100]), seq=10 ** 9)
    assert ei.value.code == -4
    corr.corr_destroy(h)


def test_delay_range_and_state_errors(env):
    torch, corr, orc = env
    s = make_config(1)
    h = corr.corr_create(s.n_ant, s.n_pol, s.n_fft, s.n_int)
    with pytest.raises(corr.CorrError) as ei:
        corr.corr_set_delays(h, [-1.0, 0, 0, 0], [0] * 4, [0] * 4)
    assert ei.value.code == -2
    with pytest.raises(corr.CorrError) as ei:
        corr.corr_read_visibilities(h, blocking=0)
    assert ei.value.code == -3
    corr.corr_set_mode(h, corr.CORR_I8, 0, 1)
    xt, n = to_device(torch, s.x)
    with pytest.raises(corr.CorrError) as ei:               # no scales yet
        corr.corr_integrate_device(h, xt, n_avail=n, stream=torch.cuda.current_stream())
    assert ei.value.code == -7
    corr.corr_set_mode(h, corr.CORR_FP32, 0, 1)
    corr.corr_set_delays(h, [0, 0, 0, 40.0], [0] * 4, [0] * 4)
    with pytest.raises(corr.CorrError) as ei:               # buffer too short for the delay
        corr.corr_integrate_device(h, xt, n_avail=n, stream=torch.cuda.current_stream())
    assert ei.value.code == -2
    corr.corr_destroy(h)


# ----------------------------------------------------------- full GMRT scale

@pytest.fixture(scope="module")
def c2_full():
    return make_config(2)      # 32 ant x 2 pol, 2048-pt FFT, 8192 spectra (~0.25 s of data)


FULL_CHANS = [0, 100, 333, 777, 1023]


def test_full_scale_fp32_sampled_channels(env, c2_full):
    torch, corr, orc = env
    s = c2_full
    r = run_gpu(env, s)
    Y, V = oracle_all(orc, s, chans=FULL_CHANS)
    e_v = vis_norm_error(r["V"][FULL_CHANS], V, s.n_ant, s.n_pol)
    # beams on a sample of frames at those channels
    Bi, Bc = orc.beams(Y, s.n_ant, s.n_pol, s.n_fft, chans=FULL_CHANS)
    e_bi, e_bc = beam_errors(r["B"][:, :, FULL_CHANS], Bi, Bc, Y, np.ones(s.n_ant), np.ones(s.n_ant), s.n_pol)
    # invariants at every channel: autos real and non-negative, RL* = conj(LR*)
    Vall = r["V"]
    for a in range(s.n_ant):
        b = a * s.n_ant - a * (a - 1) // 2
        assert np.all(Vall[:, b, 0].real >= 0) and np.all(Vall[:, b, 3].real >= 0)
        assert np.allclose(Vall[:, b, 1], np.conj(Vall[:, b, 2]), rtol=1e-5, atol=1e-3 * np.abs(Vall[:, b, 0]).max())
    print(f"full scale fp32: vis {e_v:.2e} beams {e_bi:.2e} {e_bc:.2e}")
    assert e_v <= FP32_TOL and e_bi <= FP32_TOL and e_bc <= FP32_TOL
    corr.corr_set_scales(r["h"], None)
    r2 = run_gpu(env, s, mode=corr.CORR_I8, handle=r["h"])
    Vi = corr.corr_read_vis_int(r["h"])
    for c in FULL_CHANS:
        q, sc = corr.corr_read_requant(r["h"], c, 1, s.n_int)
        Vo, _ = orc.xint(q, sc[:, c:c + 1].astype(np.float64), s.n_ant, s.n_pol)
        assert np.array_equal(Vi[c], Vo[0].astype(np.int32)), c
    e_i8 = vis_norm_error(r2["V"][FULL_CHANS], V, s.n_ant, s.n_pol)
    print(f"full scale i8 vs FP64: {e_i8:.2e}")
    assert e_i8 <= 5e-2
    assert math.isfinite(e_i8)
    # the FP32 X-engine on the tensor cores: 64 chunks of 128 frames, the same FP32 bound
    r3 = run_gpu(env, s, mode=corr.CORR_FP32TC, handle=r["h"])
    e_tc = vis_norm_error(r3["V"][FULL_CHANS], V, s.n_ant, s.n_pol)
    print(f"full scale fp32tc vs FP64: {e_tc:.2e}")
    assert e_tc <= FP32_TOL
    assert np.array_equal(r3["B"], r["B"])
    corr.corr_destroy(r["h"])


def test_rail_value_inputs(env):
    """int8 edge values in the raw samples: -128 (which the generator never produces) and long
    saturated runs of +-127 at every input (a strong burst), through the FP32, FP32TC and int8
    forms.  The largest spectral value then reaches N/2 x 128 x 2 = 2^18 at N = 2048, the bound
    the FP32TC split's 2^-3 scale keeps below fp16's range."""
    torch, corr, orc = env
    s = make_config(2, n_ant=8, n_pol=2, n_fft=2048, n_int=32, seed=3009)
    x = s.x.copy()
    rng = np.random.default_rng(3010)
    n = x.shape[1]
    x[:, 5000:5000 + 3 * 2048] = -128                        # three whole frames at -128 everywhere
    for i in range(x.shape[0]):                              # +-127 runs of 1-4 frames, random signs
        for _ in range(4):
            t0 = int(rng.integers(0, n - 4 * 2048))
            x[i, t0:t0 + int(rng.integers(2048, 4 * 2048))] = 127 if rng.random() < 0.5 else -127
    x[:, ::97] = -128                                        # scattered -128 samples
    s.x = x
    assert (s.x == -128).sum() > 0
    chans = [0, 1, 100, 333, 512, 1023]
    Yall = orc.fengine(s.x, s.n_ant, s.n_pol, s.n_fft, s.n_int, s.delay, s.phi0, s.rate)
    Y = Yall[:, :, chans]
    V = orc.xengine(Y, s.n_ant, s.n_pol)
    Bi_all, Bc_all = orc.beams(Yall, s.n_ant, s.n_pol, s.n_fft)
    # a frame of constant samples has power only at DC, so a per-channel relative beam error is not
    # defined in its other channels: beams are judged relative to the larger of their own value and
    # the frame's mean power over all channels (the scale of an FP32 FFT's rounding, by Parseval)
    frame_scale = np.maximum(Bi_all, Bi_all.mean(axis=1, keepdims=True))
    res = {}
    for mode, name in ((corr.CORR_FP32, "fp32"), (corr.CORR_FP32TC, "fp32tc")):
        r = run_gpu(env, s, mode=mode, want_spec=(0, s.n_fft // 2))
        e_v = vis_norm_error(r["V"][chans], V, s.n_ant, s.n_pol)
        Yg = r["Y"][:, :, chans]
        e_y = max(float(np.abs(Yg[i] - Y[i]).max() / np.abs(Y[i]).max()) for i in range(s.n_in))
        e_bi = float(np.max(np.abs(r["B"][0] - Bi_all) / frame_scale))
        e_bc = float(np.max(np.abs(r["B"][1] - Bc_all) / np.maximum(Bc_all, s.n_ant * frame_scale)))
        print(f"rails {name}: vis {e_v:.2e} spectra {e_y:.2e} beams (per frame scale) {e_bi:.2e} {e_bc:.2e}")
        assert e_v <= FP32_TOL and e_y <= FP32_TOL and e_bi <= FP32_TOL and e_bc <= FP32_TOL
        res[name] = r
        if name == "fp32":
            corr.corr_set_scales(r["h"], None)
            r8 = run_gpu(env, s, mode=corr.CORR_I8, handle=r["h"])
            Vi = corr.corr_read_vis_int(r["h"])
            for c in chans:
                q, sc = corr.corr_read_requant(r["h"], c, 1, s.n_int)
                Vo, _ = orc.xint(q, sc[:, c:c + 1].astype(np.float64), s.n_ant, s.n_pol)
                assert np.array_equal(Vi[c], Vo[0].astype(np.int32)), c
            assert np.isfinite(r8["V"]).all()
        corr.corr_destroy(r["h"])
