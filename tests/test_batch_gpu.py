"""Several uneven sub-arrays in one graph-captured launch (corr_batch_*): every sub-array's
integer visibilities equal the oracle's int64 MAC on its own requantised spectra, the batch
agrees with the single-handle path (to rare +-1 requantisation flips), the graph replays correctly with new samples and frame
counters, and the autotuner's stage choice leaves the results unchanged."""
import numpy as np
import pytest

from fxhelp import vis_norm_error
from synth import make_config

pytestmark = pytest.mark.gpu

# (n_ant, n_pol, n_fft, n_int): uneven antenna counts and FFT sizes; 64 x 2 exercises the
# two row blocks of a 256-row Gram, the 4096-point FFT the cluster-paired F-engine CTAs
SUBS = [(4, 2, 512, 64), (8, 2, 1024, 48), (16, 2, 2048, 32), (64, 2, 256, 32), (6, 2, 4096, 32)]
CHANS = [0, 1, 57, 100, 1023, 1024, 2047]


@pytest.fixture(scope="module")
def env(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0910_1517_gb300 import build, corr
    build.build()
    corr.load()
    return torch, corr, orc


def _dev(torch, x):
    n_in, n = x.shape
    xt = torch.zeros((n_in, ((n + 15) // 16) * 16 + 16), dtype=torch.int8, device="cuda")
    xt[:, :n] = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return xt, n


def _handles(torch, corr, seeds, mode):
    """Handles with delays set and scales calibrated by one FP32 integration each."""
    hs, streams, xs = [], [], []
    st = torch.cuda.current_stream()
    for (na, npol, nfft, nint), seed in zip(SUBS, seeds):
        s = make_config(2, n_ant=na, n_pol=npol, n_fft=nfft, n_int=nint, seed=seed)
        h = corr.corr_create(na, npol, nfft, nint)
        corr.corr_set_delays(h, s.delay, s.phi0, s.rate)
        xt, n = _dev(torch, s.x)
        corr.corr_integrate_device(h, xt, n_avail=n, stream=st)
        corr.corr_set_scales(h, None)
        corr.corr_set_mode(h, mode, 0, 1)
        hs.append(h)
        streams.append(s)
        xs.append((xt, n))
    return hs, streams, xs


def _check_exact(corr, orc, h, s):
    Vi = corr.corr_read_vis_int(h)
    for c in CHANS:
        if c >= s.n_fft // 2:
            continue
        q, sc = corr.corr_read_requant(h, c, 1, s.n_int)
        Vo, _ = orc.xint(q, sc[:, c:c + 1].astype(np.float64), s.n_ant, s.n_pol)
        assert np.array_equal(Vi[c], Vo[0].astype(np.int32)), (s.n_ant, c)
    return Vi


def test_batch_int8_exact_matches_oracle_and_single_handle(env):
    torch, corr, orc = env
    hs, streams, xs = _handles(torch, corr, [701, 702, 703, 704, 705], corr.CORR_I8)
    st = torch.cuda.current_stream()
    b = corr.corr_batch_create(hs)
    try:
        corr.corr_batch_integrate_device(b, [x for x, _ in xs], n_avail=[n for _, n in xs], stream=st)
        batch_vi = [_check_exact(corr, orc, h, s) for h, s in zip(hs, streams)]
        batch_q = [corr.corr_read_requant(h, 0, s.n_fft // 2, s.n_int)[0] for h, s in zip(hs, streams)]
        # the same integrations one handle at a time: exact against the oracle on their own int8
        # spectra, and those spectra equal the batch's but for rare +-1 flips where the two
        # F-engine kernels (the batched launch and the single-handle warp-FFT kernel) round a
        # requantised value that sits within an FP32 ulp of a rounding tie differently
        for h, s, (xt, n), qb in zip(hs, streams, xs, batch_q):
            corr.corr_integrate_device(h, xt, n_avail=n, stream=st)
            _check_exact(corr, orc, h, s)
            qs = corr.corr_read_requant(h, 0, s.n_fft // 2, s.n_int)[0]
            d = np.abs(qs.astype(np.int16) - qb.astype(np.int16))
            print(f"batch vs single {s.n_ant} ant {s.n_fft}-pt: {int((d > 0).sum())} of {d.size} int8 values differ")
            assert d.max() <= 1 and (d > 0).mean() <= 1e-4
        # replay the graph with other samples and a later frame counter
        for s_old, h, (xt, n) in zip(streams, hs, xs):
            s2 = make_config(2, n_ant=s_old.n_ant, n_pol=s_old.n_pol, n_fft=s_old.n_fft, n_int=s_old.n_int,
                             seed=s_old.recipe["seed"] + 50)
            xt[:, :n] = torch.from_numpy(s2.x).cuda()
        g0 = [3 * s.n_int for s in streams]
        corr.corr_batch_integrate_device(b, [x for x, _ in xs], n_avail=[n for _, n in xs], g0=g0, stream=st)
        for s_old, h, (xt, n), g in zip(streams, hs, xs, g0):
            s2 = make_config(2, n_ant=s_old.n_ant, n_pol=s_old.n_pol, n_fft=s_old.n_fft, n_int=s_old.n_int,
                             seed=s_old.recipe["seed"] + 50)
            _check_exact(corr, orc, h, s2)
            # the handles keep the delay model they were given; only the samples are new
            # the replay used the new samples and frame counter: the FP64 spectra with that g0,
            # requantised with the GPU's scales, give the same visibilities up to rare +-1 flips
            ch = CHANS[:3]
            Y = orc.fengine(s2.x, s2.n_ant, s2.n_pol, s2.n_fft, s2.n_int, s_old.delay, s_old.phi0, s_old.rate,
                            g0=g, chans=ch)
            _, sc = corr.corr_read_requant(h, 0, 0, s2.n_int)
            sc64 = sc[:, ch].astype(np.float64)
            _, Vq = orc.xint(orc.requant(Y, sc64), sc64, s2.n_ant, s2.n_pol)
            Vg = corr.corr_read_visibilities(h).astype(np.complex128)[ch]
            e = vis_norm_error(Vg, Vq, s2.n_ant, s2.n_pol)
            print(f"batch replay {s2.n_ant} ant {s2.n_fft}-pt: vs oracle requantisation {e:.2e}, "
                  f"vs FP64 {vis_norm_error(Vg, orc.xengine(Y, s2.n_ant, s2.n_pol), s2.n_ant, s2.n_pol):.2e}")
            assert e < 2e-3
    finally:
        corr.corr_batch_destroy(b)
        for h in hs:
            corr.corr_destroy(h)


def test_batch_replays_with_new_sample_buffers(env):
    """Later calls may pass other sample buffers: the graph's F-engine nodes take the new pointers
    (the 4096-point sub-array, whose F-engine runs in 2-CTA clusters, captures the graph again),
    and switching back to the first buffers gives their results again."""
    torch, corr, orc = env
    hs, streams, xs = _handles(torch, corr, [711, 712, 713, 714, 715], corr.CORR_I8)
    st = torch.cuda.current_stream()
    b = corr.corr_batch_create(hs)
    try:
        corr.corr_batch_integrate_device(b, [x for x, _ in xs], n_avail=[n for _, n in xs], stream=st)
        first = [corr.corr_read_vis_int(h) for h in hs]
        news = [make_config(2, n_ant=s.n_ant, n_pol=s.n_pol, n_fft=s.n_fft, n_int=s.n_int, seed=s.recipe["seed"] + 60)
                for s in streams]
        xs2 = [_dev(torch, s2.x) for s2 in news]        # other allocations: other pointers
        assert all(a.data_ptr() != c.data_ptr() for (a, _), (c, _) in zip(xs, xs2))
        corr.corr_batch_integrate_device(b, [x for x, _ in xs2], n_avail=[n for _, n in xs2], stream=st)
        for h, s, s2, v in zip(hs, streams, news, first):
            _check_exact(corr, orc, h, s2)
            assert not np.array_equal(corr.corr_read_vis_int(h), v)
            # the new buffers were read: the FP64 spectra of the new samples (the handle's own delay
            # model), requantised with the GPU's scales, give the same visibilities up to rare flips
            ch = CHANS[:3]
            Y = orc.fengine(s2.x, s.n_ant, s.n_pol, s.n_fft, s.n_int, s.delay, s.phi0, s.rate, chans=ch)
            _, sc = corr.corr_read_requant(h, 0, 0, s.n_int)
            sc64 = sc[:, ch].astype(np.float64)
            _, Vq = orc.xint(orc.requant(Y, sc64), sc64, s.n_ant, s.n_pol)
            Vg = corr.corr_read_visibilities(h).astype(np.complex128)[ch]
            assert vis_norm_error(Vg, Vq, s.n_ant, s.n_pol) < 2e-3, (s.n_ant, s.n_fft)
        corr.corr_batch_integrate_device(b, [x for x, _ in xs], n_avail=[n for _, n in xs], stream=st)
        for h, v in zip(hs, first):
            assert np.array_equal(corr.corr_read_vis_int(h), v)
    finally:
        corr.corr_batch_destroy(b)
        for h in hs:
            corr.corr_destroy(h)


def test_batch_autotune_keeps_results(env):
    torch, corr, orc = env
    hs, streams, xs = _handles(torch, corr, [801, 802, 803, 804, 805], corr.CORR_I8)
    st = torch.cuda.current_stream()
    b = corr.corr_batch_create(hs)
    try:
        corr.corr_batch_integrate_device(b, [x for x, _ in xs], n_avail=[n for _, n in xs], stream=st)
        before = [corr.corr_read_vis_int(h) for h in hs]
        ks, ms = corr.corr_batch_tune(b, len(hs))
        print("tuned frames per stage", ks.tolist(), "ms", [round(float(v), 4) for v in ms])
        assert all(k >= 32 for k in ks) and all(m > 0 for m in ms)
        corr.corr_batch_integrate_device(b, [x for x, _ in xs], n_avail=[n for _, n in xs], stream=st)
        for h, v in zip(hs, before):
            assert np.array_equal(corr.corr_read_vis_int(h), v)
    finally:
        corr.corr_batch_destroy(b)
        for h in hs:
            corr.corr_destroy(h)


def test_batch_fp32_matches_single_handle(env):
    torch, corr, orc = env
    hs, streams, xs = _handles(torch, corr, [901, 902, 903, 904, 905], corr.CORR_FP32)
    st = torch.cuda.current_stream()
    single = []
    for h, (xt, n) in zip(hs, xs):
        corr.corr_integrate_device(h, xt, n_avail=n, stream=st)
        single.append(corr.corr_read_visibilities(h).astype(np.complex128))
    b = corr.corr_batch_create(hs)
    try:
        corr.corr_batch_integrate_device(b, [x for x, _ in xs], n_avail=[n for _, n in xs], stream=st)
        for h, s, v in zip(hs, streams, single):
            vb = corr.corr_read_visibilities(h).astype(np.complex128)
            assert vis_norm_error(vb, v, s.n_ant, s.n_pol) <= 1e-6
    finally:
        corr.corr_batch_destroy(b)
        for h in hs:
            corr.corr_destroy(h)


def test_batch_with_the_64_antenna_4096_point_subarray(env):
    """Config 4's largest sub-array, (64 ant, 2 pol, 4096-pt), at 256 spectra beside a small one:
    the two-item 256-row Gram with the cluster-paired 4096-point F-engine.  Integer visibilities
    equal the oracle's int64 MAC on the exported int8 spectra; against the FP64 oracle on raw
    samples the int8 form stays within its quantisation bound (1e-2, as the single-handle test)."""
    torch, corr, orc = env
    subs = [(64, 2, 4096, 256, 721), (8, 2, 512, 256, 722)]
    st = torch.cuda.current_stream()
    hs, streams, xs = [], [], []
    for na, npol, nfft, nint, seed in subs:
        s = make_config(2, n_ant=na, n_pol=npol, n_fft=nfft, n_int=nint, seed=seed)
        h = corr.corr_create(na, npol, nfft, nint)
        corr.corr_set_delays(h, s.delay, s.phi0, s.rate)
        xt, n = _dev(torch, s.x)
        corr.corr_integrate_device(h, xt, n_avail=n, stream=st)
        corr.corr_set_scales(h, None)
        corr.corr_set_mode(h, corr.CORR_I8, 0, 1)
        hs.append(h)
        streams.append(s)
        xs.append((xt, n))
    b = corr.corr_batch_create(hs)
    try:
        corr.corr_batch_integrate_device(b, [x for x, _ in xs], n_avail=[n for _, n in xs], stream=st)
        for h, s in zip(hs, streams):
            _check_exact(corr, orc, h, s)
            ch = [c for c in (0, 1, 100, 1023, 1024, 2047) if c < s.n_fft // 2]
            Y = orc.fengine(s.x, s.n_ant, s.n_pol, s.n_fft, s.n_int, s.delay, s.phi0, s.rate, chans=ch)
            Vg = corr.corr_read_visibilities(h).astype(np.complex128)[ch]
            e = vis_norm_error(Vg, orc.xengine(Y, s.n_ant, s.n_pol), s.n_ant, s.n_pol)
            print(f"batch {s.n_ant} ant {s.n_fft}-pt x {s.n_int}: int8 vs FP64 {e:.2e}")
            assert e <= 1e-2
    finally:
        corr.corr_batch_destroy(b)
        for h in hs:
            corr.corr_destroy(h)
