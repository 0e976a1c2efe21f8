"""Multiple phased beams with full-polar products or voltages (Sec. 2.2, 5) on the GPU against
the FP64 oracle on the same seeded inputs; the coherent-weight beam reproduces the coherent beam."""
import numpy as np
import pytest

from synth import make_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(orc):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0910_1517_gb300 import build, corr
    build.build()
    corr.load()
    return torch, corr, orc


def _weights(n_beams, n_ant, nch, seed):
    rng = np.random.default_rng(seed)
    g = rng.uniform(0.3, 1.2, (n_beams, n_ant, 1))
    return g * np.exp(1j * rng.uniform(-np.pi, np.pi, (n_beams, n_ant, nch)))


def _run(env, s, W, products, avg, mode=0):
    torch, corr, _ = env
    h = corr.corr_create(s.n_ant, s.n_pol, s.n_fft, s.n_int)
    corr.corr_set_delays(h, s.delay, s.phi0, s.rate)
    corr.corr_set_mode(h, mode, 0, 1)
    corr.corr_set_multibeam(h, W, products, avg)
    n = s.x.shape[1]
    xt = torch.zeros((s.n_in, ((n + 15) // 16) * 16 + 16), dtype=torch.int8, device="cuda")
    xt[:, :n] = torch.from_numpy(np.ascontiguousarray(s.x)).cuda()
    corr.corr_integrate_device(h, xt, n_avail=n, stream=torch.cuda.current_stream())
    B = corr.corr_read_multibeam(h, W.shape[0], s.n_int // avg).astype(np.float64)
    beams = corr.corr_read_beams(h).astype(np.float64)
    corr.corr_destroy(h)
    return B, beams


def _err(B, Bo, products):
    """Errors relative to each (beam, channel)'s mean beam power over the integration (single-frame
    powers are exponentially distributed, so point-wise relative errors would judge near-zero
    values): voltages against its square root."""
    if products == 1:
        p = (Bo ** 2).sum(axis=-1).mean(axis=1, keepdims=True)[..., None]
        return float((np.abs(B - Bo) / np.sqrt(p)).max())
    p = (Bo[..., 0] + Bo[..., 1]).mean(axis=1, keepdims=True)[..., None]
    return float((np.abs(B - Bo) / p).max())


@pytest.mark.parametrize("n_beams,products,avg", [
    (12, 0, 1), (12, 0, 4), (3, 0, 64), (1, 0, 128), (64, 0, 32), (12, 1, 1), (48, 0, 1), (33, 1, 1)])
def test_multibeam_matches_oracle(env, n_beams, products, avg):
    torch, corr, orc = env
    s = make_config(2, n_ant=8, n_fft=512, n_int=128, seed=7000 + n_beams + avg)
    W = _weights(n_beams, s.n_ant, s.n_fft // 2, 70 + n_beams)
    B, _ = _run(env, s, W, products, avg)
    Y = orc.fengine(s.x, s.n_ant, s.n_pol, s.n_fft, s.n_int, s.delay, s.phi0, s.rate)
    Bo = orc.multibeam(Y, s.n_ant, s.n_pol, W.astype(np.complex64).astype(np.complex128), products, avg)
    e = _err(B, Bo, products)
    print(f"multibeam n_beams {n_beams} products {products} avg {avg}: {e:.2e}")
    assert e <= 1e-5


@pytest.mark.parametrize("n_ant,n_pol,n_fft,n_beams,products,avg", [
    (32, 2, 2048, 16, 0, 32),      # GMRT-scale antennas, 16 beams: the CUDA-core form
    (32, 2, 2048, 40, 0, 32),      # the same with 40 beams: the tensor-core form, 8-frame K-blocks
    (32, 2, 4096, 64, 0, 128),     # 4-frame K-blocks, 64 beams, windows across stages (tensor cores)
    (5, 1, 1024, 30, 1, 1),        # one polarisation, K padded, voltages (tensor cores)
    (72, 1, 512, 30, 0, 8)])       # K = 144 > 128: the CUDA-core form even with 30 beams
def test_multibeam_shapes_match_oracle(env, n_ant, n_pol, n_fft, n_beams, products, avg):
    torch, corr, orc = env
    s = make_config(2, n_ant=n_ant, n_pol=n_pol, n_fft=n_fft, n_int=256, seed=7300 + n_ant + n_fft)
    W = _weights(n_beams, s.n_ant, s.n_fft // 2, 73 + n_beams)
    B, _ = _run(env, s, W, products, avg)
    chans = [0, 1, 77, s.n_fft // 2 - 1]
    Y = orc.fengine(s.x, s.n_ant, s.n_pol, s.n_fft, s.n_int, s.delay, s.phi0, s.rate, chans=chans)
    Bo = orc.multibeam(Y, s.n_ant, s.n_pol, W[:, :, chans].astype(np.complex64).astype(np.complex128), products, avg)
    e = _err(B[:, :, chans], Bo, products)
    print(f"multibeam {n_ant}x{n_pol} N {n_fft} beams {n_beams} products {products} avg {avg}: {e:.2e}")
    assert e <= 1e-5


def test_multibeam_coherent_weights_reproduce_the_coherent_beam_and_fp32tc(env):
    torch, corr, orc = env
    s = make_config(2, n_ant=8, n_fft=512, n_int=128, seed=7100)
    W = np.ones((2, s.n_ant, s.n_fft // 2), complex)     # beam 0: the default coherent beam (all antennas, unit gains)
    W[1, :4] = 0.0                                        # beam 1: antennas 4-7 only
    B, beams = _run(env, s, W, 0, 1)
    coh = beams[1]
    assert np.allclose(B[0, ..., 0] + B[0, ..., 1], coh, rtol=1e-5, atol=1e-6 * coh.max())
    B2, _ = _run(env, s, W, 0, 1, mode=corr_mode(env, "FP32TC"))
    assert np.array_equal(B2, B)                          # the same FP32 spectra in both FP32 forms


def corr_mode(env, name):
    return getattr(env[1], "CORR_" + name)


def test_multibeam_arguments(env):
    torch, corr, orc = env
    h = corr.corr_create(4, 2, 256, 64)
    W = np.ones((2, 4, 128), complex)
    try:
        for products, avg in ((0, 3), (0, 128), (1, 2), (5, 1)):
            with pytest.raises(corr.CorrError) as ei:
                corr.corr_set_multibeam(h, W, products, avg)
            assert ei.value.code == -1
        with pytest.raises(corr.CorrError) as ei:
            corr.corr_set_multibeam(h, np.ones((65, 4, 128), complex), 0, 1)
        assert ei.value.code == -1
        with pytest.raises(corr.CorrError) as ei:
            corr.corr_read_multibeam(h, 2, 64)
        assert ei.value.code == -7                        # off
        corr.corr_set_multibeam(h, W, 0, 1)
        corr.corr_set_scales(h, np.ones((8, 128), np.float32))
        corr.corr_set_mode(h, corr.CORR_I8, 0, 1)
        s = make_config(1, n_fft=256, n_int=64)
        xt = torch.zeros((8, ((s.x.shape[1] + 15) // 16) * 16 + 16), dtype=torch.int8, device="cuda")
        xt[:, :s.x.shape[1]] = torch.from_numpy(np.ascontiguousarray(s.x)).cuda()
        with pytest.raises(corr.CorrError) as ei:         # no FP32 spectra in the int8 form
            corr.corr_integrate_device(h, xt, n_avail=s.x.shape[1], stream=torch.cuda.current_stream())
        assert ei.value.code == -7
    finally:
        corr.corr_destroy(h)
