"""ADC-format 4-bit ingest (Sec. 2.3.1, 2.3.2) on the GPU: packed card streams give exactly the
spectra, visibilities and beams of the oracle-unpacked int8 rows, through the device entry
point and through the streaming push (uneven chunks)."""
import numpy as np
import pytest

from synth import make_config

pytestmark = pytest.mark.gpu

N_ANT, N_POL, N_FFT, N_INT = 8, 2, 512, 64


@pytest.fixture(scope="module")
def env(orc):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0910_1517_gb300 import build, corr
    build.build()
    corr.load()
    return torch, corr, orc


def _packed(seed=8800, n_int=N_INT, extra=0):
    s = make_config(2, n_ant=N_ANT, n_pol=N_POL, n_fft=N_FFT, n_int=n_int, seed=seed)
    x4 = np.clip(np.rint(s.x.astype(np.float64) / 5.0), -8, 7).astype(np.int8)   # 4-bit samples
    n = x4.shape[1]
    nib = (x4.astype(np.int16) & 0xF).astype(np.uint8)
    packed = np.zeros((s.n_in // 4, 2 * n + extra), np.uint8)
    for c in range(s.n_in // 4):
        packed[c, 0:2 * n:2] = nib[4 * c] | (nib[4 * c + 1] << 4)
        packed[c, 1:2 * n:2] = nib[4 * c + 2] | (nib[4 * c + 3] << 4)
    return s, packed, n


def _handle(corr, s):
    h = corr.corr_create(s.n_ant, s.n_pol, s.n_fft, s.n_int)
    corr.corr_set_delays(h, s.delay, s.phi0, s.rate)
    return h


def test_device_4bit_integration_equals_the_unpacked_rows(env):
    torch, corr, orc = env
    s, packed, n = _packed(extra=6)
    rows = orc.unpack4(packed, n)
    h4, h8 = _handle(corr, s), _handle(corr, s)
    try:
        pt = torch.from_numpy(packed).cuda()
        corr.corr_integrate_4bit_device(h4, pt, n, stream=torch.cuda.current_stream())
        xt = torch.zeros((s.n_in, ((n + 15) // 16) * 16 + 16), dtype=torch.int8, device="cuda")
        xt[:, :n] = torch.from_numpy(rows).cuda()
        corr.corr_integrate_device(h8, xt, n_avail=n, stream=torch.cuda.current_stream())
        assert np.array_equal(corr.corr_read_visibilities(h4), corr.corr_read_visibilities(h8))
        assert np.array_equal(corr.corr_read_beams(h4), corr.corr_read_beams(h8))
        assert np.array_equal(corr.corr_read_spectra(h4, 0, N_FFT // 2, s.n_int),
                              corr.corr_read_spectra(h8, 0, N_FFT // 2, s.n_int))
        # and against the FP64 oracle on the unpacked rows
        from fxhelp import vis_norm_error
        Y = orc.fengine(rows, s.n_ant, s.n_pol, s.n_fft, s.n_int, s.delay, s.phi0, s.rate, chans=[1, 77, 200])
        V = orc.xengine(Y, s.n_ant, s.n_pol)
        assert vis_norm_error(corr.corr_read_visibilities(h4)[[1, 77, 200]].astype(np.complex128), V,
                              s.n_ant, s.n_pol) <= 1e-5
    finally:
        corr.corr_destroy(h4)
        corr.corr_destroy(h8)


def test_streaming_4bit_push_equals_the_int8_push(env):
    torch, corr, orc = env
    s, packed, n = _packed(8900, n_int=3 * N_INT)
    rows = orc.unpack4(packed, n)
    body = N_INT * N_FFT
    got = {}
    for kind in ("4bit", "int8"):
        h = corr.corr_create(s.n_ant, s.n_pol, s.n_fft, N_INT)
        try:
            corr.corr_set_delays(h, s.delay, s.phi0, s.rate)
            cuts = [0, 777, 20001, body + 5, 2 * body + 2048]
            for a, b in zip(cuts[:-1], cuts[1:]):
                if kind == "4bit":
                    corr.corr_push_samples_4bit(h, np.ascontiguousarray(packed[:, 2 * a:2 * b]), b - a, seq=a)
                else:
                    corr.corr_push_samples(h, np.ascontiguousarray(rows[:, a:b]), seq=a)
            got[kind] = (corr.corr_read_visibilities(h), corr.corr_read_beams(h))
        finally:
            corr.corr_destroy(h)
    assert np.array_equal(got["4bit"][0], got["int8"][0]) and np.array_equal(got["4bit"][1], got["int8"][1])


def test_device_4bit_from_a_pointer_off_16_byte_boundaries(env):
    # packed rows starting 2 bytes past an aligned address with an odd row pitch (in 2-byte
    # units): the unpack's 2-byte load path for every card, 16-byte loads for none
    torch, corr, orc = env
    s, packed, n = _packed(8810)
    rows = orc.unpack4(packed, n)
    h4, h8 = _handle(corr, s), _handle(corr, s)
    try:
        width = 2 * n + (2 if n % 2 == 0 else 4)          # = 2 (mod 4)
        big = torch.zeros((packed.shape[0], width), dtype=torch.uint8, device="cuda")
        big[:, 2:2 + 2 * n] = torch.from_numpy(packed).cuda()
        view = big[:, 2:2 + 2 * n]
        assert view.data_ptr() % 16 == 2 and view.stride(0) % 4 == 2
        corr.corr_integrate_4bit_device(h4, view, n, stream=torch.cuda.current_stream())
        xt = torch.zeros((s.n_in, ((n + 15) // 16) * 16 + 16), dtype=torch.int8, device="cuda")
        xt[:, :n] = torch.from_numpy(rows).cuda()
        corr.corr_integrate_device(h8, xt, n_avail=n, stream=torch.cuda.current_stream())
        assert np.array_equal(corr.corr_read_visibilities(h4), corr.corr_read_visibilities(h8))
        assert np.array_equal(corr.corr_read_beams(h4), corr.corr_read_beams(h8))
    finally:
        corr.corr_destroy(h4)
        corr.corr_destroy(h8)


def test_streaming_pushes_mixing_4bit_and_int8(env):
    # 4-bit pushes (unpacked on their own stream) and int8 pushes (copied on the copy stream)
    # interleaved on one handle, at cuts that leave every output alignment: the rings see the
    # same samples in the same order as with int8 pushes alone
    torch, corr, orc = env
    s, packed, n = _packed(8950, n_int=3 * N_INT)
    rows = orc.unpack4(packed, n)
    body = N_INT * N_FFT
    cuts = [0, 5, 4099, 4100, 17000, body - 3, body + 9, 2 * body + 1, 2 * body + 2048]
    got = {}
    for kind in ("mixed", "int8"):
        h = corr.corr_create(s.n_ant, s.n_pol, s.n_fft, N_INT)
        try:
            corr.corr_set_delays(h, s.delay, s.phi0, s.rate)
            for j, (a, b) in enumerate(zip(cuts[:-1], cuts[1:])):
                if kind == "mixed" and j % 2 == 0:
                    corr.corr_push_samples_4bit(h, np.ascontiguousarray(packed[:, 2 * a:2 * b]), b - a, seq=a)
                else:
                    corr.corr_push_samples(h, np.ascontiguousarray(rows[:, a:b]), seq=a)
            got[kind] = (corr.corr_read_visibilities(h), corr.corr_read_beams(h))
        finally:
            corr.corr_destroy(h)
    assert np.array_equal(got["mixed"][0], got["int8"][0]) and np.array_equal(got["mixed"][1], got["int8"][1])


def test_4bit_arguments(env):
    torch, corr, orc = env
    h = corr.corr_create(3, 1, 256, 16)               # 3 inputs: not whole cards
    try:
        with pytest.raises(corr.CorrError) as ei:
            corr.corr_push_samples_4bit(h, np.zeros((1, 64), np.uint8), 32, seq=0)
        assert ei.value.code == -1
    finally:
        corr.corr_destroy(h)
    h = corr.corr_create(2, 2, 256, 16)
    try:
        with pytest.raises(corr.CorrError) as ei:      # ld < 2 n
            corr.corr_push_samples_4bit(h, np.zeros((1, 64), np.uint8), 40, seq=0)
        assert ei.value.code == -1
    finally:
        corr.corr_destroy(h)
