"""Streaming ingest with two sample rings and a ring of host output slots: every integration
launched by corr_push_samples lands in its slot with exactly the visibilities and beams that
corr_integrate_device gives for the same samples and frame counter, while the pushes of later
samples overlap the correlation of earlier ones; slot reuse and not-yet-launched integrations
are reported."""
import numpy as np
import pytest

from synth import make_config

pytestmark = pytest.mark.gpu

N_ANT, N_POL, N_FFT, N_INT, N_INTEG = 8, 2, 512, 64, 5
MAX_DELAY = 2048


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0910_1517_gb300 import build, corr
    build.build()
    corr.load()
    return torch, corr


def _stream():
    body = N_INT * N_FFT
    s = make_config(2, n_ant=N_ANT, n_pol=N_POL, n_fft=N_FFT, n_int=N_INTEG * N_INT, seed=4242)
    assert s.x.shape[1] >= N_INTEG * body + MAX_DELAY
    return s, body


def _scales(torch, corr, s, body):
    """Requantisation scales from one FP32 integration of the stream's start."""
    h = corr.corr_create(N_ANT, N_POL, N_FFT, N_INT)
    try:
        corr.corr_set_delays(h, s.delay, s.phi0, s.rate)
        n = body + MAX_DELAY
        xt = torch.zeros((s.n_in, ((n + 15) // 16) * 16 + 16), dtype=torch.int8, device="cuda")
        xt[:, :n] = torch.from_numpy(np.ascontiguousarray(s.x[:, :n])).cuda()
        corr.corr_integrate_device(h, xt, n_avail=n, stream=torch.cuda.current_stream())
        corr.corr_set_scales(h, None)
        corr.corr_set_mode(h, corr.CORR_I8, 0, 1)
        corr.corr_integrate_device(h, xt, n_avail=n, stream=torch.cuda.current_stream())
        _, sc = corr.corr_read_requant(h, 0, 0, N_INT)
        return np.ascontiguousarray(sc, dtype=np.float32)
    finally:
        corr.corr_destroy(h)


def _reference(torch, corr, s, body, j, mode=0, scales=None):
    """Integration j on its own, straight from device memory."""
    h = corr.corr_create(N_ANT, N_POL, N_FFT, N_INT)
    try:
        corr.corr_set_delays(h, s.delay, s.phi0, s.rate)
        if scales is not None:
            corr.corr_set_scales(h, scales)
        corr.corr_set_mode(h, mode, 0, 1)
        n = body + MAX_DELAY
        xt = torch.zeros((s.n_in, ((n + 15) // 16) * 16 + 16), dtype=torch.int8, device="cuda")
        xt[:, :n] = torch.from_numpy(np.ascontiguousarray(s.x[:, j * body:j * body + n])).cuda()
        corr.corr_integrate_device(h, xt, n_avail=n, g0=j * N_INT, stream=torch.cuda.current_stream())
        return corr.corr_read_visibilities(h), corr.corr_read_beams(h)
    finally:
        corr.corr_destroy(h)


@pytest.mark.parametrize("mode", [0, 1], ids=["fp32", "i8"])
def test_output_ring_matches_direct_integrations(env, mode):
    torch, corr = env
    s, body = _stream()
    scales = _scales(torch, corr, s, body) if mode == corr.CORR_I8 else None
    n_bl = N_ANT * (N_ANT + 1) // 2
    n_slots = 3
    vis = torch.empty((n_slots, N_FFT // 2, n_bl, N_POL ** 2, 2), dtype=torch.float32).pin_memory()
    beams = torch.empty((n_slots, 2, N_INT, N_FFT // 2), dtype=torch.float32).pin_memory()
    h = corr.corr_create(N_ANT, N_POL, N_FFT, N_INT)
    try:
        corr.corr_set_max_delay(h, MAX_DELAY)
        corr.corr_set_delays(h, s.delay, s.phi0, s.rate)
        if scales is not None:
            corr.corr_set_scales(h, scales)
        corr.corr_set_mode(h, mode, 0, 1)
        corr.corr_set_output_ring(h, vis.numpy(), beams.numpy(), n_slots)
        with pytest.raises(corr.CorrError) as ei:
            corr.corr_wait_output(h, 0)
        assert ei.value.code == -3                       # nothing launched yet
        got = {}
        # uneven chunks, several integrations per push at times
        cuts = [0, 5000, 40000, 41000, 3 * body + 17, 4 * body + MAX_DELAY - 1, N_INTEG * body + MAX_DELAY]
        nxt = 0
        for a, b in zip(cuts[:-1], cuts[1:]):
            corr.corr_push_samples(h, np.ascontiguousarray(s.x[:, a:b]), seq=a)
            while True:                                  # collect every integration launched so far
                try:
                    slot = corr.corr_wait_output(h, nxt)
                except corr.CorrError as e:
                    assert e.code == -3
                    break
                got[nxt] = (vis[slot].numpy().copy(), beams[slot].numpy().copy())
                nxt += 1
        assert sorted(got) == list(range(N_INTEG))
        with pytest.raises(corr.CorrError) as ei:
            corr.corr_wait_output(h, 0)                  # its slot now holds integration 3
        assert ei.value.code == -7
        for j in range(N_INTEG):
            V_ref, B_ref = _reference(torch, corr, s, body, j, mode, scales)
            V, B = got[j]
            assert np.array_equal(V.reshape(-1), V_ref.view(np.float32).reshape(-1)), j
            assert np.array_equal(B.reshape(B_ref.shape), B_ref), j
        # the last launched integration is also what corr_read_visibilities returns
        assert np.array_equal(corr.corr_read_visibilities(h).view(np.float32).reshape(-1),
                              got[N_INTEG - 1][0].reshape(-1))
    finally:
        corr.corr_destroy(h)


def test_output_ring_arguments(env):
    torch, corr = env
    h = corr.corr_create(4, 2, 256, 16)
    try:
        with pytest.raises(corr.CorrError) as ei:
            corr.corr_wait_output(h, 0)
        assert ei.value.code == -7                       # no ring
        v = np.zeros((1, 128, 10, 4, 2), np.float32)
        with pytest.raises(corr.CorrError) as ei:
            corr.corr_set_output_ring(h, v, None, 0)
        assert ei.value.code == -1
        corr.corr_set_output_ring(h, v, None, 1)
        with pytest.raises(corr.CorrError) as ei:       # double-buffered outputs: not in a batch
            corr.corr_batch_create([h])
        assert ei.value.code == -7
        corr.corr_set_output_ring(h, None)
        b = corr.corr_batch_create([h])
        try:
            with pytest.raises(corr.CorrError) as ei:   # nor a ring on a batch member
                corr.corr_set_output_ring(h, v, None, 1)
            assert ei.value.code == -7
        finally:
            corr.corr_batch_destroy(b)
        corr.corr_set_output_ring(h, v, None, 1)        # free again once the batch is gone
        corr.corr_set_output_ring(h, None)
    finally:
        corr.corr_destroy(h)
