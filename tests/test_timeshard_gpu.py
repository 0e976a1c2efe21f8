"""A time-split integration on the GPU path (Sec. 2.3.2): the GPU correlator on each rank's
frames (a handle per slice, the slice's samples with the delay overlap, its global first frame
for the fringe phase), summed on the host by reduce_visibilities (ranks as threads over an
in-process store; their kernels never wait on one another).  FP32: the sum matches the FP64
oracle on the whole integration within the FP32 bound; int8: the summed integer visibilities
equal the oracle's exact MAC over the slices' own requantised spectra."""
import threading

import numpy as np
import pytest

from fxhelp import vis_norm_error
from synth import make_config

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world", [2, 3])
def test_time_split_integration_on_the_gpu(orc, world):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.distributed as dist

    from paper_0910_1517_gb300 import build, corr, timeshard
    build.build()
    corr.load()
    n_int = 128 if world == 2 else 144
    s = make_config(2, n_ant=8, n_pol=2, n_fft=512, n_int=n_int, seed=5151)
    tail = s.x.shape[1] - n_int * s.n_fft
    st = torch.cuda.current_stream()
    # one set of requantisation scales for every slice: from an FP32 pass over the whole integration
    h = corr.corr_create(s.n_ant, s.n_pol, s.n_fft, n_int)
    try:
        corr.corr_set_delays(h, s.delay, s.phi0, s.rate)
        xt = torch.zeros((s.n_in, ((s.x.shape[1] + 15) // 16) * 16 + 16), dtype=torch.int8, device="cuda")
        xt[:, :s.x.shape[1]] = torch.from_numpy(s.x).cuda()
        corr.corr_integrate_device(h, xt, n_avail=s.x.shape[1], stream=st)
        corr.corr_set_scales(h, None)
        corr.corr_set_mode(h, corr.CORR_I8, 0, 1)
        corr.corr_integrate_device(h, xt, n_avail=s.x.shape[1], stream=st)
        _, scales = corr.corr_read_requant(h, 0, 0, n_int)
    finally:
        corr.corr_destroy(h)
    parts = {}
    for r in range(world):
        t0, nt = timeshard.frame_slice(n_int, world, r)
        a0, na = timeshard.sample_slice(n_int, s.n_fft, world, r, tail)
        hr = corr.corr_create(s.n_ant, s.n_pol, s.n_fft, nt)
        try:
            corr.corr_set_delays(hr, s.delay, s.phi0, s.rate)
            corr.corr_set_scales(hr, scales)
            xs = torch.zeros((s.n_in, ((na + 15) // 16) * 16 + 16), dtype=torch.int8, device="cuda")
            xs[:, :na] = torch.from_numpy(np.ascontiguousarray(s.x[:, a0:a0 + na])).cuda()
            corr.corr_integrate_device(hr, xs, n_avail=na, g0=t0, stream=st)
            v32 = corr.corr_read_visibilities(hr)
            corr.corr_set_mode(hr, corr.CORR_I8, 0, 1)
            corr.corr_integrate_device(hr, xs, n_avail=na, g0=t0, stream=st)
            parts[r] = (v32, corr.corr_read_vis_int(hr), corr.corr_read_requant(hr, 0, s.n_fft // 2, nt)[0])
        finally:
            corr.corr_destroy(hr)
    store = dist.HashStore()
    sums = {}

    def rank(r):
        sums[r] = (timeshard.reduce_visibilities(parts[r][0], store, 0, world, r, timeout_s=30.0),
                   timeshard.reduce_visibilities(parts[r][1], store, 0, world, r, timeout_s=30.0, prefix="int"))

    th = [threading.Thread(target=rank, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=120)
    assert sorted(sums) == list(range(world))
    Y = orc.fengine(s.x, s.n_ant, s.n_pol, s.n_fft, n_int, s.delay, s.phi0, s.rate)
    e = vis_norm_error(sums[0][0].astype(np.complex128), orc.xengine(Y, s.n_ant, s.n_pol), s.n_ant, s.n_pol)
    q = np.concatenate([parts[r][2] for r in range(world)], axis=1)          # the slices' int8 spectra
    Vi_o, _ = orc.xint(q, scales.astype(np.float64), s.n_ant, s.n_pol)
    print(f"time split over {world} slices: FP32 vs FP64 {e:.2e}")
    assert e <= 1e-5
    assert np.array_equal(sums[0][1], Vi_o.astype(np.int32))
    for r in range(1, world):
        assert np.array_equal(sums[r][0], sums[0][0]) and np.array_equal(sums[r][1], sums[0][1])
