"""corr_integrate_static -- the entry point that allocates nothing, for callers that may not
allocate device memory while they run -- must give the same visibilities and beams as the
handle-based corr_integrate_device on the same samples, and match the FP64 oracle, on
consecutive calls that reuse its static scratch array (including a non-blocking call followed
by a blocking one on the same stream).  Collected last so that a failure here stops a -x run
only after every other test has run."""
import numpy as np
import pytest

from fxhelp import vis_norm_error
from synth import make_config

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the FP32-path tolerance of the parity tests


def _device_rows(torch, x):
    n_in, n = x.shape
    ld = ((n + 15) // 16) * 16 + 16
    xt = torch.zeros((n_in, ld), dtype=torch.int8, device="cuda")
    xt[:, :n] = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return xt, n


def _beam_error(B, B_ref, n_ant):
    # incoherent: relative; coherent: normalised by its Cauchy-Schwarz bound n_ant * B_inc
    return max(float(np.max(np.abs(B[0] - B_ref[0]) / np.maximum(B_ref[0], 1e-30))),
               float(np.max(np.abs(B[1] - B_ref[1]) / np.maximum(n_ant * B_ref[0], 1e-30))))


def test_static_entry_matches_handle_path_and_oracle_on_calls_in_a_row(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0910_1517_gb300 import build, corr
    build.build()
    corr.load()
    cases = [make_config(1),                                                 # integer delays, fringes
             make_config(2, n_ant=6, n_pol=2, n_fft=512, n_int=64, seed=77),    # fractional delays
             make_config(2, n_ant=4, n_pol=1, n_fft=4096, n_int=64, seed=78)]   # the 4096-point FFT
    stream = torch.cuda.current_stream()
    for s in cases:
        xt, n = _device_rows(torch, s.x)
        h = corr.corr_create(s.n_ant, s.n_pol, s.n_fft, s.n_int)
        try:
            corr.corr_set_delays(h, s.delay, s.phi0, s.rate)
            corr.corr_integrate_device(h, xt, n_avail=n, stream=stream)
            V_ref = corr.corr_read_visibilities(h).astype(np.complex128)
            B_ref = corr.corr_read_beams(h).astype(np.float64)
        finally:
            corr.corr_destroy(h)
        # the FP64 oracle on the same samples (unit gains, every antenna in both beams)
        Y = orc.fengine(s.x, s.n_ant, s.n_pol, s.n_fft, s.n_int, s.delay, s.phi0, s.rate)
        V_o = orc.xengine(Y, s.n_ant, s.n_pol)
        B_inc, B_coh = orc.beams(Y, s.n_ant, s.n_pol, s.n_fft)
        B_o = np.stack([B_inc, B_coh])
        n_bl = s.n_ant * (s.n_ant + 1) // 2
        vis = torch.full((s.n_fft // 2, n_bl, s.n_pol ** 2, 2), float("nan"), device="cuda")
        beams = torch.full((2, s.n_int, s.n_fft // 2), float("nan"), device="cuda")
        # a non-blocking call, then a blocking one on the same stream (the documented way to
        # serialise calls); the second overwrites the first's outputs with the same values
        corr.corr_integrate_static(s.n_ant, s.n_pol, s.n_fft, s.n_int, xt, vis, beams, s.delay, s.phi0,
                                   s.rate, n_avail=n, stream=stream, blocking=0)
        corr.corr_integrate_static(s.n_ant, s.n_pol, s.n_fft, s.n_int, xt, vis, beams, s.delay, s.phi0,
                                   s.rate, n_avail=n, stream=stream, blocking=1)
        v = vis.cpu().numpy()
        V = v[..., 0].astype(np.float64) + 1j * v[..., 1]
        B = beams.cpu().numpy().astype(np.float64)
        e_v = vis_norm_error(V, V_ref, s.n_ant, s.n_pol)
        e_b = _beam_error(B, B_ref, s.n_ant)
        e_vo = vis_norm_error(V, V_o, s.n_ant, s.n_pol)
        e_bo = _beam_error(B, B_o, s.n_ant)
        print(f"static ({s.n_ant} ant, {s.n_fft}-pt): vs handle vis {e_v:.2e} beams {e_b:.2e}; "
              f"vs oracle vis {e_vo:.2e} beams {e_bo:.2e}")
        assert np.isfinite(V).all() and np.isfinite(B).all()
        assert e_v <= TOL and e_b <= TOL
        assert e_vo <= TOL and e_bo <= TOL
