"""Self-polar (total-intensity) mode, corr_set_mode(..., CORR_POL_SELF, ...): the products RR*
and LL* only (Sec. 2.1 sizes the MAC for these two, Sec. 2.3.2 names the mode).  Every X-engine
form against the FP64 oracle's self-polar MAC (exact on the exported int8 spectra for CORR_I8),
and against the pp entries of the same form's full-polar output."""
import numpy as np
import pytest

from fxhelp import vis_norm_error, vis_self_norm_error
from synth import make_config

pytestmark = pytest.mark.gpu

TOL = 1e-5           # the FP32-path bound (FP32 and FP32TC)
CASES = [dict(n_ant=8, n_pol=2, n_fft=512, n_int=64, seed=611),     # 2 antenna blocks per polarisation
         dict(n_ant=5, n_pol=2, n_fft=1024, n_int=48, seed=612),    # ragged antenna block
         dict(n_ant=32, n_pol=2, n_fft=256, n_int=32, seed=613),    # the GMRT array's 32 antennas
         dict(n_ant=3, n_pol=1, n_fft=256, n_int=32, seed=614)]     # one polarisation: self = full


@pytest.fixture(scope="module")
def env(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0910_1517_gb300 import build, corr
    build.build()
    corr.load()
    return torch, corr, orc


def _run(env, c):
    torch, corr, orc = env
    s = make_config(2, **c)
    n_in, n = s.x.shape
    xt = torch.zeros((n_in, ((n + 15) // 16) * 16 + 16), dtype=torch.int8, device="cuda")
    xt[:, :n] = torch.from_numpy(s.x).cuda()
    st = torch.cuda.current_stream()
    h = corr.corr_create(s.n_ant, s.n_pol, s.n_fft, s.n_int)
    out = {}
    try:
        corr.corr_set_delays(h, s.delay, s.phi0, s.rate)
        corr.corr_integrate_device(h, xt, n_avail=n, stream=st)          # FP32 calibration for the scales
        corr.corr_set_scales(h, None)
        for mode in (corr.CORR_FP32, corr.CORR_FP32TC, corr.CORR_I8, corr.CORR_F16):
            for pm in (corr.CORR_POL_FULL, corr.CORR_POL_SELF):
                corr.corr_set_mode(h, mode, pm, 1)
                corr.corr_integrate_device(h, xt, n_avail=n, stream=st)
                V = corr.corr_read_visibilities(h).astype(np.complex128)
                Vi = corr.corr_read_vis_int(h) if mode == corr.CORR_I8 else None
                q = corr.corr_read_requant(h, 0, s.n_fft // 2, s.n_int)[0] if mode == corr.CORR_I8 else None
                out[(mode, pm)] = (V, Vi, q)
        Y = orc.fengine(s.x, s.n_ant, s.n_pol, s.n_fft, s.n_int, s.delay, s.phi0, s.rate)
    finally:
        corr.corr_destroy(h)
    return s, out, Y


@pytest.mark.parametrize("c", CASES, ids=lambda c: f"{c['n_ant']}x{c['n_pol']}-{c['n_fft']}")
def test_self_polar_matches_oracle_in_every_form(env, c):
    torch, corr, orc = env
    s, out, Y = _run(env, c)
    nb, npol = s.n_ant * (s.n_ant + 1) // 2, s.n_pol
    Vs_o = orc.xengine_self(Y, s.n_ant, s.n_pol)
    for mode, name in ((corr.CORR_FP32, "fp32"), (corr.CORR_FP32TC, "fp32tc")):
        V = out[(mode, corr.CORR_POL_SELF)][0]
        assert V.shape == (s.n_fft // 2, nb, npol)
        e = vis_self_norm_error(V, Vs_o, s.n_ant, s.n_pol)
        Vf = out[(mode, corr.CORR_POL_FULL)][0]
        e_full = vis_norm_error(Vf, orc.xengine(Y, s.n_ant, s.n_pol), s.n_ant, s.n_pol)
        pp = np.stack([Vf[:, :, p * npol + p] for p in range(npol)], axis=-1)
        e_pp = vis_self_norm_error(V, pp, s.n_ant, s.n_pol)
        print(f"{name} self-polar {s.n_ant}x{s.n_pol}: vs oracle {e:.2e} (full-polar {e_full:.2e}), "
              f"vs own full-polar pp {e_pp:.2e}")
        assert e <= TOL and e_pp <= TOL
    # int8: the integer sums equal the oracle's exact self-polar MAC on the GPU's own spectra,
    # and the pp entries of the full-polar integers
    _, Vi, q = out[(corr.CORR_I8, corr.CORR_POL_SELF)]
    Vis_o = orc.xint_self(q, s.n_ant, s.n_pol)
    assert Vi.shape == (s.n_fft // 2, nb, npol, 2)
    assert np.array_equal(Vi, Vis_o.astype(np.int32))
    _, Vif, qf = out[(corr.CORR_I8, corr.CORR_POL_FULL)]
    assert np.array_equal(q, qf)
    assert np.array_equal(Vi, np.stack([Vif[:, :, p * npol + p] for p in range(npol)], axis=2))
    # FP16: the same Gram as the full-polar form, its pp entries
    Vh = out[(corr.CORR_F16, corr.CORR_POL_SELF)][0]
    Vhf = out[(corr.CORR_F16, corr.CORR_POL_FULL)][0]
    assert np.array_equal(Vh, np.stack([Vhf[:, :, p * npol + p] for p in range(npol)], axis=-1))


def test_polmode_arguments_and_the_output_ring(env):
    torch, corr, orc = env
    h = corr.corr_create(4, 2, 512, 64)
    try:
        with pytest.raises(corr.CorrError) as ei:
            corr.corr_set_mode(h, corr.CORR_FP32, 2, 1)
        assert ei.value.code == -1
        corr.corr_set_mode(h, corr.CORR_FP32, corr.CORR_POL_SELF, 1)
        assert corr.corr_info(h)["n_prod"] == 2
        corr.corr_set_mode(h, corr.CORR_FP32, corr.CORR_POL_FULL, 1)
        assert corr.corr_info(h)["n_prod"] == 4
    finally:
        corr.corr_destroy(h)
