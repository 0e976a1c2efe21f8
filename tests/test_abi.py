"""CPU-side checks of the boundary: the library builds and loads, exports every
symbol include/corr.h declares, the binding covers exactly those, and the
argument validation that runs before any CUDA call rejects bad sizes."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in ("corr.h", "rfi.h"):
        src = open(os.path.join(ROOT, "include", hdr)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b((?:corr|rfi)_[a-z_0-9]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_0910_1517_gb300 import build, corr
    build.build()
    return corr.load()


def test_header_declares_the_north_star_calls():
    d = _declared()
    for name in ("corr_create", "corr_set_delays", "corr_push_samples", "corr_read_visibilities",
                 "corr_read_beams"):
        assert name in d


def test_library_exports_every_declared_symbol(lib):
    from paper_0910_1517_gb300 import corr
    out = subprocess.run(["nm", "-D", "--defined-only", corr.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT ((?:corr|rfi)_[a-z_0-9]+)$", out, flags=re.M))
    assert _declared() <= exported, _declared() - exported
    assert set(corr.SIGNATURES) == _declared()
    for name in _declared():
        assert hasattr(lib, name)


def test_binding_has_no_fallback(tmp_path, monkeypatch):
    from paper_0910_1517_gb300 import corr
    monkeypatch.setattr(corr, "_lib", None)
    monkeypatch.setattr(corr, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        corr.load()


@pytest.mark.parametrize("args", [
    (0, 2, 512, 64),       # no antennas
    (4, 3, 512, 64),       # bad polarisation count
    (4, 2, 500, 64),       # n_fft not a power of two
    (4, 2, 8192, 64),      # n_fft above the supported range
    (4, 2, 512, 60),       # n_int not a multiple of 16
    (65, 2, 512, 64),      # more than 128 inputs
])
def test_create_rejects_bad_sizes_before_touching_cuda(lib, args):
    from paper_0910_1517_gb300 import corr
    with pytest.raises(corr.CorrError) as ei:
        corr.corr_create(*args)
    assert ei.value.code == -1
    assert corr.corr_last_error()


def test_null_handle_is_rejected(lib):
    from paper_0910_1517_gb300 import corr
    with pytest.raises(corr.CorrError):
        corr.corr_set_mode(None, 0, 0, 1)


def test_dedisperser_smear_matches_the_oracle_on_the_host(lib):
    # corr_dd_smear_samples is host arithmetic: the cold-plasma smear across the band
    from oracle import dedisp
    from paper_0910_1517_gb300 import corr
    for dm, f_lo, bw in ((30.0, 1780.0 / 3.0, 100.0 / 3.0), (71.0398, 316.67, 16.66), (0.0, 600.0, 10.0)):
        assert corr.corr_dd_smear_samples(dm, f_lo, bw) == pytest.approx(dedisp.smear_samples(dm, f_lo, bw),
                                                                          rel=1e-12, abs=1e-9)
    assert corr.corr_dd_smear_samples(1.0, 600.0, -1.0) == -1.0


@pytest.mark.parametrize("args,code", [
    ((100, 1024, 512, 1024, 2.0, 593.3, 33.3, 256), -1),     # n_chan not a power of two
    ((256, 8192, 512, 1024, 2.0, 593.3, 33.3, 256), -1),     # fft_frames above 4096
    ((256, 1024, 1024, 1024, 2.0, 593.3, 33.3, 256), -1),    # overlap = fft_frames
    ((256, 1024, 512, 0, 2.0, 593.3, 33.3, 256), -1),        # no push room
    ((256, 1024, 512, 1024, 2.0, 593.3, -33.3, 256), -1),    # lower sideband
    ((256, 1024, 512, 1024, -1.0, 593.3, 33.3, 256), -1),    # negative DM
    ((256, 1024, 512, 1024, 2.0, 593.3, 33.3, 3), -1),       # avg not a power of two
    ((256, 1024, 511, 1024, 2.0, 593.3, 33.3, 512), -1),     # avg does not divide the block step (513 x 256)
    ((256, 1024, 64, 1024, 2.0, 593.3, 33.3, 256), -2),      # overlap below the smear
])
def test_dedisperser_create_rejects_bad_arguments_before_any_cuda_call(lib, args, code):
    from paper_0910_1517_gb300 import corr
    with pytest.raises(corr.CorrError) as ei:
        corr.corr_dd_create(*args)
    assert ei.value.code == code


def _static_call(lib, n_ant=4, n_pol=2, n_fft=512, n_int=64, delay=None, phi0=None, rate=None, n_avail=None):
    """corr_integrate_static with fake, never dereferenced device addresses: every case below is
    refused by the host-side checks that run before the first CUDA call."""
    import ctypes

    import numpy as np
    d = np.zeros(n_ant) if delay is None else np.asarray(delay, dtype=np.float64)
    f = None if phi0 is None else np.asarray(phi0, dtype=np.float64)
    w = None if rate is None else np.asarray(rate, dtype=np.float64)
    ptr = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
    fake = ctypes.c_void_p(4096)
    n_avail = n_int * n_fft + 4096 if n_avail is None else n_avail
    ld = ((n_avail + 15) // 16) * 16
    return lib.corr_integrate_static(n_ant, n_pol, n_fft, n_int, fake, ld, n_avail, 0, ptr(d), ptr(f), ptr(w),
                                     fake, fake, None, 1)


@pytest.mark.parametrize("kw,code", [
    ({"delay": [0.0, 0.0, 3e9, 0.0]}, -2),                       # rounds beyond 2e9 samples
    ({"delay": [0.0, -1.0, 0.0, 0.0]}, -2),                      # negative
    ({"delay": [0.0, float("nan"), 0.0, 0.0]}, -2),              # not finite
    ({"rate": [0.0, float("nan"), 0.0, 0.0]}, -1),               # fringe rate not finite
    ({"phi0": [float("inf"), 0.0, 0.0, 0.0]}, -1),               # fringe phase not finite
    ({"n_ant": 65, "delay": [0.0] * 65}, -1),                    # more antennas than the static tables hold
    ({"n_ant": 64, "n_fft": 2048, "n_int": 8192, "delay": [0.0] * 64}, -2),   # beyond the 32 MiB scratch
    ({"delay": [0.0, 0.0, 5000.0, 0.0], "n_avail": 64 * 512 + 100}, -2),     # samples short of the delay
])
def test_static_entry_refuses_bad_arguments_before_any_cuda_call(lib, kw, code):
    from paper_0910_1517_gb300 import corr
    assert _static_call(lib, **kw) == code
    assert corr.corr_last_error()
