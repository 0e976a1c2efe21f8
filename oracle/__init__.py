"""FP64 CPU oracle for the GMRT software backend's FX correlator and beamformer.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package; the product path (``paper_0910_1517_gb300``) never does.  The
arithmetic lives in ``fx_oracle.c`` (plain C, double precision, direct DFT);
this module only builds it with gcc and marshals numpy arrays through ctypes (the
dedispersion stage, whose steps are FFTs, is numpy in ``dedisp.py``).

Functions and the passage each follows (Roy et al., arXiv:0910.1517):
  fengine   -- integer delay, real DFT, FSTC + fringe phasor (Sec. 2.1, Eq. 2)
  xengine   -- MAC over N(N+1)/2 baselines x n_pol^2 products (Sec. 2.1)
  xengine_self, xint_self -- the self-polar (total-intensity) MAC: products RR*, LL* only
            (Sec. 2.1, 2.3.2), in FP64 and exactly on requantised spectra
  beams     -- incoherent and coherent array beams (Sec. 2.2, 4.3)
  multibeam -- several phased beams with full-polar products or voltages (Sec. 2.2, 5)
  requant   -- 8-bit requantisation of spectra (precision form; Sec. 4.1 analogue)
  xint      -- exact integer MAC on requantised spectra (Sec. 4.1)
  mad_flag  -- median-absolute-deviation flagger (Sec. 5, Eq. 3-4)
  unpack4   -- ADC-format ingest of the 4-bit, 33 MHz mode: demultiplex 4 inputs per card and
            sign-extend each 4-bit sample to 8 bits (Sec. 2.3.1, 2.3.2)
  mad_blank -- the time-domain voltage blanker built on it (Sec. 5): flagged raw samples
            replaced by pre-computed Gaussian noise scaled by the block's MAD / 0.6745
  coherent_dedisperse (dedisp.py, numpy FP64) -- coherent dedispersion of the phased-array
            voltage beam (Sec. 5): per-frame inverse FFT to the baseband series, overlap-save
            multiplication by the inverse ISM chirp, detection of both polarisations, averaging
  fft_fengine (cpu_fft_baseline.c) -- not an oracle: the bench's second CPU baseline,
            the same F-engine with an FP32 radix-2 FFT (pinned to ``fengine``)
  power_dumps, patch_stats, rfi_forward, rfi_loss_grad (rfi_oracle.c) -- the RFI
            stage: 1 ms auto-power dumps, per-patch Eq. 3-4 statistics and flags,
            and the learned flagger's forward pass, BCE loss and exact gradient
All of them are pinned by the ``-m "not gpu"`` tests in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "fx_oracle.c"), os.path.join(_HERE, "rfi_oracle.c"),
         os.path.join(_HERE, "cpu_fft_baseline.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile fx_oracle.c into liboracle.so with gcc + OpenMP (no FMA contraction)."""
    newest = max(os.path.getmtime(f) for f in _SRCS)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
            "-std=c11"] + _SRCS + ["-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        L.oracle_fengine.argtypes = [i32, i32, i32, i32, P, i64, i64, P, P, P, i64, P, i32, P]
        L.oracle_xengine.argtypes = [i32, i32, i32, i32, P, P]
        L.oracle_beams.argtypes = [i32, i32, i32, i32, i32, P, P, P, P, P, P, i32, P]
        L.oracle_requant.argtypes = [i32, i32, i32, P, P, P]
        L.oracle_xint.argtypes = [i32, i32, i32, i32, P, P, P, P]
        L.oracle_xengine_self.argtypes = [i32, i32, i32, i32, P, P]
        L.oracle_xint_self.argtypes = [i32, i32, i32, i32, P, P]
        L.oracle_mad_flag.argtypes = [i32, P, f64, P, P, P]
        L.oracle_threads.argtypes = []
        L.oracle_n_baselines.argtypes = [i32]
        L.oracle_rfi_n_params.argtypes = []
        L.oracle_power_dumps.argtypes = [i32, i32, i32, i32, P, P]
        L.oracle_patch_stats.argtypes = [i32, i32, P, f64, P, P, P, P]
        L.oracle_rfi_forward.argtypes = [i32, i32, i32, P, P, P]
        L.oracle_rfi_loss_grad.argtypes = [i32, i32, i32, P, P, P, P, P]
        L.oracle_unpack4.argtypes = [i32, i64, P, i64, P]
        L.oracle_multibeam.argtypes = [i32, i32, i32, i32, P, i32, P, i32, i32, P]
        L.oracle_mad_blank.argtypes = [i32, i64, P, i64, i32, f64, P, i32, P, P]
        L.cpu_fft_fengine.argtypes = [i32, i32, i32, i32, P, i64, i64, P, P, P, i64, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def n_baselines(n_ant: int) -> int:
    return n_ant * (n_ant + 1) // 2


def threads() -> int:
    return int(lib().oracle_threads())


def fengine(x, n_ant, n_pol, n_fft, n_frames, delay, phi0, rate, g0=0, chans=None):
    """Spectra Y[i][t][c] (complex128) after integer delay, DFT and the Eq. 2 phasor.

    x: int8 [n_in][n_avail] (rows may be strided); delay/phi0/rate: per antenna.
    """
    x = np.asarray(x)
    assert x.dtype == np.int8 and x.ndim == 2 and x.shape[0] == n_ant * n_pol
    if x.strides[1] != 1:
        x = np.ascontiguousarray(x)
    d = np.ascontiguousarray(delay, dtype=np.float64)
    f0 = np.ascontiguousarray(phi0, dtype=np.float64)
    w = np.ascontiguousarray(rate, dtype=np.float64)
    assert d.shape == f0.shape == w.shape == (n_ant,)
    if chans is None:
        ch, nch, chp = None, n_fft // 2, None
    else:
        ch = np.ascontiguousarray(chans, dtype=np.int32)
        nch, chp = len(ch), _p(ch)
    Y = np.zeros((n_ant * n_pol, n_frames, nch, 2), dtype=np.float64)
    rc = lib().oracle_fengine(n_ant, n_pol, n_fft, n_frames, _p(x), x.strides[0], x.shape[1],
                              _p(d), _p(f0), _p(w), int(g0), chp, nch, _p(Y))
    _check(rc, "fengine")
    return Y[..., 0] + 1j * Y[..., 1]


def fft_fengine(x, n_ant, n_pol, n_fft, n_frames, delay, phi0, rate, g0=0):
    """The bench's CPU FFT baseline (cpu_fft_baseline.c): the F-engine of ``fengine`` with
    an FP32 radix-2 FFT in place of the FP64 DFT; spectra Y[i][t][k] (complex128), all k."""
    x = np.asarray(x)
    assert x.dtype == np.int8 and x.ndim == 2 and x.shape[0] == n_ant * n_pol
    if x.strides[1] != 1:
        x = np.ascontiguousarray(x)
    d = np.ascontiguousarray(delay, dtype=np.float64)
    f0 = np.ascontiguousarray(phi0, dtype=np.float64)
    w = np.ascontiguousarray(rate, dtype=np.float64)
    Y = np.zeros((n_ant * n_pol, n_frames, n_fft // 2, 2), dtype=np.float64)
    rc = lib().cpu_fft_fengine(n_ant, n_pol, n_fft, n_frames, _p(x), x.strides[0], x.shape[1],
                               _p(d), _p(f0), _p(w), int(g0), _p(Y))
    _check(rc, "fft_fengine")
    return Y[..., 0] + 1j * Y[..., 1]


def _as_ri(Y):
    Y = np.asarray(Y)
    out = np.empty(Y.shape + (2,), dtype=np.float64)
    out[..., 0] = Y.real
    out[..., 1] = Y.imag
    return out


def xengine(Y, n_ant, n_pol):
    """Visibilities V[c][b][p*n_pol+q] (complex128), baselines a <= a' row-major."""
    n_in, n_frames, nch = Y.shape
    assert n_in == n_ant * n_pol
    Yr = _as_ri(Y)
    V = np.zeros((nch, n_baselines(n_ant), n_pol * n_pol, 2), dtype=np.float64)
    _check(lib().oracle_xengine(n_ant, n_pol, nch, n_frames, _p(Yr), _p(V)), "xengine")
    return V[..., 0] + 1j * V[..., 1]


def xengine_self(Y, n_ant, n_pol):
    """Self-polar visibilities V[c][b][p] (complex128): products Y_ap conj(Y_a'p) only."""
    n_in, n_frames, nch = Y.shape
    assert n_in == n_ant * n_pol
    Yr = _as_ri(Y)
    V = np.zeros((nch, n_baselines(n_ant), n_pol, 2), dtype=np.float64)
    _check(lib().oracle_xengine_self(n_ant, n_pol, nch, n_frames, _p(Yr), _p(V)), "xengine_self")
    return V[..., 0] + 1j * V[..., 1]


def xint_self(q, n_ant, n_pol):
    """Exact int64 self-polar MAC on int8 spectra q [n_in][n_frames][n_ch][2]: [c][b][p][2]."""
    q = np.ascontiguousarray(q, dtype=np.int8)
    n_in, n_frames, nch, _ = q.shape
    assert n_in == n_ant * n_pol
    Vi = np.zeros((nch, n_baselines(n_ant), n_pol, 2), dtype=np.int64)
    _check(lib().oracle_xint_self(n_ant, n_pol, nch, n_frames, _p(q), _p(Vi)), "xint_self")
    return Vi


def beams(Y, n_ant, n_pol, n_fft, gain=None, theta=None, inc_mask=None, coh_mask=None,
          beam_avg=1, chans=None):
    """(B_inc, B_coh), each [n_frames/beam_avg][n_chans] float64."""
    n_in, n_frames, nch = Y.shape
    Yr = _as_ri(Y)
    g = np.ones(n_ant) if gain is None else np.ascontiguousarray(gain, dtype=np.float64)
    th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64)
    if th is not None:
        assert th.shape == (n_ant, n_fft // 2)
    im = np.ones(n_ant, np.uint8) if inc_mask is None else np.ascontiguousarray(inc_mask, dtype=np.uint8)
    cm = np.ones(n_ant, np.uint8) if coh_mask is None else np.ascontiguousarray(coh_mask, dtype=np.uint8)
    ch = None if chans is None else np.ascontiguousarray(chans, dtype=np.int32)
    n_out = n_frames // beam_avg
    B = np.zeros((2, n_out, nch), dtype=np.float64)
    rc = lib().oracle_beams(n_ant, n_pol, n_fft, nch, n_frames, _p(Yr),
                            None if ch is None else _p(ch), _p(g),
                            None if th is None else _p(th), _p(im), _p(cm), beam_avg, _p(B))
    _check(rc, "beams")
    return B[0], B[1]


def unpack4(packed, n):
    """ADC-format 4-bit ingest: card rows packed uint8 [n_cards][>= 2n] -> int8 rows [4 n_cards][n]."""
    packed = np.asarray(packed)
    assert packed.dtype == np.uint8 and packed.ndim == 2
    if packed.strides[1] != 1:
        packed = np.ascontiguousarray(packed)
    out = np.zeros((4 * packed.shape[0], n), dtype=np.int8)
    _check(lib().oracle_unpack4(packed.shape[0], n, _p(packed), packed.strides[0], _p(out)), "unpack4")
    return out


def multibeam(Y, n_ant, n_pol, w, products=0, avg=1):
    """Phased beams [n_beams][n_frames/avg][n_chans][4] (float64) from spectra Y [n_in][t][c] and
    complex weights w [n_beams][n_ant][n_chans]: full-polar products (0) or voltages (1)."""
    n_in, n_frames, nch = Y.shape
    w = np.asarray(w)
    nb = w.shape[0]
    assert n_in == n_ant * n_pol and w.shape == (nb, n_ant, nch)
    wr = _as_ri(w.astype(np.complex128))
    out = np.zeros((nb, n_frames // avg, nch, 4), dtype=np.float64)
    _check(lib().oracle_multibeam(n_ant, n_pol, nch, n_frames, _p(_as_ri(Y)), nb, _p(wr), products, avg, _p(out)),
           "multibeam")
    return out


def requant(Y, scale):
    """q[i][t][c][2] int8 = clamp(rint(Y * s[i][c]), +-127) per real component."""
    n_in, n_frames, nch = Y.shape
    Yr = _as_ri(Y)
    s = np.ascontiguousarray(scale, dtype=np.float64)
    assert s.shape == (n_in, nch)
    q = np.zeros(Yr.shape, dtype=np.int8)
    _check(lib().oracle_requant(n_in, n_frames, nch, _p(Yr), _p(s), _p(q)), "requant")
    return q


def xint(q, scale, n_ant, n_pol):
    """Exact integer visibilities (int64 [c][b][pp][2]) and their descaled FP64 values."""
    q = np.ascontiguousarray(q, dtype=np.int8)
    n_in, n_frames, nch, two = q.shape
    assert two == 2 and n_in == n_ant * n_pol
    s = np.ascontiguousarray(scale, dtype=np.float64)
    nbl, npp = n_baselines(n_ant), n_pol * n_pol
    Vi = np.zeros((nch, nbl, npp, 2), dtype=np.int64)
    V = np.zeros((nch, nbl, npp, 2), dtype=np.float64)
    _check(lib().oracle_xint(n_ant, n_pol, nch, n_frames, _p(q), _p(s), _p(Vi), _p(V)), "xint")
    return Vi, V[..., 0] + 1j * V[..., 1]


def mad_flag(x, M):
    """(flags uint8 [n], median, MAD) per Eq. 3 and Eq. 4."""
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    f = np.zeros(x.size, dtype=np.uint8)
    med, mad = ctypes.c_double(), ctypes.c_double()
    rc = lib().oracle_mad_flag(x.size, _p(x), float(M), _p(f), ctypes.byref(med), ctypes.byref(mad))
    _check(rc, "mad_flag")
    return f, med.value, mad.value


def mad_blank(x, block, M, noise):
    """Time-domain voltage blanker (Sec. 5, Eq. 3-4) on int8 rows x [n_in][n]: (blanked rows,
    stats int32 [n_in][n_blocks][4] = 2 med, 4 MAD, floor(2 M MAD / 0.6745), samples replaced)."""
    x = np.asarray(x)
    assert x.dtype == np.int8 and x.ndim == 2
    if x.strides[1] != 1:
        x = np.ascontiguousarray(x)
    g = np.ascontiguousarray(noise, dtype=np.float32)
    n_in, n = x.shape
    assert g.ndim == 2 and g.shape[0] == n_in
    nb = (n + block - 1) // block
    out = np.zeros((n_in, n), dtype=np.int8)
    st = np.zeros((n_in, nb, 4), dtype=np.int32)
    _check(lib().oracle_mad_blank(n_in, n, _p(x), x.strides[0], int(block), float(M), _p(g), g.shape[1],
                                  _p(out), _p(st)), "mad_blank")
    return out, st


# ------------------------------------------------------------------ RFI stage

def rfi_n_params() -> int:
    return int(lib().oracle_rfi_n_params())


def power_dumps(Y, dump):
    """P[i][d][k] = sum over each dump of `dump` frames of |Y|^2 (float64)."""
    n_in, n_frames, nch = Y.shape
    Yr = _as_ri(Y)
    P = np.zeros((n_in, n_frames // dump, nch), dtype=np.float64)
    _check(lib().oracle_power_dumps(n_in, n_frames, nch, dump, _p(Yr), _p(P)), "power_dumps")
    return P


def patch_stats(x, M=5.0):
    """Per patch (leading axis): median, MAD, Eq. 4 flags and log-compressed network input."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    B = x.shape[0]
    n = int(np.prod(x.shape[1:]))
    med, mad = np.zeros(B), np.zeros(B)
    flags = np.zeros(x.shape, dtype=np.uint8)
    z = np.zeros(x.shape, dtype=np.float64)
    _check(lib().oracle_patch_stats(B, n, _p(x), float(M), _p(med), _p(mad), _p(flags), _p(z)), "patch_stats")
    return med, mad, flags, z


def rfi_forward(params, x):
    """Logits [B][H][W] of the 1->16->32->16->1 network for inputs x [B][H][W]."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    p = np.ascontiguousarray(params, dtype=np.float64)
    assert p.size == rfi_n_params()
    B, H, W = x.shape
    out = np.zeros((B, H, W), dtype=np.float64)
    _check(lib().oracle_rfi_forward(B, H, W, _p(p), _p(x), _p(out)), "rfi_forward")
    return out


def rfi_loss_grad(params, x, mask):
    """(mean BCE loss, d loss / d params) of the network on inputs x and masks."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    p = np.ascontiguousarray(params, dtype=np.float64)
    B, H, W = x.shape
    g = np.zeros(p.size, dtype=np.float64)
    loss = ctypes.c_double()
    _check(lib().oracle_rfi_loss_grad(B, H, W, _p(p), _p(x), _p(m), ctypes.byref(loss), _p(g)), "rfi_loss_grad")
    return loss.value, g


from .dedisp import coherent_dedisperse  # noqa: E402  (numpy oracle, Sec. 5)
