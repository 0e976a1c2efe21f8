"""Thin Python binding of the C ABI in include/corr.h (argument marshalling only).

Every function below has the name of the C entry point it calls and does no
arithmetic of its own: numpy arrays and torch tensors are turned into raw
pointers, shapes are computed from the handle's sizes, and a negative return
code becomes a ``CorrError`` carrying ``corr_last_error()``.  The library is
the in-tree ``libgb300corr.so``; there is no fallback if it is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgb300corr.so")

CORR_FP32, CORR_I8, CORR_F16, CORR_FP32TC = 0, 1, 2, 3
CORR_POL_FULL, CORR_POL_SELF = 0, 1
CODES = {0: "CORR_OK", -1: "CORR_E_INVAL", -2: "CORR_E_RANGE", -3: "CORR_E_AGAIN", -4: "CORR_E_DATALOSS",
         -5: "CORR_E_CUDA", -6: "CORR_E_NOMEM", -7: "CORR_E_STATE", -8: "CORR_E_TIMEOUT"}

# every symbol include/corr.h declares, with its ctypes signature
_P, _I, _L = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
SIGNATURES = {
    "corr_create": ([ctypes.POINTER(ctypes.c_void_p), _I, _I, _I, _I], _I),
    "corr_destroy": ([_P], _I),
    "corr_last_error": ([], ctypes.c_char_p),
    "corr_set_mode": ([_P, _I, _I, _I], _I),
    "corr_set_max_delay": ([_P, _I], _I),
    "corr_set_delays": ([_P, _P, _P, _P], _I),
    "corr_set_beam_weights": ([_P, _P, _P, _P, _P], _I),
    "corr_set_scales": ([_P, _P], _I),
    "corr_push_samples": ([_P, _P, _L, _L], _I),
    "corr_push_samples_device": ([_P, _P, _L, _L, _P], _I),
    "corr_set_output_ring": ([_P, _P, _P, _I], _I),
    "corr_wait_output": ([_P, _L, ctypes.POINTER(ctypes.c_int)], _I),
    "corr_integrate_device": ([_P, _P, _L, _L, _L, _P], _I),
    "corr_read_visibilities": ([_P, _P, _I], _I),
    "corr_read_beams": ([_P, _P, _I], _I),
    "corr_read_vis_int": ([_P, _P, _I], _I),
    "corr_read_requant": ([_P, _I, _I, _P, _P], _I),
    "corr_read_spectra": ([_P, _I, _I, _P], _I),
    "corr_device_outputs": ([_P, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                             ctypes.POINTER(ctypes.c_void_p)], _I),
    "corr_info": ([_P, _P], _I),
    "corr_set_timing": ([_P, _I], _I),
    "corr_stage_times": ([_P, _P, ctypes.POINTER(ctypes.c_int)], _I),
    "corr_integrate_static": ([_I, _I, _I, _I, _P, _L, _L, _L, _P, _P, _P, _P, _P, _P, _I], _I),
    "corr_set_power_dump": ([_P, _I], _I),
    "corr_set_xengine_stage": ([_P, _I], _I),
    "corr_batch_create": ([ctypes.POINTER(ctypes.c_void_p), _I, _P], _I),
    "corr_batch_destroy": ([_P], _I),
    "corr_batch_integrate_device": ([_P, _P, _P, _P, _P, _P], _I),
    "corr_batch_tune": ([_P, _P, _P], _I),
    "corr_read_power": ([_P, _P, ctypes.POINTER(ctypes.c_void_p)], _I),
    "corr_set_blanker": ([_P, ctypes.c_double, _I, _P, _I], _I),
    "corr_set_multibeam": ([_P, _I, _P, _I, _I], _I),
    "corr_push_samples_4bit": ([_P, _P, _L, _L, _L], _I),
    "corr_integrate_4bit_device": ([_P, _P, _L, _L, _L, _P], _I),
    "corr_read_multibeam": ([_P, _P, _I], _I),
    "corr_read_blank_stats": ([_P, _P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)], _I),
    "corr_wait_selftest": ([ctypes.POINTER(ctypes.c_longlong)], _I),
    "corr_dd_smear_samples": ([ctypes.c_double, ctypes.c_double, ctypes.c_double], ctypes.c_double),
    "corr_dd_create": ([ctypes.POINTER(ctypes.c_void_p), _I, _I, _I, _I, ctypes.c_double, ctypes.c_double,
                        ctypes.c_double, _I], _I),
    "corr_dd_push_device": ([_P, _P, _L, _P, _L, ctypes.POINTER(ctypes.c_int64), _P], _I),
    "corr_dd_set_timing": ([_P, _I], _I),
    "corr_dd_stage_times": ([_P, _P, ctypes.POINTER(ctypes.c_int)], _I),
    "corr_dd_reset": ([_P], _I),
    "corr_dd_destroy": ([_P], _I),
    # include/rfi.h
    "rfi_n_params": ([], _I),
    "rfi_create": ([ctypes.POINTER(ctypes.c_void_p), _I], _I),
    "rfi_create_fp32": ([ctypes.POINTER(ctypes.c_void_p), _I], _I),
    "rfi_destroy": ([_P], _I),
    "rfi_set_params": ([_P, _P], _I),
    "rfi_get_params": ([_P, _P], _I),
    "rfi_loss_grad": ([_P, _P, _P, _I, ctypes.POINTER(ctypes.c_float), _P, _P], _I),
    "rfi_train_step": ([_P, _P, _P, _I, ctypes.c_float, ctypes.POINTER(ctypes.c_float), _P], _I),
    "rfi_infer": ([_P, _P, _I, _P, _P], _I),
    "rfi_patches": ([_P, _I, _I, _I, ctypes.c_float, _P, _P, _P, _P], _I),
}

_lib = None


class CorrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{CODES.get(code, code)}: {msg}")
        self.code = code


def load():
    """Load libgb300corr.so (built by paper_0910_1517_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_0910_1517_gb300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _ok(rc: int, allow=()):
    if rc != 0 and rc not in allow:
        raise CorrError(rc, load().corr_last_error().decode())
    return rc


def _ptr(a):
    """Raw data pointer of a numpy array, torch tensor or integer address (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    return ctypes.c_void_p(a.data_ptr())


CUDA_STREAM_LEGACY = 1   # cudaStreamLegacy: the legacy default stream


def _stream(s):
    """cudaStream_t of a torch stream or raw handle; torch's default stream (handle 0) is
    the legacy default stream, which the C ABI spells cudaStreamLegacy (NULL means the
    handle's own stream there)."""
    if s is None:
        return None
    h = s if isinstance(s, int) else s.cuda_stream
    return ctypes.c_void_p(h if h else CUDA_STREAM_LEGACY)


def corr_create(n_ant: int, n_pol: int, n_fft: int, n_int: int):
    h = ctypes.c_void_p()
    _ok(load().corr_create(ctypes.byref(h), n_ant, n_pol, n_fft, n_int))
    return h


def corr_destroy(h):
    return _ok(load().corr_destroy(h))


def corr_last_error() -> str:
    return load().corr_last_error().decode()


def corr_set_mode(h, xmode: int, polmode: int = 0, beam_avg: int = 1):
    return _ok(load().corr_set_mode(h, xmode, polmode, beam_avg))


def corr_set_max_delay(h, max_delay: int):
    return _ok(load().corr_set_max_delay(h, max_delay))


def corr_set_delays(h, delay, phi0, rate):
    d = np.ascontiguousarray(delay, dtype=np.float64)
    f = np.ascontiguousarray(phi0, dtype=np.float64)
    w = np.ascontiguousarray(rate, dtype=np.float64)
    return _ok(load().corr_set_delays(h, _ptr(d), _ptr(f), _ptr(w)))


def corr_set_beam_weights(h, gain=None, theta=None, inc_mask=None, coh_mask=None):
    g = None if gain is None else np.ascontiguousarray(gain, dtype=np.float32)
    t = None if theta is None else np.ascontiguousarray(theta, dtype=np.float32)
    im = None if inc_mask is None else np.ascontiguousarray(inc_mask, dtype=np.uint8)
    cm = None if coh_mask is None else np.ascontiguousarray(coh_mask, dtype=np.uint8)
    return _ok(load().corr_set_beam_weights(h, _ptr(g), _ptr(t), _ptr(im), _ptr(cm)))


def corr_set_scales(h, scale=None):
    s = None if scale is None else np.ascontiguousarray(scale, dtype=np.float32)
    return _ok(load().corr_set_scales(h, _ptr(s)))


def corr_push_samples(h, x, seq: int, allow_dataloss: bool = False):
    """x: host int8 [n_in][n] (numpy array or pinned CPU tensor), rows contiguous."""
    n = x.shape[1]
    allow = (-4,) if allow_dataloss else ()
    return _ok(load().corr_push_samples(h, _ptr(x), n, seq), allow)


def corr_push_samples_4bit(h, packed, n: int, seq: int, allow_dataloss: bool = False):
    """packed: host uint8 [n_in/4][ld] ADC card rows (4 inputs x 4 bits per 2 bytes), n samples."""
    ld = packed.strides[0] if isinstance(packed, np.ndarray) else packed.stride(0)
    allow = (-4,) if allow_dataloss else ()
    return _ok(load().corr_push_samples_4bit(h, _ptr(packed), ld, n, seq), allow)


def corr_integrate_4bit_device(h, packed, n_avail: int, g0: int = 0, stream=None):
    """packed: device uint8 tensor [n_in/4][ld] of ADC card rows; n_avail samples per input."""
    return _ok(load().corr_integrate_4bit_device(h, _ptr(packed), packed.stride(0), n_avail, g0, _stream(stream)))


def corr_push_samples_device(h, x, seq: int, stream=None):
    return _ok(load().corr_push_samples_device(h, _ptr(x), x.shape[1], seq, _stream(stream)))


def corr_set_output_ring(h, vis, beams=None, n_slots=None):
    """vis: pinned float32 [n_slots][n_chan][n_bl][npp][2] (numpy/tensor) or None to remove the
    ring; beams: pinned float32 [n_slots][2][n_int/beam_avg][n_chan] or None; n_slots defaults
    to vis.shape[0]."""
    if vis is None:
        return _ok(load().corr_set_output_ring(h, None, None, 0))
    n = vis.shape[0] if n_slots is None else n_slots
    return _ok(load().corr_set_output_ring(h, _ptr(vis), _ptr(beams), n))


def corr_wait_output(h, index: int) -> int:
    """Block until streaming integration `index` is in its host slot; returns the slot."""
    slot = ctypes.c_int(-1)
    _ok(load().corr_wait_output(h, index, ctypes.byref(slot)))
    return slot.value


def corr_integrate_device(h, x, n_avail=None, g0: int = 0, stream=None, ld=None):
    """x: device int8 tensor [n_in][ld]; ld (bytes) defaults to the row stride."""
    if ld is None:
        ld = x.stride(0)
    if n_avail is None:
        n_avail = x.shape[1]
    return _ok(load().corr_integrate_device(h, _ptr(x), ld, n_avail, g0, _stream(stream)))


def _info(h):
    out = np.zeros(6, dtype=np.int64)
    _ok(load().corr_info(h, _ptr(out)))
    return out


def corr_info(h) -> dict:
    v = _info(h)
    return dict(n_in=int(v[0]), n_bl=int(v[1]), n_chan=int(v[2]), n_prod=int(v[3]), n_beam=int(v[4]),
                completed=int(v[5]))


def corr_read_visibilities(h, out=None, blocking: int = 1):
    i = corr_info(h)
    if out is None:
        out = np.empty((i["n_chan"], i["n_bl"], i["n_prod"]), dtype=np.complex64)
    _ok(load().corr_read_visibilities(h, _ptr(out), blocking))
    return out


def corr_read_beams(h, out=None, blocking: int = 1):
    i = corr_info(h)
    if out is None:
        out = np.empty((2, i["n_beam"], i["n_chan"]), dtype=np.float32)
    _ok(load().corr_read_beams(h, _ptr(out), blocking))
    return out


def corr_read_vis_int(h, blocking: int = 1):
    i = corr_info(h)
    out = np.empty((i["n_chan"], i["n_bl"], i["n_prod"], 2), dtype=np.int32)
    _ok(load().corr_read_vis_int(h, _ptr(out), blocking))
    return out


def corr_read_requant(h, k0: int, nk: int, n_int: int):
    i = corr_info(h)
    q = np.empty((i["n_in"], n_int, nk, 2), dtype=np.int8)
    s = np.empty((i["n_in"], i["n_chan"]), dtype=np.float32)
    _ok(load().corr_read_requant(h, k0, nk, _ptr(q), _ptr(s)))
    return q, s


def corr_read_spectra(h, k0: int, nk: int, n_int: int):
    i = corr_info(h)
    out = np.empty((i["n_in"], n_int, nk), dtype=np.complex64)
    _ok(load().corr_read_spectra(h, k0, nk, _ptr(out)))
    return out


def corr_device_outputs(h):
    v, b, s = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _ok(load().corr_device_outputs(h, ctypes.byref(v), ctypes.byref(b), ctypes.byref(s)))
    return v.value, b.value, s.value


def corr_set_timing(h, enable: int = 1):
    return _ok(load().corr_set_timing(h, int(enable)))


def corr_stage_times(h):
    """(ms summed per stage [set-up, F-engine, X-engine, beam averaging], integrations summed)."""
    ms = np.zeros(4, dtype=np.float32)
    n = ctypes.c_int()
    _ok(load().corr_stage_times(h, _ptr(ms), ctypes.byref(n)))
    return ms.astype(np.float64), int(n.value)


def corr_integrate_static(n_ant, n_pol, n_fft, n_int, x, vis, beams, delay, phi0=None, rate=None,
                          n_avail=None, g0: int = 0, stream=None, blocking: int = 1):
    """One FP32 integration with no allocation: x device int8 [n_in][ld], vis and beams device
    float32 tensors of [n_chan][n_bl][n_pol^2][2] and [2][n_int][n_chan]."""
    d = np.ascontiguousarray(delay, dtype=np.float64)
    f = None if phi0 is None else np.ascontiguousarray(phi0, dtype=np.float64)
    w = None if rate is None else np.ascontiguousarray(rate, dtype=np.float64)
    n_avail = x.shape[1] if n_avail is None else n_avail
    return _ok(load().corr_integrate_static(n_ant, n_pol, n_fft, n_int, _ptr(x), x.stride(0), n_avail, g0,
                                            _ptr(d), _ptr(f), _ptr(w), _ptr(vis), _ptr(beams),
                                            _stream(stream), blocking))


def corr_set_power_dump(h, dump: int):
    return _ok(load().corr_set_power_dump(h, dump))


def corr_power_device(h):
    """Device address of the power-dump buffer [n_in][n_dump][n_chan] float32."""
    dev = ctypes.c_void_p()
    _ok(load().corr_read_power(h, None, ctypes.byref(dev)))
    return dev.value


CORR_BEAM_FULLPOL, CORR_BEAM_VOLTAGE = 0, 1


def corr_set_multibeam(h, weights=None, products: int = 0, avg: int = 1):
    """Phased beams from complex weights [n_beams][n_ant][n_chan] (None: off)."""
    if weights is None:
        return _ok(load().corr_set_multibeam(h, 0, None, 0, 1))
    w = np.asarray(weights)
    wr = np.ascontiguousarray(np.stack([w.real, w.imag], axis=-1), dtype=np.float32)
    return _ok(load().corr_set_multibeam(h, w.shape[0], _ptr(wr), int(products), int(avg)))


def corr_read_multibeam(h, n_beams: int, n_out: int, blocking: int = 1):
    """The last integration's beams [n_beams][n_out = n_int/avg][n_chan][4] float32."""
    i = corr_info(h)
    out = np.empty((n_beams, n_out, i["n_chan"], 4), dtype=np.float32)
    _ok(load().corr_read_multibeam(h, _ptr(out), blocking))
    return out


def corr_set_blanker(h, M: float, block: int = 0, noise=None):
    """Time-domain voltage blanker (M = 0: off); noise float32 [n_in][L] standard normal."""
    if M == 0:
        return _ok(load().corr_set_blanker(h, 0.0, 0, None, 0))
    g = np.ascontiguousarray(noise, dtype=np.float32)
    return _ok(load().corr_set_blanker(h, float(M), int(block), _ptr(g), g.shape[1]))


def corr_read_blank_stats(h):
    """(stats int32 [n_in][n_blocks][4] = 2 med, 4 MAD, T2, replaced; samples covered per row)."""
    nb, ns = ctypes.c_int64(), ctypes.c_int64()
    _ok(load().corr_read_blank_stats(h, None, ctypes.byref(nb), ctypes.byref(ns)))
    out = np.empty((corr_info(h)["n_in"], nb.value, 4), dtype=np.int32)
    _ok(load().corr_read_blank_stats(h, _ptr(out), None, None))
    return out, int(ns.value)


def corr_read_power_host(h, n_dump: int):
    i = corr_info(h)
    out = np.empty((i["n_in"], n_dump, i["n_chan"]), dtype=np.float32)
    _ok(load().corr_read_power(h, _ptr(out), None))
    return out


# ------------------------------------------------------------------ rfi.h

def rfi_n_params() -> int:
    return int(load().rfi_n_params())


def rfi_create(max_batch: int):
    n = ctypes.c_void_p()
    _ok(load().rfi_create(ctypes.byref(n), max_batch))
    return n


def rfi_create_fp32(max_batch: int):
    n = ctypes.c_void_p()
    _ok(load().rfi_create_fp32(ctypes.byref(n), max_batch))
    return n


def rfi_destroy(net):
    return _ok(load().rfi_destroy(net))


def rfi_set_params(net, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == rfi_n_params()
    return _ok(load().rfi_set_params(net, _ptr(p)))


def rfi_get_params(net):
    p = np.empty(rfi_n_params(), dtype=np.float32)
    _ok(load().rfi_get_params(net, _ptr(p)))
    return p


def rfi_loss_grad(net, x, mask, B: int, stream=None):
    """(loss, grad float32 [n_params]) of a batch; x fp16 and mask uint8 device tensors."""
    loss = ctypes.c_float()
    g = np.empty(rfi_n_params(), dtype=np.float32)
    _ok(load().rfi_loss_grad(net, _ptr(x), _ptr(mask), B, ctypes.byref(loss), _ptr(g), _stream(stream)))
    return float(loss.value), g


def rfi_train_step(net, x, mask, B: int, lr: float, want_loss: bool = False, stream=None):
    loss = ctypes.c_float()
    _ok(load().rfi_train_step(net, _ptr(x), _ptr(mask), B, lr, ctypes.byref(loss) if want_loss else None,
                              _stream(stream)))
    return float(loss.value) if want_loss else None


def rfi_infer(net, x, B: int, prob, stream=None):
    return _ok(load().rfi_infer(net, _ptr(x), B, _ptr(prob), _stream(stream)))


def rfi_patches(power, n_in: int, n_dump: int, n_chan: int, M: float, x=None, flags=None, stats=None, stream=None):
    return _ok(load().rfi_patches(_ptr(power), n_in, n_dump, n_chan, M, _ptr(x), _ptr(flags), _ptr(stats),
                                  _stream(stream)))


def corr_set_xengine_stage(h, ks: int):
    return _ok(load().corr_set_xengine_stage(h, ks))


def corr_batch_create(handles):
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    b = ctypes.c_void_p()
    _ok(load().corr_batch_create(ctypes.byref(b), len(handles), arr))
    return b


def corr_batch_destroy(b):
    return _ok(load().corr_batch_destroy(b))


def corr_batch_integrate_device(b, xs, n_avail=None, g0=None, stream=None):
    """xs: device int8 tensors [n_in_s][ld_s], one per sub-array."""
    n = len(xs)
    ptrs = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    lds = np.ascontiguousarray([x.stride(0) for x in xs], dtype=np.int64)
    na = np.ascontiguousarray(n_avail if n_avail is not None else [x.shape[1] for x in xs], dtype=np.int64)
    g = None if g0 is None else np.ascontiguousarray(g0, dtype=np.int64)
    return _ok(load().corr_batch_integrate_device(b, ptrs, _ptr(lds), _ptr(na), _ptr(g), _stream(stream)))


def corr_batch_tune(b, n_sub: int):
    """(chosen frames-per-stage, their X-engine ms) per sub-array."""
    ks = np.zeros(n_sub, dtype=np.int32)
    ms = np.zeros(n_sub, dtype=np.float32)
    _ok(load().corr_batch_tune(b, _ptr(ks), _ptr(ms)))
    return ks, ms


def corr_dd_smear_samples(dm: float, f_lo: float, bw: float) -> float:
    return load().corr_dd_smear_samples(dm, f_lo, bw)


def corr_dd_create(n_chan: int, fft_frames: int, overlap_frames: int, max_push_frames: int, dm: float, f_lo: float,
                   bw: float, avg: int):
    d = ctypes.c_void_p()
    _ok(load().corr_dd_create(ctypes.byref(d), n_chan, fft_frames, overlap_frames, max_push_frames, dm, f_lo, bw,
                              avg))
    return d


def corr_dd_push_device(d, spec, out, stream=None) -> int:
    """spec: device float32 tensor [n_frames][n_chan][4] (X re, X im, Y re, Y im), contiguous;
    out: device float32 tensor receiving the outputs of the blocks this push completes.
    Returns their count."""
    n = ctypes.c_int64(0)
    _ok(load().corr_dd_push_device(d, _ptr(spec), spec.shape[0], _ptr(out), out.numel(), ctypes.byref(n),
                                   _stream(stream)))
    return n.value


def corr_dd_set_timing(d, on: bool):
    return _ok(load().corr_dd_set_timing(d, 1 if on else 0))


def corr_dd_stage_times(d):
    """(ms[5] summed over the timed pushes: ring copy, A, B, C, D; number of timed pushes)"""
    ms = np.zeros(5, np.float32)
    n = ctypes.c_int(0)
    _ok(load().corr_dd_stage_times(d, _ptr(ms), ctypes.byref(n)))
    return ms, n.value


def corr_dd_reset(d):
    return _ok(load().corr_dd_reset(d))


def corr_dd_destroy(d):
    return _ok(load().corr_dd_destroy(d))


def corr_wait_selftest() -> int:
    """Run the bounded-wait self-test; returns the clock cycles the wait took before giving up."""
    c = ctypes.c_longlong(0)
    _ok(load().corr_wait_selftest(ctypes.byref(c)))
    return c.value
