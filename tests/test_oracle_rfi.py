"""Pins for the RFI-stage oracle: network forward pass against closed forms and scipy's
2-D correlation, loss and gradient against closed forms and central finite differences,
patch statistics against numpy's median, power dumps against a numpy reduction."""
import math

import numpy as np
import pytest


def _zero_params(orc):
    return np.zeros(orc.rfi_n_params())


def _offsets():
    """Offsets of W1 b1 W2 b2 W3 b3 W4 b4 in the flat parameter vector."""
    out, o = {}, 0
    for name, n in (("W1", 16 * 1 * 9), ("b1", 16), ("W2", 32 * 16 * 9), ("b2", 32), ("W3", 16 * 32 * 9),
                    ("b3", 16), ("W4", 16), ("b4", 1)):
        out[name] = (o, n)
        o += n
    return out, o


def test_parameter_count(orc):
    offs, total = _offsets()
    assert orc.rfi_n_params() == total == 9441


def test_forward_bias_only_and_identity_chain(orc):
    offs, _ = _offsets()
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 9, 7))
    p = _zero_params(orc)
    p[offs["b4"][0]] = 0.37
    assert np.allclose(orc.rfi_forward(p, x), 0.37, rtol=0, atol=1e-15)
    # centre taps of channel 0 through every layer, head reads channel 0: logit = relu(x)
    p = _zero_params(orc)
    p[offs["W1"][0] + 4] = 1.0                      # W1[0][0][1][1]
    p[offs["W2"][0] + 4] = 1.0                      # W2[0][0][1][1]
    p[offs["W3"][0] + 4] = 1.0                      # W3[0][0][1][1]
    p[offs["W4"][0]] = 1.0
    assert np.allclose(orc.rfi_forward(p, x), np.maximum(x, 0.0), rtol=0, atol=1e-15)


def test_first_layer_is_same_padded_cross_correlation(orc):
    scipy_signal = pytest.importorskip("scipy.signal")
    offs, _ = _offsets()
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 10, 12))
    K = rng.normal(size=(3, 3))
    p = _zero_params(orc)
    p[offs["W1"][0]:offs["W1"][0] + 9] = K.ravel()
    p[offs["W2"][0] + 4] = 1.0
    p[offs["W3"][0] + 4] = 1.0
    p[offs["W4"][0]] = 1.0
    ref = np.maximum(scipy_signal.correlate2d(x[0], K, mode="same", boundary="fill", fillvalue=0.0), 0.0)
    assert np.abs(orc.rfi_forward(p, x)[0] - ref).max() < 1e-12


def test_loss_and_head_gradient_at_zero_parameters(orc):
    offs, _ = _offsets()
    rng = np.random.default_rng(2)
    x = rng.normal(size=(3, 8, 8))
    m = (rng.random((3, 8, 8)) < 0.2).astype(np.uint8)
    loss, g = orc.rfi_loss_grad(_zero_params(orc), x, m)
    assert abs(loss - math.log(2.0)) < 1e-13                       # p = 1/2 everywhere
    assert abs(g[offs["b4"][0]] - np.mean(0.5 - m)) < 1e-15       # dL/db4 = mean(p - m)
    assert np.all(g[:offs["W4"][0]] == 0.0)                         # nothing upstream of a zero head


@pytest.mark.parametrize("seed", [3, 4])
def test_gradient_matches_central_differences(orc, seed):
    rng = np.random.default_rng(seed)
    B, H, W = 2, 8, 8
    x = rng.normal(size=(B, H, W))
    m = (rng.random((B, H, W)) < 0.3).astype(np.uint8)
    p = rng.normal(scale=0.3, size=orc.rfi_n_params())
    offs, _ = _offsets()
    p[offs["b1"][0]:offs["b1"][0] + 16] += 0.2        # keep most units active
    loss, g = orc.rfi_loss_grad(p, x, m)
    pick = []
    for name, (o, n) in offs.items():
        pick += list(rng.choice(np.arange(o, o + n), size=min(n, 12), replace=False))
    eps = 1e-6
    checked = 0
    for j in pick:
        pp, pm = p.copy(), p.copy()
        pp[j] += eps
        pm[j] -= eps
        fd = (orc.rfi_loss_grad(pp, x, m)[0] - orc.rfi_loss_grad(pm, x, m)[0]) / (2 * eps)
        scale = max(abs(fd), abs(g[j]), 1e-7)
        assert abs(fd - g[j]) <= 1e-5 * scale + 1e-9, (j, fd, g[j])
        checked += 1
    assert checked >= 80


def test_patch_stats_against_numpy_median(orc):
    rng = np.random.default_rng(5)
    x = rng.gamma(4.0, size=(5, 64, 64))
    x[0, 3, 4] = 500.0
    med, mad, flags, z = orc.patch_stats(x, M=5.0)
    for b in range(5):
        m = np.median(x[b])
        d = np.median(np.abs(x[b] - m))
        assert med[b] == m and mad[b] == d
        assert np.array_equal(flags[b], (np.abs(x[b] - m) > 5.0 * d / 0.6745).astype(np.uint8))
    assert flags[0, 3, 4] == 1
    u = (x[1] - med[1]) / (mad[1] / 0.6745)
    assert np.allclose(z[1], np.sign(u) * np.log1p(np.abs(u)), rtol=1e-14, atol=1e-14)


def test_power_dumps_against_numpy(orc):
    rng = np.random.default_rng(6)
    Y = rng.normal(size=(3, 64, 5)) + 1j * rng.normal(size=(3, 64, 5))
    P = orc.power_dumps(Y, 32)
    ref = (np.abs(Y) ** 2).reshape(3, 2, 32, 5).sum(axis=2)
    assert np.allclose(P, ref, rtol=1e-14)
