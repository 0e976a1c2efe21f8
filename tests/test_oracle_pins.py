"""Pins for the FP64 oracle: each test ties an oracle function to something other
than itself -- hand-worked values, a library routine on a special case, a closed
form, an invariant, or brute force on a tiny input -- so that a dropped term, a
wrong sign or index, or a transposed operand fails at least one of them.
"""
import cmath
import math
import os

import numpy as np
import pytest

from synth import make_config, make_streams

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _zero(n):
    return np.zeros(n, dtype=np.float64)


# ---------------------------------------------------------------- DFT (Sec. 2.1)

def test_dft_hand_worked_values(orc):
    """Hand-computed DFTs of short frames (golden/dft_hand.txt)."""
    with open(os.path.join(GOLDEN, "dft_hand.txt")) as f:
        rows = [ln for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) >= 8
    for ln in rows:
        n_s, samp_s, exp_s = ln.split("|")
        N = int(n_s)
        x = np.array([int(v) for v in samp_s.split()], dtype=np.int8)[None, :]
        Y = orc.fengine(x, 1, 1, N, 1, _zero(1), _zero(1), _zero(1))[0, 0]
        for item in exp_s.split(";"):
            k, re, im = item.split()
            assert abs(Y[int(k)] - complex(float(re), float(im))) < 1e-12, (ln, k, Y)


@pytest.mark.parametrize("N", [8, 16, 64, 512, 2048])
def test_dft_matches_numpy_rfft(orc, N):
    """Zero delay and zero fringe reduce the F-stage to a plain real DFT."""
    rng = np.random.default_rng(N)
    n_frames = 3
    x = rng.integers(-127, 128, size=(2, n_frames * N), dtype=np.int8)
    Y = orc.fengine(x, 1, 2, N, n_frames, _zero(1), _zero(1), _zero(1))
    for i in range(2):
        for t in range(n_frames):
            ref = np.fft.rfft(x[i, t * N:(t + 1) * N].astype(np.float64))[: N // 2]
            scale = np.abs(ref).max()
            assert np.abs(Y[i, t] - ref).max() <= 1e-12 * scale


def test_dft_bruteforce_tiny(orc):
    """N = 8 against a nested Python sum over cmath.exp."""
    x = np.array([[3, -1, 4, -1, 5, -9, 2, 6]], dtype=np.int8)
    Y = orc.fengine(x, 1, 1, 8, 1, _zero(1), _zero(1), _zero(1))[0, 0]
    for k in range(4):
        s = sum(int(x[0, n]) * cmath.exp(-2j * math.pi * k * n / 8) for n in range(8))
        assert abs(Y[k] - s) < 1e-12


def test_parseval_unnormalised(orc):
    """sum x^2 = (|X0|^2 + 2 sum_{0<k<N/2} |Xk|^2 + |X_{N/2}|^2) / N for the unnormalised DFT."""
    rng = np.random.default_rng(5)
    N = 256
    x = rng.integers(-100, 100, size=(1, N), dtype=np.int8)
    Y = orc.fengine(x, 1, 1, N, 1, _zero(1), _zero(1), _zero(1))[0, 0]
    xf = x[0].astype(np.float64)
    nyq = np.sum(xf * (-1.0) ** np.arange(N))
    lhs = np.sum(xf ** 2)
    rhs = (abs(Y[0]) ** 2 + 2 * np.sum(np.abs(Y[1:]) ** 2) + nyq ** 2) / N
    assert abs(lhs - rhs) <= 1e-10 * lhs


# ---------------------------------------------------------- delays (Sec. 2.1)

@pytest.mark.parametrize("D", [0, 1, 5, 17])
def test_integer_delay_impulse(orc, D):
    """An impulse at n0 seen through integer delay D lands at n0 - D: X[k] = A e^{-2 pi i k (n0-D)/N}."""
    N, n0, A = 64, 40, 7
    x = np.zeros((1, N + 32), dtype=np.int8)
    x[0, n0] = A
    Y = orc.fengine(x, 1, 1, N, 1, np.array([float(D)]), _zero(1), _zero(1))[0, 0]
    k = np.arange(N // 2)
    ref = A * np.exp(-2j * np.pi * k * (n0 - D) / N)
    assert np.abs(Y - ref).max() < 1e-12


def test_integer_part_rounds_half_up(orc):
    """tau = 2.5 -> D = 3, tau_f = -0.5; tau = 2.49 -> D = 2.  Checked on an impulse."""
    N, n0 = 32, 10
    x = np.zeros((1, N + 8), dtype=np.int8)
    x[0, n0] = 1
    k = np.arange(N // 2)
    for tau, D in ((2.5, 3), (2.49, 2), (0.0, 0), (3.5, 4)):
        Y = orc.fengine(x, 1, 1, N, 1, np.array([tau]), _zero(1), _zero(1))[0, 0]
        tf = tau - D
        ref = np.exp(-2j * np.pi * k * (n0 - D) / N) * np.exp(2j * np.pi * k * tf / N)
        assert np.abs(Y - ref).max() < 1e-12, tau


def test_delay_out_of_range_is_an_error(orc):
    x = np.zeros((1, 64), dtype=np.int8)
    with pytest.raises(ValueError):
        orc.fengine(x, 1, 1, 64, 1, np.array([1.0]), _zero(1), _zero(1))
    with pytest.raises(ValueError):
        orc.fengine(x, 1, 1, 32, 1, np.array([-1.0]), _zero(1), _zero(1))


def test_fstc_cancels_a_fractional_delay_on_a_tone(orc):
    """A bin-centred cosine delayed by a fractional tau has X[k0] = (A N/2) e^{-2 pi i k0 tau / N};
    the FSTC factor e^{+2 pi i k0 tau_f / N} must bring it back to a real positive value."""
    N, k0, A = 512, 37, 100.0
    n = np.arange(2 * N)
    for tau in (0.3, -0.4, 0.49):
        x = np.rint(A * np.cos(2 * np.pi * k0 * (n - tau) / N)).astype(np.int8)[None, :]
        Y0 = orc.fengine(x, 1, 1, N, 1, _zero(1), _zero(1), _zero(1))[0, 0, k0]
        Yc = orc.fengine(x, 1, 1, N, 1, np.array([tau]), _zero(1), _zero(1))[0, 0, k0]
        # before correction the tone carries the delay phase, after it is gone
        assert abs(cmath.phase(Y0) + 2 * math.pi * k0 * tau / N) < 2e-3
        assert abs(cmath.phase(Yc)) < 2e-3
        assert abs(abs(Yc) - A * N / 2) < 1e-3 * A * N / 2


def test_fstc_recovers_injected_delay_as_phase_slope(orc):
    """Sky signal reaching antenna 1 tau samples late: the uncorrected cross-spectrum
    V_01 has phase slope +2 pi tau / N over channels; the corrected one is flat."""
    N, n_int, tau = 256, 256, 0.37
    x = make_streams(2, 1, n_int * N + 8, n_fft=N, sigma=20.0, rho=0.9, sky_delay=[0.0, tau], seed=11)
    k = np.arange(N // 2)
    sel = slice(4, N // 2 - 4)
    for applied, expect in ((0.0, tau), (tau, 0.0)):
        Y = orc.fengine(x, 2, 1, N, n_int, np.array([0.0, applied]), _zero(2), _zero(2))
        V = orc.xengine(Y, 2, 1)[:, 1, 0]           # baseline (0,1)
        ph = np.unwrap(np.angle(V[sel]))
        slope = np.polyfit(k[sel], ph, 1)[0]
        est = slope * N / (2 * np.pi)
        assert abs(est - expect) < 0.02, (applied, est)


# ------------------------------------------------------- fringe (Eq. 2)

def _golden_washing():
    out = []
    with open(os.path.join(GOLDEN, "fringe_washing.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                n, dw, fac = ln.split()
                out.append((int(n), float(dw), float(fac)))
    return out


def test_fringe_washing_closed_form_golden():
    """The golden washing factors agree with the closed form they were taken from."""
    for n, dw, fac in _golden_washing():
        assert abs(abs(math.sin(n * dw / 2) / (n * math.sin(dw / 2))) - fac) < 1e-5


def test_fringe_tone_cross_visibility_closed_form(orc):
    """Noise-free tone, identical periodic raw streams, integer delays D_a and fringe
    rates w_a: V_ab[k0] = |X|^2 e^{2 pi i k0 (D_a - D_b)/N} sum_t e^{-i (phi_a - phi_b)(g0 + t)}."""
    N, k0, A, n_int, g0 = 512, 37, 8.0, 64, 1000
    D = np.array([0.0, 1.0, 2.0, 3.0])
    w = np.array([0.0, 0.01, 0.02, 0.03])
    f0 = np.array([0.0, 0.5, -1.0, 2.0])
    n = np.arange(n_int * N + 8)
    tone = np.rint(A * np.cos(2 * np.pi * k0 * n / N)).astype(np.int8)
    x = np.repeat(tone[None, :], 4, axis=0)
    # |X[k0]|^2 of one period, by brute force
    X = sum(float(tone[m]) * cmath.exp(-2j * math.pi * k0 * m / N) for m in range(N))
    Y = orc.fengine(x, 4, 1, N, n_int, D, f0, w, g0=g0)
    V = orc.xengine(Y, 4, 1)
    washing = {round(dw, 2): fac for _, dw, fac in _golden_washing()}
    b = 0
    for a in range(4):
        for a2 in range(a, 4):
            t = np.arange(n_int) + g0
            geo = np.sum(np.exp(-1j * ((f0[a] - f0[a2]) + (w[a] - w[a2]) * t)))
            ref = abs(X) ** 2 * cmath.exp(2j * math.pi * k0 * (D[a] - D[a2]) / N) * geo
            got = V[k0, b, 0]
            assert abs(got - ref) <= 1e-9 * abs(X) ** 2 * n_int, (a, a2)
            dw = round(abs(w[a2] - w[a]), 2)
            if dw in washing:
                assert abs(abs(got) / (abs(X) ** 2 * n_int) - washing[dw]) < 2e-5
            b += 1


def test_fringe_phase_uses_global_frame_counter(orc):
    """Spectra of frames [g0, g0+n) equal the corresponding frames of a run from frame 0."""
    N, n_int = 64, 8
    rng = np.random.default_rng(3)
    x = rng.integers(-50, 50, size=(2, 3 * n_int * N + 4), dtype=np.int8)
    d, f0, w = np.array([2.3]), np.array([0.7]), np.array([0.05])
    full = orc.fengine(x, 1, 2, N, 3 * n_int, d, f0, w, g0=0)
    part = orc.fengine(x[:, n_int * N:], 1, 2, N, n_int, d, f0, w, g0=n_int)
    assert np.abs(part - full[:, n_int:2 * n_int]).max() < 1e-9


# -------------------------------------------------------- MAC (Sec. 2.1)

def test_tiny_everything_bruteforce(orc):
    """n_ant = 2, n_pol = 2, N = 8, two frames, fractional delays, fringe: the whole F and X
    chain against hand-expanded sums over the definitions."""
    N, n_int, n_ant, n_pol = 8, 2, 2, 2
    rng = np.random.default_rng(42)
    x = rng.integers(-127, 128, size=(4, n_int * N + 3), dtype=np.int8)
    tau = [1.3, 2.6]
    f0 = [0.4, -1.1]
    w = [0.2, -0.35]
    g0 = 5
    Y = orc.fengine(x, n_ant, n_pol, N, n_int, np.array(tau), np.array(f0), np.array(w), g0=g0)
    V = orc.xengine(Y, n_ant, n_pol)
    Yb = {}
    for a in range(n_ant):
        D = math.floor(tau[a] + 0.5)
        tf = tau[a] - D
        for p in range(n_pol):
            i = a * n_pol + p
            for t in range(n_int):
                for k in range(N // 2):
                    s = 0j
                    for m in range(N):
                        s += int(x[i, t * N + D + m]) * cmath.exp(-2j * math.pi * k * m / N)
                    ph = 2 * math.pi * k * tf / N - (f0[a] + w[a] * (g0 + t))
                    Yb[i, t, k] = s * cmath.exp(1j * ph)
                    assert abs(Y[i, t, k] - Yb[i, t, k]) < 1e-9
    b = 0
    for a in range(n_ant):
        for a2 in range(a, n_ant):
            for p in range(n_pol):
                for q in range(n_pol):
                    for k in range(N // 2):
                        s = sum(Yb[a * n_pol + p, t, k] * Yb[a2 * n_pol + q, t, k].conjugate()
                                for t in range(n_int))
                        assert abs(V[k, b, p * n_pol + q] - s) < 1e-8
            b += 1
    assert b == 3


def test_visibility_matrix_hermitian_psd_autos(orc):
    s = make_config(1, n_int=16)
    Y = orc.fengine(s.x, s.n_ant, s.n_pol, s.n_fft, s.n_int, s.delay, s.phi0, s.rate)
    V = orc.xengine(Y, s.n_ant, s.n_pol)
    n_in, na, npol = s.n_in, s.n_ant, s.n_pol
    bl = {}
    b = 0
    for a in range(na):
        for a2 in range(a, na):
            bl[a, a2] = b
            b += 1
    for k in (0, 5, 37, 200):
        M = np.zeros((n_in, n_in), complex)
        for a in range(na):
            for a2 in range(a, na):
                for p in range(npol):
                    for q in range(npol):
                        v = V[k, bl[a, a2], p * npol + q]
                        M[a * npol + p, a2 * npol + q] = v
                        M[a2 * npol + q, a * npol + p] = np.conj(v)
        for a in range(na):
            d = bl[a, a]
            for p in range(npol):
                auto = V[k, d, p * npol + p]
                assert auto.imag == 0.0 and auto.real >= 0.0
            # RL* and LR* of one antenna are exact conjugates
            assert V[k, d, 1] == np.conj(V[k, d, 2])
        ev = np.linalg.eigvalsh(M)
        assert ev.min() >= -1e-12 * np.trace(M).real


def test_tone_power_and_correlated_noise_statistics(orc):
    """Tiny configuration: the tone channel's auto power and the noise coherence
    match their expectations within five standard errors."""
    s = make_config(1, n_int=512, tail=3)
    N, n_int = s.n_fft, s.n_int
    Y = orc.fengine(s.x, s.n_ant, s.n_pol, N, n_int, s.delay, s.phi0, s.rate)
    V = orc.xengine(Y, s.n_ant, s.n_pol)
    sig2 = 20.0 ** 2 + 1.0 / 12.0           # sample variance incl. rounding
    A = 8.0
    auto37 = V[37, 0, 0].real
    expect = n_int * ((A * N / 2) ** 2 + N * sig2)
    se = n_int ** 0.5 * (2 * (A * N / 2) ** 2 * N * sig2) ** 0.5 + (n_int ** 0.5) * N * sig2
    assert abs(auto37 - expect) < 5 * se
    # coherence away from the tone: rho * sigma^2 / (sigma^2 + 1/12) times fringe washing
    rho = 0.3 * 400.0 / sig2
    ch = np.r_[2:30, 45:250]
    b = {(0, 1): 1, (0, 2): 2, (1, 2): 5}
    for (a, a2), bi in b.items():
        dw = abs(s.rate[a2] - s.rate[a])
        wash = abs(np.mean(np.exp(-1j * (s.rate[a] - s.rate[a2]) * np.arange(n_int))))
        coh = V[ch, bi, 0] / np.sqrt(V[ch, bl_auto(a, 4), 0].real * V[ch, bl_auto(a2, 4), 0].real)
        est = abs(np.mean(coh))
        se = (1 - rho ** 2) / math.sqrt(n_int * len(ch))
        assert abs(est - rho * wash) < 5 * se + 1e-3, (a, a2, dw, est, rho * wash)


def bl_auto(a, n_ant):
    return a * n_ant - a * (a - 1) // 2


# ---------------------------------------------------------- beams (Sec. 2.2)

def test_beams_single_antenna_and_identical_inputs(orc):
    rng = np.random.default_rng(9)
    N, n_int, na = 64, 4, 5
    one = rng.integers(-60, 60, size=(2, n_int * N), dtype=np.int8)
    x = np.tile(one, (na, 1))                         # every antenna sees the same voltages
    z = _zero(na)
    Y = orc.fengine(x, na, 2, N, n_int, z, z, z)
    Bi, Bc = orc.beams(Y, na, 2, N)
    assert np.allclose(Bc, na * Bi, rtol=1e-12, atol=0)         # coherent gain n_a over incoherent
    m = np.zeros(na, np.uint8)
    m[2] = 1
    Bi1, Bc1 = orc.beams(Y, na, 2, N, inc_mask=m, coh_mask=m)
    assert np.allclose(Bi1, Bc1, rtol=1e-12, atol=0)            # one antenna: both beams equal
    P = np.abs(Y[4]) ** 2 + np.abs(Y[5]) ** 2
    assert np.allclose(Bi1, P, rtol=1e-12, atol=0)
    g = np.linspace(0.5, 1.5, na)
    Bi2, Bc2 = orc.beams(Y, na, 2, N, gain=g)
    assert np.allclose(Bi2, np.sum(g ** 2) * P, rtol=1e-12)
    assert np.allclose(Bc2, np.sum(g) ** 2 * P, rtol=1e-12)


def test_coherent_beam_phase_calibration_rephases(orc):
    """Antenna a sees the common voltages D_a samples late; uncorrected delays leave
    a phase e^{-2 pi i k D_a/N} per channel, and theta_{a,k} = +2 pi k D_a / N restores
    the full coherent gain B_coh = n_a B_inc."""
    N, n_int, na = 128, 3, 4
    rng = np.random.default_rng(1)
    base = rng.integers(-60, 60, size=(n_int * N + 16,), dtype=np.int8)
    Dl = [0, 1, 2, 5]
    # periodic per frame so that the shift is circular within each frame
    fr = rng.integers(-60, 60, size=(N,), dtype=np.int8)
    per = np.tile(fr, n_int + 1)
    x = np.stack([np.roll(per, d)[: n_int * N + 4] for d in Dl])   # x_a[n] = per[n - D_a]
    z = _zero(na)
    Y = orc.fengine(x, na, 1, N, n_int, z, z, z)
    k = np.arange(N // 2)
    theta = np.stack([2 * np.pi * k * d / N for d in Dl])
    Bi, Bc = orc.beams(Y, na, 1, N, theta=theta)
    assert np.allclose(Bc, na * Bi, rtol=1e-10)
    Bi0, Bc0 = orc.beams(Y, na, 1, N)
    assert np.mean(Bc0) < 0.6 * na * np.mean(Bi0)
    del base


def test_beam_independent_noise_expectations_and_averaging(orc):
    """Independent noise: E[B_coh] = E[B_inc]; beam_avg = m averages m raw frames."""
    s = make_config(1, n_int=64, tail=3)
    s2 = make_streams(4, 2, 64 * 512 + 3, n_fft=512, sigma=20.0, rho=0.0, seed=77)
    z = _zero(4)
    Y = orc.fengine(s2, 4, 2, 512, 64, z, z, z)
    Bi, Bc = orc.beams(Y, 4, 2, 512)
    r = Bc.mean() / Bi.mean()
    assert abs(r - 1.0) < 5 * math.sqrt(2.0 / Bi.size) * 2
    Bi8, Bc8 = orc.beams(Y, 4, 2, 512, beam_avg=8)
    assert np.allclose(Bi8, Bi.reshape(8, 8, -1).mean(axis=1), rtol=1e-12)
    assert np.allclose(Bc8, Bc.reshape(8, 8, -1).mean(axis=1), rtol=1e-12)
    del s


# ------------------------------------------------ requantisation / integer MAC

def test_requant_rounding_and_clamp(orc):
    vals = np.array([0.5, 1.5, 2.5, -0.5, -1.5, 126.5, 127.49, 127.6, 300.0, -300.0, -127.5, 3.2])
    Y = (vals + 1j * vals[::-1])[None, None, :]
    q = orc.requant(Y, np.ones((1, vals.size)))
    exp_re = [0, 2, 2, 0, -2, 126, 127, 127, 127, -127, -127, 3]
    assert q[0, 0, :, 0].tolist() == exp_re
    assert q[0, 0, :, 1].tolist() == exp_re[::-1]
    rng = np.random.default_rng(2)
    Y = rng.normal(0, 40, size=(3, 5, 7)) + 1j * rng.normal(0, 40, size=(3, 5, 7))
    s = rng.uniform(0.5, 2.0, size=(3, 7))
    q = orc.requant(Y, s)
    ref = np.clip(np.rint(Y.real * s[:, None, :]), -127, 127)
    assert np.array_equal(q[..., 0], ref.astype(np.int8))


def test_xint_exact_against_bruteforce_and_int64_matmul(orc):
    rng = np.random.default_rng(8)
    na, npol, nf, nch = 3, 2, 40, 5
    q = rng.integers(-127, 128, size=(na * npol, nf, nch, 2), dtype=np.int8)
    s = rng.uniform(0.1, 1.0, size=(na * npol, nch))
    Vi, V = orc.xint(q, s, na, npol)
    # brute force, one baseline
    a, a2, p, qq, c = 0, 2, 1, 0, 3
    i, j = a * npol + p, a2 * npol + qq
    sr = sum(int(q[i, t, c, 0]) * int(q[j, t, c, 0]) + int(q[i, t, c, 1]) * int(q[j, t, c, 1]) for t in range(nf))
    si = sum(int(q[i, t, c, 1]) * int(q[j, t, c, 0]) - int(q[i, t, c, 0]) * int(q[j, t, c, 1]) for t in range(nf))
    b = 2
    assert Vi[c, b, p * npol + qq].tolist() == [sr, si]
    # library int64 matmul for all of them
    z = q[..., 0].astype(np.int64) + 1j * 0
    qc = q[..., 0].astype(np.int64), q[..., 1].astype(np.int64)
    for c in range(nch):
        R = qc[0][:, :, c] @ qc[0][:, :, c].T + qc[1][:, :, c] @ qc[1][:, :, c].T
        I = qc[1][:, :, c] @ qc[0][:, :, c].T - qc[0][:, :, c] @ qc[1][:, :, c].T
        b = 0
        for a in range(na):
            for a2 in range(a, na):
                for p in range(npol):
                    for qq in range(npol):
                        i, j = a * npol + p, a2 * npol + qq
                        assert Vi[c, b, p * npol + qq, 0] == R[i, j]
                        assert Vi[c, b, p * npol + qq, 1] == I[i, j]
                        d = s[i, c] * s[j, c]
                        assert abs(V[c, b, p * npol + qq] - complex(R[i, j], I[i, j]) / d) <= 1e-12 * abs(complex(R[i, j], I[i, j]) / d) + 1e-300
                b += 1
    del z


def test_xint_descaled_equals_xengine_on_dequantised(orc):
    rng = np.random.default_rng(4)
    q = rng.integers(-127, 128, size=(4, 30, 6, 2), dtype=np.int8)
    s = rng.uniform(0.2, 3.0, size=(4, 6))
    _, V = orc.xint(q, s, 2, 2)
    Yd = (q[..., 0] + 1j * q[..., 1]) / s[:, None, :]
    V2 = orc.xengine(Yd, 2, 2)
    assert np.abs(V - V2).max() <= 1e-12 * np.abs(V2).max()


def test_self_polar_mac_is_the_same_polarisation_products(orc):
    # the self-polar (total-intensity) MAC keeps exactly the pp products of the full-polar one
    # (itself pinned above), and a hand-written nested sum on a tiny input fixes one of them
    rng = np.random.default_rng(12)
    na, npol, nf, nch = 3, 2, 17, 4
    Y = rng.standard_normal((na * npol, nf, nch)) + 1j * rng.standard_normal((na * npol, nf, nch))
    Vf = orc.xengine(Y, na, npol)
    Vs = orc.xengine_self(Y, na, npol)
    assert Vs.shape == (nch, na * (na + 1) // 2, npol)
    for p in range(npol):
        assert np.array_equal(Vs[:, :, p], Vf[:, :, p * npol + p])
    a, a2, p, c = 1, 2, 1, 3
    ref = sum(Y[a * npol + p, t, c] * np.conj(Y[a2 * npol + p, t, c]) for t in range(nf))
    b = na + (a2 - a)                      # baselines (0,0) (0,1) (0,2) (1,1) (1,2) ...
    assert abs(Vs[c, b, p] - ref) <= 1e-12 * abs(ref)
    # one polarisation: self-polar is the full-polar MAC
    assert np.array_equal(orc.xengine_self(Y[:na], na, 1)[:, :, 0], orc.xengine(Y[:na], na, 1)[:, :, 0])
    # the integer form equals the full integer MAC's pp entries
    q = rng.integers(-127, 128, size=(na * npol, nf, nch, 2), dtype=np.int8)
    Vi, _ = orc.xint(q, np.ones((na * npol, nch)), na, npol)
    Vis = orc.xint_self(q, na, npol)
    for p in range(npol):
        assert np.array_equal(Vis[:, :, p], Vi[:, :, p * npol + p])


# -------------------------------------------------------------- MAD (Eq. 3-4)

def test_mad_flag_tiny_and_gaussian(orc):
    x = np.array([1.0, 2.0, 3.0, 4.0, 100.0])
    f, med, mad = orc.mad_flag(x, 3.0)
    assert med == 3.0 and mad == 1.0                   # |x-3| = 2 1 0 1 97 -> median 1
    assert f.tolist() == [0, 0, 0, 0, 1]               # threshold 3 * 1 / 0.6745 = 4.45
    x = np.array([1.0, 2.0, 4.0, 10.0])
    f, med, mad = orc.mad_flag(x, 2.5)
    assert med == 3.0 and mad == 1.5                   # |x-3| = 2 1 1 7 -> (1+2)/2
    assert f.tolist() == [0, 0, 0, 1]                  # 7 > 2.5 * 1.5 / 0.6745 = 5.56
    rng = np.random.default_rng(0)
    g = rng.normal(3.0, 7.0, size=200001)
    f, med, mad = orc.mad_flag(g, 3.0)
    assert abs(mad / 0.6745 - 7.0) < 0.05               # MAD / 0.6745 estimates sigma
    assert abs(f.mean() - 2 * (1 - 0.99865)) < 5e-4    # P(|z| > 3) = 0.0027


def test_cpu_fft_baseline_matches_the_dft_oracle(orc):
    """The bench's second CPU baseline (FP32 radix-2 FFT in place of the FP64 DFT) computes
    the oracle's spectra to FP32 accuracy, delays and fringes included."""
    for cfg, kw in ((1, {}), (2, dict(n_ant=4, n_fft=256, n_int=8, seed=77))):
        s = make_config(cfg, **kw)
        Y = orc.fengine(s.x, s.n_ant, s.n_pol, s.n_fft, s.n_int, s.delay, s.phi0, s.rate, g0=5)
        Yf = orc.fft_fengine(s.x, s.n_ant, s.n_pol, s.n_fft, s.n_int, s.delay, s.phi0, s.rate, g0=5)
        for i in range(s.n_in):
            assert np.abs(Yf[i] - Y[i]).max() <= 1e-5 * np.abs(Y[i]).max(), (cfg, i)


# ------------------------------------------------ time-domain voltage blanker (Sec. 5, Eq. 3-4)

def _noise_rows(n_in, L, seed):
    return np.random.default_rng(seed).standard_normal((n_in, L)).astype(np.float32)


def test_mad_blank_blocks_follow_eq3_eq4_per_block(orc):
    """Each block's median, MAD and flag count are those of the Eq. 3-4 flagger on that block
    (the ragged last block included); an impulse far above M sigma is always replaced."""
    rng = np.random.default_rng(11)
    n, block, M = 5000, 2048, 3.0
    x = np.clip(np.rint(rng.normal(0, 20, (3, n))), -127, 127).astype(np.int8)
    x[0, 100] = 120
    x[2, 4500:4510] = -127
    out, st = orc.mad_blank(x, block, M, _noise_rows(3, 1024, 5))
    for i in range(3):
        for b in range(3):
            seg = x[i, b * block:(b + 1) * block].astype(np.float64)
            f, med, mad = orc.mad_flag(seg, M)
            assert st[i, b, 0] == 2 * med and st[i, b, 1] == 4 * mad and st[i, b, 3] == f.sum()
            assert st[i, b, 2] == math.floor(2 * (M * mad / 0.6745))
            kept = f == 0
            assert np.array_equal(out[i, b * block:(b + 1) * block][kept], x[i, b * block:(b + 1) * block][kept])
    assert out[0, 100] != 120 and np.all(out[2, 4500:4510] != -127)
    assert st[2, 2, 3] >= 10                       # the last (904-sample) block holds the burst


def test_mad_blank_clean_gaussian_is_left_alone_at_large_M(orc):
    x = np.clip(np.rint(np.random.default_rng(3).normal(0, 20, (2, 8192))), -127, 127).astype(np.int8)
    out, st = orc.mad_blank(x, 4096, 50.0, _noise_rows(2, 256, 1))
    assert np.array_equal(out, x) and st[..., 3].sum() == 0


def test_mad_blank_replacement_noise_statistics_and_independence(orc):
    """Replaced samples are robust-sigma Gaussian noise (mean ~0, std ~ MAD/0.6745), drawn from
    each input's own table row: identical inputs with different rows get different noise."""
    rng = np.random.default_rng(21)
    n, block = 1 << 16, 4096
    row = np.clip(np.rint(rng.normal(0, 20, n)), -127, 127).astype(np.int8)
    row[::16] = 127                                 # 1 in 16 samples is an outlier
    x = np.stack([row, row])
    out, st = orc.mad_blank(x, block, 2.5, _noise_rows(2, 1 << 16, 9))
    rep0 = out[0, ::16].astype(np.float64)
    sigma = (st[0, :, 1] / 4.0 / 0.6745).mean()
    assert abs(rep0.mean()) < 0.1 * sigma and abs(rep0.std() / sigma - 1) < 0.05
    assert np.mean(out[0, ::16] != out[1, ::16]) > 0.9


def test_mad_blank_noise_index_is_the_row_position_mod_L(orc):
    """Replacement noise for row position p comes from table entry p mod L."""
    n, L = 3000, 64
    x = np.clip(np.rint(np.random.default_rng(8).normal(0, 20, (1, n))), -127, 127).astype(np.int8)
    hits = [5, 69, 133, 1029, 6, 70]                # 5 mod 64 (blocks 0 and 1), and 6 mod 64
    x[0, hits] = 127
    g = np.zeros((1, L), np.float32)
    g[0, 5] = 1.0                                   # only table entry 5 is non-zero
    out, st = orc.mad_blank(x, 1024, 3.0, g)
    sig0, sig1 = st[0, 0, 1] / 4.0 / 0.6745, st[0, 1, 1] / 4.0 / 0.6745
    assert out[0, 5] == out[0, 69] == out[0, 133] == round(sig0) != 0
    assert out[0, 1029] == round(sig1)
    assert out[0, 6] == out[0, 70] == 0


# ------------------------------------------------ multiple phased beams, full polar (Sec. 2.2, 5)

def test_multibeam_reduces_to_the_coherent_beam_and_to_autocorrelations(orc):
    """A beam with the coherent beam's weights has RR* + LL* equal to the (pinned) coherent beam;
    a beam with one unit weight has the per-frame autocorrelation products of that antenna; the
    voltage form is the weighted sum itself and its products are the full-polar form."""
    s = make_config(1, n_int=16)
    nch = s.n_fft // 2
    Y = orc.fengine(s.x, s.n_ant, s.n_pol, s.n_fft, s.n_int, s.delay, s.phi0, s.rate)
    rng = np.random.default_rng(5)
    gain = rng.uniform(0.5, 1.5, s.n_ant)
    theta = rng.uniform(-np.pi, np.pi, (s.n_ant, nch))
    coh = np.array([1, 0, 1, 1], np.uint8)
    w0 = (gain * coh)[:, None] * np.exp(1j * theta)
    w1 = np.zeros((s.n_ant, nch), complex)
    w1[2] = 1.0
    W = np.stack([w0, w1])
    B = orc.multibeam(Y, s.n_ant, s.n_pol, W, 0, 4)
    _, Bc = orc.beams(Y, s.n_ant, s.n_pol, s.n_fft, gain=gain, theta=theta, coh_mask=coh, beam_avg=4)
    assert np.allclose(B[0, ..., 0] + B[0, ..., 1], Bc, rtol=1e-12)
    V1 = np.stack([orc.xengine(Y[:, t:t + 1], s.n_ant, s.n_pol) for t in range(s.n_int)])  # per-frame V
    b = 2 * s.n_ant - 2 * (2 - 1) // 2                  # baseline (2, 2), row-major over a <= a'
    auto = V1[:, :, b]                                  # [t][c][pq]
    avg = auto.reshape(4, 4, nch, 4).mean(axis=1)
    assert np.allclose(B[1, ..., 0], avg[..., 0].real) and np.allclose(B[1, ..., 1], avg[..., 3].real)
    assert np.allclose(B[1, ..., 2], avg[..., 1].real) and np.allclose(B[1, ..., 3], avg[..., 1].imag)
    U = orc.multibeam(Y, s.n_ant, s.n_pol, W, 1, 1)
    u0, u1 = U[..., 0] + 1j * U[..., 1], U[..., 2] + 1j * U[..., 3]
    assert np.allclose(u0[1], Y[2 * 2 + 0]) and np.allclose(u1[1], Y[2 * 2 + 1])
    F = orc.multibeam(Y, s.n_ant, s.n_pol, W, 0, 1)
    assert np.allclose(F[..., 0], np.abs(u0) ** 2) and np.allclose(F[..., 2] + 1j * F[..., 3], u0 * np.conj(u1))


def test_multibeam_linearity_and_single_polarisation(orc):
    s = make_config(2, n_ant=3, n_fft=64, n_int=8, seed=9)
    Y = orc.fengine(s.x, s.n_ant, s.n_pol, s.n_fft, s.n_int, s.delay, s.phi0, s.rate)
    rng = np.random.default_rng(2)
    w = rng.standard_normal((2, s.n_ant, 32)) + 1j * rng.standard_normal((2, s.n_ant, 32))
    U = orc.multibeam(Y, s.n_ant, s.n_pol, w, 1, 1)
    U2 = orc.multibeam(Y, s.n_ant, s.n_pol, 2.5j * w, 1, 1)
    z, z2 = U[..., 0] + 1j * U[..., 1], U2[..., 0] + 1j * U2[..., 1]
    assert np.allclose(z2, 2.5j * z)
    Y1 = Y[0::2]                                        # pol 0 only: a single-polarisation array
    F = orc.multibeam(Y1, s.n_ant, 1, w, 0, 2)
    assert np.all(F[..., 1] == 0) and np.all(F[..., 2] == 0) and np.all(F[..., 3] == 0)
    assert np.allclose(F[..., 0], orc.multibeam(Y, s.n_ant, s.n_pol, w, 0, 2)[..., 0])


# ------------------------------------------------ ADC-format 4-bit ingest (Sec. 2.3.1, 2.3.2)

def test_unpack4_hand_worked_bytes(orc):
    # card 0, sample 0: 0x7F -> input 0 = -1 (0xF), input 1 = 7; 0x80 -> input 2 = 0, input 3 = -8
    # sample 1: 0x21 -> 1, 2; 0xE9 -> -7 (0x9), -2 (0xE)
    p = np.array([[0x7F, 0x80, 0x21, 0xE9]], np.uint8)
    out = orc.unpack4(p, 2)
    assert out.tolist() == [[-1, 1], [7, 2], [0, -7], [-8, -2]]


def test_unpack4_round_trip_and_card_demux(orc):
    rng = np.random.default_rng(4)
    x = rng.integers(-8, 8, (12, 1001)).astype(np.int8)     # 3 cards of 4 inputs
    nib = (x.astype(np.int16) & 0xF).astype(np.uint8)
    packed = np.zeros((3, 2 * 1001 + 6), np.uint8)            # rows with slack: ld > 2n
    for c in range(3):
        packed[c, 0:2002:2] = nib[4 * c] | (nib[4 * c + 1] << 4)
        packed[c, 1:2002:2] = nib[4 * c + 2] | (nib[4 * c + 3] << 4)
    assert np.array_equal(orc.unpack4(packed, 1001), x)
