"""GPU tests of the RFI stage against the FP64 oracle, and of what the learned flagger gains.

Tolerances: power dumps are FP32 sums of FP32 spectra (relative 1e-5); patch medians and
MADs are selections (exact up to the FP32 midpoint, relative 1e-6), flags agree except for
values within 1e-5 of the threshold; the network runs with FP16 weights and activations,
so its probabilities are compared to 2e-3 and its gradients element by element to 1e-2 in
units of their layer's largest gradient (and each layer's norm to 1e-2), against the oracle on
the same FP16-rounded parameters and inputs; the FP32 build of the same kernels meets 1e-5
element by element (relative on entries of at least a tenth of their layer's largest, and in
units of that largest everywhere).
"""
import numpy as np
import pytest

from synth import make_config

pytestmark = pytest.mark.gpu

OFFS = {"W1": (0, 144), "b1": (144, 16), "W2": (160, 4608), "b2": (4768, 32), "W3": (4800, 4608),
        "b3": (9408, 16), "W4": (9424, 16), "b4": (9440, 1)}


@pytest.fixture(scope="module")
def env(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0910_1517_gb300 import build, corr
    build.build()
    corr.load()
    return torch, corr, orc


def he_init(seed):
    rng = np.random.default_rng(seed)
    p = np.zeros(9441)
    for name, fan_in in (("W1", 9), ("W2", 16 * 9), ("W3", 32 * 9), ("W4", 16)):
        o, n = OFFS[name]
        p[o:o + n] = rng.normal(scale=np.sqrt(2.0 / fan_in), size=n)
    for name in ("b1", "b2", "b3"):
        o, n = OFFS[name]
        p[o:o + n] = 0.05
    return p


def test_power_dumps_match_oracle(env):
    torch, corr, orc = env
    s = make_config(2, n_ant=4, n_pol=2, n_fft=512, n_int=128, seed=51)
    h = corr.corr_create(s.n_ant, s.n_pol, s.n_fft, s.n_int)
    try:
        corr.corr_set_delays(h, s.delay, s.phi0, s.rate)
        corr.corr_set_power_dump(h, 32)
        n = s.x.shape[1]
        xt = torch.zeros((s.n_in, ((n + 15) // 16) * 16 + 16), dtype=torch.int8, device="cuda")
        xt[:, :n] = torch.from_numpy(s.x).cuda()
        corr.corr_integrate_device(h, xt, n_avail=n, stream=torch.cuda.current_stream())
        P = corr.corr_read_power_host(h, s.n_int // 32).astype(np.float64)
    finally:
        corr.corr_destroy(h)
    Y = orc.fengine(s.x, s.n_ant, s.n_pol, s.n_fft, s.n_int, s.delay, s.phi0, s.rate)
    Pr = orc.power_dumps(Y, 32)
    e = float(np.max(np.abs(P - Pr) / Pr))
    print(f"power dumps: max relative error {e:.2e}")
    assert e <= 1e-5


def test_patch_statistics_and_mad_flags_match_oracle(env):
    torch, corr, orc = env
    rng = np.random.default_rng(7)
    n_in, n_dump, n_chan = 3, 128, 128
    P = rng.gamma(32.0, size=(n_in, n_dump, n_chan)).astype(np.float32)
    P[0, 5, 7] *= 3.0
    P[2, 70:90, 3] *= 1.6
    Pd = torch.from_numpy(P).cuda()
    B = n_in * (n_dump // 64) * (n_chan // 64)
    x = torch.empty((B, 64, 64), dtype=torch.float16, device="cuda")
    fl = torch.empty((B, 64, 64), dtype=torch.uint8, device="cuda")
    st = torch.empty((B, 2), dtype=torch.float32, device="cuda")
    corr.rfi_patches(Pd, n_in, n_dump, n_chan, 5.0, x, fl, st, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    pat = P.reshape(n_in, n_dump // 64, 64, n_chan // 64, 64).transpose(0, 1, 3, 2, 4).reshape(B, 64, 64)
    med, mad, flags, z = orc.patch_stats(pat.astype(np.float64), M=5.0)
    stg = st.cpu().numpy().astype(np.float64)
    assert np.allclose(stg[:, 0], med, rtol=1e-6) and np.allclose(stg[:, 1], mad, rtol=1e-6)
    thr = 5.0 * mad / 0.6745
    dev = np.abs(pat - med[:, None, None])
    near = np.abs(dev - thr[:, None, None]) <= 1e-5 * thr[:, None, None]
    fg = fl.cpu().numpy()
    assert np.array_equal(fg[~near], flags[~near])
    assert fg[0, 5, 7] == 1
    zg = x.float().cpu().numpy()
    assert np.max(np.abs(zg - z) / np.maximum(1.0, np.abs(z))) <= 2e-3


def _grad_errors(grad_g, grad_r, floor=0.1):
    """Per layer: the largest relative error over the entries at least `floor` of the layer's
    largest magnitude, the largest absolute error over every entry in units of that magnitude
    (a wrong sign or a swapped index on any entry that matters fails it), and the relative norm
    error of the layer."""
    out = {}
    for name, (o, n) in OFFS.items():
        gr, gg = grad_r[o:o + n], grad_g[o:o + n].astype(np.float64)
        big = float(np.abs(gr).max())
        sel = np.abs(gr) >= floor * big
        out[name] = (float((np.abs(gg - gr)[sel] / np.abs(gr[sel])).max()), float(np.abs(gg - gr).max() / big),
                     float(np.linalg.norm(gg - gr) / np.linalg.norm(gr)))
    return out


def _network_vs_oracle(env, create, p_gpu):
    torch, corr, orc = env
    B = 2
    rng = np.random.default_rng(11)
    p = he_init(3)
    x = rng.normal(size=(B, 64, 64)).astype(np.float16)
    m = (rng.random((B, 64, 64)) < 0.1).astype(np.uint8)
    m[0, 10:30, 20] = 1
    net = create(8)
    try:
        corr.rfi_set_params(net, p)
        xt = torch.from_numpy(x).cuda()
        mt = torch.from_numpy(m).cuda()
        prob = torch.empty((B, 64, 64), dtype=torch.float32, device="cuda")
        corr.rfi_infer(net, xt, B, prob, stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        pg = prob.cpu().numpy()
        loss_g, grad_g = corr.rfi_loss_grad(net, xt, mt, B, stream=torch.cuda.current_stream())
    finally:
        corr.rfi_destroy(net)
    pr_ = p_gpu(p)                                            # the parameters the GPU computes with
    logits = orc.rfi_forward(pr_, x.astype(np.float64))
    pr = 1.0 / (1.0 + np.exp(-logits))
    e_p = float(np.max(np.abs(pg - pr)))
    loss_r, grad_r = orc.rfi_loss_grad(pr_, x.astype(np.float64), m)
    e_loss = abs(loss_g - loss_r) / loss_r
    return e_p, e_loss, _grad_errors(grad_g, grad_r)


def test_network_forward_and_gradients_match_oracle(env):
    # FP16 weights and activations (the flagger): against the oracle on the same FP16-rounded
    # parameters and inputs.  Every stored activation is rounded to 2^-11 relative and a rounding
    # can flip a ReLU mask, so an entry that is a sum over 8192 pixels with cancellation has no
    # useful relative bound; the bound is per entry in units of its layer's largest gradient
    # (measured <= 2.7e-3) and on each layer's norm (measured <= 4e-3), both <= 1e-2
    torch, corr, orc = env
    e_p, e_loss, errs = _network_vs_oracle(env, corr.rfi_create, lambda p: p.astype(np.float16).astype(np.float64))
    print(f"network fp16: prob {e_p:.2e} loss {e_loss:.2e} grads (rel >= 10% of max, abs, norm) " +
          " ".join(f"{k}:{v[0]:.1e},{v[1]:.1e},{v[2]:.1e}" for k, v in errs.items()))
    assert e_p <= 2e-3 and e_loss <= 2e-3
    assert max(v[1] for v in errs.values()) <= 1e-2 and max(v[2] for v in errs.values()) <= 1e-2


def test_network_fp32_build_matches_oracle_to_1e5(env):
    # the same kernels with FP32 weights and activations: only FP32 accumulation remains
    torch, corr, orc = env
    e_p, e_loss, errs = _network_vs_oracle(env, corr.rfi_create_fp32,
                                           lambda p: p.astype(np.float32).astype(np.float64))
    print(f"network fp32: prob {e_p:.2e} loss {e_loss:.2e} grads (rel >= 10% of max, abs, norm) " +
          " ".join(f"{k}:{v[0]:.1e},{v[1]:.1e},{v[2]:.1e}" for k, v in errs.items()))
    assert e_p <= 1e-5 and e_loss <= 1e-5
    assert max(v[0] for v in errs.values()) <= 1e-5 and max(v[1] for v in errs.values()) <= 1e-5


def _dataset(torch, corr, n_integrations, seed, n_fft=2048, n_int=2048, n_in=16):
    """Power-dump patches, Eq. 4 flags and masks from streams with injected RFI, correlated
    by the F-engine itself (CORR_FP32, 32-frame dumps)."""
    from synth.rfi import patch_masks, rfi_streams
    h = corr.corr_create(n_in // 2, 2, n_fft, n_int)
    corr.corr_set_power_dump(h, 32)
    xs, fs, ms = [], [], []
    n_dump, n_chan = n_int // 32, n_fft // 2
    B = n_in * (n_dump // 64) * (n_chan // 64)
    stream = torch.cuda.current_stream()
    try:
        for j in range(n_integrations):
            x, mask = rfi_streams(n_in, n_fft, n_int, seed=seed + j)
            corr.corr_integrate_device(h, x, n_avail=n_int * n_fft, stream=stream)
            Pdev = corr.corr_power_device(h)
            xp = torch.empty((B, 64, 64), dtype=torch.float16, device="cuda")
            fl = torch.empty((B, 64, 64), dtype=torch.uint8, device="cuda")
            corr.corr_read_visibilities(h)                      # waits for the integration
            corr.rfi_patches(Pdev, n_in, n_dump, n_chan, 5.0, xp, fl, None, stream=stream)
            torch.cuda.synchronize()
            xs.append(xp)
            fs.append(fl)
            ms.append(patch_masks(mask))
    finally:
        corr.corr_destroy(h)
    return torch.cat(xs), torch.cat(fs), torch.cat(ms)


def rates(flags, mask):
    f = flags.bool()
    m = mask.bool()
    miss = float((m & ~f).sum()) / max(1, int(m.sum()))
    false = float((f & ~m).sum()) / max(1, int((~m).sum()))
    return miss, false


def test_learned_flagger_beats_mad_on_held_out_patches(env):
    torch, corr, orc = env
    xtr, ftr, mtr = _dataset(torch, corr, 24, seed=100)         # 24 x 256 = 6144 patches
    xte, fte, mte = _dataset(torch, corr, 4, seed=900)          # held out
    net = corr.rfi_create(256)
    try:
        corr.rfi_set_params(net, he_init(1))
        g = torch.Generator(device="cuda").manual_seed(0)
        stream = torch.cuda.current_stream()
        losses = []
        for epoch in range(8):
            perm = torch.randperm(xtr.shape[0], generator=g, device="cuda")
            for b0 in range(0, xtr.shape[0] - 255, 256):
                idx = perm[b0:b0 + 256]
                loss = corr.rfi_train_step(net, xtr[idx].contiguous(), mtr[idx].contiguous(), 256, 2e-3,
                                           want_loss=(b0 == 0), stream=stream)
                if loss is not None:
                    losses.append(loss)
        prob = torch.empty(xte.shape, dtype=torch.float32, device="cuda")
        for b0 in range(0, xte.shape[0], 256):
            nb = min(256, xte.shape[0] - b0)
            corr.rfi_infer(net, xte[b0:b0 + nb].contiguous(), nb, prob[b0:b0 + nb], stream=stream)
        torch.cuda.synchronize()
    finally:
        corr.rfi_destroy(net)
    cnn = rates(prob > 0.5, mte)
    mad = rates(fte, mte)
    occ = float(mte.float().mean())
    print(f"occupancy {occ:.3f}; loss by epoch {['%.4f' % v for v in losses]}; "
          f"CNN miss {cnn[0]:.3f} false {cnn[1]:.4f}; MAD miss {mad[0]:.3f} false {mad[1]:.4f}")
    assert losses[-1] < losses[0]
    assert 0.01 < occ < 0.12
    # the learned flagger finds more of the interference without flagging more clean data
    assert cnn[0] < mad[0] and cnn[1] <= max(2 * mad[1], 2e-3)
