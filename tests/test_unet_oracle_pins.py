"""Pins of the masking-network oracle (Sec. III-D, Eq. 10-12, Tab. II) to things other than itself:
bf16 rounding values fixed by the format, the 3x3 convolution as a brute-force sum over taps,
BatchNorm statistics against numpy's mean and variances, the bilinear x2 weights worked out by
hand, max-pool routing, closed forms of the head and of the first Adam step, the [up, skip]
channel order of the decoder, and float64 central differences of the whole network with the
bf16 roundings switched off."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import unet_oracle as U  # noqa: E402

F = torch.nn.functional


def test_bf16_round_to_nearest_even_values():
    # bf16 keeps 8 significant bits: the spacing at 1 is 2^-7
    x = torch.tensor([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7, 1 + 2 ** -8 + 2 ** -20, -3.0 - 2 ** -7,
                      2.0 ** -130], dtype=torch.float64)
    want = [1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, 1 + 2 ** -7, -3.0, 2.0 ** -130]
    got = U.bf16(x)
    assert got.tolist() == want
    # the rounding is straight-through for the gradient
    y = x.clone().requires_grad_(True)
    (U.bf16(y) * torch.arange(7.0, dtype=torch.float64)).sum().backward()
    assert y.grad.tolist() == list(range(7))


def _conv3x3_bruteforce(x, w):
    b, ci, h, wd = x.shape
    co = w.shape[0]
    out = np.zeros((b, co, h, wd))
    xp = np.zeros((b, ci, h + 2, wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    for o in range(co):
        for dy in range(3):
            for dx in range(3):
                out[:, o] += np.einsum("bchw,c->bhw", xp[:, :, dy:dy + h, dx:dx + wd], w[o, :, dy, dx])
    return out


@pytest.mark.parametrize("scale", [1.0, 1e-3])   # 1e-3: batch variance near eps, where its place shows
def test_conv_bn_relu_is_bruteforce_conv_then_numpy_batchnorm(scale):
    rng = np.random.default_rng(3)
    x = scale * rng.standard_normal((2, 3, 6, 5))
    p = {"l.w": torch.from_numpy(rng.standard_normal((4, 3, 3, 3))),
         "l.gamma": torch.from_numpy(rng.uniform(0.5, 1.5, 4)), "l.beta": torch.from_numpy(rng.uniform(-.3, .3, 4))}
    st = {"l.mean": torch.zeros(4, dtype=torch.float64), "l.var": torch.ones(4, dtype=torch.float64)}
    xb = U.bf16(torch.from_numpy(x))
    got = U.conv_bn_relu(xb, p, st, "l", training=True).numpy()
    wb = U.bf16(p["l.w"]).numpy()
    y = _conv3x3_bruteforce(xb.numpy(), wb)
    mean = y.mean(axis=(0, 2, 3))
    var = y.var(axis=(0, 2, 3))                       # population variance for the batch statistics
    pre = (y - mean[None, :, None, None]) / np.sqrt(var[None, :, None, None] + U.EPS)
    pre = pre * p["l.gamma"].numpy()[None, :, None, None] + p["l.beta"].numpy()[None, :, None, None]
    want = U.bf16(torch.from_numpy(np.maximum(pre, 0))).numpy()
    assert np.max(np.abs(got - want)) <= 1e-2 * np.max(np.abs(want))   # at most one bf16 step apart
    assert np.mean(got == want) > 0.98
    # running statistics: momentum 0.1, unbiased variance
    n = y.shape[0] * y.shape[2] * y.shape[3]
    assert np.allclose(st["l.mean"].numpy(), 0.1 * mean, rtol=1e-12, atol=1e-14)
    assert np.allclose(st["l.var"].numpy(), 0.9 + 0.1 * y.var(axis=(0, 2, 3), ddof=1), rtol=1e-12)
    assert n == 60
    # evaluation mode uses the running statistics
    got_eval = U.conv_bn_relu(xb, p, st, "l", training=False).numpy()
    pre_e = (y - st["l.mean"].numpy()[None, :, None, None]) / np.sqrt(st["l.var"].numpy()[None, :, None, None] + U.EPS)
    pre_e = pre_e * p["l.gamma"].numpy()[None, :, None, None] + p["l.beta"].numpy()[None, :, None, None]
    want_e = U.bf16(torch.from_numpy(np.maximum(pre_e, 0))).numpy()
    assert np.max(np.abs(got_eval - want_e)) <= 1e-2 * np.max(np.abs(want_e))


def test_bilinear_x2_weights_by_hand():
    # align_corners=False: output o samples input (o + 0.5)/2 - 0.5, clamped at both ends
    a = np.array([1.0, 4.0, 2.0, 8.0])
    want = np.array([1.0, 0.75 * 1 + 0.25 * 4, 0.25 * 1 + 0.75 * 4, 0.75 * 4 + 0.25 * 2, 0.25 * 4 + 0.75 * 2,
                     0.75 * 2 + 0.25 * 8, 0.25 * 2 + 0.75 * 8, 8.0])
    x = torch.from_numpy(np.outer([1.0, 1.0], a))[None, None]          # [1, 1, 2, 4], constant along y
    got = U.up2(x)[0, 0].numpy()   # the oracle's own step (these values are exact in bf16)
    assert got.shape == (4, 8)
    assert np.allclose(got, want[None, :], rtol=0, atol=1e-15)


def test_maxpool_routes_the_gradient_to_the_window_maximum():
    x = torch.tensor([[[[1.0, 5.0, 2.0, 2.0], [3.0, 0.0, 7.0, 1.0]]]], dtype=torch.float64, requires_grad=True)
    y = U.down2(x)
    assert y.detach().numpy().ravel().tolist() == [5.0, 7.0]
    (y * torch.tensor([[[[10.0, 20.0]]]], dtype=torch.float64)).sum().backward()
    assert x.grad.numpy().ravel().tolist() == [0, 10, 0, 0, 0, 0, 20, 0]


def test_head_with_zero_weight_gives_sigmoid_of_bias_and_masks_multiply():
    ch = (4, 8)
    p = U.init_params(ch, seed=2)
    p["head.w"] = torch.zeros_like(p["head.w"])
    p["head.b"] = torch.tensor([0.3, -1.2], dtype=torch.float64)
    rng = np.random.default_rng(0)
    f = torch.from_numpy(rng.random((2, 8, 8)))
    g = torch.from_numpy(rng.random((2, 8, 8)))
    fo, go, m = U.masked(p, U.init_state(ch), f, g, ch, training=True)
    s = [1 / (1 + math.exp(-0.3)), 1 / (1 + math.exp(1.2))]
    assert np.allclose(m[:, 0].numpy(), s[0], rtol=0, atol=1e-15)
    assert np.allclose(m[:, 1].numpy(), s[1], rtol=0, atol=1e-15)
    assert np.allclose(fo.numpy(), f.numpy() * s[0], rtol=1e-15) and np.allclose(go.numpy(), g.numpy() * s[1], rtol=1e-15)


def test_layer_list_follows_the_unet_pattern():
    names = U.conv_layers((8, 16, 32, 64))
    assert [n for n, _, _ in names] == ["enc0a", "enc0b", "enc1a", "enc1b", "enc2a", "enc2b", "enc3a", "enc3b",
                                        "dec2a", "dec2b", "dec1a", "dec1b", "dec0a", "dec0b"]
    assert names[0][1:] == (2, 8) and names[8][1:] == (64 + 32, 32) and names[12][1:] == (16 + 8, 8)


def test_six_level_layer_list_reproduces_tab2():
    """The oracle's layer list for channels (8, 16, 32, 64, 128, 256) against every (c_i, c_o) that
    Tab. II prints, including the 384/192/96/48/24-channel decoder concatenations, and the head."""
    import os
    rows = [ln.split() for ln in open(os.path.join(os.path.dirname(__file__), "golden", "tab2_network.txt"))
            if ln.strip() and not ln.startswith("#")]
    layers = U.conv_layers((8, 16, 32, 64, 128, 256))
    enc = [(int(r[1]), int(r[2]), int(r[3]), int(r[4])) for r in rows if r[0] == "enc"]
    dec = [(int(r[1]), int(r[2]), int(r[3]), int(r[4])) for r in rows if r[0] == "dec"]
    head = [(int(r[1]), int(r[2])) for r in rows if r[0] == "head"]
    assert len(layers) == 2 * (len(enc) + len(dec))
    got = [(a[1], a[2], b[1], b[2]) for a, b in zip(layers[0::2], layers[1::2])]
    assert got == enc + dec
    p = U.init_params((8, 16, 32, 64, 128, 256), seed=1)
    assert tuple(p["head.w"].shape[:2]) == (head[0][1], head[0][0])
    for name, ci, co in layers:
        assert tuple(p[name + ".w"].shape) == (co, ci, 3, 3)


def test_decoder_concatenates_up_then_skip():
    # with the weights on the first (upsampled) input channels of every decoder conv zeroed, the
    # masks no longer depend on the deepest level; zeroing the skip channels instead keeps the
    # dependence -- which fixes the [up, skip] order against the weight layout
    ch = (4, 8, 8)
    rng = np.random.default_rng(5)
    f = torch.from_numpy(rng.random((2, 16, 16)))
    g = torch.from_numpy(rng.random((2, 16, 16)))

    def masks(p):
        return U.forward(p, U.init_state(ch), f, g, ch, training=True)

    for zero_up, expect_independent in ((True, True), (False, False)):
        p = U.init_params(ch, seed=4)
        for i in range(len(ch) - 2, -1, -1):
            w = p[f"dec{i}a.w"]
            deeper = ch[i + 1]
            if zero_up:
                w[:, :deeper] = 0
            else:
                w[:, deeper:] = 0
        m0 = masks(p)
        p2 = {k: v.clone() for k, v in p.items()}
        p2["enc2b.w"] = torch.from_numpy(rng.standard_normal(p["enc2b.w"].shape))
        m1 = masks(p2)
        same = torch.equal(m0, m1)
        assert same == expect_independent


def test_first_adam_step_closed_form():
    p = {"a": torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64)}
    g = {"a": torch.tensor([0.2, -3.0, 1e-9], dtype=torch.float64)}
    m = {"a": torch.zeros(3, dtype=torch.float64)}
    v = {"a": torch.zeros(3, dtype=torch.float64)}
    out = U.adam(p, g, m, v, step=1, lr=1e-3)
    # bias-corrected first step: m_hat = g, v_hat = g^2, so the update is lr g / (|g| + eps)
    want = p["a"] - 1e-3 * g["a"] / (g["a"].abs() + 1e-8)
    assert torch.allclose(out["a"], want, rtol=1e-14, atol=0)


def test_network_gradient_matches_central_differences_without_bf16(monkeypatch):
    monkeypatch.setattr(U, "bf16", lambda x: x)
    ch = (4, 8)
    p = U.init_params(ch, seed=7)
    rng = np.random.default_rng(8)
    for k in p:
        if k.endswith(".gamma"):
            p[k] = torch.from_numpy(rng.uniform(0.5, 1.5, p[k].shape))
        if k.endswith(".beta"):
            p[k] = torch.from_numpy(rng.uniform(-0.3, 0.3, p[k].shape))
    f = torch.from_numpy(rng.random((2, 8, 8)))
    g = torch.from_numpy(rng.random((2, 8, 8)))
    dft = torch.from_numpy(rng.standard_normal((2, 8, 8)))
    dgt = torch.from_numpy(rng.standard_normal((2, 8, 8)))
    st = U.init_state(ch)
    gr = U.grads(p, st, f, g, dft, dgt, ch)

    def loss(q):
        fo, go, _ = U.masked(q, U.init_state(ch), f, g, ch, training=True)
        return float((fo * dft).sum() + (go * dgt).sum())

    h = 1e-6
    for name, idx in (("enc0a.w", (1, 0, 2, 1)), ("enc1b.w", (3, 5, 0, 0)), ("dec0a.w", (2, 9, 1, 2)),
                      ("enc1a.gamma", (6,)), ("dec0b.beta", (0,)), ("head.w", (1, 3, 0, 0)), ("head.b", (0,))):
        qp = {k: v.clone() for k, v in p.items()}
        qm = {k: v.clone() for k, v in p.items()}
        qp[name][idx] += h
        qm[name][idx] -= h
        fd = (loss(qp) - loss(qm)) / (2 * h)
        an = float(gr[name][idx])
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, fd, an)


def test_first_convolution_sees_bf16_scans():
    """The two scans enter the network rounded to bf16 (the CUDA path's operand type): scans that
    differ only below bf16's resolution give identical masks."""
    ch = (4, 8)
    p = U.init_params(ch, seed=4)
    rng = np.random.default_rng(5)
    f = torch.from_numpy(rng.random((2, 8, 8)))
    g = torch.from_numpy(rng.random((2, 8, 8)))
    m1 = U.forward(p, U.init_state(ch), f, g, ch, training=True)
    m2 = U.forward(p, U.init_state(ch), U.bf16(f), U.bf16(g), ch, training=True)
    assert torch.equal(m1, m2) and not torch.equal(f, U.bf16(f))
