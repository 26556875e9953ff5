"""Pins of the denoiser oracle (CPU, no GPU): each oracle function against something other
than itself -- hand-checked values, brute-force loops, a library convolution, adjointness,
finite differences, closed forms."""
import numpy as np
import pytest
import torch

from oracle import denoiser as od


def test_bf16_round_values():
    # 8 significant bits: the neighbours of 1 are 1 - 2^-8 and 1 + 2^-7
    cases = [
        (1.0, 1.0),
        (1.0 + 2.0 ** -8, 1.0),                       # halfway, ties to even (mantissa 0)
        (1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -6),       # halfway, ties to even (mantissa 2)
        (1.0 + 2.0 ** -8 + 2.0 ** -20, 1.0 + 2.0 ** -7),
        (-1.0 - 2.0 ** -8 - 2.0 ** -20, -1.0 - 2.0 ** -7),
        (2.0 - 2.0 ** -9, 2.0),                       # carry into the exponent
        (3.0e38, None),                               # FP32's exponent range stays finite
        (0.0, 0.0),
    ]
    for v, want in cases:
        got = float(od.bf16_round(torch.tensor([v], dtype=torch.float64))[0])
        if want is None:
            assert abs(got - v) / v < 2 ** -8 and np.isfinite(got)
        else:
            assert got == want, (v, got, want)


def _brute_conv(x, w, b):
    n, D, H, W, C = x.shape
    O = w.shape[1]
    y = np.zeros((n, D, H, W, O))
    for i in range(n):
        for z in range(D):
            for yy in range(H):
                for xx in range(W):
                    for o in range(O):
                        s = b[o]
                        for t in range(27):
                            dz, dy, dx = t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1
                            zz, y2, x2 = z + dz, yy + dy, xx + dx
                            if 0 <= zz < D and 0 <= y2 < H and 0 <= x2 < W:
                                for c in range(C):
                                    s += x[i, zz, y2, x2, c] * w[t, o, c]
                        y[i, z, yy, xx, o] = s
    return y


def test_conv3d_against_brute_force():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(2, 3, 4, 5, 2))
    w = rng.normal(size=(27, 3, 2))
    b = rng.normal(size=3)
    got = od.conv3d(torch.tensor(x), torch.tensor(w), torch.tensor(b)).numpy()
    assert np.allclose(got, _brute_conv(x, w, b), rtol=1e-12, atol=1e-12)


def test_conv3d_against_library_convolution():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(2, 6, 5, 7, 4))
    w = rng.normal(size=(27, 5, 4))
    got = od.conv3d(torch.tensor(x), torch.tensor(w)).numpy()
    # library layout: channels first, weight [cout, cin, kz, ky, kx], cross-correlation
    wl = torch.tensor(w).reshape(3, 3, 3, 5, 4).permute(3, 4, 0, 1, 2)
    ref = torch.nn.functional.conv3d(torch.tensor(x).permute(0, 4, 1, 2, 3), wl, padding=1)
    assert np.allclose(got, ref.permute(0, 2, 3, 4, 1).numpy(), rtol=1e-12, atol=1e-12)


def test_pool_and_upsample_are_adjoint():
    rng = np.random.default_rng(5)
    x = torch.tensor(rng.normal(size=(2, 4, 6, 8, 3)))
    y = torch.tensor(rng.normal(size=(2, 2, 3, 4, 3)))
    lhs = float((od.avg_pool2(x) * y).sum())
    rhs = float((x * od.upsample2(y)).sum()) / 8
    assert lhs == pytest.approx(rhs, rel=1e-12)
    c = torch.full((1, 4, 4, 4, 2), 3.5, dtype=torch.float64)
    assert torch.all(od.avg_pool2(c) == 3.5) and od.upsample2(od.avg_pool2(c)).shape == c.shape
    u = od.upsample2(y)
    assert torch.all(u[:, 1::2, 0::2, 1::2] == y)


def _random_params(rng, scale=1.0, head=True):
    p = np.zeros(od.param_count())
    k = 0
    for ci, co in od.LAYERS:
        fan = 27 * ci
        p[k:k + 27 * co * ci] = rng.normal(size=27 * co * ci) * np.sqrt(2.0 / fan) * scale
        k += 27 * co * ci
        p[k:k + co] = rng.normal(size=co) * 0.05
        k += co
    if head:
        p[k:k + 16] = rng.normal(size=16) * 0.3
        p[k + 16] = 0.1
    return p


def test_zero_head_returns_the_input():
    rng = np.random.default_rng(6)
    p = _random_params(rng, head=False)
    x = rng.normal(size=(1, 4, 4, 8))
    y = od.forward(p, x, bf16=True).numpy()
    assert np.array_equal(y, x)


def test_channel0_network_is_relu_pool_upsample():
    """Every 3x3x3 convolution passes channel 0 through its centre tap (weight 1, no bias),
    the head reads channel 0 with weight 1: the U-Net then computes exactly
    y = x + up(up(pool(pool(relu(x))))) -- the first ReLU clips the input, later ones see
    non-negative maps, each pooling averages 2x2x2 blocks, each upsampling repeats a voxel
    2x2x2, and channel 0 of each concatenation is the upsampled path."""
    flat = torch.zeros(od.param_count(), dtype=torch.float64)
    p = od.unpack(flat)
    for name in od.NAMES:
        p[name + ".w"][13, 0, 0] = 1.0                   # tap 13 = (dz, dy, dx) = (0, 0, 0)
    p["hw"][0] = 1.0
    x = np.random.default_rng(9).normal(size=(1, 8, 8, 8))
    y = od.forward(flat, x, bf16=False).numpy()

    def pool(a):
        n, D, H, W = a.shape
        return a.reshape(n, D // 2, 2, H // 2, 2, W // 2, 2).mean(axis=(2, 4, 6))

    def up(a):
        return a.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)

    assert np.allclose(y, x + up(up(pool(pool(np.maximum(x, 0))))), rtol=0, atol=1e-12)


def test_first_layer_against_brute_force():
    """the input layer sees the input as channel 0 of 16 zero-padded channels"""
    rng = np.random.default_rng(7)
    p = od.unpack(_random_params(rng))
    x = rng.normal(size=(1, 2, 3, 4))
    x16 = np.zeros(x.shape + (16,))
    x16[..., 0] = x
    ref = np.maximum(_brute_conv(x16, p["e1a.w"].numpy(), p["e1a.b"].numpy()), 0)
    got = torch.relu(od.conv3d(torch.tensor(x16), p["e1a.w"], p["e1a.b"])).numpy()
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_feature_channels_enter_the_first_layer():
    """with features, channels 1..k of the input layer carry them (brute force)"""
    rng = np.random.default_rng(17)
    p = od.unpack(_random_params(rng))
    x = rng.normal(size=(1, 2, 3, 4))
    aux = rng.normal(size=(1, 2, 2, 3, 4))
    x16 = np.zeros(x.shape + (16,))
    x16[..., 0] = x
    x16[..., 1] = aux[:, 0]
    x16[..., 2] = aux[:, 1]
    ref = np.maximum(_brute_conv(x16, p["e1a.w"].numpy(), p["e1a.b"].numpy()), 0)
    got = torch.relu(od.conv3d(torch.tensor(x16), p["e1a.w"], p["e1a.b"])).numpy()
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)
    # and the network sees them: changing a feature changes the output
    pp = _random_params(rng)
    xv = rng.normal(size=(1, 4, 4, 4))
    av = rng.normal(size=(1, 2, 4, 4, 4))
    y0 = od.forward(pp, xv, bf16=False, aux=av).numpy()
    av[0, 1, 1, 1, 1] += 1.0
    assert not np.allclose(od.forward(pp, xv, bf16=False, aux=av).numpy(), y0)


def test_features_values():
    media = np.array([(0.0, 0.0, 1.0, 1.0), (0.01, 10.0, 0.9, 1.37), (0.1, 5.0, 0.5, 1.4)])
    labels = np.array([0, 1, 2, 7], dtype=np.uint8)
    f = od.features(labels, media)
    assert np.allclose(f[0], [np.log10(1e-4) + 2, 0.0, 1.0, -2.0])
    assert np.allclose(f[1], [-3.0, 0.0, np.log10(2.5), -3.0])


def test_forward_equivariant_under_shifts_of_four():
    """pooling twice makes the network equivariant under shifts by multiples of 4 voxels,
    up to the receptive field's reach of the zero-padded boundary"""
    rng = np.random.default_rng(8)
    p = _random_params(rng)
    x = rng.normal(size=(1, 4, 4, 64))
    xs = np.roll(x, 4, axis=3)
    y = od.forward(p, x, bf16=False).numpy()
    ys = od.forward(p, xs, bf16=False).numpy()
    # far from both x boundaries (receptive field < 24 voxels) the outputs agree
    assert np.allclose(ys[..., 28:36], y[..., 24:32], rtol=1e-10, atol=1e-10)
    assert not np.allclose(ys[..., 0:8], y[..., 0:8])


def test_gradients_against_finite_differences():
    rng = np.random.default_rng(9)
    p = _random_params(rng)
    x = rng.normal(size=(1, 4, 4, 8))
    t = x + 0.3 * rng.normal(size=x.shape)
    aux = rng.normal(size=(1, 2) + x.shape[1:])
    loss, g = od.loss_and_grads(p, x, t, bf16=False, aux=aux)
    # parameters in every layer, the biases and the head
    idx = []
    k = 0
    for ci, co in od.LAYERS:
        idx += [k + int(rng.integers(0, 27 * co * ci)), k + 27 * co * ci + int(rng.integers(0, co))]
        k += 27 * co * ci + co
    idx += [k + 3, k + 16]
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        lp = float(((od.forward(pp, x, bf16=False, aux=aux) - torch.tensor(t)) ** 2).mean())
        lm = float(((od.forward(pm, x, bf16=False, aux=aux) - torch.tensor(t)) ** 2).mean())
        fd = (lp - lm) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9), i


def test_loss_is_the_voxel_mean_with_its_closed_form_head_gradient():
    """With the head's weights at zero the output is x + hb, so the loss
    mean((x + hb - t)^2) and its gradient d/dhb = 2 mean(x + hb - t) follow in closed
    form, while every other parameter's gradient is zero."""
    rng = np.random.default_rng(11)
    p = _random_params(rng, head=False)
    p[-1] = 0.25                                        # hb
    x = rng.normal(size=(2, 4, 4, 8))
    t = rng.normal(size=(2, 4, 4, 8))
    loss, g = od.loss_and_grads(p, x, t, bf16=False)
    e = x + 0.25 - t
    assert abs(loss - float(np.mean(e * e))) < 1e-12
    assert abs(g[-1] - 2.0 * float(np.mean(e))) < 1e-12
    assert np.all(g[:-17] == 0.0)                       # the head weights are zero


def test_adam_first_step_closed_form():
    """with zero moments the first bias-corrected step moves each parameter by
    lr * g / (|g| + eps) ~ lr * sign(g)"""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p, m, v = od.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 1e-2)
    assert np.allclose(p[:3], -1e-2 * np.sign(g[:3]), rtol=1e-4)
    assert p[3] == 0.0
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_encode_decode_inverse_and_log_rms():
    phi = np.array([0.0, 1e-9, 1e-4, 2.0])
    x = od.encode(phi)
    assert x[0] == pytest.approx((-8 + 4) / 2)
    assert np.allclose(od.decode(x), phi, rtol=1e-12, atol=1e-20)
    ref = np.array([1.0, 1e-3, 1e-8, 0.0])
    # voxels below 1e-6 of the maximum are outside the mask
    err = od.log_rms(np.array([10.0, 1e-2, 5.0, 7.0]), ref)
    assert err == pytest.approx(np.sqrt(np.mean(np.log10([(10 + 1e-8) / (1 + 1e-8), (1e-2 + 1e-8) / (1e-3 + 1e-8)]) ** 2)),
                                rel=1e-9)


def test_study_log_rms_matches_oracle_definition():
    """the product's evaluation metric (paper_1711_03244_gb300.denoise.log_rms) against the
    oracle's restatement on random maps with zeros and a masked tail"""
    from paper_1711_03244_gb300 import denoise as dn
    rng = np.random.default_rng(21)
    ref = 10.0 ** rng.uniform(-9, 0, size=(8, 8, 8))
    ref[0, 0, :4] = 0.0
    phi = ref * 10.0 ** rng.normal(0, 0.3, size=ref.shape)
    phi[1, 1, :5] = 0.0
    assert dn.log_rms(phi, ref) == pytest.approx(od.log_rms(phi, ref), rel=1e-12)
    assert dn.log_rms(ref, ref) == 0.0
