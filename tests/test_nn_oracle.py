"""Pins of the denoiser oracle (oracle/nn.py): convolution against an
independent formulation, gradients against finite differences, BF16 rounding
against torch."""

import numpy as np
import pytest

from oracle import nn


def test_conv3x3_matches_direct_sum():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 5, 6, 3))
    w = rng.normal(size=(4, 9, 3))
    b = rng.normal(size=4)
    y = nn.conv3x3(x, w, b)
    # one output element written out by hand
    n, yy, xx, co = 1, 0, 5, 2
    acc = b[co]
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if 0 <= yy + dy < 5 and 0 <= xx + dx < 6:
                acc += x[n, yy + dy, xx + dx] @ w[co, 3 * (dy + 1) + (dx + 1)]
    assert abs(y[n, yy, xx, co] - acc) < 1e-12
    # against scipy's correlation, channel by channel
    from scipy.signal import correlate2d

    for co in range(4):
        ref = sum(correlate2d(x[0, :, :, ci], w[co, :, ci].reshape(3, 3), mode="same") for ci in range(3)) + b[co]
        np.testing.assert_allclose(y[0, :, :, co], ref, atol=1e-12)


def test_conv_gradients_are_adjoints():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 4, 5, 3))
    w = rng.normal(size=(4, 9, 3))
    gy = rng.normal(size=(2, 4, 5, 4))
    # <conv(x, w), gy> = <x, dgrad(gy, w)> = <w, wgrad(x, gy)>
    lhs = np.sum(nn.conv3x3(x, w) * gy)
    assert abs(lhs - np.sum(x * nn.conv3x3_dgrad(gy, w))) < 1e-10
    assert abs(lhs - np.sum(w * nn.conv3x3_wgrad(x, gy))) < 1e-10


def test_pool_and_upsample_backward_are_adjoints():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1, 4, 6, 2))
    y, arg = nn.pool_fwd(x)
    g = rng.normal(size=y.shape)
    gx = nn.pool_bwd(arg, g, x.shape)
    eps = 1e-6
    # the pooled maximum moves with its argmax input only
    x2 = x + eps * gx
    assert abs(np.sum(nn.pool_fwd(x2)[0] * g) - np.sum(y * g) - eps * np.sum(gx * gx)) < 1e-9
    u = rng.normal(size=(1, 3, 2, 2))
    gu = rng.normal(size=(1, 6, 4, 2))
    assert abs(np.sum(nn.up_fwd(u) * gu) - np.sum(u * nn.up_bwd(gu))) < 1e-12


@pytest.mark.slow
def test_unet_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    weights = nn.random_weights(4)
    net = nn.UNet(weights, bf16=False)
    noisy = rng.uniform(0.5, 1.5, size=(1, 16, 16))
    clean = noisy + 0.1 * rng.normal(size=noisy.shape)
    loss, grads = net.loss_and_grads(noisy, clean)
    eps = 1e-5
    for layer in (0, 4, 7, 8, 12, 14):
        w, b = weights[layer]
        for _ in range(2):
            idx = tuple(rng.integers(0, s) for s in w.shape)
            wp = [(ww.copy(), bb.copy()) for ww, bb in weights]
            wm = [(ww.copy(), bb.copy()) for ww, bb in weights]
            wp[layer][0][idx] += eps
            wm[layer][0][idx] -= eps
            fd = (nn.UNet(wp).loss_and_grads(noisy, clean)[0] - nn.UNet(wm).loss_and_grads(noisy, clean)[0]) / (2 * eps)
            assert abs(fd - grads[layer][0][idx]) <= 1e-6 + 1e-4 * abs(fd), (layer, idx, fd, grads[layer][0][idx])
        j = int(rng.integers(0, len(b)))
        bp = [(ww.copy(), bb.copy()) for ww, bb in weights]
        bm = [(ww.copy(), bb.copy()) for ww, bb in weights]
        bp[layer][1][j] += eps
        bm[layer][1][j] -= eps
        fd = (nn.UNet(bp).loss_and_grads(noisy, clean)[0] - nn.UNet(bm).loss_and_grads(noisy, clean)[0]) / (2 * eps)
        assert abs(fd - grads[layer][1][j]) <= 1e-6 + 1e-4 * abs(fd)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(5).normal(size=1000) * 10.0 ** np.random.default_rng(6).integers(-5, 5, 1000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(nn.bf16_round(x), ref)
