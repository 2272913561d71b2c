"""Learned denoiser on the tcgen05 tensor cores vs the FP64 numpy oracle.

Convolution kernels: the GPU multiplies BF16 values exactly and sums in FP32,
so against an FP64 sum of the same BF16 inputs the error is the FP32
summation's (<= 1e-5 relative here).  Whole-network gradients: the oracle
rounds to BF16 at the points where the GPU stores BF16; the rest of the
difference is FP32 vs FP64 arithmetic and rare one-ulp flips of a BF16
rounding, so per-layer gradients must agree to 5e-2 relative L2 (median over
layers 1.5e-2, cosine > 0.998); the deepest layers see only 8 x 8 pixels per
image, where one flipped BF16 rounding weighs most.
"""

import numpy as np
import pytest

from oracle import nn

pytestmark = pytest.mark.gpu


def _bf(torch, a):
    return torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).cuda()


@pytest.mark.parametrize("shape", [(2, 16, 24, 16, 32), (1, 10, 13, 32, 48), (1, 8, 8, 384, 128), (2, 9, 16, 64, 256),
                                   (1, 4, 4, 16, 16), (2, 7, 80, 32, 32), (1, 5, 150, 96, 16)])
def test_conv3x3_forward_parity(gpu, shape):
    torch = pytest.importorskip("torch")
    n, h, w, cin, cout = shape
    rng = np.random.default_rng(sum(shape))
    x = nn.bf16_round(rng.normal(size=(n, h, w, cin)))
    wt = nn.bf16_round(rng.normal(size=(cout, 9, cin)) / np.sqrt(9 * cin))
    b = rng.normal(size=cout).astype(np.float32)
    ref = nn.conv3x3(x, wt, b.astype(np.float64))
    y = gpu.conv3x3(_bf(torch, x), _bf(torch, wt), torch.tensor(b).cuda(), relu=False, out_f32=True)
    got = y.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    # fused ReLU and BF16 store
    yb = gpu.conv3x3(_bf(torch, x), _bf(torch, wt), torch.tensor(b).cuda(), relu=True, out_f32=False)
    gotb = yb.to(torch.float32).cpu().numpy().astype(np.float64)
    refb = nn.bf16_round(np.maximum(ref, 0.0))
    mism = np.abs(gotb - refb) > 1e-6 * np.abs(refb).max()
    assert mism.mean() < 1e-3  # only where FP32 vs FP64 sums round to different BF16 neighbours
    assert np.abs(gotb - refb).max() <= 2 ** -7 * np.abs(refb).max()


@pytest.mark.parametrize("shape", [(2, 12, 20, 32, 64), (1, 16, 16, 384, 128), (3, 5, 7, 16, 32)])
def test_conv3x3_weight_gradient_parity(gpu, shape):
    torch = pytest.importorskip("torch")
    n, h, w, cin, cout = shape
    rng = np.random.default_rng(7 + sum(shape))
    x = nn.bf16_round(rng.normal(size=(n, h, w, cin)))
    dy = nn.bf16_round(rng.normal(size=(n, h, w, cout)))
    ref = nn.conv3x3_wgrad(x, dy)
    for splits in (1, 5):
        got = gpu.conv3x3_wgrad(_bf(torch, x), _bf(torch, dy), splits=splits).cpu().numpy().astype(np.float64)
        assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max(), splits


def test_conv3x3_input_gradient_via_adjoint_weights(gpu):
    """The input gradient is the forward kernel run with flipped, transposed weights."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    gy = nn.bf16_round(rng.normal(size=(2, 8, 12, 64)))
    w = nn.bf16_round(rng.normal(size=(64, 9, 32)))
    wt = w.transpose(2, 1, 0)[:, ::-1, :]  # [cin][tap][cout] flipped in space
    got = gpu.conv3x3(_bf(torch, gy), _bf(torch, np.ascontiguousarray(wt))).cpu().numpy()
    ref = nn.conv3x3_dgrad(gy, w)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def _smooth_fields(rng, n, h, w):
    yy, xx = np.mgrid[0:h, 0:w] / h
    out = []
    for _ in range(n):
        a, b, c, d = rng.uniform(0.5, 2.0, 4)
        out.append(1.0 + 0.5 * np.sin(a * 3 * xx + b) * np.cos(c * 3 * yy + d))
    return np.array(out)


def test_denoiser_gradients_match_oracle(gpu):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(12)
    H = W = 64
    weights = nn.random_weights(5)
    c = gpu.Context(0)
    c.denoise_init(H, W, 2, seed=1)
    for i, (w, b) in enumerate(weights):
        c.denoise_set_layer(i, w, b)
    clean = _smooth_fields(rng, 2, H, W)
    noisy = clean * rng.gamma(20.0, 1 / 20.0, size=clean.shape)
    loss = c.denoise_train_step(torch.tensor(noisy, dtype=torch.float32).cuda(),
                                torch.tensor(clean, dtype=torch.float32).cuda(), lr=0.0)
    ref_net = nn.UNet([(nn.bf16_round(w), b.astype(np.float32).astype(np.float64)) for w, b in weights], bf16=True)
    ref_loss, grads = ref_net.loss_and_grads(noisy.astype(np.float32).astype(np.float64),
                                             clean.astype(np.float32).astype(np.float64))
    assert abs(loss / ref_loss - 1.0) < 1e-2, (loss, ref_loss)
    errs = []
    for i in range(15):
        _, _, gw, gb = c.denoise_layer(i)
        rw, rb = grads[i]
        ew = np.linalg.norm(gw - rw) / max(np.linalg.norm(rw), 1e-30)
        eb = np.linalg.norm(gb - rb) / max(np.linalg.norm(rb), 1e-30)
        cos = float(np.sum(gw * rw) / (np.linalg.norm(gw) * np.linalg.norm(rw)))
        errs.append(ew)
        assert ew < 5e-2 and eb < 5e-2 and cos > 0.998, (i, ew, eb, cos)
    assert np.median(errs) < 1.5e-2, errs


def test_denoiser_learns_and_checkpoints(gpu, tmp_path):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(13)
    H = W = 64
    c = gpu.Context(0)
    c.denoise_init(H, W, 8, seed=3)
    clean = _smooth_fields(rng, 64, H, W)
    noisy = clean * rng.gamma(8.0, 1 / 8.0, size=clean.shape)
    tc = torch.tensor(clean, dtype=torch.float32).cuda()
    tn = torch.tensor(noisy, dtype=torch.float32).cuda()
    losses = []
    for step in range(120):
        k = (step * 8) % 64
        losses.append(c.denoise_train_step(tn[k : k + 8], tc[k : k + 8], lr=1e-3))
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:10]), (losses[:10], losses[-10:])
    out = c.denoise_infer(tn).cpu().numpy()
    err_noisy = np.linalg.norm(noisy - clean) / np.linalg.norm(clean)
    err_out = np.linalg.norm(out - clean) / np.linalg.norm(clean)
    assert err_out < 0.7 * err_noisy, (err_out, err_noisy)
    path = tmp_path / "den.bin"
    c.denoise_save(path)
    c2 = gpu.Context(0)
    c2.denoise_load(path, max_batch=8)
    out2 = c2.denoise_infer(tn).cpu().numpy()
    np.testing.assert_array_equal(out, out2)
    # the denoiser as the smoothing step of mc_smooth_upsample
    c.set_options(denoise_mode=1)
    up = c.smooth_upsample(tn[:2], [0.0, 3.0], [0.0, 3.0], W, H)
    np.testing.assert_allclose(up.cpu().numpy(), out[:2], rtol=1e-5, atol=1e-6)
