"""ORACLE -- test infrastructure only (see oracle/__init__.py).

Plain numpy FP64 restatement of the learned scatter denoiser: 3x3 'same'
convolutions (NHWC, weights [cout][9][cin] with tap = 3 (dy+1) + (dx+1)),
their input and weight gradients written from the definition of the
convolution, 2x2 max pooling (first maximum of each window), nearest 2x
up-sampling, channel concatenation [up, skip], the residual U-Net of
paper_2201_13191_gb300's denoiser (4 levels, 32 base channels), mean
normalisation, the mean-squared-error loss and its full backward pass.

With bf16=True the activations, the masked gradients fed to each layer's
weight/input gradient and the weights are rounded to BF16 at the points
where the GPU stores them in BF16 (round to nearest even), so the GPU can
be compared against the same arithmetic; with bf16=False everything is FP64
(this mode is pinned against finite differences).
"""

from __future__ import annotations

import numpy as np

CIN = [16, 32, 32, 64, 64, 128, 128, 256, 384, 128, 192, 64, 96, 32, 32]
COUT = [32, 32, 64, 64, 128, 128, 256, 256, 128, 128, 64, 64, 32, 32, 16]
LEVEL = [0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0, 0]


def bf16_round(x):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_bits(x):
    """BF16 bit patterns (uint16) of x (round to nearest even)."""
    f = np.asarray(bf16_round(x), dtype=np.float32)
    return (f.view(np.uint32) >> 16).astype(np.uint16)


def conv3x3(x, w, b=None):
    """y[n,y,x,co] = sum_{dy,dx,ci} x[n,y+dy,x+dx,ci] w[co, 3(dy+1)+(dx+1), ci] + b[co], zero padded."""
    n, h, wd, cin = x.shape
    cout = w.shape[0]
    xp = np.zeros((n, h + 2, wd + 2, cin))
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((n, h, wd, cout))
    for tap in range(9):
        dy, dx = tap // 3, tap % 3
        y += np.einsum("nhwc,oc->nhwo", xp[:, dy : dy + h, dx : dx + wd], w[:, tap, :])
    if b is not None:
        y += b
    return y


def conv3x3_wgrad(x, gy):
    """dL/dw[co, tap, ci] = sum over pixels of gy[p, co] x[p + tap, ci]."""
    n, h, wd, cin = x.shape
    xp = np.zeros((n, h + 2, wd + 2, cin))
    xp[:, 1:-1, 1:-1] = x
    gw = np.zeros((gy.shape[-1], 9, cin))
    for tap in range(9):
        dy, dx = tap // 3, tap % 3
        gw[:, tap, :] = np.einsum("nhwo,nhwc->oc", gy, xp[:, dy : dy + h, dx : dx + wd])
    return gw


def conv3x3_dgrad(gy, w):
    """dL/dx[p, ci] = sum_{tap, co} gy[p - tap, co] w[co, tap, ci] (adjoint of conv3x3)."""
    n, h, wd, cout = gy.shape
    cin = w.shape[2]
    gx = np.zeros((n, h + 2, wd + 2, cin))
    for tap in range(9):
        dy, dx = tap // 3, tap % 3
        gx[:, dy : dy + h, dx : dx + wd] += np.einsum("nhwo,oc->nhwc", gy, w[:, tap, :])
    return gx[:, 1:-1, 1:-1]


def pool_fwd(x):
    n, h, w, c = x.shape
    blocks = x.reshape(n, h // 2, 2, w // 2, 2, c).transpose(0, 1, 3, 5, 2, 4).reshape(n, h // 2, w // 2, c, 4)
    return blocks.max(axis=-1), blocks.argmax(axis=-1)  # argmax: first maximum in order (0,0),(0,1),(1,0),(1,1)


def pool_bwd(arg, gy, shape):
    n, h, w, c = shape
    g = np.zeros((n, h // 2, w // 2, c, 4))
    np.put_along_axis(g, arg[..., None], gy[..., None], axis=-1)
    return g.reshape(n, h // 2, w // 2, c, 2, 2).transpose(0, 1, 4, 2, 5, 3).reshape(n, h, w, c)


def up_fwd(x):
    return x.repeat(2, axis=1).repeat(2, axis=2)


def up_bwd(g):
    n, h, w, c = g.shape
    return g.reshape(n, h // 2, 2, w // 2, 2, c).sum(axis=(2, 4))


class UNet:
    """Weights: list of (w [cout][9][cin], b [cout]) float64."""

    def __init__(self, weights, bf16=False):
        self.W = [(np.asarray(w, dtype=np.float64), np.asarray(b, dtype=np.float64)) for w, b in weights]
        self.bf16 = bf16

    def _r(self, x):
        return bf16_round(x) if self.bf16 else x

    def _conv(self, i, x, relu=True):
        w, b = self.W[i]
        y = conv3x3(x, self._r(w), b)
        return np.maximum(y, 0.0) if relu else y

    def forward(self, img):
        """img [n][h][w] -> (net output channel 0 [n][h][w], scale [n], cache)."""
        s = np.maximum(img.mean(axis=(1, 2)), 1e-30)
        x0 = np.zeros(img.shape + (16,))
        x0[..., 0] = img / s[:, None, None]
        x0 = self._r(x0)
        c = {"in0": x0, "s": s}
        r = self._r
        c["a0a"] = r(self._conv(0, x0))
        c["s0"] = r(self._conv(1, c["a0a"]))
        c["p0"], c["arg0"] = pool_fwd(c["s0"])
        c["a1a"] = r(self._conv(2, c["p0"]))
        c["s1"] = r(self._conv(3, c["a1a"]))
        c["p1"], c["arg1"] = pool_fwd(c["s1"])
        c["a2a"] = r(self._conv(4, c["p1"]))
        c["s2"] = r(self._conv(5, c["a2a"]))
        c["p2"], c["arg2"] = pool_fwd(c["s2"])
        c["a3a"] = r(self._conv(6, c["p2"]))
        c["a3b"] = r(self._conv(7, c["a3a"]))
        c["cat2"] = np.concatenate([up_fwd(c["a3b"]), c["s2"]], axis=-1)
        c["u2a"] = r(self._conv(8, c["cat2"]))
        c["u2b"] = r(self._conv(9, c["u2a"]))
        c["cat1"] = np.concatenate([up_fwd(c["u2b"]), c["s1"]], axis=-1)
        c["u1a"] = r(self._conv(10, c["cat1"]))
        c["u1b"] = r(self._conv(11, c["u1a"]))
        c["cat0"] = np.concatenate([up_fwd(c["u1b"]), c["s0"]], axis=-1)
        c["u0a"] = r(self._conv(12, c["cat0"]))
        c["u0b"] = r(self._conv(13, c["u0a"]))
        c["out"] = self._conv(14, c["u0b"], relu=False)
        return c["out"][..., 0], s, c

    def denoise(self, img):
        out0, s, _ = self.forward(img)
        return img + s[:, None, None] * out0

    def loss_and_grads(self, noisy, clean):
        """Mean squared error of the normalised residual prediction and its gradients."""
        out0, s, c = self.forward(noisy)
        d = noisy / s[:, None, None] + out0 - clean / s[:, None, None]
        loss = float(np.mean(d * d))
        g_out = np.zeros(c["out"].shape)
        g_out[..., 0] = 2.0 * d / d.size
        grads = [None] * 15
        r = self._r

        def back(i, x, y, gy, relu=True):
            gm = gy * (y > 0) if relu else gy
            gm = r(gm)
            grads[i] = (conv3x3_wgrad(x, gm), gm.sum(axis=(0, 1, 2)))
            return conv3x3_dgrad(gm, r(self.W[i][0]))

        g = back(14, c["u0b"], None, g_out, relu=False)
        g = back(13, c["u0a"], c["u0b"], g)
        g = back(12, c["cat0"], c["u0a"], g)
        g_up, g_s0 = g[..., :64], g[..., 64:]
        g = back(11, c["u1a"], c["u1b"], up_bwd(g_up))
        g = back(10, c["cat1"], c["u1a"], g)
        g_up, g_s1 = g[..., :128], g[..., 128:]
        g = back(9, c["u2a"], c["u2b"], up_bwd(g_up))
        g = back(8, c["cat2"], c["u2a"], g)
        g_up, g_s2 = g[..., :256], g[..., 256:]
        g = back(7, c["a3a"], c["a3b"], up_bwd(g_up))
        g = back(6, c["p2"], c["a3a"], g)
        g_s2 = g_s2 + pool_bwd(c["arg2"], g, c["s2"].shape)
        g = back(5, c["a2a"], c["s2"], g_s2)
        g = back(4, c["p1"], c["a2a"], g)
        g_s1 = g_s1 + pool_bwd(c["arg1"], g, c["s1"].shape)
        g = back(3, c["a1a"], c["s1"], g_s1)
        g = back(2, c["p0"], c["a1a"], g)
        g_s0 = g_s0 + pool_bwd(c["arg0"], g, c["s0"].shape)
        g = back(1, c["a0a"], c["s0"], g_s0)
        back(0, c["in0"], c["a0a"], g)
        return loss, grads


def random_weights(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    out = []
    for i, (ci, co) in enumerate(zip(CIN, COUT)):
        fan = 9 * (1 if i == 0 else ci)
        w = rng.normal(0, np.sqrt(2.0 / fan) * (0.1 if i == 14 else 1.0) * scale, size=(co, 9, ci))
        b = rng.normal(0, 0.01, size=co)
        out.append((w, b))
    return out
