"""Pins of the U-Net reference: the weight-offset convention of its 3x3x3
convolution (an impulse reproduces the weight of the opposite offset), the
pooling/upsampling adjoint identity, the flat parameter layout, and the
gradient against central finite differences on a tiny network."""
import numpy as np
import torch

from oracle import unet as U


def test_conv_offset_convention():
    # output at v sums input at v + o_k with o_k = (k//9 - 1, k//3 % 3 - 1, k % 3 - 1)
    for k in (0, 4, 13, 17, 26):
        w = torch.zeros(27, 1, 1, dtype=torch.float64)
        w[k, 0, 0] = 1.0
        x = torch.zeros(1, 1, 5, 5, 5, dtype=torch.float64)
        x[0, 0, 2, 2, 2] = 1.0
        y = U.conv3(x, w, None, False)[0, 0]
        dz, dy, dx = k // 9 - 1, k // 3 % 3 - 1, k % 3 - 1
        assert y[2 - dz, 2 - dy, 2 - dx] == 1.0 and y.sum() == 1.0


def test_pool_upsample_adjoint():
    g = torch.Generator().manual_seed(0)
    a = torch.rand(1, 3, 2, 2, 2, generator=g, dtype=torch.float64)
    b = torch.rand(1, 3, 4, 4, 4, generator=g, dtype=torch.float64)
    up = torch.nn.functional.interpolate(a, scale_factor=2, mode="nearest")
    pool = torch.nn.functional.avg_pool3d(b, 2)
    assert torch.allclose((up * b).sum(), 8 * (a * pool).sum())


def test_layout_sizes():
    ch = (16, 32)
    names = [n for n, _ in U.layout(2, 2, ch)]
    assert names[:4] == ["enc0.1.w", "enc0.1.b", "enc0.2.w", "enc0.2.b"]
    assert names[-2:] == ["head.w", "head.b"]
    n = sum(int(np.prod(s)) for _, s in U.layout(2, 2, ch))
    assert n == 27 * 16 * 16 + 16 + 27 * 16 * 16 + 16 + 27 * 16 * 32 + 32 + 27 * 32 * 32 + 32 \
        + 27 * 48 * 16 + 16 + 27 * 16 * 16 + 16 + 16 * 2 + 2


def test_gradient_finite_differences():
    ch, in_ch, out_ch = (16, 16), 2, 2
    n = sum(int(np.prod(s)) for _, s in U.layout(in_ch, out_ch, ch))
    g = torch.Generator().manual_seed(1)
    flat = 0.1 * torch.randn(n, generator=g, dtype=torch.float64)
    x = torch.rand(1, 4, 4, 4, in_ch, generator=g, dtype=torch.float64)
    t = torch.rand(1, 4, 4, 4, out_ch, generator=g, dtype=torch.float64)
    m = (torch.rand(1, 4, 4, 4, generator=g) > 0.3).to(torch.uint8)
    loss, grad, _ = U.loss_and_grads(flat, x, t, m, in_ch, out_ch, ch)
    rng = np.random.default_rng(2)
    for i in rng.choice(n, 12, replace=False):
        e = torch.zeros(n, dtype=torch.float64)
        e[i] = 1e-6
        lp = U.masked_mse(U.forward(U.unflatten(flat + e, in_ch, out_ch, ch), x, in_ch, out_ch, ch), t, m)
        lm = U.masked_mse(U.forward(U.unflatten(flat - e, in_ch, out_ch, ch), x, in_ch, out_ch, ch), t, m)
        fd = (lp - lm).item() / 2e-6
        assert abs(fd - grad[i].item()) <= 1e-6 * max(1.0, abs(fd))
