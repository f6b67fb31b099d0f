"""FP64 CPU reference of the warm-start U-Net (plain PyTorch CPU ops).

TEST INFRASTRUCTURE ONLY.  Rebuilds, from the flat parameter vector of
om_unet, the network the CUDA path evaluates -- per level two 3x3x3
convolutions with ReLU, 2x average pooling down, nearest 2x upsampling and
(upsampled, skip) channel concatenation up, a 1x1 head -- and differentiates
the masked mean-squared error with autograd.  `round_bf16` rounds the inputs,
weights and every stored activation to BF16 at the points where the CUDA
path stores BF16, so the two differ only by accumulation order.

Conventions pinned in tests/test_oracle_unet.py: the 3x3x3 weight index
k = 9 (dz+1) + 3 (dy+1) + (dx+1) over (z, y, x) = (D, H, W) and the
correlation sign (output at v sums input at v + offset).
"""
import torch
import torch.nn.functional as F

IN_PAD = 16  # the input is zero-padded to 16 channels


def layout(in_ch, out_ch, ch):
    """[(name, shape)] of the flat parameter vector, in order."""
    L = len(ch)
    out = []
    for l in range(L):
        cin = IN_PAD if l == 0 else ch[l - 1]
        out += [(f"enc{l}.1.w", (27, cin, ch[l])), (f"enc{l}.1.b", (ch[l],)),
                (f"enc{l}.2.w", (27, ch[l], ch[l])), (f"enc{l}.2.b", (ch[l],))]
    for l in range(L - 2, -1, -1):
        out += [(f"dec{l}.1.w", (27, ch[l + 1] + ch[l], ch[l])), (f"dec{l}.1.b", (ch[l],)),
                (f"dec{l}.2.w", (27, ch[l], ch[l])), (f"dec{l}.2.b", (ch[l],))]
    out += [("head.w", (ch[0], out_ch)), ("head.b", (out_ch,))]
    return out


def unflatten(flat, in_ch, out_ch, ch):
    p, off = {}, 0
    for name, shape in layout(in_ch, out_ch, ch):
        n = 1
        for s in shape:
            n *= s
        p[name] = flat[off:off + n].reshape(shape)
        off += n
    assert off == flat.numel()
    return p


def _bf16(t, on):
    return t.to(torch.bfloat16).to(t.dtype) if on else t


def conv3(x, w, b, rb):
    """x [B, C, D, H, W]; w [27, cin, cout] -> torch weight [cout, cin, 3, 3, 3]."""
    wt = _bf16(w, rb).reshape(3, 3, 3, w.shape[1], w.shape[2]).permute(4, 3, 0, 1, 2)
    return F.conv3d(x, wt, b, padding=1)


def forward(p, x, in_ch, out_ch, ch, round_bf16=False):
    """x [B, D, H, W, in_ch] float64 -> y [B, D, H, W, out_ch]."""
    rb = round_bf16
    B, D, H, W, _ = x.shape
    x0 = torch.zeros(B, IN_PAD, D, H, W, dtype=x.dtype)
    x0[:, :in_ch] = x.permute(0, 4, 1, 2, 3)
    x0 = _bf16(x0, rb)
    L = len(ch)
    s = []
    inp = x0
    for l in range(L):
        if l > 0:
            inp = _bf16(F.avg_pool3d(s[l - 1], 2), rb)
        a = _bf16(F.relu(conv3(inp, p[f"enc{l}.1.w"], p[f"enc{l}.1.b"], rb)), rb)
        s.append(_bf16(F.relu(conv3(a, p[f"enc{l}.2.w"], p[f"enc{l}.2.b"], rb)), rb))
    h = s[L - 1]
    for l in range(L - 2, -1, -1):
        u = F.interpolate(h, scale_factor=2, mode="nearest")
        bl = _bf16(F.relu(conv3(torch.cat([u, s[l]], dim=1), p[f"dec{l}.1.w"], p[f"dec{l}.1.b"], rb)), rb)
        h = _bf16(F.relu(conv3(bl, p[f"dec{l}.2.w"], p[f"dec{l}.2.b"], rb)), rb)
    y = torch.einsum("bcdhw,co->bdhwo", h, p["head.w"]) + p["head.b"]
    return y


def masked_mse(y, t, m):
    keep = (m != 0).to(y.dtype)[..., None]
    cnt = keep.sum() * y.shape[-1]
    return (((y - t) * keep) ** 2).sum() / cnt


def loss_and_grads(flat, x, t, m, in_ch, out_ch, ch, round_bf16=False):
    """Masked MSE and its gradient w.r.t. the flat parameter vector (FP64)."""
    w = flat.detach().clone().to(torch.float64).requires_grad_(True)
    p = unflatten(w, in_ch, out_ch, ch)
    y = forward(p, x.to(torch.float64), in_ch, out_ch, ch, round_bf16)
    loss = masked_mse(y, t.to(torch.float64), m)
    loss.backward()
    return loss.item(), w.grad.detach(), y.detach()
