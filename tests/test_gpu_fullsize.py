"""Parity at the benchmark's full size, in the configuration bench.py times:
the 256^3 porosity-0.35 sweep structure, FP32 storage, autotuned launch
variants, graph-replayed windows.  The oracle cannot run 5e6 nodes, but the
state of a node after s steps depends only on the nodes within s cells, so
the oracle runs s steps on a periodic crop of half-width s + 1 around each
sampled node (from the same initial populations) and its centre must match
the GPU field there."""
import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def _structure(om):
    from paper_1410_1921_gb300 import warmstart as W
    cfg = S.sweep_structure(0.35)
    dom, mask, tr, d = W.structure(cfg)
    return cfg, dom, tr, d


def _crop(a, c, h):
    """Periodic crop of the last three axes of a around c (half-width h)."""
    idx = [np.arange(c[k] - h, c[k] + h + 1) % a.shape[-3 + k] for k in range(3)]
    return a[..., idx[0][:, None, None], idx[1][None, :, None], idx[2][None, None, :]]


def _samples(tr_np, n, seed):
    pts = np.argwhere(tr_np)
    return pts[np.random.default_rng(seed).choice(len(pts), n, replace=False)]


@pytest.mark.timeout(900)
def test_fullsize_flow_sampled(orc, om):
    cfg, dom, tr, d = _structure(om)
    shape = cfg.shape
    N = tr.numel()
    steps = 3
    w = torch.tensor(orc.weights19(), dtype=torch.float64, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(5)
    # deviations representable in FP32, so the stored state is exactly f0
    dev = (1e-3 * (torch.rand(19, N, generator=g, device="cuda", dtype=torch.float32) - 0.5)).double()
    f0 = (w[:, None] + dev) * tr.double()[None]
    ns = om.NodeSet(tr, dom)
    tau, gforce = 1.0, 1e-6
    fl = om.Flow(ns, om.flow_params(tau=tau, body_force=gforce, precision=om.OM_F32, check_every=100))
    fl.set_populations(f0.reshape(-1))
    fl.step(steps)
    u = torch.empty(3 * N, dtype=torch.float32, device="cuda")
    fl.get_velocity(u)
    torch.cuda.synchronize()
    tr_np = tr.cpu().numpy().reshape(shape)
    ux = u[:N].cpu().numpy().reshape(shape)
    h = steps + 1
    pts = _samples(tr_np, 40, 11)
    f0v = f0.view(19, *shape)
    for p in pts:
        idx = [torch.arange(p[k] - h, p[k] + h + 1, device="cuda") % shape[k] for k in range(3)]
        fc = f0v[:, idx[0][:, None, None], idx[1][None, :, None], idx[2][None, None, :]].cpu().numpy()
        mc = _crop(tr_np, p, h)
        f1 = orc.flow_step(mc, fc, tau, gforce, steps)
        ref = orc.flow_velocity(mc, f1, gforce)[0][h, h, h]
        assert abs(ux[tuple(p)] - ref) <= 64 * U32 * 1e-3 * steps + 1e-9, p


@pytest.mark.timeout(900)
def test_fullsize_diffusion_sampled(orc, om):
    cfg, dom, tr, d = _structure(om)
    shape = cfg.shape
    N = tr.numel()
    steps = 3
    a = torch.tensor([0.25] + [0.125] * 6, dtype=torch.float64, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(6)
    c0 = torch.rand(N, generator=g, device="cuda", dtype=torch.float32).double()
    g0 = a[:, None] * c0[None] * tr.double()[None]
    ns = om.NodeSet(tr, dom)
    df = om.Diffusion(ns, d, om.diff_params(precision=om.OM_F32, check_every=100))
    df.set_populations(g0.reshape(-1))
    df.step(steps)
    c = torch.empty(N, dtype=torch.float32, device="cuda")
    df.get_fields(c, None)
    torch.cuda.synchronize()
    tr_np = tr.cpu().numpy().reshape(shape)
    cg = c.cpu().numpy().reshape(shape)
    d_np = d.cpu().numpy().reshape(shape)
    h = steps + 1
    pts = _samples(tr_np, 40, 12)
    g0v = g0.view(7, *shape)
    for p in pts:
        if p[0] < h or p[0] >= shape[0] - h:
            continue  # the x faces are Dirichlet, not periodic: keep crops inside
        idx = [torch.arange(p[k] - h, p[k] + h + 1, device="cuda") % shape[k] for k in range(3)]
        gc = g0v[:, idx[0][:, None, None], idx[1][None, :, None], idx[2][None, None, :]].cpu().numpy()
        mc = _crop(tr_np, p, h)
        oc = orc.omega_field(mc, _crop(d_np, p, h))
        g1 = orc.diff_step(mc, gc, oc, 1.0, 0.0, steps)
        ref = orc.diff_fields(mc, g1, oc)[0][h, h, h]
        assert abs(cg[tuple(p)] - ref) <= 64 * U32 * steps + 1e-9, p


# ------------------------------------------------------------------ the 512^3 16-bit configuration
# The precision workload at its full size (512^3, porosity 0.30, <d> 40 nm):
# FP16 and BF16 population storage, FP32 collision, autotuned launch
# variants.  Initial states are chosen (nearly) representable in the storage
# (flow deviations on the 16-bit grid of the scaled format; diffusion at
# local equilibrium), so the sampled nodes differ from the oracle only by
# the storage rounding of each step (and of the import):
# at most half an ulp of the stored deviation per population, i.e.
# |dev| 2^-8 (FP16: 11-bit significand; BF16: 8-bit, taken for both) summed
# over the populations of a node and the steps.
def _large(om):
    from paper_1410_1921_gb300 import warmstart as W
    cfg = S.large_structure()
    dom, mask, tr, d = W.structure(cfg)
    return cfg, dom, tr, d


@pytest.mark.timeout(900)
@pytest.mark.parametrize("prec,bits", [("OM_F16DEV", 11), ("OM_BF16DEV", 8)])
def test_512_16bit_flow_sampled(orc, om, prec, bits):
    cfg, dom, tr, d = _large(om)
    shape = cfg.shape
    N = tr.numel()
    steps = 3
    up = 1024.0 if prec == "OM_F16DEV" else 1.0
    w = torch.tensor(orc.weights19(), dtype=torch.float64, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(7)
    dev = 1e-3 * (torch.rand(19, N, generator=g, device="cuda", dtype=torch.float32) - 0.5)
    q = dev * up
    q = (q.half() if prec == "OM_F16DEV" else q.bfloat16()).double() / up  # on the storage grid
    f0 = (w[:, None] + q) * tr.double()[None]
    del dev
    ns = om.NodeSet(tr, dom)
    tau, gforce = 1.0, 1e-6
    fl = om.Flow(ns, om.flow_params(tau=tau, body_force=gforce, precision=getattr(om, prec), check_every=100))
    fl.set_populations(f0.reshape(-1))
    fl.step(steps)
    u = torch.empty(3 * N, dtype=torch.float32, device="cuda")
    fl.get_velocity(u)
    torch.cuda.synchronize()
    tr_np = tr.cpu().numpy().reshape(shape)
    ux = u[:N].cpu().numpy().reshape(shape)
    h = steps + 1
    pts = _samples(tr_np, 30, 13)
    f0v = f0.view(19, *shape)
    tol = steps * 19 * 2e-3 * 2.0 ** -bits + 1e-9  # |dev| stays below ~2e-3
    for p in pts:
        idx = [torch.arange(p[k] - h, p[k] + h + 1, device="cuda") % shape[k] for k in range(3)]
        fc = f0v[:, idx[0][:, None, None], idx[1][None, :, None], idx[2][None, None, :]].cpu().numpy()
        mc = _crop(tr_np, p, h)
        f1 = orc.flow_step(mc, fc, tau, gforce, steps)
        ref = orc.flow_velocity(mc, f1, gforce)[0][h, h, h]
        assert abs(ux[tuple(p)] - ref) <= tol, p


@pytest.mark.timeout(900)
@pytest.mark.parametrize("prec,bits", [("OM_F16DEV", 11), ("OM_BF16DEV", 8)])
def test_512_16bit_diffusion_sampled(orc, om, prec, bits):
    cfg, dom, tr, d = _large(om)
    shape = cfg.shape
    N = tr.numel()
    steps = 3
    a = torch.tensor([0.25] + [0.125] * 6, dtype=torch.float64, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(8)
    c0 = torch.rand(N, generator=g, device="cuda", dtype=torch.float32).double()
    g0 = a[:, None] * c0[None] * tr.double()[None]
    ns = om.NodeSet(tr, dom)
    df = om.Diffusion(ns, d, om.diff_params(precision=getattr(om, prec), check_every=100))
    df.set_populations(g0.reshape(-1))
    del g0
    df.step(steps)
    c = torch.empty(N, dtype=torch.float32, device="cuda")
    df.get_fields(c, None)
    torch.cuda.synchronize()
    tr_np = tr.cpu().numpy().reshape(shape)
    cg = c.cpu().numpy().reshape(shape)
    d_np = d.cpu().numpy().reshape(shape)
    c0v = c0.view(*shape)
    h = steps + 1
    pts = _samples(tr_np, 30, 14)
    # deviations a_i |C_nb - C| <= 1/4; one more rounding for the import into the storage
    tol = (steps + 1) * 7 * 0.25 * 2.0 ** -bits + 1e-6
    for p in pts:
        if p[0] < h or p[0] >= shape[0] - h:
            continue
        idx = [torch.arange(p[k] - h, p[k] + h + 1, device="cuda") % shape[k] for k in range(3)]
        cc = c0v[idx[0][:, None, None], idx[1][None, :, None], idx[2][None, None, :]].cpu().numpy()
        mc = _crop(tr_np, p, h)
        gc = np.array([0.25] + [0.125] * 6)[:, None, None, None] * cc[None] * mc[None]
        oc = orc.omega_field(mc, _crop(d_np, p, h))
        g1 = orc.diff_step(mc, gc, oc, 1.0, 0.0, steps)
        ref = orc.diff_fields(mc, g1, oc)[0][h, h, h]
        assert abs(cg[tuple(p)] - ref) <= tol, p
