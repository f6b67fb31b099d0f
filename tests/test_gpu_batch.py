"""Batched solves (om_batch_*): many structures advanced together over a
work list of tiles, a check window replayed from a captured graph of
per-step launches or run as one persistent cooperative launch per group
with grid barriers between steps, and per-structure early retirement.
Parity with the oracle per step (random populations, FP64 and FP32) and at
convergence, identical bits in both window modes, structures without nodes,
and the bounded barrier wait."""
import numpy as np
import pytest
import torch

import synthetic as S
from conftest import recon_args

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to("cuda") if dtype is None else t.to("cuda", dtype)


MASKS = [lambda: S.blob_mask((14, 19, 37), 11, n=7), lambda: S.random_mask((9, 33, 35), 0.7, 3),
         lambda: S.square_duct(5, 6), lambda: np.ones((4, 5, 3), np.uint8)]


def _rand_flow(orc, m, seed):
    w = orc.weights19()
    return w[:, None, None, None] * (1 + 0.1 * S.random_field((19,) + m.shape, seed, -1, 1)) * m


def _rand_diff(m, seed):
    a = np.array([0.25] + [0.125] * 6)
    c = S.random_field(m.shape, seed, 0.0, 1.0)
    return a[:, None, None, None] * c[None] * (1 + 0.2 * S.random_field((7,) + m.shape, seed + 1, -1, 1)) * m


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("steps", [1, 2, 10])
def test_batch_flow_steps_match_oracle(orc, om, prec, steps):
    masks = [f() for f in MASKS]
    P = om.OM_F64 if prec == "f64" else om.OM_F32
    tau, g = 0.83, 3e-4
    b = om.Batch([om.domain(m.shape) for m in masks], [_dev(m) for m in masks],
                 flow=om.flow_params(tau=tau, body_force=g, precision=P))
    f0 = [_rand_flow(orc, m, 7 * k + steps) for k, m in enumerate(masks)]
    for k, f in enumerate(f0):
        b.set_populations(0, k, _dev(f))
    b.step(0, steps)
    for k, m in enumerate(masks):
        out = torch.empty(19 * m.size, dtype=torch.float64, device="cuda")
        b.get_populations(0, k, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape((19,) + m.shape)
        ref = orc.flow_step(m, f0[k], tau, g, steps)
        dev = np.abs(f0[k] - orc.weights19()[:, None, None, None] * m).max()
        tol = 1e-13 * steps if prec == "f64" else 64 * U32 * dev * steps + 1e-12
        assert np.abs(got - ref).max() <= tol, k


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("steps", [1, 2, 10])
def test_batch_diffusion_steps_match_oracle(orc, om, prec, steps):
    masks = [f() for f in MASKS]
    P = om.OM_F64 if prec == "f64" else om.OM_F32
    ds = [(S.random_field(m.shape, 40 + k, 3.0, 90.0) * m).astype(np.float32) for k, m in enumerate(masks)]
    b = om.Batch([om.domain(m.shape) for m in masks], [_dev(m) for m in masks], [_dev(d) for d in ds],
                 diff=om.diff_params(c_in=0.9, c_out=0.2, precision=P))
    g0 = [_rand_diff(m, 3 * k + steps) for k, m in enumerate(masks)]
    for k, g in enumerate(g0):
        b.set_populations(1, k, _dev(g))
    b.step(1, steps)
    for k, m in enumerate(masks):
        out = torch.empty(7 * m.size, dtype=torch.float64, device="cuda")
        b.get_populations(1, k, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape((7,) + m.shape)
        ref = orc.diff_step(m, g0[k], orc.omega_field(m, ds[k]), 0.9, 0.2, steps)
        tol = 1e-13 * steps if prec == "f64" else 64 * U32 * np.abs(g0[k]).max() * steps + 1e-12
        assert np.abs(got - ref).max() <= tol, k


def _structures(orc):
    # reconstructed transport sets whose oracle solves converge in seconds
    cfgs = [S.small_structure(s).with_(shape=shape) for s, shape in [(3, (16, 24, 20)), (10, (24, 16, 16)),
                                                                    (11, (24, 16, 16))]]
    out = []
    for cfg in cfgs:
        _, mask, *_ = orc.reconstruct(*recon_args(cfg))
        _, tr, _ = orc.label18(mask)
        d, _ = orc.chord13(mask, cfg.dx_nm, counts=False)
        out.append((tr, d))
    out.append((np.zeros((6, 7, 8), np.uint8), np.zeros((6, 7, 8), np.float32)))  # nothing percolates
    return out


@pytest.mark.timeout(600)
def test_batch_in_l2_groups_steps_match_oracle(orc, om):
    # three structures of ~6e5 nodes: their FP64 flow populations take ~93 MB
    # and their FP64 diffusion fields ~41 MB each, so no two fit in one L2
    # group (80 MB) and every item runs in a group of its own; a window of 5
    # steps is taken group after group and must equal the oracle's steps
    masks = [S.random_mask((72, 96, 96), 0.9, 40 + k) for k in range(3)]
    tau, g = 0.9, 2e-4
    rng = np.random.default_rng(5)
    d = [(10 + 50 * rng.random(m.shape) * m).astype(np.float32) for m in masks]
    b = om.Batch([om.domain(m.shape) for m in masks], [_dev(m) for m in masks], [_dev(x) for x in d],
                 flow=om.flow_params(tau=tau, body_force=g, precision=om.OM_F64),
                 diff=om.diff_params(precision=om.OM_F64, c_in=0.9, c_out=0.1))
    f0 = [_rand_flow(orc, m, 70 + k) for k, m in enumerate(masks)]
    g0 = [_rand_diff(m, 80 + k) for k, m in enumerate(masks)]
    for k in range(3):
        b.set_populations(0, k, _dev(f0[k]))
        b.set_populations(1, k, _dev(g0[k]))
    b.step(0, 5)
    b.step(1, 5)
    for k, m in enumerate(masks):
        out = torch.empty(19 * m.size, dtype=torch.float64, device="cuda")
        b.get_populations(0, k, out)
        ref = orc.flow_step(m, f0[k], tau, g, 5)
        assert np.abs(out.cpu().numpy().reshape(ref.shape) - ref).max() <= 5e-13, k
        out = torch.empty(7 * m.size, dtype=torch.float64, device="cuda")
        b.get_populations(1, k, out)
        ref = orc.diff_step(m, g0[k], orc.omega_field(m, d[k]), 0.9, 0.1, 5)
        assert np.abs(out.cpu().numpy().reshape(ref.shape) - ref).max() <= 5e-13, k


@pytest.mark.timeout(900)
def test_batch_solves_match_oracle(orc, om):
    st = _structures(orc)
    doms = [om.domain(t.shape, 2.0) for t, _ in st]
    ref = []
    for tr, d in st[:-1]:
        rc1, kL, *_ = orc.flow_solve(tr, tau=1.0, g=1e-6, tol=1e-8, K=100, max_steps=200000)
        rc2, D, *_ = orc.diff_solve(tr, orc.omega_field(tr, d), 1.0, 0.0, tol=1e-8, K=100, max_steps=400000)
        assert rc1 == 0 and rc2 == 0
        ref.append((kL, D))
    # FP32 rounding puts a floor of ~1e-7 under the relative-change measures
    # (sums of |du|, |dC| over all nodes); checking every 2000 steps against
    # 1e-6 asks for a rate of change of 5e-10 per step, close to the
    # oracle's 1e-10
    for P, K, tol, rel in ((om.OM_F64, 100, 1e-8, 1e-9), (om.OM_F32, 2000, 1e-6, 1e-5)):
        b = om.Batch(doms, [_dev(t) for t, _ in st], [_dev(d) for _, d in st],
                     flow=om.flow_params(conv_tol=tol, check_every=K, max_steps=400000, precision=P),
                     diff=om.diff_params(conv_tol=tol, check_every=K, max_steps=400000, precision=P))
        kl, _, info_f, st_f = b.solve(0)
        dl, mean_dl, info_d, st_d = b.solve(1)
        assert st_f[-1] == om.OM_ENOPERC and st_d[-1] == om.OM_ENOPERC
        steps = set()
        for k, (kL, D) in enumerate(ref):
            assert st_f[k] == om.OM_OK and st_d[k] == om.OM_OK
            assert kl[k] == pytest.approx(kL, rel=rel)
            assert dl[k] == pytest.approx(D, rel=rel)
            steps.add(info_d[k].steps)
        assert len(steps) > 1  # structures retire at their own check
        b.close()


@pytest.mark.timeout(300)
def test_batch_matches_single_structure_solver(orc, om):
    st = _structures(orc)[1:3]
    doms = [om.domain(t.shape, 2.0) for t, _ in st]
    b = om.Batch(doms, [_dev(t) for t, _ in st], flow=om.flow_params(conv_tol=1e-6))
    kl, _, info, status = b.solve(0)
    for k, (tr, _) in enumerate(st):
        ns = om.NodeSet(_dev(tr), doms[k])
        s1, k1, i1 = om.Flow(ns, om.flow_params(conv_tol=1e-6)).solve()
        assert status[k] == om.OM_OK and s1 == om.OM_OK
        assert kl[k] == pytest.approx(k1, rel=1e-6)
        assert abs(info[k].steps - i1.steps) <= 100


# ------------------------------------------------------------------ persistent windows
def _window_run(om, masks, d, prec, mode, K=100, windows=12):
    """Populations of both models after a solve that runs `windows` whole
    windows (a test of 0 is never met) in window mode `mode`."""
    b = om.Batch([om.domain(m.shape) for m in masks], [_dev(m) for m in masks], [_dev(x) for x in d],
                 flow=om.flow_params(conv_tol=0.0, check_every=K, max_steps=K * windows, precision=prec),
                 diff=om.diff_params(conv_tol=0.0, check_every=K, max_steps=K * windows, precision=prec))
    b.set_window_mode(0, mode)
    b.set_window_mode(1, mode)
    kl, _, _, st_f = b.solve(0)
    dl, _, _, st_d = b.solve(1)
    pops = []
    for model, q in ((0, 19), (1, 7)):
        for k, m in enumerate(masks):
            out = torch.empty(q * m.size, dtype=torch.float64, device="cuda")
            b.get_populations(model, k, out)
            pops.append(out.cpu().numpy())
    b.close()
    return kl, dl, st_f, st_d, pops


# A persistent window (one cooperative launch per group, grid barriers
# between steps) does per step exactly the node updates of the per-step
# launches, so both modes give the same bits, in every storage format, for
# small items packed into one group and for items of a group of their own
# with more tiles than the grid has blocks.
@pytest.mark.timeout(600)
@pytest.mark.parametrize("prec", ["OM_F64", "OM_F32", "OM_F16DEV"])
def test_persistent_windows_equal_graph_windows(orc, om, prec):
    st = _structures(orc)
    masks = [t for t, _ in st] + [S.random_mask((72, 96, 96), 0.9, 41)]
    rng = np.random.default_rng(9)
    d = [x for _, x in st] + [(10 + 50 * rng.random(masks[-1].shape) * masks[-1]).astype(np.float32)]
    P = getattr(om, prec)
    a = _window_run(om, masks, d, P, 0)
    b = _window_run(om, masks, d, P, 1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert list(a[2]) == list(b[2]) and list(a[3]) == list(b[3])
    assert a[2][-2] == om.OM_ENOPERC  # the item without nodes stays out of both
    for x, y in zip(a[4], b[4]):
        assert np.array_equal(x, y)


def test_default_window_mode_times_both_and_matches(orc, om):
    # mode -1: the first two windows of the first solve run one in each mode
    st = _structures(orc)
    masks = [t for t, _ in st]
    d = [x for _, x in st]
    a = _window_run(om, masks, d, om.OM_F32, 0, windows=6)
    b = _window_run(om, masks, d, om.OM_F32, -1, windows=6)
    for x, y in zip(a[4], b[4]):
        assert np.array_equal(x, y)


# The grid barrier's waits are bounded: a barrier that expects one block more
# than the launch has can never complete, every wait gives up after its poll
# limit, the status reports it, the launch ends and the context stays usable.
def test_grid_barrier_wait_is_bounded(om):
    import time
    assert om.om_barrier_selftest(2 * 152, 200, 0, 20_000_000) == om.OM_OK
    t = time.perf_counter()
    assert om.om_barrier_selftest(8, 3, 1, 20_000) == om.OM_ETIMEOUT
    assert time.perf_counter() - t < 10.0
    x = torch.arange(10, device="cuda", dtype=torch.float32)
    assert float(x.sum()) == 45.0
    assert om.om_barrier_selftest(64, 10, 0, 20_000_000) == om.OM_OK
    with pytest.raises(om.OmError):
        om.om_barrier_selftest(10 ** 6, 1, 0, 1000)  # more blocks than can be resident


# ------------------------------------------------------------------ the 150-structure set at full size
# The batched configuration bench.py times (all structures of the
# 150-structure set with transport pores in one batch, L2 groups and solo
# groups, tuned launch shapes, FP32): random states in three items of
# different sizes, three steps of the whole batch, and nodes sampled in
# those items against the oracle on periodic crops around them (the state of
# a node after s steps depends only on nodes within s cells).
@pytest.mark.timeout(1200)
def test_150_set_batch_sampled(orc, om):
    from paper_1410_1921_gb300 import warmstart as W
    items = []
    for cfg in S.batch_structures():
        dom, mask, tr, d = W.structure(cfg)
        if int(tr.sum().item()) > 0:
            items.append((cfg, dom, tr, d))
    doms = [it[1] for it in items]
    tau, gforce = 1.0, 1e-6
    b = om.Batch(doms, [it[2] for it in items], [it[3] for it in items],
                 flow=om.flow_params(tau=tau, body_force=gforce, precision=om.OM_F32),
                 diff=om.diff_params(precision=om.OM_F32))
    sizes = np.array([int(it[2].sum().item()) for it in items])
    picks = [int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 2]), int(np.argmax(sizes))]
    w = torch.tensor(orc.weights19(), dtype=torch.float64, device="cuda")
    f0s = {}
    for k in picks:
        tr = items[k][2]
        gen = torch.Generator(device="cuda").manual_seed(100 + k)
        dev = (1e-3 * (torch.rand(19, tr.numel(), generator=gen, device="cuda", dtype=torch.float32) - 0.5)).double()
        f0s[k] = (w[:, None] + dev) * tr.double()[None]
        b.set_populations(0, k, f0s[k].reshape(-1))
    steps = 3
    b.step(0, steps)
    h = steps + 1
    for k in picks:
        cfg, dom, tr, _ = items[k]
        shape = cfg.shape
        out = torch.empty(19 * tr.numel(), dtype=torch.float64, device="cuda")
        b.get_populations(0, k, out)
        got = out.view(19, *shape)
        tr_np = tr.cpu().numpy().reshape(shape)
        f0v = f0s[k].view(19, *shape)
        pts = np.argwhere(tr_np)
        pts = pts[np.random.default_rng(k).choice(len(pts), min(12, len(pts)), replace=False)]
        for p in pts:
            idx = [torch.arange(p[a] - h, p[a] + h + 1, device="cuda") % shape[a] for a in range(3)]
            fc = f0v[:, idx[0][:, None, None], idx[1][None, :, None], idx[2][None, None, :]].cpu().numpy()
            mc = tr_np[np.ix_(*[np.arange(p[a] - h, p[a] + h + 1) % shape[a] for a in range(3)])]
            ref = orc.flow_step(mc, fc, tau, gforce, steps)[:, h, h, h]
            gv = got[:, p[0], p[1], p[2]].cpu().numpy()
            assert np.abs(gv - ref).max() <= 64 * U32 * 1e-3 * steps + 1e-12, (k, p)
    b.close()


@pytest.mark.timeout(900)
def test_batch_extrapolated_restarts_match_oracle(orc, om):
    # the batch's per-structure extrapolated restarts (OM_ACCEL_EXTRAPOLATE):
    # each structure lands on the oracle's tightly converged D_eff, in fewer
    # steps than the plain batch, in FP64 and FP32 storage
    st = _structures(orc)
    doms = [om.domain(t.shape, 2.0) for t, _ in st]
    ref = []
    for tr, d in st[:-1]:
        rc, D, *_ = orc.diff_solve(tr, orc.omega_field(tr, d), 1.0, 0.0, tol=1e-11, K=100, max_steps=3_000_000)
        assert rc == 0
        ref.append(D)
    for P, tol, rel in ((om.OM_F64, 1e-10, 1e-8), (om.OM_F32, 1e-7, 1e-5)):
        total = {}
        for accel in (om.OM_ACCEL_NONE, om.OM_ACCEL_EXTRAPOLATE):
            b = om.Batch(doms, [_dev(t) for t, _ in st], [_dev(d) for _, d in st],
                         diff=om.diff_params(conv_tol=tol, check_every=1000, max_steps=3_000_000, precision=P,
                                             accel=accel))
            dl, _, info, status = b.solve(1)
            b.close()
            assert status[-1] == om.OM_ENOPERC
            for k, D in enumerate(ref):
                assert status[k] == om.OM_OK
                assert dl[k] == pytest.approx(D, rel=rel), (P, accel, k)
            total[accel] = sum(i.steps for i in info[:-1])
        assert total[om.OM_ACCEL_EXTRAPOLATE] < 0.8 * total[om.OM_ACCEL_NONE], total


# Launch variants 2 and 3 run each structure large enough for a group of its
# own in the single-structure solver's forms: 2 (flow) in the batch's copies
# of its fastest ones (odd steps on a resident grid striding over the nodes,
# even steps two nodes per thread), 3 (flow and diffusion) in that solver's
# own sweeps on the item's slice of the arena (its arena offset a multiple of
# 32), with the launch variants tuned for the item's size.  All do the same per-node arithmetic
# as the one-thread-per-node sweeps, so they give the same bits, in every
# storage format.  In single precision the solve enters each structure's
# rebased mode on the way (its relative change passes 1e-4), as
# om_flow_solve does.
def _variant_run(om, masks, prec, variant, K=100, windows=6):
    rng = np.random.default_rng(9)
    d = [(10 + 50 * rng.random(m.shape) * m).astype(np.float32) for m in masks]
    b = om.Batch([om.domain(m.shape) for m in masks], [_dev(m) for m in masks], [_dev(x) for x in d],
                 flow=om.flow_params(conv_tol=0.0, check_every=K, max_steps=K * windows, precision=prec,
                                     variant=variant),
                 diff=om.diff_params(conv_tol=0.0, check_every=K, max_steps=K * windows, precision=prec,
                                     variant=variant))
    kl, _, _, st = b.solve(0)
    dl, _, _, sd = b.solve(1)
    b.step(0, 3)  # and an odd count of single steps
    b.step(1, 3)
    pops = []
    for model, q in ((0, 19), (1, 7)):
        for k, m in enumerate(masks):
            out = torch.empty(q * m.size, dtype=torch.float64, device="cuda")
            b.get_populations(model, k, out)
            pops.append(out.cpu().numpy())
    b.close()
    return np.concatenate([kl, dl]), list(st) + list(sd), pops


@pytest.mark.timeout(600)
@pytest.mark.parametrize("prec", ["OM_F64", "OM_F32", "OM_BF16DEV"])
def test_large_structure_forms_equal_plain_sweeps(om, prec):
    # items 1 and 3 have > 2^19 nodes (groups of their own); the node counts
    # before item 3 sum to an odd number (its offset is rounded up)
    masks = [S.random_mask((9, 33, 35), 0.7, 3), S.random_mask((72, 96, 96), 0.9, 41),
             S.random_mask((5, 7, 9), 0.6, 1), S.random_mask((64, 96, 96), 0.9, 7)]
    nf = [int(m.sum()) for m in masks]
    assert nf[1] >= 1 << 19 and nf[3] >= 1 << 19
    assert nf[0] % 2 == 0 and sum(nf[:3]) % 2 == 1
    P = getattr(om, prec)
    a = _variant_run(om, masks, P, 0)
    for v in (2, 3):
        b = _variant_run(om, masks, P, v)
        assert np.array_equal(a[0], b[0]) and list(a[1]) == list(b[1])
        for x, y in zip(a[2], b[2]):
            assert np.array_equal(x, y)


@pytest.mark.timeout(600)
def test_batch_rebased_mode_per_structure_matches_single_solver(om):
    masks = [S.random_mask((72, 96, 96), 0.9, 41), S.blob_mask((14, 19, 37), 11, n=7),
             S.random_mask((9, 33, 35), 0.7, 3)]
    doms = [om.domain(m.shape) for m in masks]
    fp = om.flow_params(conv_tol=1e-6, precision=om.OM_F32)
    b = om.Batch(doms, [_dev(m) for m in masks], flow=fp)
    kl, _, info, status = b.solve(0)
    b.close()
    for k, m in enumerate(masks):
        ns = om.NodeSet(_dev(m), doms[k])
        fl = om.Flow(ns, fp)
        s1, k1, i1 = fl.solve()
        fl.close()
        ns.close()
        assert status[k] == om.OM_OK and s1 == om.OM_OK
        assert kl[k] == pytest.approx(k1, rel=1e-6)
        assert abs(info[k].steps - i1.steps) <= 100


# om_batch_get_field: each item's u_x (flow) and C (diffusion) in its voxel
# layout, the moments of the item's own populations (om_batch_get_populations)
# at any time parity, zero off the node set.
@pytest.mark.parametrize("prec", ["OM_F64", "OM_F32"])
def test_batch_fields_are_the_moments_of_the_populations(orc, om, prec):
    st = _structures(orc)
    masks = [t for t, _ in st]
    P = getattr(om, prec)
    g = 1e-6
    b = om.Batch([om.domain(m.shape) for m in masks], [_dev(m) for m in masks], [_dev(x) for _, x in st],
                 flow=om.flow_params(body_force=g, precision=P), diff=om.diff_params(precision=P))
    ex = np.array([e[0] for e in orc.velocities19()], np.float64)
    for steps in (200, 1):
        b.step(0, steps)
        b.step(1, steps)
        for k, m in enumerate(masks):
            N = m.size
            f = torch.empty(19 * N, dtype=torch.float64, device="cuda")
            b.get_populations(0, k, f)
            u = torch.empty(N, dtype=torch.float32, device="cuda")
            b.get_field(0, k, u)
            ux = (ex[:, None] * f.view(19, N).cpu().numpy()).sum(0) + 0.5 * g
            on = m.reshape(-1) > 0
            assert np.allclose(u.cpu().numpy()[on], ux[on], rtol=1e-6, atol=1e-12)
            assert not u.cpu().numpy()[~on].any()
            q = torch.empty(7 * N, dtype=torch.float64, device="cuda")
            b.get_populations(1, k, q)
            c = torch.empty(N, dtype=torch.float32, device="cuda")
            b.get_field(1, k, c)
            assert np.allclose(c.cpu().numpy()[on], q.view(7, N).cpu().numpy().sum(0)[on], rtol=1e-6, atol=1e-12)
            assert not c.cpu().numpy()[~on].any()
    b.close()
