"""Two-level warm start of the diffusion (om_coarsen2_dev, om_prolong2_dev):
the coarsening and the prolongation against plain numpy restatements of
their definitions (bit for bit, odd and even extents), and a fine solve
started from the prolonged coarse solution: the same D_eff as the cold solve
under the same test, in fewer steps."""
import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to("cuda") if dtype is None else t.to("cuda", dtype)


def _coarsen_ref(m, d):
    nx, ny, nz = m.shape
    cx, cy, cz = (nx + 1) // 2, (ny + 1) // 2, (nz + 1) // 2
    mc = np.zeros((cx, cy, cz), np.uint8)
    dc = np.zeros((cx, cy, cz), np.float32)
    for X in range(cx):
        for Y in range(cy):
            for Z in range(cz):
                blk = m[2 * X:2 * X + 2, 2 * Y:2 * Y + 2, 2 * Z:2 * Z + 2]
                dd = d[2 * X:2 * X + 2, 2 * Y:2 * Y + 2, 2 * Z:2 * Z + 2]
                cnt = int(blk.sum())
                mc[X, Y, Z] = 1 if 2 * cnt >= blk.size else 0
                s = 0.0
                for v, f in zip(blk.ravel(), dd.ravel()):
                    if v:
                        s += float(f)
                dc[X, Y, Z] = np.float32(s / cnt) if cnt else 0.0
    return mc, dc


@pytest.mark.parametrize("shape,seed", [((8, 6, 10), 1), ((9, 7, 5), 2), ((1, 4, 3), 3), ((15, 16, 17), 4)])
def test_coarsen_matches_definition(om, shape, seed):
    m = S.random_mask(shape, 0.55, seed)
    d = (S.random_field(shape, seed + 10, 3.0, 90.0) * m).astype(np.float32)
    dom = om.domain(shape)
    dc, mc, dcd = om.om_coarsen2_dev(_dev(m), dom, _dev(d))
    ref_m, ref_d = _coarsen_ref(m, d)
    assert (dc.nx, dc.ny, dc.nz) == ref_m.shape and dc.dx_nm == 2 * dom.dx_nm
    assert np.array_equal(mc.cpu().numpy().reshape(ref_m.shape), ref_m)
    assert np.array_equal(dcd.cpu().numpy().reshape(ref_d.shape), ref_d)


@pytest.mark.parametrize("shape,seed,q", [((8, 6, 10), 5, 7), ((9, 7, 5), 6, 19)])
def test_prolong_matches_definition(om, shape, seed, q):
    dom = om.domain(shape)
    dc = om.om_coarse_domain(dom)
    cshape = (dc.nx, dc.ny, dc.nz)
    mc = S.random_mask(cshape, 0.6, seed)
    g = S.random_field((q,) + cshape, seed + 1, 0.0, 0.2) * mc
    out = torch.empty(int(np.prod(shape)), dtype=torch.float32, device="cuda")
    om.om_prolong2_dev(_dev(g), q, _dev(mc), dom, 0.9, 0.1, out)
    got = out.cpu().numpy().reshape(shape)
    ref = np.zeros(shape, np.float32)
    for x in range(shape[0]):
        for y in range(shape[1]):
            for z in range(shape[2]):
                X, Y, Z = x // 2, y // 2, z // 2
                if mc[X, Y, Z]:
                    s = 0.0
                    for i in range(q):
                        s += float(g[i, X, Y, Z])
                    ref[x, y, z] = np.float32(s)
                else:
                    ref[x, y, z] = np.float32(0.9 + (0.1 - 0.9) * (x + 0.5) / shape[0])
    assert np.array_equal(got, ref)
    # departure from C_lin, plus a strided correction
    corr = S.random_field((int(np.prod(shape)), 2), seed + 2, -0.05, 0.05).astype(np.float32)
    om.om_prolong2_dev(_dev(g), q, _dev(mc), dom, 0.9, 0.1, out, corr_dev=_dev(corr), corr_stride=2, departure=True)
    # the FP64 value of the same steps, rounded once
    exact = np.zeros(shape)
    for xx in range(shape[0]):
        for y in range(shape[1]):
            for z in range(shape[2]):
                X, Y, Z = xx // 2, y // 2, z // 2
                cl = 0.9 + (0.1 - 0.9) * (xx + 0.5) / shape[0]
                if mc[X, Y, Z]:
                    s = 0.0
                    for i in range(q):
                        s += float(g[i, X, Y, Z])
                    v = s - cl
                else:
                    v = cl - cl
                v += float(corr[(xx * shape[1] + y) * shape[2] + z, 0])
                exact[xx, y, z] = v
    assert np.array_equal(out.cpu().numpy().reshape(shape), exact.astype(np.float32))


@pytest.mark.timeout(600)
def test_two_level_warm_start_keeps_result_and_saves_steps(om):
    from paper_1410_1921_gb300 import warmstart as W
    cfg = S.sweep_structure(0.35, edge=64)
    dom, mask, tr, d = W.structure(cfg)
    dp = om.diff_params(precision=om.OM_F32, conv_tol=1e-5, check_every=1000, max_steps=2_000_000)
    ns = om.NodeSet(tr, dom)
    st0, D0, info0 = om.Diffusion(ns, d, dp).solve()
    # coarse level: coarsen, keep the transport set, solve, carry the concentration back
    dc, mc, d_c = om.om_coarsen2_dev(tr, dom, d)
    tr_c = torch.empty_like(mc)
    om.om_label_connectivity_dev(mc, dc, None, tr_c)
    ns_c = om.NodeSet(tr_c, dc)
    dfc = om.Diffusion(ns_c, d_c, dp)
    st_c, _, info_c = dfc.solve()
    nc = dc.nx * dc.ny * dc.nz
    g_c = torch.empty(7 * nc, dtype=torch.float64, device="cuda")
    dfc.get_populations(g_c)
    c = torch.empty(dom.nx * dom.ny * dom.nz, dtype=torch.float32, device="cuda")
    om.om_prolong2_dev(g_c, 7, tr_c, dom, dp.c_in, dp.c_out, c)
    df = om.Diffusion(ns, d, dp)
    df.init_concentration(c)
    st1, D1, info1 = df.solve()
    print(f"cold {info0.steps} steps, coarse {info_c.steps} steps on {ns_c.n_nodes} nodes, warm {info1.steps} steps")
    assert st0 == st1 == st_c == om.OM_OK
    assert D1 == pytest.approx(D0, rel=2e-3)  # both stop on the same test, from different sides
    assert info1.steps < 0.8 * info0.steps  # measured 92k against 134k


@pytest.mark.timeout(600)
def test_two_level_flow_warm_start_keeps_result(om):
    # the coarse flow with 4x the body force has about the fine lattice's
    # velocities (k scales with the square of the lattice spacing); its u_x
    # carried to the fine nodes starts the fine solve, which iterates to the
    # same test and the same permeability
    from paper_1410_1921_gb300 import warmstart as W
    cfg = S.sweep_structure(0.35, edge=64)
    dom, mask, tr, d = W.structure(cfg)
    g = 1e-6
    fp = om.flow_params(body_force=g, precision=om.OM_F32, conv_tol=1e-5, check_every=1000, max_steps=1_000_000)
    ns = om.NodeSet(tr, dom)
    st0, k0, info0 = om.Flow(ns, fp).solve()
    dc, tr_c, _ = W.coarse_level(dom, tr, d)
    ns_c = om.NodeSet(tr_c, dc)
    flc = om.Flow(ns_c, om.flow_params(body_force=4 * g, precision=om.OM_F32, conv_tol=1e-4, check_every=1000,
                                       max_steps=1_000_000))
    st_c, _, info_c = flc.solve()
    nc = dc.nx * dc.ny * dc.nz
    f_c = torch.empty(19 * nc, dtype=torch.float64, device="cuda")
    flc.get_populations(f_c)
    u = torch.empty(dom.nx * dom.ny * dom.nz, dtype=torch.float32, device="cuda")
    om.om_prolong2_ux_dev(f_c, tr_c, dom, 4 * g, 1.0, u)
    fl = om.Flow(ns, fp)
    fl.init_velocity(u)
    st1, k1, info1 = fl.solve()
    print(f"flow cold {info0.steps} steps, coarse {info_c.steps}, warm {info1.steps}; k {k0:.6e} {k1:.6e}")
    assert st0 == st1 == st_c == om.OM_OK
    assert k1 == pytest.approx(k0, rel=2e-3)
