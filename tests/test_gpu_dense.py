"""The dense population layout (om_flow_params.layout / om_diff_params.layout
= OM_LAYOUT_DENSE) through the host-buffer C ABI.

Every voxel of the box is stored and a node's neighbours follow by address
arithmetic and the node mask; each node's update is the sparse sweeps' own,
so the layouts must agree bit for bit on every field after the same steps:
the results of a solve differ only by the rounding order of the FP64
observable sums (checked at 1e-12, with equal step counts).  Against the
oracle: the 48^3 workload's stored converged values (tests/golden/cfg1.json,
oracle only) at 1e-10 in FP64 and 1e-5 in FP32, as the sparse layout."""
import json
import os

import numpy as np
import pytest

import synthetic as S
from conftest import recon_params

pytestmark = pytest.mark.gpu


def _porous(om, seed, shape=(36, 24, 28), p=0.85):
    mask = S.random_mask(shape, p, seed)
    dom = om.domain(shape, 2.0)
    d, _ = om.om_local_pore_diameter(mask, dom, om.OM_PORE_CHORD13)
    return dom, mask, d


def _solve_both(om, dom, mask, d, prec, layout, accel=0):
    fp = om.flow_params(conv_tol=1e-6, check_every=100, max_steps=400_000, precision=prec, layout=layout)
    f = om.om_solve_permeability(mask, dom, fp, want_ux=True)
    dp = om.diff_params(conv_tol=1e-6, check_every=100, max_steps=1_000_000, precision=prec, layout=layout,
                        accel=accel)
    g = om.om_solve_knudsen(mask, d, dom, dp, want_c=True)
    return f, g


@pytest.mark.timeout(600)
@pytest.mark.parametrize("prec", ["OM_F64", "OM_F32"])
@pytest.mark.parametrize("seed", [3, 8])
def test_dense_layout_equals_sparse(om, prec, seed):
    dom, mask, d = _porous(om, seed)
    P = getattr(om, prec)
    for accel in (0, 1):
        (fs, gs), (fd, gd) = (_solve_both(om, dom, mask, d, P, om.OM_LAYOUT_SPARSE, accel),
                              _solve_both(om, dom, mask, d, P, om.OM_LAYOUT_DENSE, accel))
        assert fs[0] == fd[0] == om.OM_OK and gs[0] == gd[0] == om.OM_OK
        assert fd[2] == pytest.approx(fs[2], rel=1e-12) and fd[3].steps == fs[3].steps
        assert gd[1] == pytest.approx(gs[1], rel=1e-12) and gd[2] == pytest.approx(gs[2], rel=1e-12)
        assert gd[3].steps == gs[3].steps and gd[3].n_nodes == gs[3].n_nodes
        assert np.array_equal(fd[4], fs[4])  # u_x, every voxel
        assert np.array_equal(gd[4], gs[4])  # C, every voxel


@pytest.mark.timeout(600)
def test_auto_layout_gives_the_same_results(om):
    # OM_LAYOUT_AUTO times both layouts where the nodes fill half the box or
    # more and solves in the faster one: the results are those of either
    dom, mask, d = _porous(om, 5, shape=(40, 32, 32), p=0.9)
    (fs, gs), (fa, ga) = (_solve_both(om, dom, mask, d, om.OM_F32, om.OM_LAYOUT_SPARSE),
                          _solve_both(om, dom, mask, d, om.OM_F32, om.OM_LAYOUT_AUTO))
    assert fa[2] == pytest.approx(fs[2], rel=1e-12) and fa[3].steps == fs[3].steps
    assert ga[1] == pytest.approx(gs[1], rel=1e-12) and ga[3].steps == gs[3].steps
    assert np.array_equal(fa[4], fs[4]) and np.array_equal(ga[4], gs[4])


@pytest.mark.timeout(900)
@pytest.mark.parametrize("seed", [1, 4])
def test_dense_layout_cfg1_against_oracle(om, seed):
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "cfg1.json")))
    row = {r["seed"]: r for r in gold["structures"]}[seed]
    fg, dg = gold["flow"], gold["diffusion"]
    cfg = S.small_structure(seed)
    dom = om.domain(cfg.shape, cfg.dx_nm)
    st, mask, eps, nsph = om.om_reconstruct(cfg.seed, dom, recon_params(om, cfg))
    d, _ = om.om_local_pore_diameter(mask, dom, om.OM_PORE_MIS)
    for prec, rel in ((om.OM_F64, 1e-10), (om.OM_F32, 1e-5)):
        fp = om.flow_params(tau=fg["tau"], body_force=fg["body_force"], conv_tol=fg["conv_tol"],
                            check_every=fg["check_every"], max_steps=2_000_000, precision=prec,
                            layout=om.OM_LAYOUT_DENSE)
        st, k, kl, info, _ = om.om_solve_permeability(mask, dom, fp)
        assert st == om.OM_OK
        assert kl == pytest.approx(row["flow"]["k_lattice"], rel=rel)
        if prec == om.OM_F64:
            assert info.steps == row["flow"]["steps"]
        dp = om.diff_params(T_K=dg["T_K"], M_kg_per_mol=dg["M_kg_per_mol"], d_ref_nm=dg["d_ref_nm"],
                            tau_ref=dg["tau_ref"], c_in=dg["c_in"], c_out=dg["c_out"], conv_tol=dg["conv_tol"],
                            check_every=dg["check_every"], max_steps=5_000_000, precision=prec,
                            layout=om.OM_LAYOUT_DENSE)
        st, D, tau, info, _ = om.om_solve_knudsen(mask, d, dom, dp)
        assert st == om.OM_OK
        assert D == pytest.approx(row["diffusion"]["D_eff_m2s"], rel=rel)
        assert tau == pytest.approx(row["diffusion"]["tortuosity"], rel=rel)
        if prec == om.OM_F64:
            assert info.steps == row["diffusion"]["steps"]


def test_dense_layout_rejections(om):
    dom, mask, d = _porous(om, 2, shape=(12, 10, 10))
    with pytest.raises(om.OmError):  # 16-bit storage is sparse only
        om.om_solve_permeability(mask, dom, om.flow_params(precision=om.OM_F16DEV, layout=om.OM_LAYOUT_DENSE))
    with pytest.raises(om.OmError):  # the paper's D3Q19 diffusion is sparse only
        om.om_solve_knudsen(mask, d, dom, om.diff_params(lattice=19, layout=om.OM_LAYOUT_DENSE))
    with pytest.raises(om.OmError):  # solver objects use the node set's layout
        import torch
        ns = om.NodeSet(torch.from_numpy(mask.reshape(-1)).cuda(), dom)
        try:
            om.Flow(ns, om.flow_params(layout=om.OM_LAYOUT_DENSE))
        finally:
            ns.close()
