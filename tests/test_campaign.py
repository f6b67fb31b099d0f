"""The paper's structure campaign (Secs. 2, 4.1-4.4): the structure grid,
the Bruggeman and Kozeny-Carman fits, and a two-structure campaign on the
GPU checked against single-structure solves."""
import math

import numpy as np
import pytest

import synthetic as S


def test_campaign_grid_follows_sec2():
    cfgs = S.campaign_structures()
    # <d> in {30, 45, 60}, porosity 0.10 .. 0.55 by 0.05, xi in {0.1, 0.2, 0.3}, five seeds
    assert len(cfgs) == 3 * 10 * 3 * 5
    assert sorted({c.mean_nm for c in cfgs}) == [30.0, 45.0, 60.0]
    assert sorted({c.porosity for c in cfgs}) == [round(0.10 + 0.05 * k, 2) for k in range(10)]
    assert sorted({c.xi for c in cfgs}) == [0.1, 0.2, 0.3]
    assert all(c.dist == 1 and c.dmin_nm == c.mean_nm - 15 and c.dmax_nm == c.mean_nm + 15 for c in cfgs)
    assert all(c.shape == (200, 200, 200) and c.dx_nm == 1.5 for c in cfgs)
    assert len({c.seed for c in cfgs}) == len(cfgs)


def test_bruggeman_fit_recovers_the_exponent():
    from paper_1410_1921_gb300 import campaign as CP
    rows = [{"porosity": e, "D_mean_m2s": 2e-6, "D_eff_m2s": 2e-6 * e ** 3.3} for e in (0.2, 0.3, 0.45)]
    assert CP.fit_bruggeman(rows) == pytest.approx(3.3, rel=1e-12)
    assert CP.bruggeman_alpha(2e-6 * 0.3 ** 1.5, 2e-6, 0.3) == pytest.approx(1.5)
    # the product's formulas against the oracle's
    from oracle import physics as PH
    assert CP.kozeny_carman(45e-9, 0.3) == pytest.approx(PH.kozeny_carman(45e-9, 0.3), rel=1e-15)
    assert CP.knudsen_diffusivity(60e-9, 323.0, 0.016) == pytest.approx(PH.knudsen_diffusivity(60e-9, 323.0, 0.016),
                                                                        rel=1e-15)


@pytest.mark.gpu
@pytest.mark.timeout(600)
def test_small_campaign_matches_single_solves(om):
    import torch
    from paper_1410_1921_gb300 import campaign as CP
    from paper_1410_1921_gb300 import warmstart as W
    cfgs = S.campaign_structures(means=(30.0,), porosities=(0.40, 0.50), xis=(0.3,), seeds=1, edge=48)
    fp = om.flow_params(conv_tol=1e-6, check_every=200, max_steps=400_000, drive=om.OM_DRIVE_PRESSURE)
    dp = om.diff_params(conv_tol=1e-6, check_every=200, max_steps=400_000)
    rows = CP.run(cfgs, fp, dp)
    solved = [r for r in rows if "k_m2" in r]
    assert solved
    for r, cfg in zip(rows, cfgs):
        if "k_m2" not in r:
            continue
        assert r["flow_status"] == om.OM_OK and r["diff_status"] == om.OM_OK
        assert r["k_m2"] > 0 and r["D_eff_m2s"] > 0 and r["tortuosity"] > 0.5
        assert 0 < r["connectivity"] <= 1 and abs(r["porosity"] - cfg.porosity) < 0.02
        # the batched diffusion equals a single solve of the same structure
        dom, mask, tr, d = W.structure(cfg)
        ns = om.NodeSet(tr, dom)
        df = om.Diffusion(ns, d, dp)
        st, Dl, _ = df.solve()
        cs2 = 0.25
        DK = CP.knudsen_diffusivity(60e-9, dp.T_K, dp.M_kg_per_mol)
        assert st == om.OM_OK and r["D_eff_m2s"] == pytest.approx(Dl * DK / (cs2 * 0.5), rel=1e-6)
        assert math.isfinite(r["alpha"]) and r["alpha"] > 1.0
        assert set(r["corrections"]) >= {"dgm", "klinkenberg", "beskok_civan", "heid"}
