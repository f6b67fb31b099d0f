"""The paper's structure campaign (Secs. 2, 4.1-4.4): the structure grid, the
results-in-physical-units entry points against the oracle's formulas, and a
campaign sub-grid solved on the GPU against the FP64 oracle's converged
values (tests/golden/campaign_small.json, written by make_campaign.py)."""
import json
import math
import os

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


@pytest.fixture(scope="module")
def lib():
    """The library's host entry points (they run on the CPU, no device)."""
    from paper_1410_1921_gb300 import build
    build.build()
    import paper_1410_1921_gb300 as P
    P.lib()
    return P


@pytest.mark.parametrize("lattice", [7, 19])
def test_structure_results_match_the_oracle_formulas(lib, lattice):
    from oracle import physics as PH
    P = lib
    dp = P.diff_params(T_K=323.0, lattice=lattice)
    DL, DLm, kL, eps, dx, dmean = 0.0123, 0.0311, 0.0456, 0.37, 1.5, 45.0
    r = P.om_structure_results_from_lattice(dx, kL, DL, DLm, eps, dmean, dp)
    D = PH.diffusivity_physical(DL, 60e-9, 323.0, 0.016, lattice)
    Dm = PH.diffusivity_physical(DLm, 60e-9, 323.0, 0.016, lattice)
    assert r["k_m2"] == pytest.approx(PH.permeability_physical(kL, dx * 1e-9), rel=1e-15)
    assert r["D_eff_m2s"] == pytest.approx(D, rel=1e-14)
    assert r["D_mean_m2s"] == pytest.approx(Dm, rel=1e-14)
    assert r["tortuosity"] == pytest.approx(PH.tortuosity(eps, Dm, D), rel=1e-14)
    assert r["alpha"] == pytest.approx(PH.bruggeman_alpha(D, Dm, eps), rel=1e-13)
    assert r["k_kc_m2"] == pytest.approx(PH.kozeny_carman(dmean * 1e-9, eps), rel=1e-14)
    with pytest.raises(P.OmError):
        P.om_structure_results_from_lattice(dx, kL, DL, DLm, 1.0, dmean, dp)


def test_bruggeman_fit_matches_the_oracle(lib):
    from oracle import physics as PH
    eps = [0.12, 0.3, 0.45, 0.51]
    Dm = [1e-6, 3e-6, 7e-7, 2e-6]
    De = [d * e ** a for d, e, a in zip(Dm, eps, (3.1, 2.7, 3.6, 2.9))]
    assert lib.om_bruggeman_fit(eps, De, Dm) == pytest.approx(PH.bruggeman_fit(eps, De, Dm), rel=1e-14)
    with pytest.raises(lib.OmError):
        lib.om_bruggeman_fit([0.3], [1e-7], [0.0])


@pytest.mark.gpu
@pytest.mark.timeout(600)
def test_campaign_subgrid_matches_the_oracle(om):
    # the campaign driver (batched diffusion, pressure-driven flow per
    # structure, FP32) on the oracle's sub-grid: porosity and connectivity
    # exactly; k, D_eff, D, tortuosity, Kozeny-Carman k within the FP32
    # bound 1e-5 relative, alpha and the fitted alpha within 1e-5 absolute
    from paper_1410_1921_gb300 import campaign as CP
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "campaign_small.json")))
    g = gold["grid"]
    cfgs = [c for c in S.campaign_structures(means=(g["mean_d_nm"],), porosities=tuple(g["porosities"]),
                                             xis=(g["xi"],), seeds=3, edge=g["edge"])
            if c.seed in {r["seed"] for r in gold["structures"]}]
    fg, dg = gold["flow"], gold["diffusion"]
    fp = om.flow_params(tau=fg["tau"], conv_tol=fg["conv_tol"], check_every=fg["check_every"], max_steps=2_000_000,
                        drive=om.OM_DRIVE_PRESSURE, delta_rho=fg["delta_rho"])
    dp = om.diff_params(T_K=dg["T_K"], M_kg_per_mol=dg["M_kg_per_mol"], conv_tol=dg["conv_tol"],
                        check_every=dg["check_every"], max_steps=3_000_000)
    rows = {r["seed"]: r for r in CP.run(cfgs, fp, dp)}
    solved = []
    for want in gold["structures"]:
        got = rows[want["seed"]]
        assert got["porosity"] == want["porosity"]
        assert got["connectivity"] == want["connectivity"]
        if "k_m2" not in want:
            assert "k_m2" not in got  # nothing percolates
            continue
        assert got["flow_status"] == om.OM_OK and got["diff_status"] == om.OM_OK
        for key in ("k_m2", "D_eff_m2s", "D_mean_m2s", "tortuosity", "k_kc_m2"):
            assert got[key] == pytest.approx(want[key], rel=1e-5), key
        assert got["alpha"] == pytest.approx(want["alpha"], abs=1e-5)
        assert math.isfinite(got["alpha"]) and set(got["corrections"]) >= {"dgm", "klinkenberg", "beskok_civan"}
        solved.append(got)
    assert len(solved) >= 2
    assert CP.fit_bruggeman(solved) == pytest.approx(gold["bruggeman_alpha_fit"], abs=1e-5)
