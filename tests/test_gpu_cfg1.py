"""The 48^3 workload end to end through the host-buffer C ABI, against the
FP64 oracle at convergence.

Five structures (48^3 at 2 nm, porosity 0.40, overlap tolerance 0.5,
d ~ Normal(20, 5) nm in [6, 40]; seeds 1..5): reconstruction (Sec. 2),
maximal-inscribed-sphere pore size, the D3Q19 body-force flow (tau = 1,
g = 1e-6) and the D3Q7 Knudsen diffusion (Eq. 12, T = 300 K, methane), both
to a relative change below 1e-6 over 100 steps, then k (Eqs. 13, 15), D_eff
(Eqs. 14, 15) and tortuosity (Eq. 16).  The expected values are in
tests/golden/cfg1.json, written by tests/golden/make_cfg1.py from the oracle
alone (the oracle takes minutes per structure, so its results are stored).

Bars: the mask is bit-exact (its SHA-256); FP64 results within 1e-10
relative with the same number of steps (the same iteration stopped by the
same test, the sums differing only in rounding order); FP32 storage within
1e-5 relative, the stated FP32 bound.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import synthetic as S
from conftest import recon_params

pytestmark = pytest.mark.gpu

SEEDS = (1, 2, 3, 4, 5)


def _gold():
    return json.load(open(os.path.join(os.path.dirname(__file__), "golden", "cfg1.json")))


def _structure(om, seed):
    cfg = S.small_structure(seed)
    dom = om.domain(cfg.shape, cfg.dx_nm)
    st, mask, eps, nsph = om.om_reconstruct(cfg.seed, dom, recon_params(om, cfg))
    assert st == om.OM_OK
    d, _ = om.om_local_pore_diameter(mask, dom, om.OM_PORE_MIS)
    return dom, mask, eps, nsph, d


@pytest.mark.timeout(900)
@pytest.mark.parametrize("seed", SEEDS)
def test_cfg1_converged_against_oracle(om, seed):
    gold = _gold()
    row = {r["seed"]: r for r in gold["structures"]}[seed]
    fg, dg = gold["flow"], gold["diffusion"]
    dom, mask, eps, nsph, d = _structure(om, seed)
    assert hashlib.sha256(np.ascontiguousarray(mask, np.uint8).tobytes()).hexdigest() == row["mask_sha256"]
    assert eps == row["porosity"] and nsph == row["n_spheres"]
    _, tr, conn = om.om_label_connectivity(mask)
    assert int(tr.sum()) == row["n_transport"] and conn == row["connectivity"]

    for prec, rel in ((om.OM_F64, 1e-10), (om.OM_F32, 1e-5)):
        fp = om.flow_params(tau=fg["tau"], body_force=fg["body_force"], conv_tol=fg["conv_tol"],
                            check_every=fg["check_every"], max_steps=2_000_000, precision=prec)
        st, k, kl, info, _ = om.om_solve_permeability(mask, dom, fp)
        assert st == om.OM_OK
        assert kl == pytest.approx(row["flow"]["k_lattice"], rel=rel)
        assert k == pytest.approx(row["flow"]["k_m2"], rel=rel)
        if prec == om.OM_F64:
            assert info.steps == row["flow"]["steps"]

        dp = om.diff_params(T_K=dg["T_K"], M_kg_per_mol=dg["M_kg_per_mol"], d_ref_nm=dg["d_ref_nm"],
                            tau_ref=dg["tau_ref"], c_in=dg["c_in"], c_out=dg["c_out"], conv_tol=dg["conv_tol"],
                            check_every=dg["check_every"], max_steps=5_000_000, precision=prec)
        st, D, tau, info, _ = om.om_solve_knudsen(mask, d, dom, dp)
        assert st == om.OM_OK
        assert D == pytest.approx(row["diffusion"]["D_eff_m2s"], rel=rel)
        assert tau == pytest.approx(row["diffusion"]["tortuosity"], rel=rel)
        if prec == om.OM_F64:
            assert info.steps == row["diffusion"]["steps"]


def test_tortuosity_averages_over_transport_nodes_gpu(om):
    # Eq. 16 on a layered channel with an isolated pocket of another pore
    # size: tortuosity = pore voxels / transport nodes exactly, and D_eff =
    # sum of the transport nodes' D_K / N (parallel conductors)
    from oracle import physics as PH
    from test_oracle_lbm import layered_slit_with_pocket
    m, d, tr = layered_slit_with_pocket()
    T, M = 300.0, 0.016
    dp = om.diff_params(T_K=T, M_kg_per_mol=M, conv_tol=1e-13, max_steps=2_000_000, precision=om.OM_F64)
    st, D, tau, info, _ = om.om_solve_knudsen(m, d.astype(np.float32), om.domain(m.shape, 1.0), dp)
    assert st == om.OM_OK
    DK = [PH.knudsen_diffusivity(float(v) * 1e-9, T, M) for v in d[tr == 1]]
    assert D == pytest.approx(sum(DK) / m.size, rel=1e-10)
    assert tau == pytest.approx(m.sum() / tr.sum(), rel=1e-10)
