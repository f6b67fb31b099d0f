"""Write campaign_small.json: a sub-grid of the paper's campaign (Sec. 2:
diameters uniform in <d> +- 15 nm, here <d> = 30 nm, overlap tolerance
0.3, porosity 0.40 and 0.50) on 32^3 boxes of 1.5 nm, solved to convergence
by the FP64 oracle the way the campaign driver solves it: the flow driven by
the paper's pressure ends (Sec. 3.3, rho = 1 +- 5e-5, tau = 1), the D3Q7
Knudsen diffusion (Eq. 12, 13-direction pore size, T = 300 K, methane), both
until the relative change over 200 steps is below 1e-6; then per structure
porosity, connectivity (Sec. 4.1), k (Eqs. 13, 15), D_eff (Eqs. 14, 15), the
mean local Knudsen diffusivity D over the transport nodes, tortuosity
(Eq. 16), the Bruggeman exponent of that structure and the Kozeny-Carman
estimate (Eq. 17); and the Bruggeman exponent fitted over the set
(Sec. 4.2).

Calls only the oracle (plus the campaign grid of synthetic.py).
Usage:  python tests/golden/make_campaign.py   (a few minutes on 4 cores)
"""
import json
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

TOL, K, DRHO = 1e-6, 200, 1e-4
T_K, M = 300.0, 0.016


def configs():
    import synthetic as S
    return [c for c in S.campaign_structures(means=(30.0,), porosities=(0.40, 0.50), xis=(0.3,), seeds=3, edge=32)
            if c.seed in (100000, 100002, 100100, 100101)]


def solve_one(cfg):
    import numpy as np

    import oracle
    from oracle import physics as PH
    rc, mask, sph, eps, _ = oracle.reconstruct(cfg.seed, cfg.shape, cfg.dx_nm, cfg.mean_nm, cfg.sd_nm, cfg.dmin_nm,
                                               cfg.dmax_nm, cfg.porosity, cfg.xi, cfg.p0, cfg.dist, cfg.max_trials)
    assert rc == 0
    _, tr, conn = oracle.label18(mask)
    row = {"seed": cfg.seed, "porosity": eps, "connectivity": conn, "n_transport": int(tr.sum())}
    if tr.sum() == 0:
        return row
    d, _ = oracle.chord13(mask, cfg.dx_nm, counts=False)
    frc, kL, *_ = oracle.flow_solve_p(tr, tau=1.0, rho_in=1.0 + DRHO / 2, rho_out=1.0 - DRHO / 2, tol=TOL, K=K,
                                      max_steps=2_000_000)
    drc, DL, *_ = oracle.diff_solve(tr, oracle.omega_field(tr, d), 1.0, 0.0, tol=TOL, K=K, max_steps=3_000_000)
    dx = cfg.dx_nm * 1e-9
    D_eff = PH.diffusivity_physical(DL, 60e-9, T_K, M, 7)
    D_mean = PH.mean_knudsen_diffusivity(np.asarray(d, np.float64)[tr == 1], T_K, M)
    row.update(flow_status=frc, diff_status=drc, k_m2=PH.permeability_physical(kL, dx), D_eff_m2s=D_eff,
               D_mean_m2s=D_mean, tortuosity=oracle.tortuosity_eq16(mask, tr, d, D_eff, T_K, M),
               alpha=PH.bruggeman_alpha(D_eff, D_mean, eps), k_kc_m2=PH.kozeny_carman(cfg.mean_nm * 1e-9, eps))
    return row


def main():
    cfgs = configs()
    with mp.get_context("spawn").Pool(len(cfgs)) as pool:
        rows = pool.map(solve_one, cfgs)
    solved = [r for r in rows if "k_m2" in r]
    from oracle import physics as PH
    out = {"_source": "written by tests/golden/make_campaign.py from the FP64 oracle alone",
           "grid": {"mean_d_nm": 30.0, "xi": 0.3, "porosities": [0.40, 0.50], "edge": 32, "dx_nm": 1.5},
           "flow": {"drive": "pressure", "delta_rho": DRHO, "tau": 1.0, "conv_tol": TOL, "check_every": K},
           "diffusion": {"lattice": 7, "T_K": T_K, "M_kg_per_mol": M, "conv_tol": TOL, "check_every": K},
           "structures": rows,
           "bruggeman_alpha_fit": PH.bruggeman_fit([r["porosity"] for r in solved], [r["D_eff_m2s"] for r in solved],
                                                   [r["D_mean_m2s"] for r in solved])}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "campaign_small.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out)[:2000])


if __name__ == "__main__":
    main()
