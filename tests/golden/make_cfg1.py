"""Write cfg1.json: the 48^3 workload (2 nm voxels, porosity 0.40, overlap
tolerance 0.5, d ~ Normal(20, 5) nm clipped to [6, 40]) solved to
convergence by the FP64 oracle, seeds 1..5.

Per structure: reconstruction (Sec. 2), transport nodes (Sec. 4.1), the
maximal-inscribed-sphere pore size, the D3Q19 body-force flow (Sec. 3.1,
tau = 1, g = 1e-6 along x) and the D3Q7 Knudsen diffusion (Sec. 3.2,
Eq. 12 with d_ref = 60 nm, tau_ref = 1; T = 300 K, methane; C = 1 / 0 at
the x ends), both run until the relative change over 100 steps is below
1e-6; then k (Eqs. 13, 15), D_eff (Eqs. 14, 15) and tortuosity (Eq. 16).

Calls only the oracle (plus the workload parameters of synthetic.py).
Usage:  python tests/golden/make_cfg1.py   (about ten minutes on 5 cores)
"""
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SEEDS = (1, 2, 3, 4, 5)
TAU, G, TOL, K = 1.0, 1e-6, 1e-6, 100
T_K, M, D_REF_NM, TAU_REF = 300.0, 0.016, 60.0, 1.0


def solve_one(seed):
    import numpy as np

    import oracle
    from oracle import physics as PH
    import synthetic as S

    cfg = S.small_structure(seed)
    t0 = time.time()
    rc, mask, sph, eps, _ = oracle.reconstruct(cfg.seed, cfg.shape, cfg.dx_nm, cfg.mean_nm, cfg.sd_nm,
                                               cfg.dmin_nm, cfg.dmax_nm, cfg.porosity, cfg.xi, cfg.p0,
                                               cfg.dist, cfg.max_trials)
    assert rc == 0
    _, tr, conn = oracle.label18(mask)
    rc, d, _ = oracle.mis(mask, cfg.dx_nm)
    assert rc == 0
    dx = cfg.dx_nm * 1e-9
    frc, kL, _, fsteps, frel, _ = oracle.flow_solve(tr, tau=TAU, g=G, tol=TOL, K=K, max_steps=2_000_000)
    omega = oracle.omega_field(tr, d, D_REF_NM, TAU_REF)
    drc, DL, _, dsteps, drel, _, _ = oracle.diff_solve(tr, omega, 1.0, 0.0, tol=TOL, K=K, max_steps=5_000_000)
    D_eff = PH.diffusivity_physical(DL, D_REF_NM * 1e-9, T_K, M, 7, TAU_REF)
    return {
        "seed": seed,
        "mask_sha256": hashlib.sha256(np.ascontiguousarray(mask, np.uint8).tobytes()).hexdigest(),
        "porosity": eps,
        "n_spheres": int(sph.shape[0]),
        "n_pore": int(mask.sum()),
        "n_transport": int(tr.sum()),
        "connectivity": conn,
        "flow": {"status": frc, "k_lattice": kL, "k_m2": PH.permeability_physical(kL, dx), "steps": fsteps,
                 "rel_change": frel},
        "diffusion": {"status": drc, "D_eff_lattice": DL, "D_eff_m2s": D_eff,
                      "tortuosity": oracle.tortuosity_eq16(mask, tr, d, D_eff, T_K, M), "steps": dsteps,
                      "rel_change": drel},
        "oracle_seconds": time.time() - t0,
    }


def main():
    with mp.get_context("spawn").Pool(len(SEEDS)) as pool:
        rows = pool.map(solve_one, SEEDS)
    out = {
        "_source": "written by tests/golden/make_cfg1.py from the FP64 oracle alone",
        "workload": "48^3 at 2 nm, porosity 0.40, overlap tolerance 0.5, d ~ N(20, 5) nm in [6, 40], "
                    "maximal inscribed sphere pore size",
        "flow": {"tau": TAU, "body_force": G, "conv_tol": TOL, "check_every": K},
        "diffusion": {"lattice": 7, "T_K": T_K, "M_kg_per_mol": M, "d_ref_nm": D_REF_NM, "tau_ref": TAU_REF,
                      "c_in": 1.0, "c_out": 0.0, "conv_tol": TOL, "check_every": K},
        "structures": rows,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cfg1.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps([(r["seed"], r["flow"]["steps"], r["diffusion"]["steps"], round(r["oracle_seconds"]))
                      for r in rows]))


if __name__ == "__main__":
    main()
