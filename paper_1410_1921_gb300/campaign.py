"""The paper's structure campaign (Secs. 2, 4.1-4.4) on the library.

Orchestration only: every step, and every formula of the paper, runs in the
library (its kernels and its C entry points).  For a list of reconstructions
(synthetic.campaign_structures draws the paper's grid) it reconstructs,
labels and sizes each structure, solves the Knudsen diffusion of all of them
together on the batched path and the flow of each one (by the paper's
pressure ends, or batched with the body force), and takes per structure from
om_structure_results_from_lattice: total porosity and connectivity
(Sec. 4.1), k (Eqs. 13, 15), D_eff (Eqs. 14, 15), tortuosity (Eq. 16), the
Bruggeman exponent of D_eff = D eps^alpha (Sec. 4.2, D the mean local
Knudsen diffusivity over the transport pores), the Kozeny-Carman estimate of
Eq. 17 with the mean pore diameter, and the apparent-permeability factors of
Sec. 4.4; fit_bruggeman is om_bruggeman_fit over the solved structures.
"""
from . import (OM_DRIVE_FORCE, OM_DRIVE_PRESSURE, OM_OK, Batch, Flow, NodeSet, diff_params, flow_params,
               om_bruggeman_fit, om_slip_correction_factors, om_structure_results_from_lattice)
from . import warmstart as W


def fit_bruggeman(rows):
    """Sec. 4.2: alpha of D_eff = D eps^alpha over the solved rows (least
    squares through the origin in log space)."""
    rows = [r for r in rows if r.get("D_eff_m2s", 0) > 0]
    return om_bruggeman_fit([r["porosity"] for r in rows], [r["D_eff_m2s"] for r in rows],
                            [r["D_mean_m2s"] for r in rows])


def run(cfgs, fp=None, dp=None, drive=OM_DRIVE_PRESSURE, T_op=323.0, mu=1.73e-5, p=17236893.0, log=None):
    """Solve the campaign; returns one dict per structure.  fp, dp: flow and
    diffusion parameters (defaults: FP32, relative change 1e-6 per 100 steps);
    T_op, mu, p: the operating point of the apparent-permeability factors
    (Sec. 4.4.3: 323 K, 1.73e-5 Pa s, 2500 psi)."""
    fp = fp or flow_params(drive=drive)
    dp = dp or diff_params()
    if drive != fp.drive:
        fp.drive = drive
    items, rows = [], []
    for cfg in cfgs:
        dom, mask, tr, d = W.structure(cfg)
        npore, ntr = int(mask.sum().item()), int(tr.sum().item())
        row = {"seed": cfg.seed, "shape": cfg.shape, "dx_nm": cfg.dx_nm, "mean_d_nm": cfg.mean_nm, "xi": cfg.xi,
               "target_porosity": cfg.porosity, "porosity": npore / tr.numel(),
               "connectivity": ntr / npore if npore else 0.0}
        rows.append(row)
        if ntr:
            items.append((row, dom, tr, d))
    if not items:
        return rows
    # diffusion: all structures together on the batched path
    b = Batch([i[1] for i in items], [i[2] for i in items], [i[3] for i in items],
              flow=fp if drive == OM_DRIVE_FORCE else None, diff=dp)
    dl, dmean, info_d, st_d = b.solve(1)
    if drive == OM_DRIVE_FORCE:
        kl, _, info_f, st_f = b.solve(0)
    b.close()
    for j, (row, dom, tr, d) in enumerate(items):
        if drive == OM_DRIVE_FORCE:
            k_l, st_k = kl[j], int(st_f[j])
        else:
            ns = NodeSet(tr, dom)
            fl = Flow(ns, fp)
            st_k, k_l, _ = fl.solve()
            fl.close()
            ns.close()
        eps = row["porosity"]
        res = om_structure_results_from_lattice(row["dx_nm"], k_l, dl[j], dmean[j], eps, row["mean_d_nm"], dp)
        row.update(flow_status=st_k, diff_status=int(st_d[j]), **res)
        if row["k_m2"] > 0 and st_k in (OM_OK,):
            row["corrections"] = om_slip_correction_factors(row["k_m2"], eps, row["D_eff_m2s"], T_op,
                                                            dp.M_kg_per_mol, mu, p)
        if log:
            log(f"{row['seed']}: eps {eps:.3f} conn {row['connectivity']:.3f} k {row['k_m2']:.3e} m2 "
                f"D_eff {row['D_eff_m2s']:.3e} m2/s tau {row['tortuosity']:.2f} alpha {row['alpha']:.2f}")
    return rows


def main(argv=None):
    """Command line: solve a sub-grid of the campaign and write one JSON
    object (the rows, the fitted Bruggeman exponent, wall time).  Run from
    the repository root, where the synthetic input generator lives:
        python -m paper_1410_1921_gb300.campaign --means 45 --porosities 0.2,0.35,0.5 --seeds 2
    """
    import argparse
    import json
    import time

    import synthetic

    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--means", default="30,45,60", help="mean pore diameters <d> in nm")
    ap.add_argument("--porosities", default=",".join(f"{0.10 + 0.05 * k:.2f}" for k in range(10)))
    ap.add_argument("--xis", default="0.1,0.2,0.3", help="overlap tolerances")
    ap.add_argument("--seeds", type=int, default=5, help="structures per configuration")
    ap.add_argument("--edge", type=int, default=200, help="box edge in voxels (1.5 nm each)")
    ap.add_argument("--drive", choices=("pressure", "force"), default="pressure")
    ap.add_argument("--extrapolate", action="store_true", help="extrapolated restarts of the diffusion")
    ap.add_argument("--out", default=None, help="JSON file (default: stdout)")
    a = ap.parse_args(argv)
    fl = lambda s: tuple(float(v) for v in s.split(","))
    cfgs = synthetic.campaign_structures(means=fl(a.means), porosities=fl(a.porosities), xis=fl(a.xis),
                                         seeds=a.seeds, edge=a.edge)
    drive = OM_DRIVE_PRESSURE if a.drive == "pressure" else OM_DRIVE_FORCE
    dp = diff_params(accel=1 if a.extrapolate else 0)
    t0 = time.time()
    rows = run(cfgs, flow_params(drive=drive), dp, drive=drive,
               log=lambda m: print(f"[{time.time() - t0:7.1f} s] {m}", flush=True))
    solved = [r for r in rows if r.get("D_eff_m2s", 0) > 0 and r.get("flow_status") == OM_OK]
    out = {"structures": len(rows), "solved": len(solved), "wall_s": time.time() - t0, "edge": a.edge,
           "drive": a.drive, "extrapolate": a.extrapolate,
           "bruggeman_alpha_fit": fit_bruggeman(solved) if len(solved) >= 2 else None,
           "rows": [{k: (list(v) if isinstance(v, tuple) else v) for k, v in r.items()} for r in rows]}
    text = json.dumps(out, indent=1, default=float)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text)
    else:
        print(text)


if __name__ == "__main__":
    main()
