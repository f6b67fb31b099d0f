"""The paper's structure campaign (Secs. 2, 4.1-4.4) on the library.

Orchestration only: every step runs in the library's kernels.  For a list
of reconstructions (synthetic.campaign_structures draws the paper's grid) it
reconstructs, labels and sizes each structure, solves the Knudsen diffusion
of all of them together on the batched path and the flow of each one (by
the paper's pressure ends, or batched with the body force), and derives per
structure: total porosity and connectivity (Sec. 4.1), k (Eqs. 13, 15),
D_eff (Eqs. 14, 15), tortuosity (Eq. 16), the Bruggeman exponent of
D_eff = D eps^alpha (Sec. 4.2, D the mean local Knudsen diffusivity over the
transport pores), the Kozeny-Carman estimate of Eq. 17 with the mean pore
diameter, and the apparent-permeability factors of Sec. 4.4.
"""
import math

import numpy as np
import torch

from . import (OM_DRIVE_FORCE, OM_DRIVE_PRESSURE, OM_ENOPERC, OM_OK, Batch, Flow, NodeSet, diff_params, flow_params,
               om_slip_correction_factors)
from . import warmstart as W

R_GAS = 8.314462618  # J / (mol K)


def knudsen_diffusivity(d_m, T_K, M):
    """Eq. 11."""
    return (d_m / 3.0) * math.sqrt(8.0 * R_GAS * T_K / (math.pi * M))


def bruggeman_alpha(D_eff, D_mean, porosity):
    """D_eff = D eps^alpha (Sec. 4.2) solved for alpha."""
    return math.log(D_eff / D_mean) / math.log(porosity)


def fit_bruggeman(rows):
    """Least-squares alpha over rows: ln(D_eff / D) = alpha ln(eps), no
    intercept."""
    x = np.array([math.log(r["porosity"]) for r in rows])
    y = np.array([math.log(r["D_eff_m2s"] / r["D_mean_m2s"]) for r in rows])
    return float((x * y).sum() / (x * x).sum())


def kozeny_carman(d_m, porosity):
    """Eq. 17 with A = d^2 / 180."""
    return (d_m * d_m / 180.0) * porosity ** 3 / (1.0 - porosity) ** 2


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
    cs2 = 1.0 / 3.0 if dp.lattice == 19 else 0.25
    DK_ref = knudsen_diffusivity(dp.d_ref_nm * 1e-9, dp.T_K, dp.M_kg_per_mol)
    to_phys = DK_ref / (cs2 * (dp.tau_ref - 0.5))  # Eq. 15 with the time step of Eqs. 11-12
    for j, (row, dom, tr, d) in enumerate(items):
        if drive == OM_DRIVE_FORCE:
            k_l, st_k = kl[j], int(st_f[j])
        else:
            ns = NodeSet(tr, dom)
            fl = Flow(ns, fp)
            st_k, k_l, _ = fl.solve()
            fl.close()
            ns.close()
        dx = row["dx_nm"] * 1e-9
        eps = row["porosity"]
        row.update(flow_status=st_k, diff_status=int(st_d[j]), k_m2=k_l * dx * dx,
                   D_eff_m2s=dl[j] * to_phys, D_mean_m2s=dmean[j] * to_phys,
                   tortuosity=eps * dmean[j] / dl[j] if dl[j] > 0 else float("inf"),
                   k_kc_m2=kozeny_carman(row["mean_d_nm"] * 1e-9, eps))
        row["alpha"] = bruggeman_alpha(row["D_eff_m2s"], row["D_mean_m2s"], eps) if dl[j] > 0 else float("nan")
        if row["k_m2"] > 0 and st_k in (OM_OK,):
            row["corrections"] = om_slip_correction_factors(row["k_m2"], eps, row["D_eff_m2s"], T_op,
                                                            dp.M_kg_per_mol, mu, p)
        if log:
            log(f"{row['seed']}: eps {eps:.3f} conn {row['connectivity']:.3f} k {row['k_m2']:.3e} m2 "
                f"D_eff {row['D_eff_m2s']:.3e} m2/s tau {row['tortuosity']:.2f} alpha {row['alpha']:.2f}")
    return rows
