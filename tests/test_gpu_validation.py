"""The validation cases of Sec. 3.5 at the paper's resolution (100^3 lattice),
on the GPU path.

Diffusion: a cube holding a solid sphere whose diameter is the side
(porosity 1 - pi/6); the paper prints D_eff/D = 0.3317 for its D3Q19 model
at 100^3.  Both diffusion lattices land within 2 % of it here (the oracle
pins the same case at 40^3, 3-4 %).

Flow: one cell of a body-centred cubic array of spheres at porosity 0.915
(Fig. 3a), pressure-driven between the x faces and periodic in y, z as in
the paper, against the fully periodic body-force solve of the same cell:
the two drives give the same permeability within 5 %.  The paper reports
that Eq. 17 (Kozeny-Carman with A = d^2/180) lies above the simulated
permeability at high porosity; the test checks that ordering.  The analytic
curve of Fig. 3(b) is not printed in the text and is not used."""
import json
import os

import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to("cuda") if dtype is None else t.to("cuda", dtype)


@pytest.mark.timeout(600)
@pytest.mark.parametrize("q,cs2", [(7, 0.25), (19, 1.0 / 3.0)])
def test_sphere_in_cube_at_100(om, q, cs2):
    gold = json.load(open(os.path.join(GOLDEN, "paper_values.json")))["sphere_in_cube"]
    m = S.sphere_in_cube(100)
    ns = om.NodeSet(_dev(m), om.domain(m.shape))
    d = _dev(np.full(m.shape, 60.0, np.float32))  # d = d_ref: tau = tau_ref = 1 everywhere
    df = om.Diffusion(ns, d, om.diff_params(precision=om.OM_F32, conv_tol=1e-6, check_every=2000,
                                            max_steps=4_000_000, lattice=q))
    st, D, info = df.solve()
    assert st == om.OM_OK
    ratio = D / (cs2 * 0.5)
    print(f"D3Q{q} sphere in cube 100^3: D_eff/D = {ratio:.4f} ({info.steps} steps)")
    assert ratio == pytest.approx(gold["D_eff_over_D"], rel=0.02)


@pytest.mark.timeout(600)
def test_bcc_array_pressure_drive_matches_body_force(om):
    m, d = S.bcc_array(100, 0.915)
    eps = float(m.mean())
    ns = om.NodeSet(_dev(m), om.domain(m.shape))
    common = dict(tau=1.0, precision=om.OM_F32, conv_tol=1e-6, check_every=2000, max_steps=2_000_000)
    st_b, k_body, info_b = om.Flow(ns, om.flow_params(body_force=1e-6, **common)).solve()
    st_p, k_press, info_p = om.Flow(ns, om.flow_params(drive=om.OM_DRIVE_PRESSURE, delta_rho=1e-4,
                                                       **common)).solve()
    assert st_b == om.OM_OK and st_p == om.OM_OK
    k_kc = d * d / 180.0 * eps ** 3 / (1.0 - eps) ** 2  # Eq. 17, lattice units
    print(f"BCC eps {eps:.4f} d {d:.2f}: k body {k_body:.2f}, pressure {k_press:.2f}, KC {k_kc:.2f}")
    assert k_press == pytest.approx(k_body, rel=0.05)
    assert k_kc > k_body  # Sec. 3.5: Eq. 17 lies above the simulation at high porosity
