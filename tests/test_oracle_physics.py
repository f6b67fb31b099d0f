"""Oracle pins for the scalar formulas: Eq. 11 against the value printed in
Sec. 4.2, Eq. 28 as the closed form of Eqs. 11, 26, 27 and 29 for a
cylinder, the operating point of Sec. 4.4.3, and Eq. 12 limits."""
import json
import math
import os

import pytest

from oracle import physics as P

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_knudsen_reference_printed_value():
    g = GOLD["knudsen_reference"]
    D = P.knudsen_diffusivity(g["d_nm"] * 1e-9, g["T_K"], g["M_kg_per_mol"])
    assert float(f"{D:.{g['digits']}g}") == g["D_K_m2_per_s"]


def test_operating_point_pressure():
    g = GOLD["operating_point"]
    psi = 6894.757293168361  # Pa per psi (NIST)
    assert g["p_psi"] * psi == pytest.approx(g["p_Pa"], rel=1e-7)


@pytest.mark.parametrize("d_nm", [2.0, 10.0, 30.0, 60.0, 200.0])
def test_cylinder_correction_eq28(d_nm):
    """Eq. 26 with k_d of Eq. 27 and D_eff = D_K of Eq. 11 equals Eq. 28 with
    Kn = lambda / r, lambda by Eq. 29 (r = d/2)."""
    g = GOLD["operating_point"]
    T, M, mu, p = g["T_K"], 0.016, g["mu_Pa_s"], g["p_Pa"]
    d = d_nm * 1e-9
    ka, fc = P.apparent_permeability(P.cylinder_permeability(d), P.knudsen_diffusivity(d, T, M), mu, p)
    Kn = P.mean_free_path(mu, p, T, M) / (d / 2)
    assert fc == pytest.approx(P.cylinder_fc(Kn), rel=1e-12)
    assert ka == pytest.approx(P.cylinder_permeability(d) * fc, rel=1e-15)


def test_tau_knudsen_eq12_limits():
    assert P.tau_knudsen(60.0) == 1.0
    assert P.tau_knudsen(0.0) == 0.5
    # lattice diffusivity proportional to the pore size (Eqs. 11-12)
    assert P.d3q7_lattice_diffusivity(P.tau_knudsen(30.0)) == pytest.approx(
        0.5 * P.d3q7_lattice_diffusivity(P.tau_knudsen(60.0)))


def test_unit_conversion_round_trip():
    # D_L,ref maps to D_K(d_ref) on either lattice: Eq. 15 with the time step
    # fixed by Eq. 12
    T, M = 300.0, 0.016
    for q in (7, 19):
        D = P.diffusivity_physical(P.lattice_diffusivity(1.0, q), 60e-9, T, M, q)
        assert D == pytest.approx(P.knudsen_diffusivity(60e-9, T, M), rel=1e-15)
    # c_s^2 of the two lattices: D3Q7 with rest weight 1/4, the D3Q19 weights
    # printed below Eq. 3 (sum of w_i e_ix^2)
    w = GOLD["weights_d3q19"]
    assert P.lattice_cs2(19) == pytest.approx(2 * w["axis"] + 8 * w["diagonal"], rel=1e-15)
    assert P.lattice_cs2(7) == 2 * 0.125
    with pytest.raises(ValueError):
        P.lattice_cs2(15)
    assert P.permeability_physical(2.0, 1.5e-9) == pytest.approx(2.0 * 2.25e-18)


def test_kozeny_carman_and_bruggeman():
    assert P.kozeny_carman(1.0, 0.5) == pytest.approx(1 / 180 * 0.125 / 0.25)
    assert P.bruggeman_alpha(0.4 ** 1.5, 1.0, 0.4) == pytest.approx(1.5)
    assert P.tortuosity(0.4, 1.0, 0.4 / 2.0) == pytest.approx(2.0)
    # Bruggeman's own law (alpha = 1.5, Sec. 4.2) is recovered exactly from
    # structures that obey it, whatever their D; a second exponent from a
    # set generated with it
    eps = [0.15, 0.3, 0.55]
    assert P.bruggeman_fit(eps, [2.0 * e ** 1.5 for e in eps], [2.0] * 3) == pytest.approx(1.5, rel=1e-13)
    Dm = [1e-6, 3e-6, 7e-7]
    assert P.bruggeman_fit(eps, [d * e ** 3.3 for d, e in zip(Dm, eps)], Dm) == pytest.approx(3.3, rel=1e-13)
    # a least-squares line: scatter about the law averages out symmetrically
    De = [2.0 * e ** 2.0 * f for e, f in zip(eps, (1.1, 1.0, 1.0))]
    a = P.bruggeman_fit(eps, De, [2.0] * 3)
    x = [math.log(e) for e in eps]
    y = [math.log(d / 2.0) for d in De]
    assert a == pytest.approx(sum(u * v for u, v in zip(x, y)) / sum(u * u for u in x), rel=1e-13)


# ------------------------------------------------------------------ slip corrections (Sec. 4.4)
def test_knudsen_corrections_agree_at_low_kn_and_part_above():
    # Sec. 4.4.3 / Fig. 10: in the Darcy regime (Kn < 0.01) the Klinkenberg,
    # Beskok-Karniadakis-Civan and cylinder (Eq. 28) corrections nearly
    # coincide; as Kn grows Klinkenberg falls away and Eq. 28 stays with
    # Beskok-Karniadakis-Civan
    for Kn in (1e-4, 1e-3, 1e-2):
        k, bk, cyl = P.klinkenberg_fc(Kn), P.beskok_civan_fc(Kn), P.cylinder_fc(Kn)
        assert abs(k - 1) < 0.05 and abs(bk - 1) < 0.05 and abs(cyl - 1) < 0.1
        assert bk == pytest.approx(k, rel=2 * Kn)
    prev = 1.0
    for Kn in (1.0, 3.0, 10.0):
        k, bk, cyl = P.klinkenberg_fc(Kn), P.beskok_civan_fc(Kn), P.cylinder_fc(Kn)
        assert abs(cyl - bk) < abs(k - bk) and abs(cyl - bk) < 0.25 * bk
        assert bk / k > prev  # Klinkenberg falls further behind as Kn grows
        prev = bk / k


def test_civan_alpha_limits():
    # Eq. 21: alpha -> 0 as Kn -> 0 (no rarefaction) and -> 1.358 as Kn -> inf
    assert P.civan_alpha(1e-12) < 1e-4
    assert P.civan_alpha(1e12) == pytest.approx(1.358, rel=1e-5)
    # Eq. 20 with b = -1 reduces to 1 + 4 Kn / (1 + Kn) when alpha is dropped
    assert P.beskok_civan_fc(1e-12) == pytest.approx(1.0, abs=1e-11)


def test_table1_units_and_limits():
    # Table 1 works in psi and mD: 1 mD, porosity 1, P = b_k psi gives f_c = 2
    k = P.M2_PER_MILLIDARCY
    for name, bk in (("heid", 11.419), ("jones_owens", 12.639), ("sampath_keighin", 13.85), ("florence", 32.766)):
        assert P.table1_bk_psi(name, 1.0, 1.0) == pytest.approx(bk)
        assert P.table1_fc(name, k, 1.0, bk * P.PA_PER_PSI) == pytest.approx(2.0)
    # the porosity forms depend on k / eps only
    assert P.table1_bk_psi("florence", 0.2, 0.2) == pytest.approx(32.766)
    # tighter rock slips more
    assert P.table1_fc("heid", 1e-21, 0.3, 1e7) > P.table1_fc("heid", 1e-18, 0.3, 1e7)


def test_eq30_characteristic_pore_size_is_the_capillary_bundle_radius():
    # a bundle of capillaries of radius r at porosity eps has k = eps r^2 / 8,
    # i.e. r = sqrt(8 k / eps): Eq. 30's constant is that relation with k in
    # mD and r in micrometres (the unit that fixes the reading of Eq. 30)
    for k, eps in ((1e-21, 0.1), (1e-19, 0.3), (1e-17, 0.5)):
        assert P.characteristic_pore_size(k, eps) == pytest.approx(math.sqrt(8 * k / eps), rel=1e-3)
