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
    # D_L,ref maps to D_K(d_ref): Eq. 15 with the time step fixed by Eq. 12
    T, M = 300.0, 0.016
    D = P.diffusivity_physical(P.d3q7_lattice_diffusivity(1.0), 60e-9, T, M)
    assert D == pytest.approx(P.knudsen_diffusivity(60e-9, T, M), rel=1e-15)
    assert P.permeability_physical(2.0, 1.5e-9) == pytest.approx(2.0 * 2.25e-18)


def test_kozeny_carman_and_bruggeman():
    assert P.kozeny_carman(1.0, 0.5) == pytest.approx(1 / 180 * 0.125 / 0.25)
    assert P.bruggeman_alpha(0.4 ** 1.5, 1.0, 0.4) == pytest.approx(1.5)
    assert P.tortuosity(0.4, 1.0, 0.4 / 2.0) == pytest.approx(2.0)
