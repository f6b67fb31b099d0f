"""Scalar formulas of arXiv:1410.1921, FP64, one function per equation.

Test infrastructure (part of the oracle).  SI units unless a name says
otherwise.
"""
import math

R_GAS = 8.314462618  # J / (mol K)


def knudsen_diffusivity(d_m, T_K, M_kg_per_mol):
    """Eq. 11: D_K = (d_p / 3) sqrt(8 R T / (pi M))."""
    return (d_m / 3.0) * math.sqrt(8.0 * R_GAS * T_K / (math.pi * M_kg_per_mol))


def tau_knudsen(d_nm, d_ref_nm=60.0, tau_ref=1.0):
    """Eq. 12: tau_g = (d_p / d_p,ref)(tau_g,ref - 1/2) + 1/2."""
    return (d_nm / d_ref_nm) * (tau_ref - 0.5) + 0.5


def lattice_cs2(q):
    """Squared lattice sound speed of the diffusion lattice: D3Q7 with rest
    weight 1/4 has c_s^2 = 1/4; the paper's D3Q19 (Sec. 3.2, the weights
    below Eq. 3) has c_s^2 = 1/3."""
    if q == 7:
        return 0.25
    if q == 19:
        return 1.0 / 3.0
    raise ValueError(f"no diffusion lattice D3Q{q}")


def lattice_diffusivity(tau, q):
    """BGK diffusion: D_L = c_s^2 (tau - 1/2) on D3Q7 or D3Q19."""
    return (tau - 0.5) * lattice_cs2(q)


def d3q7_lattice_diffusivity(tau):
    """BGK diffusion on D3Q7 with rest weight 1/4: c_s^2 = 1/4, D_L = (tau - 1/2)/4."""
    return lattice_diffusivity(tau, 7)


def d3q19_viscosity(tau):
    """Eq. 8 with c_s^2 = 1/3: nu = (tau - 1/2)/3 (lattice units)."""
    return (tau - 0.5) / 3.0


def permeability_physical(k_lattice, dx_m):
    """Eq. 15: k_P / l_P^2 = k_L / l_L^2 with one lattice length = dx."""
    return k_lattice * dx_m * dx_m


def diffusivity_physical(D_lattice, d_ref_m, T_K, M, q, tau_ref=1.0):
    """Eq. 15 with the time step fixed by the reference pore: D_L,ref of the
    lattice q maps to D_K(d_ref) (Eqs. 11-12), so D_P = D_L * D_K,ref / D_L,ref.
    The lattice must be named: D_L,ref = c_s^2 (tau_ref - 1/2) depends on it."""
    return D_lattice * knudsen_diffusivity(d_ref_m, T_K, M) / lattice_diffusivity(tau_ref, q)


def tortuosity(porosity, D_mean, D_eff):
    """Eq. 16: D_eff = D eps / tortuosity."""
    return porosity * D_mean / D_eff


def mean_knudsen_diffusivity(d_nm_values, T_K, M):
    """The D of Eq. 16 for a structure with local pore sizes: Eq. 11 applied
    node by node (d in nm) and averaged over the nodes given -- the transport
    nodes, the ones the diffusion runs on."""
    n = 0
    acc = 0.0
    for d in d_nm_values:
        acc += knudsen_diffusivity(float(d) * 1e-9, T_K, M)
        n += 1
    return acc / n


def bruggeman_alpha(D_eff, D_ref, porosity):
    """Sec. 4.2: D_eff = D eps^alpha  ->  alpha = ln(D_eff/D)/ln(eps)."""
    return math.log(D_eff / D_ref) / math.log(porosity)


def bruggeman_fit(porosities, D_effs, D_means):
    """Sec. 4.2: the exponent alpha of D_eff = D eps^alpha fitted over a set
    of structures by least squares on ln(D_eff / D) = alpha ln(eps) (a line
    through the origin)."""
    sxy = sxx = 0.0
    for e, De, Dm in zip(porosities, D_effs, D_means):
        x = math.log(e)
        sxy += x * math.log(De / Dm)
        sxx += x * x
    return sxy / sxx


def kozeny_carman(d_m, porosity):
    """Eq. 17 with A = d^2/180."""
    return (d_m * d_m / 180.0) * porosity ** 3 / (1.0 - porosity) ** 2


def apparent_permeability(k_d, D_eff, mu, p):
    """Eq. 26: k_a = k_d f_c, f_c = 1 + D_eff mu / (k_d p).  Returns (k_a, f_c)."""
    fc = 1.0 + D_eff * mu / (k_d * p)
    return k_d * fc, fc


def cylinder_permeability(d_m):
    """Eq. 27: k_d = (d_p/2)^2 / 8."""
    return (d_m / 2.0) ** 2 / 8.0


def mean_free_path(mu, p, T_K, M):
    """Eq. 29: lambda = (mu/p) sqrt(pi R T / (2 M))."""
    return (mu / p) * math.sqrt(math.pi * R_GAS * T_K / (2.0 * M))


def cylinder_fc(Kn):
    """Eq. 28: f_c = 1 + (64 / (3 pi)) Kn."""
    return 1.0 + 64.0 / (3.0 * math.pi) * Kn


# ------------------------------------------------------------------ slip corrections (Sec. 4.4.1, 4.4.3)
PA_PER_PSI = 6894.757293168361      # NIST
M2_PER_MILLIDARCY = 9.869233e-16    # 1 D = 9.869233e-13 m^2 (NIST)


def klinkenberg_fc(Kn):
    """Eqs. 18-19 with c = 1: f_c = 1 + b_k/P = 1 + 4 Kn."""
    return 1.0 + 4.0 * Kn


def civan_alpha(Kn):
    """Eq. 21: alpha(Kn) = 1.358 / (1 + 0.170 Kn^-0.4348)."""
    return 1.358 / (1.0 + 0.170 * Kn ** -0.4348)


def beskok_civan_fc(Kn, b=-1.0):
    """Eq. 20 with Eq. 21: f_c = (1 + alpha Kn)(1 + 4 Kn / (1 - b Kn)), b = -1 (slip flow)."""
    return (1.0 + civan_alpha(Kn) * Kn) * (1.0 + 4.0 * Kn / (1.0 - b * Kn))


def table1_bk_psi(name, k_md, porosity):
    """Table 1: Klinkenberg slippage factor b_k (psi) from k_d (mD) and porosity."""
    if name == "heid":
        return 11.419 * k_md ** -0.39
    if name == "jones_owens":
        return 12.639 * k_md ** -0.33
    if name == "sampath_keighin":
        return 13.85 * (k_md / porosity) ** -0.53
    if name == "florence":
        return 32.766 * (k_md / porosity) ** -0.5  # membrane beta
    raise ValueError(name)


def table1_fc(name, k_m2, porosity, p_Pa):
    """Eq. 18 with a Table 1 slippage factor: f_c = 1 + b_k / P (b_k, P in psi)."""
    return 1.0 + table1_bk_psi(name, k_m2 / M2_PER_MILLIDARCY, porosity) / (p_Pa / PA_PER_PSI)


def characteristic_pore_size(k_m2, porosity):
    """Eq. 30: r = 8.886e-2 (k / eps)^0.5 with k in mD, read with r in
    micrometres (the capillary-bundle radius sqrt(8 k / eps) in those units;
    the printed nm is off by 1000); returned in m."""
    return 8.886e-2 * (k_m2 / M2_PER_MILLIDARCY / porosity) ** 0.5 * 1e-6
