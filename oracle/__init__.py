"""FP64 CPU oracle for the pore-scale LB method of arXiv:1410.1921.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py.  The product package never imports it, and it
imports nothing from the product package.

The heavy loops live in om_oracle.c (plain C, one loop per definition); this
module marshals numpy arrays into it and holds the scalar formulas of the
paper (physics.py).
"""
import ctypes as C

import numpy as np

from . import build as _build
from . import physics  # noqa: F401  (re-exported)

_lib = None

ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_EINFEASIBLE, ORC_ENOPERC, ORC_ENOTCONVERGED = 0, 1, 2, 4, 5, 6

_u8p = C.POINTER(C.c_uint8)
_i32p = C.POINTER(C.c_int32)
_f32p = C.POINTER(C.c_float)
_f64p = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
_u64p = C.POINTER(C.c_uint64)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        L.orc_splitmix64_next.restype = C.c_uint64
        L.orc_splitmix64_next.argtypes = [_u64p]
        L.orc_uniform.restype = C.c_double
        L.orc_uniform.argtypes = [_u64p]
        L.orc_lens_volume.restype = C.c_double
        L.orc_lens_volume.argtypes = [C.c_double] * 3
        L.orc_sphere_volume.restype = C.c_double
        L.orc_sphere_volume.argtypes = [C.c_double]
        L.orc_reconstruct.restype = C.c_int
        L.orc_reconstruct.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                      C.c_double, C.c_double, C.c_double, C.c_int, C.c_double,
                                      C.c_double, C.c_double, C.c_int64, _u8p, _f64p, C.c_int64,
                                      _i64p, _f64p, _i64p]
        L.orc_label18.restype = C.c_int
        L.orc_label18.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, _i32p, _u8p, _f64p]
        L.orc_chord13.restype = None
        L.orc_chord13.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_double, _f32p, _i32p]
        L.orc_mis.restype = C.c_int
        L.orc_mis.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_double, _f32p, _i32p]
        L.orc_q_matrix.argtypes = [_f64p]
        L.orc_qinv_matrix.argtypes = [_f64p]
        L.orc_velocities19.argtypes = [_i32p]
        L.orc_w19.restype = C.c_double
        L.orc_w19.argtypes = [C.c_int]
        L.orc_opp19.restype = C.c_int
        L.orc_opp19.argtypes = [C.c_int]
        L.orc_meq.argtypes = [C.c_double] * 4 + [_f64p]
        L.orc_rates.argtypes = [C.c_double, _f64p]
        L.orc_mrt_collide_node.argtypes = [_f64p, C.c_double, C.c_double, _f64p]
        L.orc_flow_step.restype = C.c_int
        L.orc_flow_step.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _f64p]
        L.orc_flow_velocity.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_double, _f64p,
                                        _f64p, _f64p, _f64p, _f64p]
        L.orc_flow_init.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, _f64p]
        L.orc_flow_solve.restype = C.c_int
        L.orc_flow_solve.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                     C.c_double, C.c_int, C.c_int64, _f64p, _f64p]
        L.orc_pressure_bc.restype = C.c_int
        L.orc_pressure_bc.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _f64p]
        L.orc_flow_step_p.restype = C.c_int
        L.orc_flow_step_p.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                      _f64p]
        L.orc_flow_solve_p.restype = C.c_int
        L.orc_flow_solve_p.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                       C.c_double, C.c_int, C.c_int64, _f64p, _f64p]
        L.orc_tau_knudsen.restype = C.c_double
        L.orc_tau_knudsen.argtypes = [C.c_double] * 3
        L.orc_diff_init.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _f64p]
        L.orc_diffq_init.restype = C.c_int
        L.orc_diffq_init.argtypes = [C.c_int, _u8p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _f64p]
        L.orc_diffq_step.restype = C.c_int
        L.orc_diffq_step.argtypes = [C.c_int, _u8p, C.c_int, C.c_int, C.c_int, _f64p, C.c_double, C.c_double,
                                     _f64p]
        L.orc_diffq_fields.restype = C.c_int
        L.orc_diffq_fields.argtypes = [C.c_int, _u8p, C.c_int, C.c_int, C.c_int, _f64p, _f64p, _f64p, _f64p]
        L.orc_diffq_solve.restype = C.c_int
        L.orc_diffq_solve.argtypes = [C.c_int, _u8p, C.c_int, C.c_int, C.c_int, _f64p, C.c_double, C.c_double,
                                      C.c_double, C.c_int, C.c_int64, _f64p, _f64p]
        L.orc_diff_step.restype = C.c_int
        L.orc_diff_step.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, _f64p, C.c_double, C.c_double,
                                    _f64p]
        L.orc_diff_fields.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, _f64p, _f64p, _f64p, _f64p]
        L.orc_diff_solve.restype = C.c_int
        L.orc_diff_solve.argtypes = [_u8p, C.c_int, C.c_int, C.c_int, _f64p, C.c_double, C.c_double,
                                     C.c_double, C.c_int, C.c_int64, _f64p, _f64p]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _u8(mask):
    return np.ascontiguousarray(mask, dtype=np.uint8)


# ---------------------------------------------------------------- random numbers
def splitmix64(seed, n):
    """First n SplitMix64 outputs from state `seed`."""
    st = C.c_uint64(seed)
    return [lib().orc_splitmix64_next(C.byref(st)) for _ in range(n)]


def uniforms(seed, n):
    st = C.c_uint64(seed)
    return np.array([lib().orc_uniform(C.byref(st)) for _ in range(n)])


def lens_volume(r1, r2, dist):
    return lib().orc_lens_volume(r1, r2, dist)


def sphere_volume(r):
    return lib().orc_sphere_volume(r)


# ---------------------------------------------------------------- reconstruction (Sec. 2)
def reconstruct(seed, shape, dx_nm, mean_nm, sd_nm, dmin_nm, dmax_nm, porosity, xi, p0=0.5,
                dist=0, max_trials=10_000_000, cap=2_000_000):
    """Returns (status, mask uint8 [nx,ny,nz], spheres [n,4] (voxel units), porosity, trials)."""
    nx, ny, nz = shape
    mask = np.zeros(nx * ny * nz, np.uint8)
    sph = np.zeros(4 * cap, np.float64)
    ns, eps, tr = C.c_int64(0), C.c_double(0), C.c_int64(0)
    rc = lib().orc_reconstruct(seed, nx, ny, nz, dx_nm, mean_nm, sd_nm, dmin_nm, dmax_nm, dist,
                               porosity, xi, p0, max_trials, _p(mask, _u8p), _p(sph, _f64p), cap,
                               C.byref(ns), C.byref(eps), C.byref(tr))
    return rc, mask.reshape(shape), sph[: 4 * ns.value].reshape(-1, 4).copy(), eps.value, tr.value


# ---------------------------------------------------------------- structure (Sec. 4.1)
def label18(mask):
    m = _u8(mask)
    labels = np.zeros(m.size, np.int32)
    tr = np.zeros(m.size, np.uint8)
    conn = C.c_double(0)
    rc = lib().orc_label18(_p(m, _u8p), *m.shape, _p(labels, _i32p), _p(tr, _u8p), C.byref(conn))
    assert rc == ORC_OK
    return labels.reshape(m.shape), tr.reshape(m.shape), conn.value


def chord13(mask, dx_nm=1.0, counts=True):
    m = _u8(mask)
    d = np.zeros(m.size, np.float32)
    cnt = np.zeros(13 * m.size, np.int32) if counts else None
    lib().orc_chord13(_p(m, _u8p), *m.shape, dx_nm, _p(d, _f32p), _p(cnt, _i32p))
    return d.reshape(m.shape), (cnt.reshape((13,) + m.shape) if counts else None)


def mis(mask, dx_nm=1.0):
    m = _u8(mask)
    d = np.zeros(m.size, np.float32)
    r2 = np.zeros(m.size, np.int32)
    rc = lib().orc_mis(_p(m, _u8p), *m.shape, dx_nm, _p(d, _f32p), _p(r2, _i32p))
    return rc, d.reshape(m.shape), r2.reshape(m.shape)


# ---------------------------------------------------------------- MRT D3Q19 (Sec. 3.1, App. A)
def q_matrix():
    Q = np.zeros(361)
    lib().orc_q_matrix(_p(Q, _f64p))
    return Q.reshape(19, 19)


def qinv_matrix():
    Qi = np.zeros(361)
    lib().orc_qinv_matrix(_p(Qi, _f64p))
    return Qi.reshape(19, 19)


def velocities19():
    e = np.zeros(57, np.int32)
    lib().orc_velocities19(_p(e, _i32p))
    return e.reshape(19, 3)


def weights19():
    return np.array([lib().orc_w19(i) for i in range(19)])


def opposite19():
    return np.array([lib().orc_opp19(i) for i in range(19)])


def meq(rho, jx, jy, jz):
    m = np.zeros(19)
    lib().orc_meq(rho, jx, jy, jz, _p(m, _f64p))
    return m


def rates(tau):
    s = np.zeros(19)
    lib().orc_rates(tau, _p(s, _f64p))
    return s


def mrt_collide_node(f, tau, g):
    f = np.ascontiguousarray(f, np.float64)
    out = np.zeros(19)
    lib().orc_mrt_collide_node(_p(f, _f64p), tau, g, _p(out, _f64p))
    return out


def flow_init(node):
    n = _u8(node)
    f = np.zeros(19 * n.size)
    lib().orc_flow_init(_p(n, _u8p), *n.shape, _p(f, _f64p))
    return f.reshape((19,) + n.shape)


def flow_step(node, f, tau, g, steps=1):
    """Advance populations f [19, nx, ny, nz] (in place copy returned)."""
    n = _u8(node)
    f = np.ascontiguousarray(f, np.float64).copy()
    for _ in range(steps):
        rc = lib().orc_flow_step(_p(n, _u8p), *n.shape, tau, g, _p(f, _f64p))
        assert rc == ORC_OK
    return f


def flow_velocity(node, f, g):
    n = _u8(node)
    f = np.ascontiguousarray(f, np.float64)
    ux, uy, uz, rho = (np.zeros(n.size) for _ in range(4))
    lib().orc_flow_velocity(_p(n, _u8p), *n.shape, g, _p(f, _f64p), _p(ux, _f64p), _p(uy, _f64p),
                            _p(uz, _f64p), _p(rho, _f64p))
    return tuple(a.reshape(n.shape) for a in (ux, uy, uz, rho))


def flow_solve(node, tau=1.0, g=1e-6, tol=1e-6, K=100, max_steps=1_000_000):
    """Returns (status, k_L, sum_ux, steps, rel_change, f)."""
    n = _u8(node)
    f = np.zeros(19 * n.size)
    out = np.zeros(4)
    rc = lib().orc_flow_solve(_p(n, _u8p), *n.shape, tau, g, tol, K, max_steps, _p(f, _f64p),
                              _p(out, _f64p))
    return rc, out[0], out[1], int(out[2]), out[3], f.reshape((19,) + n.shape)


def pressure_bc(node, f, rho_in, rho_out):
    """The boundary replacement of the pressure-driven flow (Sec. 3.3) on a
    copy of f [19, nx, ny, nz]."""
    n = _u8(node)
    f = np.ascontiguousarray(f, np.float64).copy()
    rc = lib().orc_pressure_bc(_p(n, _u8p), *n.shape, rho_in, rho_out, _p(f, _f64p))
    assert rc == ORC_OK
    return f


def flow_step_p(node, f, tau, rho_in, rho_out, steps=1):
    """Advance the pressure-driven flow (a copy of f is returned)."""
    n = _u8(node)
    f = np.ascontiguousarray(f, np.float64).copy()
    for _ in range(steps):
        rc = lib().orc_flow_step_p(_p(n, _u8p), *n.shape, tau, rho_in, rho_out, _p(f, _f64p))
        assert rc == ORC_OK
    return f


def flow_solve_p(node, tau=1.0, rho_in=1.00005, rho_out=0.99995, tol=1e-6, K=100, max_steps=1_000_000):
    """Pressure-driven solve.  Returns (status, k_L, <u_x>, steps, rel_change, f)."""
    n = _u8(node)
    f = np.zeros(19 * n.size)
    out = np.zeros(4)
    rc = lib().orc_flow_solve_p(_p(n, _u8p), *n.shape, tau, rho_in, rho_out, tol, K, max_steps, _p(f, _f64p),
                                _p(out, _f64p))
    return rc, out[0], out[1], int(out[2]), out[3], f.reshape((19,) + n.shape)


# ---------------------------------------------------------------- BGK D3Q7 (Sec. 3.2)
def tau_knudsen(d_nm, d_ref_nm=60.0, tau_ref=1.0):
    return lib().orc_tau_knudsen(d_nm, d_ref_nm, tau_ref)


def omega_field(node, d_nm, d_ref_nm=60.0, tau_ref=1.0):
    """omega = 1/tau_g per voxel by Eq. 12 (0 off the node set)."""
    n = _u8(node)
    d = np.asarray(d_nm, np.float64)
    om = np.zeros(n.shape)
    idx = np.nonzero(n)
    for v in zip(*idx):
        om[v] = 1.0 / tau_knudsen(float(d[v]), d_ref_nm, tau_ref)
    return om


def diff_init(node, cin=1.0, cout=0.0, q=7):
    """a_i C_lin(x) on the node set, q = 7 (D3Q7) or 19 (the paper's D3Q19)."""
    n = _u8(node)
    g = np.zeros(q * n.size)
    assert lib().orc_diffq_init(q, _p(n, _u8p), *n.shape, cin, cout, _p(g, _f64p)) == ORC_OK
    return g.reshape((q,) + n.shape)


def diff_step(node, g, omega, cin=1.0, cout=0.0, steps=1):
    """Advance g [q, nx, ny, nz] (q = 7 or 19, from its shape); a copy."""
    n = _u8(node)
    g = np.ascontiguousarray(g, np.float64).copy()
    q = g.shape[0]
    om = np.ascontiguousarray(omega, np.float64)
    for _ in range(steps):
        rc = lib().orc_diffq_step(q, _p(n, _u8p), *n.shape, _p(om, _f64p), cin, cout, _p(g, _f64p))
        assert rc == ORC_OK
    return g


def diff_fields(node, g, omega):
    n = _u8(node)
    g = np.ascontiguousarray(g, np.float64)
    om = np.ascontiguousarray(omega, np.float64)
    Cf, J = np.zeros(n.size), np.zeros(n.size)
    assert lib().orc_diffq_fields(g.shape[0], _p(n, _u8p), *n.shape, _p(om, _f64p), _p(g, _f64p), _p(Cf, _f64p),
                                  _p(J, _f64p)) == ORC_OK
    return Cf.reshape(n.shape), J.reshape(n.shape)


def diff_solve(node, omega, cin=1.0, cout=0.0, tol=1e-6, K=100, max_steps=1_000_000, q=7):
    """Returns (status, D_eff_L, sum_Jx, steps, rel_change, sum_C, g)."""
    n = _u8(node)
    om = np.ascontiguousarray(omega, np.float64)
    g = np.zeros(q * n.size)
    out = np.zeros(5)
    rc = lib().orc_diffq_solve(q, _p(n, _u8p), *n.shape, _p(om, _f64p), cin, cout, tol, K, max_steps,
                               _p(g, _f64p), _p(out, _f64p))
    return rc, out[0], out[1], int(out[2]), out[3], out[4], g.reshape((q,) + n.shape)


# ---------------------------------------------------------------- results in physical units (Eqs. 15, 16)
def tortuosity_eq16(pore_mask, transport, d_nm, D_eff_m2s, T_K, M_kg_per_mol):
    """Eq. 16, tortuosity = eps D / D_eff, with eps the total porosity (pore
    voxels over all voxels, dead-end and isolated pores included) and D the
    local Knudsen diffusivity of Eq. 11 averaged over the transport nodes (the
    nodes the diffusion runs on), d in nm."""
    pore = np.asarray(pore_mask) != 0
    tr = np.asarray(transport) != 0
    eps = float(pore.sum()) / pore.size
    D_mean = physics.mean_knudsen_diffusivity(np.asarray(d_nm, np.float64)[tr], T_K, M_kg_per_mol)
    return physics.tortuosity(eps, D_mean, D_eff_m2s)
