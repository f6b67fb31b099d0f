"""Python binding of libom.so, the GB300 library of include/om.h.

Argument marshalling only: every entry point below calls the C function of
the same name, and all computation runs in the library's CUDA kernels.
Host arrays are numpy; device arrays are torch CUDA tensors (torch is used
for device memory and streams).  The library must have been built
(paper_1410_1921_gb300.build.build()); there is no fallback.

Method: Chen, Kang, Zhang & Tao, arXiv:1410.1921 -- pore-sphere
reconstruction (Sec. 2), 18-neighbour labelling and pore size (Sec. 4.1),
D3Q19 MRT flow (Sec. 3.1, App. A) and D3Q7 Knudsen diffusion (Sec. 3.2),
permeability / diffusivity / tortuosity / apparent permeability (Eqs. 13-16,
26).
"""
import ctypes as C
import os

import numpy as np

from .build import LIB

OM_OK, OM_EINVAL, OM_ENOMEM, OM_ECUDA, OM_EINFEASIBLE, OM_ENOPERC, OM_ENOTCONVERGED, OM_ETIMEOUT = range(8)
OM_F64, OM_F32, OM_F16DEV, OM_BF16DEV = range(4)
OM_PORE_CHORD13, OM_PORE_MIS = 0, 1
OM_DRIVE_FORCE, OM_DRIVE_PRESSURE = 0, 1
OM_ACCEL_NONE, OM_ACCEL_EXTRAPOLATE = 0, 1
OM_LAYOUT_AUTO, OM_LAYOUT_SPARSE, OM_LAYOUT_DENSE = 0, 1, 2
STATUS_NAMES = ["OM_OK", "OM_EINVAL", "OM_ENOMEM", "OM_ECUDA", "OM_EINFEASIBLE", "OM_ENOPERC",
                "OM_ENOTCONVERGED", "OM_ETIMEOUT"]


class OmError(RuntimeError):
    def __init__(self, fn, status, msg):
        self.status = status
        super().__init__(f"{fn}: {STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")


class om_domain(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("dx_nm", C.c_double)]


class om_recon_params(C.Structure):
    _fields_ = [("mean_d_nm", C.c_double), ("sd_d_nm", C.c_double), ("dmin_nm", C.c_double),
                ("dmax_nm", C.c_double), ("dist", C.c_int32), ("porosity", C.c_double),
                ("overlap_tol", C.c_double), ("p_overlap", C.c_double), ("max_trials", C.c_int64)]


class om_flow_params(C.Structure):
    _fields_ = [("tau", C.c_double), ("body_force", C.c_double), ("conv_tol", C.c_double),
                ("check_every", C.c_int32), ("max_steps", C.c_int64), ("precision", C.c_int32),
                ("variant", C.c_int32), ("drive", C.c_int32), ("delta_rho", C.c_double), ("layout", C.c_int32)]


class om_diff_params(C.Structure):
    _fields_ = [("T_K", C.c_double), ("M_kg_per_mol", C.c_double), ("d_ref_nm", C.c_double),
                ("tau_ref", C.c_double), ("c_in", C.c_double), ("c_out", C.c_double),
                ("conv_tol", C.c_double), ("check_every", C.c_int32), ("max_steps", C.c_int64),
                ("precision", C.c_int32), ("variant", C.c_int32), ("lattice", C.c_int32), ("accel", C.c_int32),
                ("layout", C.c_int32)]


class om_slip_corrections(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("lambda_m", "r_m", "Kn", "dgm", "klinkenberg", "beskok_civan", "heid",
                                           "jones_owens", "sampath_keighin", "florence")]


class om_structure_results(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("k_m2", "D_eff_m2s", "D_mean_m2s", "tortuosity", "alpha", "k_kc_m2")]


class om_run_info(C.Structure):
    _fields_ = [("steps", C.c_int64), ("n_nodes", C.c_int64), ("rel_change", C.c_double),
                ("mass", C.c_double), ("seconds", C.c_double), ("mlups", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp, _u8p, _i32p, _f32p, _f64p, _i64p = (C.c_void_p, C.POINTER(C.c_uint8), C.POINTER(C.c_int32),
                                         C.POINTER(C.c_float), C.POINTER(C.c_double),
                                         C.POINTER(C.c_int64))

# name -> argtypes (restype om_status = int)
_SIGS = {
    "om_reconstruct": [C.c_uint64, om_domain, C.POINTER(om_recon_params), _vp, _f64p, _i64p],
    "om_reconstruct_dev": [C.c_uint64, om_domain, C.POINTER(om_recon_params), _vp, _f64p, _i64p, _vp],
    "om_label_connectivity": [_vp, om_domain, _vp, _vp, _f64p],
    "om_label_connectivity_dev": [_vp, om_domain, _vp, _vp, _f64p, _vp],
    "om_label_connectivity_noalloc": [_vp, om_domain, _vp, _vp, _f64p, _vp],
    "om_local_pore_diameter": [_vp, om_domain, C.c_int32, _vp, _vp],
    "om_local_pore_diameter_dev": [_vp, om_domain, C.c_int32, _vp, _vp, _vp],
    "om_solve_permeability": [_vp, om_domain, C.POINTER(om_flow_params), _f64p, _f64p,
                              C.POINTER(om_run_info), _vp],
    "om_solve_knudsen": [_vp, _vp, om_domain, C.POINTER(om_diff_params), _f64p, _f64p,
                         C.POINTER(om_run_info), _vp],
    "om_apparent_permeability": [C.c_double, C.c_double, C.c_double, C.c_double, _f64p, _f64p],
    "om_structure_results_from_lattice": [C.c_double] * 6 + [C.POINTER(om_diff_params),
                                                             C.POINTER(om_structure_results)],
    "om_bruggeman_fit": [C.c_int64, _vp, _vp, _vp, _f64p],
    "om_slip_correction_factors": [C.c_double] * 7 + [C.POINTER(om_slip_corrections)],
    "om_nodeset_create": [_vp, om_domain, _vp, C.POINTER(_vp)],
    "om_nodeset_count": [_vp, _i64p],
    "om_nodeset_voxels": [_vp, _vp, _vp],
    "om_nodeset_destroy": [_vp],
    "om_flow_create": [_vp, C.POINTER(om_flow_params), _vp, C.POINTER(_vp)],
    "om_flow_step": [_vp, C.c_int64, _vp],
    "om_flow_observe": [_vp, _f64p, _vp],
    "om_flow_solve": [_vp, _f64p, C.POINTER(om_run_info), _vp],
    "om_flow_get_populations": [_vp, _vp, _vp],
    "om_flow_set_populations": [_vp, _vp, _vp],
    "om_flow_get_velocity": [_vp, _vp, _vp],
    "om_flow_time": [_vp, _i64p],
    "om_flow_destroy": [_vp],
    "om_diff_create": [_vp, _vp, C.POINTER(om_diff_params), _vp, C.POINTER(_vp)],
    "om_diff_step": [_vp, C.c_int64, _vp],
    "om_diff_observe": [_vp, _f64p, _vp],
    "om_diff_solve": [_vp, _f64p, C.POINTER(om_run_info), _vp],
    "om_diff_get_populations": [_vp, _vp, _vp],
    "om_diff_set_populations": [_vp, _vp, _vp],
    "om_diff_get_fields": [_vp, _vp, _vp, _vp],
    "om_diff_time": [_vp, _i64p],
    "om_diff_destroy": [_vp],
    "om_coarse_domain": [om_domain, C.POINTER(om_domain)],
    "om_coarsen2_dev": [_vp, _vp, om_domain, _vp, _vp, _vp],
    "om_prolong2_dev": [_vp, C.c_int32, _vp, om_domain, C.c_double, C.c_double, _vp, C.c_int64, C.c_int32, _vp, _vp],
    "om_unet_pack_structure3": [_vp, _vp, C.c_double, _vp, C.c_int64, _vp, _vp],
    "om_prolong2_ux_dev": [_vp, _vp, om_domain, C.c_double, C.c_double, _vp, _vp],
    "om_flow_state_size": [_vp, _i64p],
    "om_flow_save_state": [_vp, _vp, C.c_int64, _vp],
    "om_flow_load_state": [_vp, _vp, C.c_int64, _vp],
    "om_diff_state_size": [_vp, _i64p],
    "om_diff_save_state": [_vp, _vp, C.c_int64, _vp],
    "om_diff_load_state": [_vp, _vp, C.c_int64, _vp],
    "om_batch_create": [C.c_int32, C.POINTER(om_domain), C.POINTER(_vp), C.POINTER(_vp),
                        C.POINTER(om_flow_params), C.POINTER(om_diff_params), _vp, C.POINTER(_vp)],
    "om_batch_step": [_vp, C.c_int32, C.c_int64, _vp],
    "om_batch_solve": [_vp, C.c_int32, _vp, _vp, _vp, _vp, _vp],
    "om_batch_set_window_mode": [_vp, C.c_int32, C.c_int32],
    "om_barrier_selftest": [C.c_int32, C.c_int32, C.c_int32, C.c_int64, C.POINTER(C.c_int32), _vp],
    "om_batch_get_populations": [_vp, C.c_int32, C.c_int32, _vp, _vp],
    "om_batch_get_field": [_vp, C.c_int32, C.c_int32, _vp, _vp],
    "om_batch_set_populations": [_vp, C.c_int32, C.c_int32, _vp, _vp],
    "om_batch_reset": [_vp, C.c_int32, _vp],
    "om_batch_init_fields": [_vp, C.c_int32, C.c_int32, _vp, C.c_int64, C.c_double, C.c_int32, _vp],
    "om_batch_destroy": [_vp],
    "om_unet_create": [C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_int32), C.c_uint64, C.POINTER(_vp)],
    "om_unet_param_count": [_vp, _i64p],
    "om_unet_get_params": [_vp, _vp, _vp],
    "om_unet_set_params": [_vp, _vp, _vp],
    "om_unet_get_grads": [_vp, _vp, _vp],
    "om_unet_forward": [_vp, _vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _vp, _vp],
    "om_unet_backward": [_vp, _vp, _vp, _vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _f64p, _vp],
    "om_unet_train_step": [_vp, _vp, _vp, _vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_float, _f64p,
                           _vp],
    "om_unet_destroy": [_vp],
    "om_unet_pack_structure": [_vp, _vp, C.c_int64, C.c_double, _vp, _vp],
    "om_flow_init_velocity": [_vp, _vp, C.c_int64, C.c_double, _vp],
    "om_diff_init_concentration": [_vp, _vp, C.c_int64, C.c_int32, _vp],
}

_lib = None


def lib():
    """Load libom.so (fails loudly when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build it with paper_1410_1921_gb300.build.build()")
        import torch  # noqa: F401  -- load PyTorch's CUDA runtime first so both share it
        L = C.CDLL(LIB)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.om_last_error.restype = C.c_char_p
        L.om_version.restype = C.c_char_p
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS) + ["om_last_error", "om_version"]


def _check(fn, st, ok=(OM_OK,)):
    if st not in ok:
        raise OmError(fn, st, lib().om_last_error().decode())
    return st


def _call(fn, *args, ok=(OM_OK,)):
    return _check(fn, getattr(lib(), fn)(*args), ok)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, C.c_void_p):
        return stream
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "host arrays must be C-contiguous"
        return C.c_void_p(a.ctypes.data)
    assert a.is_contiguous(), "device tensors must be contiguous"
    return C.c_void_p(a.data_ptr())


def domain(shape, dx_nm=1.0):
    nx, ny, nz = shape
    return om_domain(nx, ny, nz, dx_nm)


def recon_params(mean_d_nm, sd_d_nm, dmin_nm, dmax_nm, porosity, overlap_tol, p_overlap=0.5, dist=0,
                 max_trials=20_000_000):
    return om_recon_params(mean_d_nm, sd_d_nm, dmin_nm, dmax_nm, dist, porosity, overlap_tol, p_overlap,
                           max_trials)


def flow_params(tau=1.0, body_force=1e-6, conv_tol=1e-6, check_every=100, max_steps=10_000_000,
                precision=OM_F32, variant=-1, drive=OM_DRIVE_FORCE, delta_rho=1e-4, layout=0):
    return om_flow_params(tau, body_force, conv_tol, check_every, max_steps, precision, variant, drive, delta_rho,
                          layout)


def diff_params(T_K=300.0, M_kg_per_mol=0.016, d_ref_nm=60.0, tau_ref=1.0, c_in=1.0, c_out=0.0,
                conv_tol=1e-6, check_every=100, max_steps=10_000_000, precision=OM_F32, variant=-1, lattice=7,
                accel=0, layout=0):
    return om_diff_params(T_K, M_kg_per_mol, d_ref_nm, tau_ref, c_in, c_out, conv_tol, check_every,
                          max_steps, precision, variant, lattice, accel, layout)


# ------------------------------------------------------------------ host-buffer entry points
def om_reconstruct(seed, dom, params):
    mask = np.zeros(dom.nx * dom.ny * dom.nz, np.uint8)
    eps, ns = C.c_double(), C.c_int64()
    st = _call("om_reconstruct", seed, dom, C.byref(params), _ptr(mask), C.byref(eps), C.byref(ns),
               ok=(OM_OK, OM_EINFEASIBLE))
    return st, mask.reshape(dom.nx, dom.ny, dom.nz), eps.value, ns.value


def om_reconstruct_dev(seed, dom, params, mask_dev, stream=None):
    eps, ns = C.c_double(), C.c_int64()
    st = _call("om_reconstruct_dev", seed, dom, C.byref(params), _ptr(mask_dev), C.byref(eps), C.byref(ns),
               _stream(stream), ok=(OM_OK, OM_EINFEASIBLE))
    return st, eps.value, ns.value


def om_label_connectivity(mask, dom=None):
    mask = np.ascontiguousarray(mask, np.uint8)
    dom = dom or domain(mask.shape)
    labels = np.zeros(mask.shape, np.int32)
    tr = np.zeros(mask.shape, np.uint8)
    conn = C.c_double()
    _call("om_label_connectivity", _ptr(mask), dom, _ptr(labels), _ptr(tr), C.byref(conn))
    return labels, tr, conn.value


def om_label_connectivity_dev(mask_dev, dom, labels_dev=None, transport_dev=None, stream=None):
    conn = C.c_double()
    _call("om_label_connectivity_dev", _ptr(mask_dev), dom, _ptr(labels_dev), _ptr(transport_dev),
          C.byref(conn), _stream(stream))
    return conn.value


def om_label_connectivity_noalloc(mask_dev, dom, labels_dev, transport_dev=None, stream=None):
    """om_label_connectivity_dev without any device allocation.

    For callers that cannot allocate device memory: their GPU memory is
    already held by another allocator (a framework's caching pool), or their
    memory plan is fixed at start-up and cudaMalloc/cudaFree (with their
    device-wide synchronisation) are not allowed later.  The scratch is a
    static 4 MiB device array, so boxes are limited to 2^24 voxels; calls
    that overlap on the GPU race on it.  labels_dev is required."""
    conn = C.c_double()
    _call("om_label_connectivity_noalloc", _ptr(mask_dev), dom, _ptr(labels_dev), _ptr(transport_dev),
          C.byref(conn), _stream(stream))
    return conn.value


def om_local_pore_diameter(mask, dom=None, mode=OM_PORE_CHORD13, witness=False):
    mask = np.ascontiguousarray(mask, np.uint8)
    dom = dom or domain(mask.shape)
    d = np.zeros(mask.shape, np.float32)
    w = None
    if witness:
        w = np.zeros(((13,) if mode == OM_PORE_CHORD13 else ()) + mask.shape, np.int32)
    _call("om_local_pore_diameter", _ptr(mask), dom, mode, _ptr(d), _ptr(w))
    return d, w


def om_local_pore_diameter_dev(mask_dev, dom, mode, d_dev, witness_dev=None, stream=None):
    _call("om_local_pore_diameter_dev", _ptr(mask_dev), dom, mode, _ptr(d_dev), _ptr(witness_dev),
          _stream(stream))


def om_solve_permeability(mask, dom, params, want_ux=False):
    mask = np.ascontiguousarray(mask, np.uint8)
    k, kl = C.c_double(), C.c_double()
    info = om_run_info()
    ux = np.zeros(mask.shape, np.float32) if want_ux else None
    st = _call("om_solve_permeability", _ptr(mask), dom, C.byref(params), C.byref(k), C.byref(kl),
               C.byref(info), _ptr(ux), ok=(OM_OK, OM_ENOTCONVERGED))
    return st, k.value, kl.value, info, ux


def om_solve_knudsen(mask, d_nm, dom, params, want_c=False):
    mask = np.ascontiguousarray(mask, np.uint8)
    d_nm = np.ascontiguousarray(d_nm, np.float32)
    D, tau = C.c_double(), C.c_double()
    info = om_run_info()
    c = np.zeros(mask.shape, np.float32) if want_c else None
    st = _call("om_solve_knudsen", _ptr(mask), _ptr(d_nm), dom, C.byref(params), C.byref(D), C.byref(tau),
               C.byref(info), _ptr(c), ok=(OM_OK, OM_ENOTCONVERGED))
    return st, D.value, tau.value, info, c


def om_slip_correction_factors(k_m2, porosity, D_eff_m2s, T_K=323.0, M_kg_per_mol=0.016, mu_Pa_s=1.73e-5,
                               p_Pa=17236893.0):
    """The correction factors of Sec. 4.4 as a dict (defaults: the operating
    point of Sec. 4.4.3, methane)."""
    out = om_slip_corrections()
    _call("om_slip_correction_factors", k_m2, porosity, D_eff_m2s, T_K, M_kg_per_mol, mu_Pa_s, p_Pa, C.byref(out))
    return {n: getattr(out, n) for n, _ in om_slip_corrections._fields_}


def om_structure_results_from_lattice(dx_nm, k_lattice, D_eff_lattice, D_mean_lattice, porosity, mean_d_nm,
                                      params):
    """k, D_eff, D, tortuosity, alpha and the Kozeny-Carman k of a structure
    from its lattice results (Eqs. 15-17, Sec. 4.2), as a dict."""
    out = om_structure_results()
    _call("om_structure_results_from_lattice", dx_nm, k_lattice, D_eff_lattice, D_mean_lattice, porosity, mean_d_nm,
          C.byref(params), C.byref(out))
    return {n: getattr(out, n) for n, _ in om_structure_results._fields_}


def om_bruggeman_fit(porosity, D_eff_m2s, D_mean_m2s):
    """Sec. 4.2: the exponent of D_eff = D eps^alpha fitted over structures."""
    arrs = [np.ascontiguousarray(a, np.float64) for a in (porosity, D_eff_m2s, D_mean_m2s)]
    alpha = C.c_double()
    _call("om_bruggeman_fit", arrs[0].size, *[_ptr(a) for a in arrs], C.byref(alpha))
    return alpha.value


def om_apparent_permeability(k_m2, D_eff_m2s, mu_Pa_s, p_Pa):
    ka, fc = C.c_double(), C.c_double()
    _call("om_apparent_permeability", k_m2, D_eff_m2s, mu_Pa_s, p_Pa, C.byref(ka), C.byref(fc))
    return ka.value, fc.value


# ------------------------------------------------------------------ solver objects (device)
class NodeSet:
    """om_nodeset: the transport voxels of a device mask, numbered in voxel order."""

    def __init__(self, nodes_dev, dom, stream=None):
        self.dom = dom
        self.h = C.c_void_p()
        _call("om_nodeset_create", _ptr(nodes_dev), dom, _stream(stream), C.byref(self.h))

    @property
    def n_nodes(self):
        n = C.c_int64()
        _call("om_nodeset_count", self.h, C.byref(n))
        return n.value

    def voxels(self, out_dev, stream=None):
        _call("om_nodeset_voxels", self.h, _ptr(out_dev), _stream(stream))

    def close(self):
        if self.h:
            lib().om_nodeset_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Flow:
    """om_flow: D3Q19 populations on a node set (om_flow_*)."""

    def __init__(self, ns, params, stream=None):
        self.ns, self.params = ns, params
        self.h = C.c_void_p()
        _call("om_flow_create", ns.h, C.byref(params), _stream(stream), C.byref(self.h))

    def step(self, n, stream=None):
        _call("om_flow_step", self.h, n, _stream(stream))

    def observe(self, stream=None):
        out = (C.c_double * 4)()
        _call("om_flow_observe", self.h, out, _stream(stream))
        return list(out)

    def solve(self, stream=None):
        kl = C.c_double()
        info = om_run_info()
        st = _call("om_flow_solve", self.h, C.byref(kl), C.byref(info), _stream(stream),
                   ok=(OM_OK, OM_ENOTCONVERGED, OM_ENOPERC))
        return st, kl.value, info

    def get_populations(self, out_dev, stream=None):
        _call("om_flow_get_populations", self.h, _ptr(out_dev), _stream(stream))

    def set_populations(self, f_dev, stream=None):
        _call("om_flow_set_populations", self.h, _ptr(f_dev), _stream(stream))

    def get_velocity(self, out_dev, stream=None):
        _call("om_flow_get_velocity", self.h, _ptr(out_dev), _stream(stream))

    def init_velocity(self, ux_dev, stride=1, scale=1.0, stream=None):
        _call("om_flow_init_velocity", self.h, _ptr(ux_dev), stride, scale, _stream(stream))

    def save_state(self, stream=None):
        """The solver's whole evolving state as a host byte array (om_flow_save_state)."""
        n = C.c_int64()
        _call("om_flow_state_size", self.h, C.byref(n))
        buf = np.empty(n.value, np.uint8)
        _call("om_flow_save_state", self.h, _ptr(buf), n.value, _stream(stream))
        return buf

    def load_state(self, buf, stream=None):
        """Continue from a state saved by save_state (om_flow_load_state)."""
        buf = np.ascontiguousarray(buf, np.uint8)
        _call("om_flow_load_state", self.h, _ptr(buf), buf.size, _stream(stream))

    @property
    def time(self):
        t = C.c_int64()
        _call("om_flow_time", self.h, C.byref(t))
        return t.value

    def close(self):
        if self.h:
            lib().om_flow_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Diffusion:
    """om_diff: D3Q7 Knudsen-diffusion populations on a node set (om_diff_*)."""

    def __init__(self, ns, d_nm_dev, params, stream=None):
        self.ns, self.params = ns, params
        self.h = C.c_void_p()
        _call("om_diff_create", ns.h, _ptr(d_nm_dev), C.byref(params), _stream(stream), C.byref(self.h))

    def step(self, n, stream=None):
        _call("om_diff_step", self.h, n, _stream(stream))

    def observe(self, stream=None):
        out = (C.c_double * 5)()
        _call("om_diff_observe", self.h, out, _stream(stream))
        return list(out)

    def solve(self, stream=None):
        D = C.c_double()
        info = om_run_info()
        st = _call("om_diff_solve", self.h, C.byref(D), C.byref(info), _stream(stream),
                   ok=(OM_OK, OM_ENOTCONVERGED))
        return st, D.value, info

    def get_populations(self, out_dev, stream=None):
        _call("om_diff_get_populations", self.h, _ptr(out_dev), _stream(stream))

    def set_populations(self, g_dev, stream=None):
        _call("om_diff_set_populations", self.h, _ptr(g_dev), _stream(stream))

    def get_fields(self, c_dev=None, jx_dev=None, stream=None):
        _call("om_diff_get_fields", self.h, _ptr(c_dev), _ptr(jx_dev), _stream(stream))

    def init_concentration(self, c_dev, stride=1, from_linear=False, stream=None):
        _call("om_diff_init_concentration", self.h, _ptr(c_dev), stride, int(from_linear), _stream(stream))

    def save_state(self, stream=None):
        """The solver's whole evolving state as a host byte array (om_diff_save_state)."""
        n = C.c_int64()
        _call("om_diff_state_size", self.h, C.byref(n))
        buf = np.empty(n.value, np.uint8)
        _call("om_diff_save_state", self.h, _ptr(buf), n.value, _stream(stream))
        return buf

    def load_state(self, buf, stream=None):
        """Continue from a state saved by save_state (om_diff_load_state)."""
        buf = np.ascontiguousarray(buf, np.uint8)
        _call("om_diff_load_state", self.h, _ptr(buf), buf.size, _stream(stream))

    @property
    def time(self):
        t = C.c_int64()
        _call("om_diff_time", self.h, C.byref(t))
        return t.value

    def close(self):
        if self.h:
            lib().om_diff_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """om_batch: many structures solved together (om_batch_*).  nodes: list of
    device uint8 node masks; d_nm: list of device float pore sizes (or None);
    doms: list of om_domain."""

    def __init__(self, doms, nodes, d_nm=None, flow=None, diff=None, stream=None):
        n = len(doms)
        self.n = n
        self._keep = (list(nodes), list(d_nm) if d_nm is not None else None)
        darr = (om_domain * n)(*doms)
        narr = (C.c_void_p * n)(*[_ptr(t) for t in nodes])
        parr = (C.c_void_p * n)(*[_ptr(t) for t in d_nm]) if d_nm is not None else None
        self.h = C.c_void_p()
        _call("om_batch_create", n, darr, narr, parr, C.byref(flow) if flow is not None else None,
              C.byref(diff) if diff is not None else None, _stream(stream), C.byref(self.h))

    def step(self, model, n, stream=None):
        _call("om_batch_step", self.h, model, n, _stream(stream))

    def solve(self, model, stream=None):
        res = np.zeros(self.n)
        aux = np.zeros(self.n)
        info = (om_run_info * self.n)()
        st = np.zeros(self.n, np.int32)
        _call("om_batch_solve", self.h, model, _ptr(res), _ptr(aux), info, _ptr(st), _stream(stream))
        return res, aux, list(info), st

    def set_window_mode(self, model, mode):
        """-1: time both window modes in the first solve; 0: graph of
        per-step launches; 1: persistent grid-barrier launches."""
        _call("om_batch_set_window_mode", self.h, model, mode)

    def get_populations(self, model, item, out_dev, stream=None):
        _call("om_batch_get_populations", self.h, model, item, _ptr(out_dev), _stream(stream))

    def get_field(self, model, item, out_dev, stream=None):
        _call("om_batch_get_field", self.h, model, item, _ptr(out_dev), _stream(stream))

    def set_populations(self, model, item, f_dev, stream=None):
        _call("om_batch_set_populations", self.h, model, item, _ptr(f_dev), _stream(stream))

    def reset(self, model, stream=None):
        _call("om_batch_reset", self.h, model, _stream(stream))

    def init_fields(self, model, item, field_dev, stride=1, scale=1.0, from_linear=False, stream=None):
        _call("om_batch_init_fields", self.h, model, item, _ptr(field_dev), stride, scale, int(from_linear),
              _stream(stream))

    def close(self):
        if self.h:
            lib().om_batch_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def om_coarse_domain(dom):
    dc = om_domain()
    _call("om_coarse_domain", dom, C.byref(dc))
    return dc


def om_coarsen2_dev(nodes_dev, dom, d_nm_dev=None, stream=None):
    """(coarse domain, coarse node mask, coarse pore sizes or None) of a
    device node mask (and pore sizes), coarsened 2x per axis."""
    import torch
    dc = om_coarse_domain(dom)
    nc = dc.nx * dc.ny * dc.nz
    nodes_c = torch.empty(nc, dtype=torch.uint8, device=nodes_dev.device)
    d_c = torch.empty(nc, dtype=torch.float32, device=nodes_dev.device) if d_nm_dev is not None else None
    _call("om_coarsen2_dev", _ptr(nodes_dev), _ptr(d_nm_dev), dom, _ptr(nodes_c), _ptr(d_c), _stream(stream))
    return dc, nodes_c, d_c


def om_prolong2_dev(g_c_dev, q, nodes_c_dev, dom, c_in, c_out, c_dev, corr_dev=None, corr_stride=1, departure=False,
                    stream=None):
    _call("om_prolong2_dev", _ptr(g_c_dev), q, _ptr(nodes_c_dev), dom, c_in, c_out, _ptr(corr_dev), corr_stride,
          int(departure), _ptr(c_dev), _stream(stream))


def om_prolong2_ux_dev(f_c_dev, nodes_c_dev, dom, body_force_c, scale, ux_dev, stream=None):
    _call("om_prolong2_ux_dev", _ptr(f_c_dev), _ptr(nodes_c_dev), dom, body_force_c, scale, _ptr(ux_dev),
          _stream(stream))


def om_unet_pack_structure3(mask_dev, d_nm_dev, d_scale, extra_dev, x_dev, stream=None):
    _call("om_unet_pack_structure3", _ptr(mask_dev), _ptr(d_nm_dev), d_scale, _ptr(extra_dev), mask_dev.numel(),
          _ptr(x_dev), _stream(stream))


def om_barrier_selftest(blocks, rounds, extra, max_polls, stream=None):
    """Status (OM_OK or OM_ETIMEOUT) of `rounds` bounded grid barriers among
    `blocks` co-resident blocks that expect `blocks + extra` arrivals."""
    st = C.c_int32()
    _call("om_barrier_selftest", blocks, rounds, extra, max_polls, C.byref(st), _stream(stream))
    return st.value


def om_unet_pack_structure(mask_dev, d_nm_dev, d_scale, x_dev, stream=None):
    _call("om_unet_pack_structure", _ptr(mask_dev), _ptr(d_nm_dev), mask_dev.numel(), d_scale, _ptr(x_dev),
          _stream(stream))


class UNet:
    """om_unet: the warm-start network (om_unet_*).  Tensors are contiguous
    float32 CUDA tensors in NDHWC layout."""

    def __init__(self, in_ch, out_ch, channels=(16, 32, 64, 128), seed=1):
        arr = (C.c_int32 * len(channels))(*channels)
        self.h = C.c_void_p()
        self.in_ch, self.out_ch = in_ch, out_ch
        _call("om_unet_create", in_ch, out_ch, len(channels), arr, seed, C.byref(self.h))

    @property
    def n_params(self):
        n = C.c_int64()
        _call("om_unet_param_count", self.h, C.byref(n))
        return n.value

    def get_params(self, out_dev, stream=None):
        _call("om_unet_get_params", self.h, _ptr(out_dev), _stream(stream))

    def set_params(self, src_dev, stream=None):
        _call("om_unet_set_params", self.h, _ptr(src_dev), _stream(stream))

    def get_grads(self, out_dev, stream=None):
        _call("om_unet_get_grads", self.h, _ptr(out_dev), _stream(stream))

    def forward(self, x, y, stream=None):
        B, D, H, W = x.shape[:4]
        _call("om_unet_forward", self.h, _ptr(x), B, D, H, W, _ptr(y), _stream(stream))

    def backward(self, x, t, m, stream=None):
        B, D, H, W = x.shape[:4]
        loss = C.c_double()
        _call("om_unet_backward", self.h, _ptr(x), _ptr(t), _ptr(m), B, D, H, W, C.byref(loss), _stream(stream))
        return loss.value

    def train_step(self, x, t, m, lr, stream=None):
        B, D, H, W = x.shape[:4]
        loss = C.c_double()
        _call("om_unet_train_step", self.h, _ptr(x), _ptr(t), _ptr(m), B, D, H, W, lr, C.byref(loss),
              _stream(stream))
        return loss.value

    def close(self):
        if self.h:
            lib().om_unet_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
