// solve.cu -- the host-buffer entry points that chain the steps of the
// method: labelling (Sec. 4.1) -> node set -> LB solve (Secs. 3.1-3.2) ->
// lattice-to-physical units (Eq. 15) -> permeability (Eq. 13), effective
// diffusivity (Eq. 14), tortuosity (Eq. 16) and apparent permeability
// (Eq. 26).
#include <cmath>

#include "common.cuh"

namespace om {
om_status label_impl(const uint8_t* mask_dev, const om_domain& d, int* labels_dev, uint8_t* transport_dev,
                     int64_t* npore, int64_t* ntrans, cudaStream_t s);
// dense.cu
bool dense_flow_supported(const om_flow_params& p);
bool dense_diff_supported(const om_diff_params& p);
om_status dense_flow_solve(const uint8_t* node_dev, const om_domain& dom, int64_t nf, const om_flow_params& p,
                           double* k_lattice, om_run_info* info, float* ux_dev, double* pair_ms, cudaStream_t s);
om_status dense_diff_solve(const uint8_t* node_dev, const float* d_nm_dev, const om_domain& dom, int64_t nf,
                           const om_diff_params& p, double* D_lattice, double* DL_sum, om_run_info* info, float* c_dev,
                           double* pair_ms, cudaStream_t s);
}

using namespace om;

namespace {

constexpr double kR = 8.314462618;  // J / (mol K), CODATA 2018
constexpr double kPi = 3.14159265358979323846;

// Eq. 11: D_K = (d / 3) sqrt(8 R T / (pi M)), d in metres
double knudsen(double d_m, double T, double M) { return d_m / 3.0 * std::sqrt(8.0 * kR * T / (kPi * M)); }

// Eq. 15 for a diffusivity: lattice units to m^2/s, the time step fixed by
// the reference pore (Eqs. 11-12) on the lattice of p
double diffusivity_to_si(double D_lattice, const om_diff_params& p) {
  const double cs2 = p.lattice == 19 ? 1.0 / 3.0 : 0.25;  // D3Q19 or D3Q7
  const double DL_ref = cs2 * (p.tau_ref - 0.5);
  const double DK_ref = knudsen(p.d_ref_nm * 1e-9, p.T_K, p.M_kg_per_mol);
  return D_lattice * DK_ref / DL_ref;
}

struct Scope {
  cudaStream_t s = nullptr;
  om_nodeset* ns = nullptr;
  om_flow* fl = nullptr;
  om_diff* df = nullptr;
  ~Scope() {
    if (fl) om_flow_destroy(fl);
    if (df) om_diff_destroy(df);
    if (ns) om_nodeset_destroy(ns);
    if (s) cudaStreamDestroy(s);
  }
};

// transport mask on the device; counts of pore and transport voxels
om_status transport_nodes(const uint8_t* mask, const om_domain& d, DevBuf<uint8_t>& tr, int64_t& np,
                          int64_t& nt, cudaStream_t s) {
  const int64_t N = voxels(d);
  DevBuf<uint8_t> m;
  DevBuf<int> lab;
  OM_TRY(m.alloc(N));
  OM_TRY(lab.alloc(N));
  OM_TRY(tr.alloc(N));
  OM_CUDA(cudaMemcpyAsync(m.p, mask, N, cudaMemcpyHostToDevice, s));
  OM_TRY(label_impl(m.p, d, lab.p, tr.p, &np, &nt, s));
  if (nt == 0) return fail(OM_ENOPERC, "no pore component spans x = 0 .. nx-1");
  return OM_OK;
}

// OM_LAYOUT_AUTO times the layouts only where the nodes fill at least this
// fraction of the box (below it the dense sweeps move more non-node lanes
// than they save in lookups)
constexpr double kDenseTryFraction = 0.5;

// one even + odd pair of the sparse solver of this node set (after a warm-up pair)
template <class Step>
om_status pair_ms_of(Step step, cudaStream_t s, double* ms_out) {
  cudaEvent_t e0, e1;
  OM_CUDA(cudaEventCreate(&e0));
  OM_CUDA(cudaEventCreate(&e1));
  om_status st = step();
  if (st == OM_OK) {
    OM_CUDA(cudaEventRecord(e0, s));
    st = step();
    OM_CUDA(cudaEventRecord(e1, s));
  }
  if (st == OM_OK) {
    OM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    OM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    *ms_out = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

}  // namespace

extern "C" om_status om_solve_permeability(const uint8_t* mask, om_domain d, const om_flow_params* params,
                                           double* k_m2, double* k_lattice, om_run_info* info, float* ux_out) {
  if (!mask || !params) return fail(OM_EINVAL, "om_solve_permeability: null pointer");
  OM_TRY(check_domain(d));
  if (params->layout < OM_LAYOUT_AUTO || params->layout > OM_LAYOUT_DENSE)
    return fail(OM_EINVAL, "om_solve_permeability: unknown layout");
  if (params->layout == OM_LAYOUT_DENSE && !dense_flow_supported(*params))
    return fail(OM_EINVAL, "om_solve_permeability: the dense layout takes FP64 or FP32 and the body force");
  Scope sc;
  OM_CUDA(cudaStreamCreateWithFlags(&sc.s, cudaStreamNonBlocking));
  DevBuf<uint8_t> tr;
  int64_t np = 0, nt = 0;
  OM_TRY(transport_nodes(mask, d, tr, np, nt, sc.s));
  OM_TRY(om_nodeset_create(tr.p, d, sc.s, &sc.ns));
  const int64_t N = voxels(d);
  om_flow_params ps = *params;  // the sparse solver's parameters
  ps.layout = OM_LAYOUT_SPARSE;
  // the layout: as asked, or for OM_LAYOUT_AUTO the faster one over an even + odd pair
  bool dense = params->layout == OM_LAYOUT_DENSE && sc.ns->wrap_links > 0;
  if (params->layout == OM_LAYOUT_AUTO && dense_flow_supported(*params) && sc.ns->wrap_links > 0 &&
      (double)nt >= kDenseTryFraction * (double)N) {
    double ms_dense = 0.0, ms_sparse = 0.0;
    // a dense layout that does not fit in memory leaves the choice to the sparse one
    if (dense_flow_solve(tr.p, d, nt, *params, nullptr, nullptr, nullptr, &ms_dense, sc.s) == OM_OK) {
      OM_TRY(om_flow_create(sc.ns, &ps, sc.s, &sc.fl));
      OM_TRY(pair_ms_of([&]() { return om_flow_step(sc.fl, 2, sc.s); }, sc.s, &ms_sparse));
      om_flow_destroy(sc.fl);  // the solve starts from rest
      sc.fl = nullptr;
      dense = ms_dense < ms_sparse;
    }
  }
  double kl = 0.0;
  om_status st;
  DevBuf<float> u;
  if (dense) {
    if (ux_out) OM_TRY(u.alloc(N));
    st = dense_flow_solve(tr.p, d, nt, *params, &kl, info, ux_out ? u.p : nullptr, nullptr, sc.s);
  } else {
    tr.release();
    OM_TRY(om_flow_create(sc.ns, &ps, sc.s, &sc.fl));
    st = om_flow_solve(sc.fl, &kl, info, sc.s);
  }
  if (st == OM_ENOPERC) {
    if (k_lattice) *k_lattice = 0.0;
    if (k_m2) *k_m2 = 0.0;
  }
  if (st != OM_OK && st != OM_ENOTCONVERGED) return st;
  const double dx = d.dx_nm * 1e-9;
  if (k_lattice) *k_lattice = kl;
  if (k_m2) *k_m2 = kl * dx * dx;  // Eq. 15
  if (ux_out) {
    if (!dense) {
      OM_TRY(u.alloc(3 * N));
      OM_TRY(om_flow_get_velocity(sc.fl, u.p, sc.s));
    }
    OM_CUDA(cudaMemcpyAsync(ux_out, u.p, N * sizeof(float), cudaMemcpyDeviceToHost, sc.s));
    OM_CUDA(cudaStreamSynchronize(sc.s));
  }
  return st;
}

extern "C" om_status om_solve_knudsen(const uint8_t* mask, const float* d_nm, om_domain d,
                                      const om_diff_params* params, double* D_eff_m2s, double* tortuosity,
                                      om_run_info* info, float* c_out) {
  if (!mask || !d_nm || !params) return fail(OM_EINVAL, "om_solve_knudsen: null pointer");
  OM_TRY(check_domain(d));
  if (!(params->T_K > 0.0) || !(params->M_kg_per_mol > 0.0))
    return fail(OM_EINVAL, "om_solve_knudsen: T_K and M_kg_per_mol must be positive");
  if (params->layout < OM_LAYOUT_AUTO || params->layout > OM_LAYOUT_DENSE)
    return fail(OM_EINVAL, "om_solve_knudsen: unknown layout");
  if (params->layout == OM_LAYOUT_DENSE && !dense_diff_supported(*params))
    return fail(OM_EINVAL, "om_solve_knudsen: the dense layout takes FP64 or FP32 and the D3Q7 lattice");
  const int64_t N = voxels(d);
  Scope sc;
  OM_CUDA(cudaStreamCreateWithFlags(&sc.s, cudaStreamNonBlocking));
  DevBuf<uint8_t> tr;
  int64_t np = 0, nt = 0;
  OM_TRY(transport_nodes(mask, d, tr, np, nt, sc.s));
  OM_TRY(om_nodeset_create(tr.p, d, sc.s, &sc.ns));
  DevBuf<float> dd;
  OM_TRY(dd.alloc(N));
  OM_CUDA(cudaMemcpyAsync(dd.p, d_nm, N * sizeof(float), cudaMemcpyHostToDevice, sc.s));
  om_diff_params ps = *params;  // the sparse solver's parameters
  ps.layout = OM_LAYOUT_SPARSE;
  // the layout: as asked, or for OM_LAYOUT_AUTO the faster one over an even + odd pair
  bool dense = params->layout == OM_LAYOUT_DENSE;
  if (params->layout == OM_LAYOUT_AUTO && dense_diff_supported(*params) && (double)nt >= kDenseTryFraction * (double)N) {
    double ms_dense = 0.0, ms_sparse = 0.0;
    if (dense_diff_solve(tr.p, dd.p, d, nt, *params, nullptr, nullptr, nullptr, nullptr, &ms_dense, sc.s) == OM_OK) {
      OM_TRY(om_diff_create(sc.ns, dd.p, &ps, sc.s, &sc.df));
      OM_TRY(pair_ms_of([&]() { return om_diff_step(sc.df, 2, sc.s); }, sc.s, &ms_sparse));
      om_diff_destroy(sc.df);  // the solve starts from the linear profile
      sc.df = nullptr;
      dense = ms_dense < ms_sparse;
    }
  }
  double Dl = 0.0, DL_sum = 0.0;
  om_status st;
  DevBuf<float> c;
  if (c_out) OM_TRY(c.alloc(N));
  if (dense) {
    st = dense_diff_solve(tr.p, dd.p, d, nt, *params, &Dl, &DL_sum, info, c_out ? c.p : nullptr, nullptr, sc.s);
    if (st != OM_OK && st != OM_ENOTCONVERGED) return st;
  } else {
    tr.release();
    OM_TRY(om_diff_create(sc.ns, dd.p, &ps, sc.s, &sc.df));
    st = om_diff_solve(sc.df, &Dl, info, sc.s);
    if (st != OM_OK && st != OM_ENOTCONVERGED) return st;
    double o[5];
    OM_TRY(om_diff_observe(sc.df, o, sc.s));
    DL_sum = o[4];
    if (c_out) OM_TRY(om_diff_get_fields(sc.df, c.p, nullptr, sc.s));
  }
  if (D_eff_m2s) *D_eff_m2s = diffusivity_to_si(Dl, *params);  // Eq. 15
  if (tortuosity) {
    const double porosity = (double)np / (double)N;
    const double DL_mean = DL_sum / (double)nt;
    *tortuosity = porosity * DL_mean / Dl;  // Eq. 16
  }
  if (c_out) {
    OM_CUDA(cudaMemcpyAsync(c_out, c.p, N * sizeof(float), cudaMemcpyDeviceToHost, sc.s));
    OM_CUDA(cudaStreamSynchronize(sc.s));
  }
  return st;
}

extern "C" om_status om_structure_results_from_lattice(double dx_nm, double k_lattice, double D_eff_lattice,
                                                       double D_mean_lattice, double porosity, double mean_d_nm,
                                                       const om_diff_params* params, om_structure_results* out) {
  if (!params || !out) return fail(OM_EINVAL, "om_structure_results_from_lattice: null pointer");
  if (!(dx_nm > 0.0) || !(porosity > 0.0) || !(porosity < 1.0) || !(mean_d_nm > 0.0))
    return fail(OM_EINVAL, "om_structure_results_from_lattice: need dx > 0, 0 < porosity < 1, mean_d > 0");
  const double dx = dx_nm * 1e-9;
  om_structure_results r{};
  r.k_m2 = k_lattice * dx * dx;                             // Eq. 15
  r.D_eff_m2s = diffusivity_to_si(D_eff_lattice, *params);  // Eq. 15
  r.D_mean_m2s = diffusivity_to_si(D_mean_lattice, *params);
  if (D_eff_lattice > 0.0) {
    r.tortuosity = porosity * D_mean_lattice / D_eff_lattice;               // Eq. 16
    r.alpha = std::log(r.D_eff_m2s / r.D_mean_m2s) / std::log(porosity);  // Sec. 4.2
  } else {
    r.tortuosity = INFINITY;
    r.alpha = NAN;
  }
  const double d = mean_d_nm * 1e-9;
  r.k_kc_m2 = (d * d / 180.0) * porosity * porosity * porosity / ((1.0 - porosity) * (1.0 - porosity));  // Eq. 17
  *out = r;
  return OM_OK;
}

extern "C" om_status om_bruggeman_fit(int64_t n, const double* porosity, const double* D_eff_m2s,
                                      const double* D_mean_m2s, double* alpha) {
  if (n < 1 || !porosity || !D_eff_m2s || !D_mean_m2s || !alpha)
    return fail(OM_EINVAL, "om_bruggeman_fit: need n >= 1 and four arrays");
  double sxy = 0.0, sxx = 0.0;
  for (int64_t k = 0; k < n; ++k) {
    if (!(porosity[k] > 0.0) || !(porosity[k] < 1.0) || !(D_eff_m2s[k] > 0.0) || !(D_mean_m2s[k] > 0.0))
      return fail(OM_EINVAL, "om_bruggeman_fit: porosities in (0, 1) and positive diffusivities");
    const double x = std::log(porosity[k]);
    sxy += x * std::log(D_eff_m2s[k] / D_mean_m2s[k]);
    sxx += x * x;
  }
  *alpha = sxy / sxx;
  return OM_OK;
}

extern "C" om_status om_apparent_permeability(double k_m2, double D_eff_m2s, double mu_Pa_s, double p_Pa,
                                              double* k_app_m2, double* f_c) {
  if (!(k_m2 > 0.0) || !(D_eff_m2s >= 0.0) || !(mu_Pa_s > 0.0) || !(p_Pa > 0.0))
    return fail(OM_EINVAL, "om_apparent_permeability: need k > 0, D_eff >= 0, mu > 0, p > 0");
  const double fc = 1.0 + D_eff_m2s * mu_Pa_s / (k_m2 * p_Pa);  // Eq. 26
  if (f_c) *f_c = fc;
  if (k_app_m2) *k_app_m2 = k_m2 * fc;
  return OM_OK;
}

extern "C" om_status om_slip_correction_factors(double k_m2, double porosity, double D_eff_m2s, double T_K,
                                                double M_kg_per_mol, double mu_Pa_s, double p_Pa,
                                                om_slip_corrections* out) {
  if (!out) return fail(OM_EINVAL, "om_slip_correction_factors: null pointer");
  if (!(k_m2 > 0.0) || !(porosity > 0.0) || !(porosity <= 1.0) || !(D_eff_m2s >= 0.0) || !(T_K > 0.0) ||
      !(M_kg_per_mol > 0.0) || !(mu_Pa_s > 0.0) || !(p_Pa > 0.0))
    return fail(OM_EINVAL, "om_slip_correction_factors: need k, porosity, T, M, mu, p > 0, porosity <= 1, D_eff >= 0");
  constexpr double kR = 8.314462618;             // J / (mol K)
  constexpr double kPi = 3.14159265358979323846;
  constexpr double kPsi = 6894.757293168361;      // Pa per psi
  constexpr double kMilliDarcy = 9.869233e-16;    // m^2 per mD
  om_slip_corrections c{};
  c.lambda_m = (mu_Pa_s / p_Pa) * std::sqrt(kPi * kR * T_K / (2.0 * M_kg_per_mol));  // Eq. 29
  const double k_md = k_m2 / kMilliDarcy;
  c.r_m = 8.886e-2 * std::sqrt(k_md / porosity) * 1e-6;  // Eq. 30: micrometres from mD (sqrt(8 k / eps))
  c.Kn = c.lambda_m / c.r_m;
  c.dgm = 1.0 + D_eff_m2s * mu_Pa_s / (k_m2 * p_Pa);  // Eq. 26
  c.klinkenberg = 1.0 + 4.0 * c.Kn;                   // Eqs. 18-19, c = 1
  const double alpha = 1.358 / (1.0 + 0.170 * std::pow(c.Kn, -0.4348));  // Eq. 21
  c.beskok_civan = (1.0 + alpha * c.Kn) * (1.0 + 4.0 * c.Kn / (1.0 + c.Kn));  // Eq. 20, b = -1
  const double p_psi = p_Pa / kPsi;
  c.heid = 1.0 + 11.419 * std::pow(k_md, -0.39) / p_psi;  // Table 1 with Eq. 18
  c.jones_owens = 1.0 + 12.639 * std::pow(k_md, -0.33) / p_psi;
  c.sampath_keighin = 1.0 + 13.85 * std::pow(k_md / porosity, -0.53) / p_psi;
  c.florence = 1.0 + 32.766 * std::pow(k_md / porosity, -0.5) / p_psi;
  *out = c;
  return OM_OK;
}
