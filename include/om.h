/*
 * om.h -- C ABI of the GB300 pore-scale transport library.
 *
 * Method: Chen, Kang, Zhang & Tao, "Lattice Boltzmann prediction of transport
 * properties in reconstructed nanostructures of organic matters in shales"
 * (arXiv:1410.1921).  The library reconstructs an organic-matter nanostructure
 * by random pore-sphere placement (Sec. 2), labels its transport pores and
 * local pore size (Sec. 4.1), runs the D3Q19 MRT flow solve (Sec. 3.1,
 * App. A) for the intrinsic permeability (Eq. 13) and the BGK Knudsen
 * diffusion solve (Sec. 3.2, Eqs. 10-12) for the effective diffusivity
 * (Eq. 14) and tortuosity (Eq. 16), and forms the apparent permeability
 * (Eq. 26).  All heavy steps run as CUDA kernels on the current device.
 *
 * Conventions for every entry point
 *  - Voxel (x, y, z) of an nx*ny*nz box is element (x*ny + y)*nz + z.  x is
 *    the flow / diffusion direction; y and z are periodic (Sec. 3.3).
 *  - A mask byte is 1 for pore, 0 for solid.
 *  - Buffers are owned by the caller.  "host" buffers are ordinary CPU
 *    memory; "device" buffers are CUDA device memory of the current device.
 *    The library allocates its own scratch and frees it before returning,
 *    except for the solver objects, which own their memory until
 *    om_*_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  *_dev calls enqueue work on it; those that return host
 *    scalars synchronise it before returning.
 *  - Every call returns an om_status.  On anything but OM_OK the outputs are
 *    undefined, except OM_ENOTCONVERGED (step cap reached), which fills
 *    every output from the last convergence check.  om_last_error() gives a
 *    message for the calling thread's most recent failure.
 *  - Scalars are SI unless the name says otherwise (nm, lattice units).
 */
#ifndef OM_H
#define OM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  OM_OK = 0,
  OM_EINVAL = 1,         /* bad argument (sizes, pointers, parameters) */
  OM_ENOMEM = 2,         /* device or host allocation failed */
  OM_ECUDA = 3,          /* a CUDA call failed; see om_last_error() */
  OM_EINFEASIBLE = 4,    /* reconstruction: trial cap hit before the porosity */
  OM_ENOPERC = 5,        /* no transport pore spans x = 0 .. nx-1; flow: or no
                          * lattice link crosses the periodic x boundary */
  OM_ENOTCONVERGED = 6,  /* step cap hit; outputs hold the last check */
  OM_ETIMEOUT = 7        /* a bounded device wait gave up */
} om_status;

/* Lattice box: nx*ny*nz voxels of edge dx_nm.  Limits: nx <= 1024,
 * ny, nz <= 2048. */
typedef struct {
  int32_t nx, ny, nz;
  double dx_nm;
} om_domain;

/* Pore-sphere placement (Sec. 2).  dist 0: diameter ~ Normal(mean_d_nm,
 * sd_d_nm) clipped to [dmin_nm, dmax_nm]; dist 1: Uniform(mean_d_nm -
 * sd_d_nm, mean_d_nm + sd_d_nm), the paper's law with sd_d_nm = 15.
 * overlap_tol is xi, p_overlap is p0; max_trials caps candidate draws. */
typedef struct {
  double mean_d_nm, sd_d_nm, dmin_nm, dmax_nm;
  int32_t dist;
  double porosity, overlap_tol, p_overlap;
  int64_t max_trials;
} om_recon_params;

/* population storage; arithmetic is FP64 for OM_F64, FP32 otherwise */
enum { OM_F64 = 0, OM_F32 = 1, OM_F16DEV = 2, OM_BF16DEV = 3 };
/* local pore size definitions */
enum { OM_PORE_CHORD13 = 0, OM_PORE_MIS = 1 };

/* D3Q19 flow (Sec. 3.1): relaxation time tau (Eq. 8), body force along x in
 * lattice units, convergence when sum|du_x| / sum|u_x| over check_every
 * steps drops below conv_tol.  Single- and half-precision solves store their
 * populations as deviations from w_i until that change falls below 1e-4,
 * then as deviations from w_i (1 + rho_ref(node)) with the per-node
 * reference moved to the node's density every check window (the velocity,
 * a small difference of populations that also carry the local density
 * deviation, keeps its precision; see flow_core.cuh). */
typedef struct {
  double tau, body_force, conv_tol;
  int32_t check_every;
  int64_t max_steps;
  int32_t precision;
  /* sweep launch variant, the same arithmetic in every one: -1 = time them
   * all at creation and keep the fastest per parity (solvers whose node
   * count lies in the same power-of-two octave as one timed before in this
   * process, with the same precision and device, reuse its choice); 0..9 =
   * force one (0/1 one thread per node without/with a register cap, 2/3 the
   * same on a resident grid striding over nodes, 4 a tighter cap, 5 the
   * resident grid two nodes deep with the next node's column-map words
   * prefetched, 6 even steps two consecutive nodes per thread with vector
   * loads and stores, odd steps as 0; 7/8/9 odd steps from the per-node
   * neighbour records, one thread per node / capped / on a resident grid,
   * even steps as 6; 10/11/12 odd steps from the records holding only the
   * populations across the collision, uncapped / capped / capped tighter,
   * even steps as 6); larger values clamp to 12.  A batch (om_batch_create)
   * takes 0..3: 0/1 one thread per node without/with a register cap, 2 as 1
   * with each structure large enough for a group of its own in the forms
   * of 2 (odd) and 6 (even), 3 as 1 with each such structure in this
   * solver's own sweeps, the variants tuned for its size (the diffusion
   * takes 0, 1 and 3) */
  int32_t variant;
  /* OM_DRIVE_FORCE: body_force along x, x periodic.  OM_DRIVE_PRESSURE
   * (Sec. 3.3): no force, x not periodic, densities 1 + delta_rho/2 and
   * 1 - delta_rho/2 on the node layers x = 0 and x = nx-1 by Guo's
   * non-equilibrium extrapolation (u_b = 2 u(b1) - u(b2) from the two inward
   * neighbours; u(b1) without b2; the rest equilibrium without b1); needs
   * nx >= 4 and 0 < |delta_rho| < 0.1.  k_lattice = nu <u_x> (nx - 1) /
   * (delta_rho / 3), <u_x> averaged over the voxels of the layers 1..nx-2,
   * on which the convergence test is also taken.  Batches accept only
   * OM_DRIVE_FORCE. */
  int32_t drive;
  double delta_rho;
  /* population layout of om_solve_permeability: OM_LAYOUT_SPARSE (the
   * fluid-node-only storage of the node set), OM_LAYOUT_DENSE (every voxel of
   * the box stored, neighbours by address arithmetic and the node mask;
   * FP64 or FP32 with the body force), or OM_LAYOUT_AUTO: where the dense
   * layout applies and the nodes fill at least half the box, the faster of
   * the two over one even + odd pair on this structure, else sparse.  Both
   * give the same update per node and step.  The solver objects
   * (om_flow_create, batches) use the sparse layout and refuse
   * OM_LAYOUT_DENSE. */
  int32_t layout;
} om_flow_params;

enum { OM_DRIVE_FORCE = 0, OM_DRIVE_PRESSURE = 1 };
enum { OM_LAYOUT_AUTO = 0, OM_LAYOUT_SPARSE = 1, OM_LAYOUT_DENSE = 2 };

/* Knudsen diffusion (Sec. 3.2): temperature, molar mass, reference pore
 * size and relaxation time of Eq. 12, inlet/outlet concentrations.
 * Convergence: every check_every steps both sum|dC| / sum|C| and the relative
 * change of the total flux sum J_x drop below conv_tol.  lattice: 7 (D3Q7,
 * c_s^2 = 1/4) or 19 (the paper's D3Q19 with the flow's velocities and
 * weights, c_s^2 = 1/3); D_L = c_s^2 (tau_g - 1/2).  Batches take 7 only. */
typedef struct {
  double T_K, M_kg_per_mol, d_ref_nm, tau_ref, c_in, c_out, conv_tol;
  int32_t check_every;
  int64_t max_steps;
  int32_t precision;
  int32_t variant; /* launch variant, -1 = autotune (see diff.cu; larger values clamp to the last) */
  int32_t lattice;
  /* OM_ACCEL_EXTRAPOLATE (not in the paper): om_diff_solve and
   * om_batch_solve restart the iteration from an extrapolated state when the
   * decay of the concentration change has settled on one mode: after three
   * consecutive check windows whose ratios rho = sum|dC| / sum|dC|_previous
   * agree to 2 % of 1 - rho, every node's concentration moves by
   * dC rho / (1 - rho) (dC its change over the last window; the stored
   * non-equilibrium parts are kept).  The LB then iterates on to the same
   * convergence test, so the fixed point and the test are those of the
   * plain solve.  OM_ACCEL_NONE: the plain iteration. */
  int32_t accel;
  /* population layout of om_solve_knudsen (see om_flow_params.layout; the
   * dense layout takes FP64 or FP32 and the D3Q7 lattice) */
  int32_t layout;
} om_diff_params;

enum { OM_ACCEL_NONE = 0, OM_ACCEL_EXTRAPOLATE = 1 };

typedef struct {
  int64_t steps;        /* LB steps taken */
  int64_t n_nodes;      /* lattice nodes (transport voxels) updated per step */
  double rel_change;    /* last convergence measure */
  double mass;          /* flow: sum of (rho - 1); diffusion: sum of C */
  double seconds;       /* wall time of the solve on the stream */
  double mlups;         /* n_nodes * steps / seconds / 1e6 */
} om_run_info;

/* ---------------------------------------------------------------- structure */

/* Sec. 2: place pore spheres with SplitMix64 stream `seed` until the pore
 * fraction reaches params->porosity.  mask: host, N bytes, written.
 * porosity_out: achieved porosity; n_spheres_out: accepted spheres.
 * Returns OM_EINFEASIBLE when max_trials draws do not reach the porosity. */
om_status om_reconstruct(uint64_t seed, om_domain d, const om_recon_params* params, uint8_t* mask,
                         double* porosity_out, int64_t* n_spheres_out);
/* as om_reconstruct, mask in device memory */
om_status om_reconstruct_dev(uint64_t seed, om_domain d, const om_recon_params* params,
                             uint8_t* mask_dev, double* porosity_out, int64_t* n_spheres_out,
                             void* stream);

/* Sec. 4.1: 18-neighbour connected-phase labelling (the D3Q19 links),
 * periodic in y and z.  labels (nullable): int32 N, the smallest voxel index
 * of the voxel's component, -1 in solid.  transport (nullable): uint8 N, 1 on
 * pores of components that touch both x = 0 and x = nx-1.
 * connectivity_out: #transport / #pore (0 when there is no pore).
 * Host buffers. */
om_status om_label_connectivity(const uint8_t* mask, om_domain d, int32_t* labels,
                                uint8_t* transport, double* connectivity_out);
om_status om_label_connectivity_dev(const uint8_t* mask_dev, om_domain d, int32_t* labels_dev,
                                    uint8_t* transport_dev, double* connectivity_out, void* stream);
/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory -- a process whose GPU memory is held by
 * another allocator (a framework's caching pool), or a service that fixes its
 * memory plan at start-up and cannot take cudaMalloc/cudaFree (and their
 * device-wide synchronisation and failure modes) later on.
 * Same results as om_label_connectivity_dev; it calls no cudaMalloc,
 * cudaFree or allocating routine.  labels_dev (int32 N) is required;
 * transport_dev nullable; device buffers owned by the caller.  Its scratch
 * is a static device array of 4 MiB + 256 B that every GPU loading the
 * library holds until exit, which limits the box to 2^24 voxels (larger ->
 * OM_EINVAL).  The first call on a device (with it current) looks up the
 * array's device address and keeps it for that CUDA context; a call under
 * another context (after a device reset, or with a caller-made context
 * current) looks it up again.  Make the first call on a device, and in each
 * new context, before any stream capture.
 * All calls share the array: calls that overlap on the GPU race. */
om_status om_label_connectivity_noalloc(const uint8_t* mask_dev, om_domain d, int32_t* labels_dev,
                                        uint8_t* transport_dev, double* connectivity_out, void* stream);

/* Local pore diameter in nm, 0 in solid.
 * mode OM_PORE_CHORD13 (Sec. 4.1): mean over 3 axis, 6 face-diagonal and 4
 *   body-diagonal directions of the all-pore line length through the voxel
 *   (wrapping in y, z, stopping at the x faces); witness (nullable) int32
 *   13*N, the cell count per direction (direction-major).
 * mode OM_PORE_MIS: diameter of the largest inscribed pore ball containing
 *   the voxel, d = dx * max(2 sqrt(r2(c)) - 1) over centres c whose ball
 *   (|v - c|^2 < r2(c), r2 = squared distance to the nearest solid voxel)
 *   holds v; witness (nullable) int32 N holds r2.  OM_EINVAL if the mask
 *   has no solid voxel.
 * Host buffers. */
om_status om_local_pore_diameter(const uint8_t* mask, om_domain d, int32_t mode, float* d_nm,
                                 int32_t* witness);
om_status om_local_pore_diameter_dev(const uint8_t* mask_dev, om_domain d, int32_t mode,
                                     float* d_nm_dev, int32_t* witness_dev, void* stream);

/* ---------------------------------------------------------------- solves */

/* Intrinsic permeability (Eq. 13) of the transport pores of `mask` (host,
 * N bytes): D3Q19 flow, halfway bounce-back at walls, periodic in y and z,
 * to convergence, driven as params->drive says: by params->body_force along
 * x with x periodic (k_lattice = nu <u_x> / g, <.> over all N voxels), or by
 * the pressure ends of om_flow_params.drive.  k_m2 = k_lattice * dx^2
 * (Eq. 15).  ux_out (nullable, host float N): u_x, 0 off the node set.
 * info (nullable).  OM_ENOPERC when no pore spans the box, or, with the
 * body-force drive, when no D3Q19 link joins a node at x = nx-1 to one at
 * x = 0: the periodic x boundary is then a wall, the steady net flux is
 * zero, and k_m2 and k_lattice are set to 0 without stepping. */
om_status om_solve_permeability(const uint8_t* mask, om_domain d, const om_flow_params* params,
                                double* k_m2, double* k_lattice, om_run_info* info, float* ux_out);

/* Effective Knudsen diffusivity (Eq. 14) and tortuosity (Eq. 16) of the
 * transport pores of `mask` with local pore sizes d_nm (host float N, nm):
 * D3Q7 BGK with tau_g from Eq. 12, fixed c_in / c_out on the half links
 * x = -1/2 and nx - 1/2, bounce-back walls, periodic y, z, to convergence.
 * D_eff_m2s = D_eff,L * D_K(d_ref) / D_L(tau_ref) (Eqs. 11, 15);
 * tortuosity = porosity * mean(D_K over nodes) / D_eff.  c_out (nullable,
 * host float N): concentration, 0 off the node set.  info nullable. */
om_status om_solve_knudsen(const uint8_t* mask, const float* d_nm, om_domain d,
                           const om_diff_params* params, double* D_eff_m2s, double* tortuosity,
                           om_run_info* info, float* c_out);

/* A structure's results in physical units from its lattice solves (the
 * arithmetic behind om_solve_permeability / om_solve_knudsen, for callers
 * that solve on the device objects or in batches):
 *   k_m2        Eq. 15: k_lattice dx^2;
 *   D_eff_m2s   Eq. 15 with the time step fixed by the reference pore
 *               (Eqs. 11-12): D_eff_lattice D_K(d_ref) / (c_s^2 (tau_ref - 1/2)),
 *               c_s^2 of params->lattice (1/4 on D3Q7, 1/3 on D3Q19);
 *   D_mean_m2s  the same conversion of D_mean_lattice, the mean lattice
 *               diffusivity over the transport nodes: the mean local Knudsen
 *               diffusivity D of Eqs. 11-12 over them;
 *   tortuosity  Eq. 16: porosity D / D_eff (porosity: pore voxels over all);
 *   alpha       Sec. 4.2: the exponent of D_eff = D porosity^alpha for this
 *               structure, ln(D_eff / D) / ln(porosity);
 *   k_kc_m2     Eq. 17 (Kozeny-Carman, A = d^2 / 180) with d = mean_d_nm.
 * Non-positive D_eff_lattice gives tortuosity +inf and alpha NaN; k_lattice
 * may be 0.  OM_EINVAL for dx_nm <= 0, porosity outside (0, 1) or a
 * non-positive mean_d_nm. */
typedef struct {
  double k_m2, D_eff_m2s, D_mean_m2s, tortuosity, alpha, k_kc_m2;
} om_structure_results;
om_status om_structure_results_from_lattice(double dx_nm, double k_lattice, double D_eff_lattice,
                                            double D_mean_lattice, double porosity, double mean_d_nm,
                                            const om_diff_params* params, om_structure_results* out);

/* Sec. 4.2: the Bruggeman exponent alpha of D_eff = D porosity^alpha fitted
 * over n structures, least squares on ln(D_eff / D) = alpha ln(porosity)
 * (a line through the origin).  Host arrays of n values; OM_EINVAL if n < 1
 * or any value is non-positive or a porosity is not below 1. */
om_status om_bruggeman_fit(int64_t n, const double* porosity, const double* D_eff_m2s, const double* D_mean_m2s,
                           double* alpha);

/* Eq. 26: k_app = k (1 + D_eff mu / (k p)); f_c the bracket. */
om_status om_apparent_permeability(double k_m2, double D_eff_m2s, double mu_Pa_s, double p_Pa,
                                   double* k_app_m2, double* f_c);

/* The correction factors f_c (k_app = k f_c) of Sec. 4.4 for a medium of
 * intrinsic permeability k_m2, porosity and effective Knudsen diffusivity
 * D_eff_m2s, for a gas of molar mass M at temperature T, pressure p and
 * viscosity mu (SI units):
 *   lambda_m     Eq. 29, lambda = (mu / p) sqrt(pi R T / (2 M));
 *   r_m          Eq. 30, r = 8.886e-2 (k / eps)^0.5 with k in mD and r in
 *                micrometres (the capillary-bundle radius sqrt(8 k / eps);
 *                the nm printed with Eq. 30 is read as a misprint);
 *   Kn           lambda / r;
 *   dgm          Eq. 26 (the dusty-gas form of this method);
 *   klinkenberg  Eqs. 18-19 with c = 1: 1 + 4 Kn;
 *   beskok_civan Eq. 20 with Eq. 21 and b = -1;
 *   heid, jones_owens, sampath_keighin, florence: Eq. 18 with the slippage
 *                factors of Table 1 (b_k in psi from k in mD; Florence et al.
 *                with the membrane beta = 32.766).
 * 1 mD = 9.869233e-16 m^2, 1 psi = 6894.757293168361 Pa.  OM_EINVAL unless
 * k, porosity, T, M, mu, p > 0, porosity <= 1 and D_eff >= 0. */
typedef struct {
  double lambda_m, r_m, Kn;
  double dgm, klinkenberg, beskok_civan;
  double heid, jones_owens, sampath_keighin, florence;
} om_slip_corrections;
om_status om_slip_correction_factors(double k_m2, double porosity, double D_eff_m2s, double T_K, double M_kg_per_mol,
                                     double mu_Pa_s, double p_Pa, om_slip_corrections* out);

/* ---------------------------------------------------------------- node set and solver objects
 * The hot loop.  A node set holds the transport voxels in lexicographic order
 * with a per-column bit map and prefix count, from which every neighbour's
 * node index is computed on the fly.  Solver objects own the populations of
 * one model on one node set and advance them with fused collide-stream
 * kernels in the AA pattern (one read and one write per population and
 * step).  All pointers device, all work on `stream`. */
typedef struct om_nodeset om_nodeset;
typedef struct om_flow om_flow;
typedef struct om_diff om_diff;

/* nodes_dev: uint8 N, 1 on lattice nodes (normally the transport mask). */
om_status om_nodeset_create(const uint8_t* nodes_dev, om_domain d, void* stream, om_nodeset** out);
om_status om_nodeset_count(const om_nodeset* ns, int64_t* n_nodes);
/* voxel index of every node (int64 n_nodes, device), for gathers */
om_status om_nodeset_voxels(const om_nodeset* ns, int64_t* voxel_dev, void* stream);
om_status om_nodeset_destroy(om_nodeset* ns);

/* f initialised to the rest state f_i = w_i (rho = 1, u = 0). */
om_status om_flow_create(const om_nodeset* ns, const om_flow_params* params, void* stream,
                         om_flow** out);
/* advance nsteps LB steps (Sec. 3.1, steps 1-5 per step) */
om_status om_flow_step(om_flow* fl, int64_t nsteps, void* stream);
/* Observables of the current state (FP64, node order): out[0] sum u_x,
 * out[1] sum |u_x - u_x at the previous observe|, out[2] sum |u_x| (the
 * pressure drive sums these three over the layers x = 1..nx-2), out[3]
 * sum (rho - 1) over all nodes.  Host out, synchronises. */
om_status om_flow_observe(om_flow* fl, double* out, void* stream);
/* Run to convergence (om_flow_params) from the current state.  Body-force
 * drive: OM_ENOPERC (k_lattice = 0, no steps) when no lattice link crosses
 * the periodic x boundary: the net flux then vanishes at steady state. */
om_status om_flow_solve(om_flow* fl, double* k_lattice, om_run_info* info, void* stream);
/* populations at the current time in the dense layout f[i*N + voxel],
 * i in the order of the App. A transformation matrix, 0 off the node set.
 * f_dev: double 19*N. */
om_status om_flow_get_populations(const om_flow* fl, double* f_dev, void* stream);
om_status om_flow_set_populations(om_flow* fl, const double* f_dev, void* stream);
/* velocity u = j + g/2 (Eq. 9 with the half force), float 3*N, 0 off nodes */
om_status om_flow_get_velocity(const om_flow* fl, float* u_dev, void* stream);
om_status om_flow_time(const om_flow* fl, int64_t* t);
om_status om_flow_destroy(om_flow* fl);

/* d_nm_dev: float N local pore size (nm) for Eq. 12; g initialised to
 * a_i C_lin(x), the linear profile between c_in and c_out. */
om_status om_diff_create(const om_nodeset* ns, const float* d_nm_dev, const om_diff_params* params,
                         void* stream, om_diff** out);
om_status om_diff_step(om_diff* df, int64_t nsteps, void* stream);
/* out[0] sum J_x (J = (1 - omega/2) sum e_x g), out[1] sum |C - C_prev|,
 * out[2] sum |C|, out[3] sum C, out[4] sum D_L over nodes.  Synchronises. */
om_status om_diff_observe(om_diff* df, double* out, void* stream);
om_status om_diff_solve(om_diff* df, double* D_eff_lattice, om_run_info* info, void* stream);
/* populations in the dense layout g[i*N + voxel], order rest,+x,-x,+y,-y,+z,-z */
om_status om_diff_get_populations(const om_diff* df, double* g_dev, void* stream);
om_status om_diff_set_populations(om_diff* df, const double* g_dev, void* stream);
/* concentration C (float N) and flux J_x (float N), 0 off nodes; either nullable */
om_status om_diff_get_fields(const om_diff* df, float* c_dev, float* jx_dev, void* stream);
om_status om_diff_time(const om_diff* df, int64_t* t);
om_status om_diff_destroy(om_diff* df);

/* ---------------------------------------------------------------- two-level warm start
 * Not in the paper: an initial state for a fine diffusion solve from a solve
 * on the structure coarsened 2x per axis; the fine LB then iterates to its
 * own convergence test, so the result stays the fine method's.
 * om_coarse_domain: the coarse domain, ceil(n/2) per axis, voxel 2 dx.
 * om_coarsen2_dev: coarse voxel (X, Y, Z) covers fine voxels 2X..2X+1 per
 * axis (clipped at an odd edge); nodes_c = 1 where at least half of those
 * are nodes of nodes_dev; d_c = mean pore size (nm) over those nodes (0 if
 * none).  d_nm_dev and d_c_dev both NULL to skip pore sizes.  uint8 / float
 * arrays of N (fine) and N_c (coarse) voxels, device, caller-owned.
 * om_prolong2_dev: fine concentration c_dev (float N) from the coarse dense
 * populations g_c_dev (double q x N_c, the layout of om_diff_get_populations
 * / om_batch_get_populations): the sum over i at the covering coarse voxel
 * where nodes_c is 1, else the linear profile C_lin(x) between c_in and
 * c_out; minus C_lin when departure != 0; plus corr_dev[v * corr_stride]
 * when corr_dev is not NULL (a learned correction).
 * om_unet_pack_structure3: the network input of the refining warm start,
 * float [N][3] = (node mask, d * d_scale, extra), extra = the prolonged
 * coarse departure.  All asynchronous on stream. */
om_status om_coarse_domain(om_domain d, om_domain* dc);
om_status om_coarsen2_dev(const uint8_t* nodes_dev, const float* d_nm_dev, om_domain d, uint8_t* nodes_c_dev,
                          float* d_c_dev, void* stream);
om_status om_prolong2_dev(const double* g_c_dev, int32_t q, const uint8_t* nodes_c_dev, om_domain d, double c_in,
                          double c_out, const float* corr_dev, int64_t corr_stride, int32_t departure, float* c_dev,
                          void* stream);
om_status om_unet_pack_structure3(const uint8_t* mask_dev, const float* d_nm_dev, double d_scale,
                                  const float* extra_dev, int64_t n, float* x_dev, void* stream);
/* Fine u_x (float N) from the coarse flow's dense populations f_c_dev (double
 * 19 x N_c, body force body_force_c along x on the coarse lattice):
 * scale * (sum_i e_ix f_i + body_force_c / 2) at the covering coarse voxel
 * where nodes_c is 1, else 0 -- the flow's initial velocity for
 * om_batch_init_fields / om_flow_init_velocity. */
om_status om_prolong2_ux_dev(const double* f_c_dev, const uint8_t* nodes_c_dev, om_domain d, double body_force_c,
                             double scale, float* ux_dev, void* stream);

/* ---------------------------------------------------------------- checkpoint and resume
 * A solver's evolving state -- its populations exactly as stored, the
 * diffusion's per-node reference concentration (FP32 and 16-bit storage),
 * the previous observables of its convergence test and its step counter --
 * as an opaque host byte image of *_state_size bytes.  Loaded into a solver
 * of the same node set, kind, precision and lattice (else OM_EINVAL, nothing
 * changed), the solver continues bit for bit as the saved one would have:
 * long diffusion runs can stop and resume.  host: caller-owned host memory
 * (pinned or pageable) of at least the size given; both calls synchronise
 * the stream. */
om_status om_flow_state_size(const om_flow* fl, int64_t* bytes);
om_status om_flow_save_state(const om_flow* fl, void* host, int64_t bytes, void* stream);
om_status om_flow_load_state(om_flow* fl, const void* host, int64_t bytes, void* stream);
om_status om_diff_state_size(const om_diff* df, int64_t* bytes);
om_status om_diff_save_state(const om_diff* df, void* host, int64_t bytes, void* stream);
om_status om_diff_load_state(om_diff* df, const void* host, int64_t bytes, void* stream);

/* ---------------------------------------------------------------- batches
 * Many independent structures (the paper's 150 reconstructions) solved
 * together.  The structures not yet converged are packed into groups whose
 * sweep footprint fits in L2 (at most 32 structures each); one launch per LB
 * step advances a whole group over a work list of 256-node tiles, a check
 * window runs its steps group after group from a captured CUDA graph, and a
 * structure leaves the work list when it converges.  Launch shapes (register
 * cap; one CTA per tile or a resident grid of 2-8 CTAs per SM; the large
 * structures' forms) are timed at creation.  The flow of each structure
 * enters the rebased mode (om_flow_solve) for its last decades: single
 * precision once its relative change falls below 1e-4, 16-bit storage from
 * the start.  om_batch_step replays the window graph for whole windows from
 * even times.  Both models share the parameters given; pass NULL for a
 * model that is not needed (d_nm_dev may then be NULL too).
 * nodes_dev[k]: uint8 N_k node mask (normally the transport set) of
 * doms[k]; d_nm_dev[k]: float N_k pore sizes (nm).  All device pointers. */
typedef struct om_batch om_batch;
om_status om_batch_create(int32_t n, const om_domain* doms, const uint8_t* const* nodes_dev,
                          const float* const* d_nm_dev, const om_flow_params* flow,
                          const om_diff_params* diff, void* stream, om_batch** out);
/* model 0 = flow, 1 = diffusion */
om_status om_batch_step(om_batch* b, int32_t model, int64_t nsteps, void* stream);
/* Run every structure of the model to its convergence test (as om_flow_solve
 * / om_diff_solve) from the current state.  Host arrays of n entries:
 * result = k_lattice (flow) or D_eff,L (diffusion); aux (nullable) = sum of
 * (rho - 1) (flow) or the mean lattice diffusivity over nodes (diffusion);
 * info (nullable; seconds and mlups are those of the whole batch); status
 * (nullable) = OM_OK, OM_ENOTCONVERGED or OM_ENOPERC (no nodes; flow: or
 * no link across the periodic x boundary, result 0) per structure.  Returns
 * OM_OK unless a call fails; OM_ETIMEOUT if a grid-barrier wait of a
 * persistent window gave up (see om_batch_set_window_mode; the batch's
 * state is then undefined).
 * Check windows run in one of two modes with identical results: the
 * captured graph of per-step launches, or one persistent cooperative launch
 * per group whose blocks meet at a grid barrier between steps (every wait
 * bounded, ~2 s).  Unless a mode was set, the first two whole windows of the
 * first solve are run one in each mode, timed, and the faster is kept. */
om_status om_batch_solve(om_batch* b, int32_t model, double* result, double* aux, om_run_info* info,
                         int32_t* status, void* stream);
/* Window mode of om_batch_solve for a model: -1 = time both (default), 0 =
 * graph of per-step launches, 1 = persistent launches.  om_batch_step always
 * replays the graph. */
om_status om_batch_set_window_mode(om_batch* b, int32_t model, int32_t mode);
/* Self-test of the bounded grid barrier: one cooperative launch of `blocks`
 * 256-thread blocks (at most what fits on the GPU at once, else OM_EINVAL)
 * meets `rounds` times at the barrier of the persistent windows, which is
 * told to expect `blocks + extra` arrivals; each wait gives up after
 * max_polls polls of ~100 ns.  *status = OM_OK when every barrier completed,
 * OM_ETIMEOUT when a wait gave up (always so for extra > 0: the barrier can
 * never complete, and the launch still ends).  Synchronises. */
om_status om_barrier_selftest(int32_t blocks, int32_t rounds, int32_t extra, int64_t max_polls, int32_t* status,
                              void* stream);
/* populations of structure `item` in the dense layout of om_flow_get_populations /
 * om_diff_get_populations (double q*N_k, device) */
om_status om_batch_get_populations(om_batch* b, int32_t model, int32_t item, double* dense_dev,
                                   void* stream);
/* the field of structure `item` in its voxel layout (float N_item, device;
 * 0 off the node set): model 0 u_x = sum_i e_ix f_i + g/2 (as
 * om_flow_get_velocity's x component), model 1 the concentration C (as
 * om_diff_get_fields) -- the solved fields a learned warm start trains on */
om_status om_batch_get_field(om_batch* b, int32_t model, int32_t item, float* field_dev, void* stream);
om_status om_batch_set_populations(om_batch* b, int32_t model, int32_t item,
                                   const double* dense_dev, void* stream);
/* back to the initial state (rest / linear profile) at time 0 */
om_status om_batch_reset(om_batch* b, int32_t model, void* stream);
/* warm start of structure `item` from a device field in its voxel layout,
 * element v at field[v * stride]: flow f = f_eq(1, (scale * field, 0, 0));
 * diffusion g = a_i C, C = field (+ C_lin(x) when from_linear != 0).  The
 * batch must be at an even time (after create, reset or a solve). */
om_status om_batch_init_fields(om_batch* b, int32_t model, int32_t item, const float* field_dev,
                               int64_t stride, double scale, int32_t from_linear, void* stream);
om_status om_batch_destroy(om_batch* b);

/* ---------------------------------------------------------------- learned warm start
 * A 3-D U-Net predicting the steady fields from the structure, trained on
 * fields the LB solves produce (the paper has no counterpart: its solves
 * start cold; the LB still runs to the same convergence test afterwards).
 * `levels` levels with channels ch[0..levels-1] (multiples of 16), two
 * 3x3x3 convolutions + ReLU per level, 2x average pooling down, nearest 2x
 * upsampling and skip concatenation up, a 1x1 head.  The 3x3x3
 * convolutions (forward and data gradient) run on the 5th-generation tensor
 * cores (tcgen05.mma, BF16 operands staged by TMA, FP32 accumulator in
 * tensor memory); FP32 master weights and Adam.  om_unet_forward and
 * om_unet_backward synchronise the stream and return OM_ETIMEOUT if a
 * convolution's bounded wait gave up (the result is then not written).
 * Tensors are FP32 NDHWC on the device: x [B][D][H][W][in_ch] (in_ch <= 16),
 * targets/outputs [B][D][H][W][out_ch], mask [B][D][H][W] (loss over
 * voxels with mask != 0).  D, H, W must be multiples of 2^(levels-1).
 * Parameters are one flat FP32 vector: per level (encoder, then decoder from
 * the bottom) W[27][c_in][c_out] and b[c_out], then the head W[c0][out], b.
 * om_unet_create draws the convolution weights He-uniform from a SplitMix64
 * stream of `seed` and sets biases and the head to zero (the first output is
 * 0: the cold start). */
typedef struct om_unet om_unet;
om_status om_unet_create(int32_t in_ch, int32_t out_ch, int32_t levels, const int32_t* ch, uint64_t seed,
                         om_unet** out);
om_status om_unet_param_count(const om_unet* u, int64_t* n);
om_status om_unet_get_params(const om_unet* u, float* dst_dev, void* stream);
om_status om_unet_set_params(om_unet* u, const float* src_dev, void* stream);
/* gradients of the last om_unet_backward / om_unet_train_step */
om_status om_unet_get_grads(const om_unet* u, float* dst_dev, void* stream);
om_status om_unet_forward(om_unet* u, const float* x, int32_t B, int32_t D, int32_t H, int32_t W, float* y,
                          void* stream);
/* forward + masked mean-squared error + gradients (no update); loss_out host */
om_status om_unet_backward(om_unet* u, const float* x, const float* target, const uint8_t* mask, int32_t B,
                           int32_t D, int32_t H, int32_t W, double* loss_out, void* stream);
/* om_unet_backward then one Adam step (beta 0.9 / 0.999, eps 1e-8) */
om_status om_unet_train_step(om_unet* u, const float* x, const float* target, const uint8_t* mask, int32_t B,
                             int32_t D, int32_t H, int32_t W, float lr, double* loss_out, void* stream);
om_status om_unet_destroy(om_unet* u);

/* U-Net input from a structure: x[v][0] = mask != 0, x[v][1] = d_nm[v] *
 * d_scale (float [N][2], device). */
om_status om_unet_pack_structure(const uint8_t* mask_dev, const float* d_nm_dev, int64_t n, double d_scale,
                                 float* x_dev, void* stream);

/* Warm starts for the solver objects from a device field in the voxel layout
 * read with a stride (element v at field[v * stride]); values off the node
 * set are ignored and the time is reset to 0.
 * flow: f_i = f_eq(rho = 1, u = (scale * field, 0, 0));
 * diffusion: g_i = a_i C with C = field, or C = C_lin(x) + field when
 * from_linear != 0. */
om_status om_flow_init_velocity(om_flow* fl, const float* ux_dev, int64_t stride, double scale, void* stream);
om_status om_diff_init_concentration(om_diff* df, const float* c_dev, int64_t stride, int32_t from_linear,
                                     void* stream);

/* ---------------------------------------------------------------- misc */
const char* om_last_error(void);
/* library version string */
const char* om_version(void);

#ifdef __cplusplus
}
#endif
#endif /* OM_H */
