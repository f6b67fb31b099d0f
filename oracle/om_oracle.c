/*
 * om_oracle.c -- plain, slow, FP64 CPU oracle for the pore-scale method of
 * Chen, Kang, Zhang & Tao, "Lattice Boltzmann prediction of transport
 * properties in reconstructed nanostructures of organic matters in shales"
 * (arXiv:1410.1921).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code, header or table with
 * the CUDA path.
 *
 * Every routine is written to be read against the paper: one loop per
 * definition, no blocking, no fusion.  All floating point is IEEE double;
 * the build passes -ffp-contract=off so no multiply-add is fused.
 *
 * Index convention: voxel (x, y, z) lives at (x*ny + y)*nz + z; x is the
 * flow / diffusion direction; y and z are periodic (Sec. 3.3).
 *
 * Parity pins (see tests/test_oracle_*.py): SplitMix64 known answers, lens
 * volume vs quadrature, reconstruction invariants, brute-force labelling /
 * chords / inscribed spheres on tiny masks, Q Q^-1 = I and the printed
 * Q^-1 table (App. A), m_eq (A1-A9) = Q f_eq, slit Poiseuille (exact),
 * square duct (series), tube (Eq. 27), mass conservation, straight-channel
 * diffusion (exact), sphere-in-cube diffusion (Sec. 3.5).  The reconstruction
 * sampler itself (diameter law, draw order, p0) is "parity unpinned" against
 * the paper: the paper prints no structure.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_EINFEASIBLE 4
#define ORC_ENOPERC 5
#define ORC_ENOTCONVERGED 6

static const double ORC_PI = 3.14159265358979323846;

static inline int64_t vidx(int x, int y, int z, int ny, int nz) {
  return ((int64_t)x * ny + y) * nz + z;
}
static inline int wrap(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

/* ======================================================================
 * 1. Random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), from
 *    its published definition.  Uniform double in [0,1) from the top 53
 *    bits.
 * ====================================================================== */
uint64_t orc_splitmix64_next(uint64_t *state) {
  uint64_t z;
  *state += 0x9E3779B97F4A7C15ULL;
  z = *state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

double orc_uniform(uint64_t *state) {
  return (double)(orc_splitmix64_next(state) >> 11) * (1.0 / 9007199254740992.0);
}

/* Pore-sphere diameter in nm.  dist 0: Normal(mean, sd) by Box-Muller
 * (two uniforms per draw, the second value discarded) clipped to
 * [dmin, dmax]; dist 1: the paper's Uniform(mean - half, mean + half) with
 * half = sd (Sec. 2: <d> +- 15 nm). */
static double orc_draw_diameter(uint64_t *st, int dist, double mean, double sd,
                                double dmin, double dmax) {
  if (dist == 1) {
    double u = orc_uniform(st);
    return (mean - sd) + (2.0 * sd) * u;
  }
  double u1 = orc_uniform(st);
  double u2 = orc_uniform(st);
  double zz = sqrt(-2.0 * log(1.0 - u1)) * cos(2.0 * ORC_PI * u2);
  double d = mean + sd * zz;
  if (d < dmin) d = dmin;
  if (d > dmax) d = dmax;
  return d;
}

/* ======================================================================
 * 2. Overlap volume of two spheres (Sec. 2, the overlap tolerance xi is the
 *    overlapped volume over a sphere's own volume).  Classical lens volume
 *    of two intersecting balls; the whole smaller ball when one contains
 *    the other; zero when they are apart.
 * ====================================================================== */
double orc_sphere_volume(double r) { return (4.0 * ORC_PI / 3.0) * (r * r * r); }

double orc_lens_volume(double r1, double r2, double dist) {
  double s = r1 + r2;
  if (dist >= s) return 0.0;
  double rmin = r1 < r2 ? r1 : r2;
  if (dist <= fabs(r1 - r2)) return orc_sphere_volume(rmin);
  double a = s - dist;
  double df = r1 - r2;
  return ORC_PI * (a * a) * (dist * dist + 2.0 * dist * s - 3.0 * (df * df)) / (12.0 * dist);
}

/* minimum-image separation in y and z, none in x (Sec. 3.3 periodicity) */
static double orc_center_distance(const double *a, const double *b, int ny, int nz) {
  double dx = a[0] - b[0];
  double dy = a[1] - b[1];
  double dz = a[2] - b[2];
  if (dy > 0.5 * ny) dy -= ny; else if (dy < -0.5 * ny) dy += ny;
  if (dz > 0.5 * nz) dz -= nz; else if (dz < -0.5 * nz) dz += nz;
  return sqrt(dx * dx + dy * dy + dz * dz);
}

/* Voxel (vx,vy,vz) lies in the ball (c, r) if its centre is within r of the
 * ball centre or of one of its periodic images shifted by -1,0,+1 periods
 * in y and in z. */
static int orc_voxel_in_ball(int vx, int vy, int vz, const double *c, double r, int ny, int nz) {
  double ddx = ((double)vx + 0.5) - c[0];
  double r2 = r * r;
  for (int ky = -1; ky <= 1; ++ky)
    for (int kz = -1; kz <= 1; ++kz) {
      double ddy = ((double)vy + 0.5) - (c[1] + (double)(ky * ny));
      double ddz = ((double)vz + 0.5) - (c[2] + (double)(kz * nz));
      double d2 = (ddx * ddx + ddy * ddy) + ddz * ddz;
      if (d2 <= r2) return 1;
    }
  return 0;
}

/* ======================================================================
 * 3. Reconstruction by random pore-sphere placement (Sec. 2, steps 1-3).
 *    spheres: caller array of 4*cap doubles (cx, cy, cz in voxel units and
 *    the radius in voxel units).  Returns ORC_EINFEASIBLE when max_trials
 *    candidate spheres have been drawn without reaching the porosity.
 * ====================================================================== */
int orc_reconstruct(uint64_t seed, int nx, int ny, int nz, double dx_nm, double mean_nm,
                    double sd_nm, double dmin_nm, double dmax_nm, int dist, double porosity,
                    double xi, double p0, int64_t max_trials, uint8_t *mask, double *spheres,
                    int64_t cap, int64_t *n_spheres, double *porosity_out, int64_t *trials_out) {
  if (nx <= 0 || ny <= 0 || nz <= 0 || dx_nm <= 0.0 || porosity <= 0.0 || porosity > 1.0)
    return ORC_EINVAL;
  int64_t N = (int64_t)nx * ny * nz;
  memset(mask, 0, (size_t)N);
  uint64_t st = seed;
  int64_t ns = 0, trials = 0, pore = 0;
  double eps = 0.0;
  while (eps < porosity) {
    if (ns >= cap) return ORC_ENOMEM;
    int must_overlap = 0;
    if (ns > 0) must_overlap = orc_uniform(&st) < p0; /* step 2: overlap required? */
    double c[3], r;
    for (;;) {
      if (trials >= max_trials) {
        *n_spheres = ns; *porosity_out = eps; *trials_out = trials;
        return ORC_EINFEASIBLE;
      }
      ++trials;
      c[0] = orc_uniform(&st) * nx;
      c[1] = orc_uniform(&st) * ny;
      c[2] = orc_uniform(&st) * nz;
      r = 0.5 * (orc_draw_diameter(&st, dist, mean_nm, sd_nm, dmin_nm, dmax_nm) / dx_nm);
      if (ns == 0) break; /* step 1: the first sphere is always placed */
      double vt = orc_sphere_volume(r);
      int touched = 0, ok = 1;
      for (int64_t s = 0; s < ns && ok; ++s) {
        const double *cs = spheres + 4 * s;
        double rs = cs[3];
        double dd = orc_center_distance(c, cs, ny, nz);
        double v = orc_lens_volume(r, rs, dd);
        if (v > 0.0) touched = 1;
        if (v / vt > xi || v / orc_sphere_volume(rs) > xi) ok = 0;
      }
      if (ok && must_overlap && !touched) ok = 0; /* step 2a */
      if (ok) break;
    }
    double *out = spheres + 4 * ns;
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = r;
    ++ns;
    /* rasterise the accepted sphere over its bounding box (y, z wrapped) */
    int x0 = (int)floor(c[0] - r) - 1, x1 = (int)ceil(c[0] + r) + 1;
    int y0 = (int)floor(c[1] - r) - 1, y1 = (int)ceil(c[1] + r) + 1;
    int z0 = (int)floor(c[2] - r) - 1, z1 = (int)ceil(c[2] + r) + 1;
    if (x0 < 0) x0 = 0;
    if (x1 > nx - 1) x1 = nx - 1;
    if (y1 - y0 + 1 > ny) { y0 = 0; y1 = ny - 1; }
    if (z1 - z0 + 1 > nz) { z0 = 0; z1 = nz - 1; }
    for (int x = x0; x <= x1; ++x)
      for (int yy = y0; yy <= y1; ++yy)
        for (int zz = z0; zz <= z1; ++zz) {
          int y = wrap(yy, ny), z = wrap(zz, nz);
          int64_t v = vidx(x, y, z, ny, nz);
          if (!mask[v] && orc_voxel_in_ball(x, y, z, c, r, ny, nz)) {
            mask[v] = 1;
            ++pore;
          }
        }
    eps = (double)pore / (double)N; /* step 3: stop once the porosity is reached */
  }
  *n_spheres = ns;
  *porosity_out = eps;
  *trials_out = trials;
  return ORC_OK;
}

/* ======================================================================
 * 4. Connected-phase labelling with the 18 neighbours of the D3Q19 lattice
 *    (Sec. 4.1).  Breadth-first search started from voxels in increasing
 *    index order, so each component's label is its smallest voxel index.
 *    Transport cells: components that contain a voxel at x = 0 and one at
 *    x = nx-1.  labels: -1 in solid.
 * ====================================================================== */
static const int N18[18][3] = {{1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},
                               {0, 0, -1}, {1, 1, 0},  {-1, 1, 0}, {1, -1, 0}, {-1, -1, 0},
                               {1, 0, 1},  {-1, 0, 1}, {1, 0, -1}, {-1, 0, -1}, {0, 1, 1},
                               {0, -1, 1}, {0, 1, -1}, {0, -1, -1}};

int orc_label18(const uint8_t *mask, int nx, int ny, int nz, int32_t *labels,
                uint8_t *transport, double *connectivity) {
  int64_t N = (int64_t)nx * ny * nz;
  int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
  if (!queue) return ORC_ENOMEM;
  for (int64_t v = 0; v < N; ++v) labels[v] = -1;
  int64_t npore = 0, ntrans = 0;
  for (int64_t s = 0; s < N; ++s) {
    if (!mask[s] || labels[s] >= 0) continue;
    int64_t head = 0, tail = 0;
    labels[s] = (int32_t)s;
    queue[tail++] = s;
    while (head < tail) {
      int64_t v = queue[head++];
      int x = (int)(v / ((int64_t)ny * nz)), y = (int)((v / nz) % ny), z = (int)(v % nz);
      for (int k = 0; k < 18; ++k) {
        int xx = x + N18[k][0];
        if (xx < 0 || xx >= nx) continue;
        int64_t w = vidx(xx, wrap(y + N18[k][1], ny), wrap(z + N18[k][2], nz), ny, nz);
        if (mask[w] && labels[w] < 0) {
          labels[w] = (int32_t)s;
          queue[tail++] = w;
        }
      }
    }
    /* does this component reach both x faces? */
    int in = 0, out = 0;
    for (int64_t q = 0; q < tail; ++q) {
      int x = (int)(queue[q] / ((int64_t)ny * nz));
      if (x == 0) in = 1;
      if (x == nx - 1) out = 1;
    }
    npore += tail;
    for (int64_t q = 0; q < tail; ++q) transport[queue[q]] = (uint8_t)(in && out);
    if (in && out) ntrans += tail;
  }
  for (int64_t v = 0; v < N; ++v)
    if (!mask[v]) transport[v] = 0;
  *connectivity = npore > 0 ? (double)ntrans / (double)npore : 0.0;
  free(queue);
  return ORC_OK;
}

/* ======================================================================
 * 5a. 13-direction chord averaging (Sec. 4.1): for each pore cell and each
 *     of 3 axis, 6 face-diagonal and 4 body-diagonal directions, the number
 *     of cells of the all-pore line through it (wrapping in y, z, stopping
 *     at the x faces, at most one period); the pore size is the mean of the
 *     13 lengths, each count times the cell's length along that direction.
 *     counts: nullable, 13*N int32 in the direction order below.
 * ====================================================================== */
static const int D13[13][3] = {{1, 0, 0},  {0, 1, 0},  {0, 0, 1},   {1, 1, 0},  {1, -1, 0},
                               {1, 0, 1},  {1, 0, -1}, {0, 1, 1},   {0, 1, -1}, {1, 1, 1},
                               {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};

static int orc_walk(const uint8_t *mask, int nx, int ny, int nz, int x, int y, int z, int ex,
                    int ey, int ez, int *returned) {
  int n = 0, cx = x, cy = y, cz = z;
  *returned = 0;
  for (;;) {
    cx += ex;
    if (cx < 0 || cx >= nx) return n;
    cy = wrap(cy + ey, ny);
    cz = wrap(cz + ez, nz);
    if (cx == x && cy == y && cz == z) { *returned = 1; return n; }
    if (!mask[vidx(cx, cy, cz, ny, nz)]) return n;
    ++n;
  }
}

void orc_chord13(const uint8_t *mask, int nx, int ny, int nz, double dx_nm, float *d_nm,
                 int32_t *counts) {
  int64_t N = (int64_t)nx * ny * nz;
  for (int64_t v = 0; v < N; ++v) {
    int x = (int)(v / ((int64_t)ny * nz)), y = (int)((v / nz) % ny), z = (int)(v % nz);
    int64_t S[3] = {0, 0, 0}; /* axis, face diagonal, body diagonal */
    for (int k = 0; k < 13; ++k) {
      int n = 0;
      if (mask[v]) {
        int ret;
        int fwd = orc_walk(mask, nx, ny, nz, x, y, z, D13[k][0], D13[k][1], D13[k][2], &ret);
        if (ret) n = 1 + fwd;
        else n = 1 + fwd + orc_walk(mask, nx, ny, nz, x, y, z, -D13[k][0], -D13[k][1], -D13[k][2], &ret);
      }
      if (counts) counts[(int64_t)k * N + v] = n;
      S[k < 3 ? 0 : (k < 9 ? 1 : 2)] += n;
    }
    if (!mask[v]) { d_nm[v] = 0.0f; continue; }
    double d = (((double)S[0] + sqrt(2.0) * (double)S[1]) + sqrt(3.0) * (double)S[2]) / 13.0;
    d_nm[v] = (float)(d * dx_nm);
  }
}

/* ======================================================================
 * 5b. Maximal inscribed sphere diameter.  r2(c): smallest squared integer
 *     distance from pore voxel c to a solid voxel (periodic in y, z; there
 *     is no solid outside the x faces).  d(v) = dx * max over pore c with
 *     |v-c|^2 < r2(c) of (2 sqrt(r2(c)) - 1).  Brute force.  r2: nullable.
 *     Returns ORC_EINVAL when the mask has no solid voxel.
 * ====================================================================== */
static int64_t orc_dist2(int x0, int y0, int z0, int x1, int y1, int z1, int ny, int nz) {
  int64_t dx = x0 - x1;
  int64_t dy = abs(y0 - y1), dz = abs(z0 - z1);
  if (ny - dy < dy) dy = ny - dy;
  if (nz - dz < dz) dz = nz - dz;
  return dx * dx + dy * dy + dz * dz;
}

int orc_mis(const uint8_t *mask, int nx, int ny, int nz, double dx_nm, float *d_nm, int32_t *r2out) {
  int64_t N = (int64_t)nx * ny * nz;
  int64_t nsolid = 0;
  for (int64_t v = 0; v < N; ++v) nsolid += !mask[v];
  if (nsolid == 0) return ORC_EINVAL;
  int64_t *r2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
  if (!r2) return ORC_ENOMEM;
  for (int64_t c = 0; c < N; ++c) {
    r2[c] = 0;
    if (!mask[c]) continue;
    int cx = (int)(c / ((int64_t)ny * nz)), cy = (int)((c / nz) % ny), cz = (int)(c % nz);
    int64_t best = INT64_MAX;
    for (int64_t s = 0; s < N; ++s) {
      if (mask[s]) continue;
      int sx = (int)(s / ((int64_t)ny * nz)), sy = (int)((s / nz) % ny), sz = (int)(s % nz);
      int64_t d2 = orc_dist2(cx, cy, cz, sx, sy, sz, ny, nz);
      if (d2 < best) best = d2;
    }
    r2[c] = best;
  }
  for (int64_t v = 0; v < N; ++v) {
    if (r2out) r2out[v] = (int32_t)r2[v];
    if (!mask[v]) { d_nm[v] = 0.0f; continue; }
    int vx = (int)(v / ((int64_t)ny * nz)), vy = (int)((v / nz) % ny), vz = (int)(v % nz);
    double best = 0.0;
    for (int64_t c = 0; c < N; ++c) {
      if (!mask[c]) continue;
      int cx = (int)(c / ((int64_t)ny * nz)), cy = (int)((c / nz) % ny), cz = (int)(c % nz);
      if (orc_dist2(vx, vy, vz, cx, cy, cz, ny, nz) < r2[c]) {
        double dd = 2.0 * sqrt((double)r2[c]) - 1.0;
        if (dd > best) best = dd;
      }
    }
    d_nm[v] = (float)(best * dx_nm);
  }
  free(r2);
  return ORC_OK;
}

/* ======================================================================
 * 6. MRT D3Q19 flow (Sec. 3.1, Eqs. 1-9, App. A), written in moment space.
 *    Q is the table of App. A; the discrete velocities e_i are read off its
 *    momentum rows 3, 5 and 7; Q^-1 is computed as Q^T diag(1/|row|^2)
 *    (the rows are orthogonal), not copied.
 * ====================================================================== */
static const int QT[19][19] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-30, -11, -11, -11, -11, -11, -11, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8},
    {12, -4, -4, -4, -4, -4, -4, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, -4, 4, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, -4, 4, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
    {0, 0, 0, 0, 0, -4, 4, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
    {0, 2, 2, -1, -1, -1, -1, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
    {0, -4, -4, 2, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
    {0, 0, 0, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
    {0, 0, 0, -2, -2, 2, 2, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, -1, 1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, -1, -1, 1, 1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, -1, -1, 1, 1}};

void orc_q_matrix(double *Q) {
  for (int k = 0; k < 19; ++k)
    for (int i = 0; i < 19; ++i) Q[k * 19 + i] = QT[k][i];
}

void orc_qinv_matrix(double *Qi) {
  for (int k = 0; k < 19; ++k) {
    double n2 = 0.0;
    for (int i = 0; i < 19; ++i) n2 += (double)(QT[k][i] * QT[k][i]);
    for (int i = 0; i < 19; ++i) Qi[i * 19 + k] = (double)QT[k][i] / n2;
  }
}

void orc_velocities19(int *e) { /* 19 x 3 */
  for (int i = 0; i < 19; ++i) {
    e[3 * i + 0] = QT[3][i];
    e[3 * i + 1] = QT[5][i];
    e[3 * i + 2] = QT[7][i];
  }
}

/* Tables derived once from QT: velocities, Eq. 3 weights by speed, the
 * opposite of each velocity, Q and Q^-1 as doubles. */
static int T_ready = 0;
static int T_e[57], T_opp[19];
static double T_w[19], T_Q[361], T_Qi[361];

static void orc_tables(void) {
  if (T_ready) return;
  orc_velocities19(T_e);
  for (int i = 0; i < 19; ++i) {
    int s = abs(T_e[3 * i]) + abs(T_e[3 * i + 1]) + abs(T_e[3 * i + 2]);
    T_w[i] = s == 0 ? 1.0 / 3.0 : (s == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    T_opp[i] = -1;
    for (int j = 0; j < 19; ++j)
      if (T_e[3 * j] == -T_e[3 * i] && T_e[3 * j + 1] == -T_e[3 * i + 1] &&
          T_e[3 * j + 2] == -T_e[3 * i + 2])
        T_opp[i] = j;
  }
  orc_q_matrix(T_Q);
  orc_qinv_matrix(T_Qi);
  T_ready = 1;
}

double orc_w19(int i) { orc_tables(); return T_w[i]; }
int orc_opp19(int i) { orc_tables(); return T_opp[i]; }

/* App. A, Eqs. A1-A9 (rho0 = 1) */
void orc_meq(double rho, double jx, double jy, double jz, double *m) {
  double jj = jx * jx + jy * jy + jz * jz;
  m[0] = rho;
  m[1] = -11.0 * rho + 19.0 * jj;
  m[2] = 3.0 * rho - 5.5 * jj;
  m[3] = jx;
  m[4] = -2.0 / 3.0 * jx;
  m[5] = jy;
  m[6] = -2.0 / 3.0 * jy;
  m[7] = jz;
  m[8] = -2.0 / 3.0 * jz;
  m[9] = 3.0 * jx * jx - jj;
  m[10] = -(3.0 * jx * jx - jj) / 2.0;
  m[11] = jy * jy - jz * jz;
  m[12] = -(jy * jy - jz * jz) / 2.0;
  m[13] = jx * jy;
  m[14] = jy * jz;
  m[15] = jx * jz;
  m[16] = 0.0;
  m[17] = 0.0;
  m[18] = 0.0;
}

/* Eq. 7 relaxation rates */
void orc_rates(double tau, double *s) {
  double sq = 8.0 * (2.0 * tau - 1.0) / (8.0 * tau - 1.0);
  for (int k = 0; k < 19; ++k) s[k] = 0.0;
  s[1] = s[2] = 1.0 / tau;
  for (int k = 9; k <= 15; ++k) s[k] = 1.0 / tau;
  s[4] = s[6] = s[8] = sq;
  s[16] = s[17] = s[18] = sq;
}

/* One node's collision in moment space (Eq. 4-5) with a body force g along
 * x: m = Q f; j* = j + g/2 enters m_eq; m* = m - S (m - m_eq) + (I - S/2) Q F
 * with F_i = 3 w_i (e_i . g); f* = Q^-1 m*. */
void orc_mrt_collide_node(const double *f, double tau, double g, double *fout) {
  double s[19], m[19], meq[19], QF[19], ms[19], F[19];
  orc_tables();
  const double *Q = T_Q, *Qi = T_Qi;
  const int *e = T_e;
  orc_rates(tau, s);
  for (int k = 0; k < 19; ++k) {
    m[k] = 0.0;
    for (int i = 0; i < 19; ++i) m[k] += Q[k * 19 + i] * f[i];
  }
  double jx = m[3] + 0.5 * g, jy = m[5], jz = m[7];
  orc_meq(m[0], jx, jy, jz, meq);
  for (int i = 0; i < 19; ++i) F[i] = 3.0 * T_w[i] * ((double)e[3 * i] * g);
  for (int k = 0; k < 19; ++k) {
    QF[k] = 0.0;
    for (int i = 0; i < 19; ++i) QF[k] += Q[k * 19 + i] * F[i];
  }
  for (int k = 0; k < 19; ++k) ms[k] = m[k] - s[k] * (m[k] - meq[k]) + (1.0 - 0.5 * s[k]) * QF[k];
  for (int i = 0; i < 19; ++i) {
    fout[i] = 0.0;
    for (int k = 0; k < 19; ++k) fout[i] += Qi[i * 19 + k] * ms[k];
  }
}

/* f: 19*N (population i of voxel v at i*N + v); node: 1 on lattice nodes.
 * Sec. 3.1 steps 1-4: collide every node in moment space, then stream in
 * velocity space with halfway bounce-back off every non-node and periodic
 * wrap in x, y and z (the body-force reading of the x boundaries). */
int orc_flow_step(const uint8_t *node, int nx, int ny, int nz, double tau, double g, double *f) {
  int64_t N = (int64_t)nx * ny * nz;
  double *fs = (double *)malloc(sizeof(double) * 19 * (size_t)N);
  if (!fs) return ORC_ENOMEM;
  int e[57], opp[19];
  orc_velocities19(e);
  for (int i = 0; i < 19; ++i) opp[i] = orc_opp19(i);
  double fin[19], fo[19];
  for (int64_t v = 0; v < N; ++v) {
    if (!node[v]) continue;
    for (int i = 0; i < 19; ++i) fin[i] = f[(int64_t)i * N + v];
    orc_mrt_collide_node(fin, tau, g, fo);
    for (int i = 0; i < 19; ++i) fs[(int64_t)i * N + v] = fo[i];
  }
  for (int64_t v = 0; v < N; ++v) {
    if (!node[v]) continue;
    int x = (int)(v / ((int64_t)ny * nz)), y = (int)((v / nz) % ny), z = (int)(v % nz);
    for (int i = 0; i < 19; ++i) {
      int64_t src = vidx(wrap(x - e[3 * i], nx), wrap(y - e[3 * i + 1], ny), wrap(z - e[3 * i + 2], nz), ny, nz);
      f[(int64_t)i * N + v] = node[src] ? fs[(int64_t)i * N + src] : fs[(int64_t)opp[i] * N + v];
    }
  }
  free(fs);
  return ORC_OK;
}

/* Eq. 9 with the half-force velocity: u = j + g/2 (rho0 = 1). */
void orc_flow_velocity(const uint8_t *node, int nx, int ny, int nz, double g, const double *f,
                       double *ux, double *uy, double *uz, double *rho) {
  int64_t N = (int64_t)nx * ny * nz;
  int e[57];
  orc_velocities19(e);
  for (int64_t v = 0; v < N; ++v) {
    double r = 0, jx = 0, jy = 0, jz = 0;
    if (node[v])
      for (int i = 0; i < 19; ++i) {
        double fi = f[(int64_t)i * N + v];
        r += fi;
        jx += e[3 * i] * fi;
        jy += e[3 * i + 1] * fi;
        jz += e[3 * i + 2] * fi;
      }
    if (ux) ux[v] = node[v] ? jx + 0.5 * g : 0.0;
    if (uy) uy[v] = jy;
    if (uz) uz[v] = jz;
    if (rho) rho[v] = r;
  }
}

void orc_flow_init(const uint8_t *node, int nx, int ny, int nz, double *f) {
  int64_t N = (int64_t)nx * ny * nz;
  for (int i = 0; i < 19; ++i)
    for (int64_t v = 0; v < N; ++v) f[(int64_t)i * N + v] = node[v] ? orc_w19(i) : 0.0;
}

/* Solve to the steady state: every K steps compare u_x with the value K
 * steps earlier; stop when sum|du_x| / sum|u_x| < tol.  Darcy (Eq. 13) with
 * the body force as the pressure gradient: k_L = nu <u_x> / g, the average
 * over all N voxels, nu = (tau - 1/2)/3 (Eq. 8).
 * out[0] k_L, out[1] sum u_x, out[2] steps, out[3] last relative change. */
int orc_flow_solve(const uint8_t *node, int nx, int ny, int nz, double tau, double g, double tol,
                   int K, int64_t max_steps, double *f, double *out) {
  int64_t N = (int64_t)nx * ny * nz;
  double *ux = (double *)malloc(sizeof(double) * (size_t)N);
  double *prev = (double *)malloc(sizeof(double) * (size_t)N);
  if (!ux || !prev) { free(ux); free(prev); return ORC_ENOMEM; }
  orc_flow_init(node, nx, ny, nz, f);
  orc_flow_velocity(node, nx, ny, nz, g, f, prev, NULL, NULL, NULL);
  int64_t n = 0;
  double rel = 1.0, sum = 0.0;
  int rc = ORC_ENOTCONVERGED;
  while (n < max_steps) {
    for (int k = 0; k < K && n < max_steps; ++k, ++n) {
      int r = orc_flow_step(node, nx, ny, nz, tau, g, f);
      if (r) { free(ux); free(prev); return r; }
    }
    orc_flow_velocity(node, nx, ny, nz, g, f, ux, NULL, NULL, NULL);
    double du = 0.0, au = 0.0;
    sum = 0.0;
    for (int64_t v = 0; v < N; ++v) {
      if (!node[v]) continue;
      du += fabs(ux[v] - prev[v]);
      au += fabs(ux[v]);
      sum += ux[v];
      prev[v] = ux[v];
    }
    rel = au > 0.0 ? du / au : 0.0;
    if (rel < tol) { rc = ORC_OK; break; }
  }
  double nu = (tau - 0.5) / 3.0;
  out[0] = nu * (sum / (double)N) / g;
  out[1] = sum;
  out[2] = (double)n;
  out[3] = rel;
  free(ux);
  free(prev);
  return rc;
}

/* ----------------------------------------------------------------------
 * Pressure-driven flow (Sec. 3.3): x is not periodic; the nodes of the
 * layers x = 0 and x = nx-1 carry the inlet and outlet densities by the
 * non-equilibrium extrapolation of Guo et al.: before each collision every
 * population of such a boundary node b is replaced by
 *     f_i(b) = f_i^eq(rho_b, u_b) + [f_i(b1) - f_i^eq(rho(b1), u(b1))],
 * b1 = b + n and b2 = b + 2n along the inward normal n = (+-1, 0, 0).  The
 * boundary velocity is extrapolated to second order, u_b = 2 u(b1) - u(b2),
 * when b1 and b2 are nodes, taken as u(b1) when only b1 is, and with no node
 * at b1 the population is the equilibrium at rest, f_i^eq(rho_b, 0).  f^eq
 * is the equilibrium whose moments are A1-A9 (j in place of rho0 u, rho0 = 1):
 *     f_i^eq = w_i (rho + 3 e_i.j + 4.5 (e_i.j)^2 - 1.5 j.j).
 * No body force acts.  Needs nx >= 4 (the inlet's b2 is not an outlet node).
 * ---------------------------------------------------------------------- */
static double orc_feq19(int i, double rho, double jx, double jy, double jz) {
  orc_tables();
  double eu = (double)T_e[3 * i] * jx + (double)T_e[3 * i + 1] * jy + (double)T_e[3 * i + 2] * jz;
  double jj = jx * jx + jy * jy + jz * jz;
  return T_w[i] * (rho + 3.0 * eu + 4.5 * eu * eu - 1.5 * jj);
}

static void orc_moments19(const double *f, int64_t N, int64_t v, double *rho, double *j) {
  orc_tables();
  double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
  for (int i = 0; i < 19; ++i) {
    double fi = f[(int64_t)i * N + v];
    r += fi;
    jx += (double)T_e[3 * i] * fi;
    jy += (double)T_e[3 * i + 1] * fi;
    jz += (double)T_e[3 * i + 2] * fi;
  }
  *rho = r;
  j[0] = jx;
  j[1] = jy;
  j[2] = jz;
}

/* Replace the populations of the boundary nodes (both faces) in place.  The
 * values of b1 and b2 are read before any boundary node is written (they are
 * interior nodes for nx >= 4). */
int orc_pressure_bc(const uint8_t *node, int nx, int ny, int nz, double rho_in, double rho_out, double *f) {
  if (nx < 4) return ORC_EINVAL;
  int64_t N = (int64_t)nx * ny * nz;
  for (int side = 0; side < 2; ++side) {
    int xb = side == 0 ? 0 : nx - 1, dir = side == 0 ? 1 : -1;
    double rho_b = side == 0 ? rho_in : rho_out;
    for (int y = 0; y < ny; ++y)
      for (int z = 0; z < nz; ++z) {
        int64_t b = vidx(xb, y, z, ny, nz);
        if (!node[b]) continue;
        int64_t b1 = vidx(xb + dir, y, z, ny, nz), b2 = vidx(xb + 2 * dir, y, z, ny, nz);
        double out[19];
        if (!node[b1]) {
          for (int i = 0; i < 19; ++i) out[i] = orc_feq19(i, rho_b, 0.0, 0.0, 0.0);
        } else {
          double r1, j1[3], ub[3];
          orc_moments19(f, N, b1, &r1, j1);
          if (node[b2]) {
            double r2, j2[3];
            orc_moments19(f, N, b2, &r2, j2);
            for (int k = 0; k < 3; ++k) ub[k] = 2.0 * j1[k] - j2[k];
          } else {
            for (int k = 0; k < 3; ++k) ub[k] = j1[k];
          }
          for (int i = 0; i < 19; ++i)
            out[i] = orc_feq19(i, rho_b, ub[0], ub[1], ub[2]) +
                     (f[(int64_t)i * N + b1] - orc_feq19(i, r1, j1[0], j1[1], j1[2]));
        }
        for (int i = 0; i < 19; ++i) f[(int64_t)i * N + b] = out[i];
      }
  }
  return ORC_OK;
}

/* One step of the pressure-driven flow: boundary replacement, collision of
 * every node (no force), streaming with halfway bounce-back off non-nodes
 * and off the x ends (those populations are replaced before the next
 * collision), periodic in y and z. */
int orc_flow_step_p(const uint8_t *node, int nx, int ny, int nz, double tau, double rho_in, double rho_out,
                    double *f) {
  int rc = orc_pressure_bc(node, nx, ny, nz, rho_in, rho_out, f);
  if (rc) return rc;
  int64_t N = (int64_t)nx * ny * nz;
  double *fs = (double *)malloc(sizeof(double) * 19 * (size_t)N);
  if (!fs) return ORC_ENOMEM;
  int e[57], opp[19];
  orc_velocities19(e);
  for (int i = 0; i < 19; ++i) opp[i] = orc_opp19(i);
  double fin[19], fo[19];
  for (int64_t v = 0; v < N; ++v) {
    if (!node[v]) continue;
    for (int i = 0; i < 19; ++i) fin[i] = f[(int64_t)i * N + v];
    orc_mrt_collide_node(fin, tau, 0.0, fo);
    for (int i = 0; i < 19; ++i) fs[(int64_t)i * N + v] = fo[i];
  }
  for (int64_t v = 0; v < N; ++v) {
    if (!node[v]) continue;
    int x = (int)(v / ((int64_t)ny * nz)), y = (int)((v / nz) % ny), z = (int)(v % nz);
    for (int i = 0; i < 19; ++i) {
      int xs = x - e[3 * i];
      int inside = xs >= 0 && xs < nx;
      int64_t src = inside ? vidx(xs, wrap(y - e[3 * i + 1], ny), wrap(z - e[3 * i + 2], nz), ny, nz) : -1;
      f[(int64_t)i * N + v] = (inside && node[src]) ? fs[(int64_t)i * N + src] : fs[(int64_t)opp[i] * N + v];
    }
  }
  free(fs);
  return ORC_OK;
}

/* Solve the pressure-driven flow to the steady state (the test of
 * orc_flow_solve on the interior layers x = 1 .. nx-2).  Darcy (Eq. 13):
 * k_L = nu <u_x> L / (dp / rho0) with dp = c_s^2 (rho_in - rho_out), L =
 * nx - 1 (the distance between the boundary layers) and <u_x> the
 * superficial velocity, the sum of u_x = j_x over the interior layers divided
 * by their voxel count (every layer carries the same flux at steady state).
 * out[0] k_L, out[1] <u_x>, out[2] steps, out[3] last relative change. */
int orc_flow_solve_p(const uint8_t *node, int nx, int ny, int nz, double tau, double rho_in, double rho_out,
                     double tol, int K, int64_t max_steps, double *f, double *out) {
  if (nx < 4) return ORC_EINVAL;
  int64_t N = (int64_t)nx * ny * nz, plane = (int64_t)ny * nz;
  double *ux = (double *)malloc(sizeof(double) * (size_t)N);
  double *prev = (double *)malloc(sizeof(double) * (size_t)N);
  if (!ux || !prev) { free(ux); free(prev); return ORC_ENOMEM; }
  orc_flow_init(node, nx, ny, nz, f);
  orc_flow_velocity(node, nx, ny, nz, 0.0, f, prev, NULL, NULL, NULL);
  int64_t n = 0;
  double rel = 1.0, sum = 0.0;
  int rc = ORC_ENOTCONVERGED;
  while (n < max_steps) {
    for (int k = 0; k < K && n < max_steps; ++k, ++n) {
      int r = orc_flow_step_p(node, nx, ny, nz, tau, rho_in, rho_out, f);
      if (r) { free(ux); free(prev); return r; }
    }
    orc_flow_velocity(node, nx, ny, nz, 0.0, f, ux, NULL, NULL, NULL);
    double du = 0.0, au = 0.0;
    sum = 0.0;
    for (int64_t v = plane; v < N - plane; ++v) {
      if (!node[v]) continue;
      du += fabs(ux[v] - prev[v]);
      au += fabs(ux[v]);
      sum += ux[v];
      prev[v] = ux[v];
    }
    rel = au > 0.0 ? du / au : 0.0;
    if (rel < tol) { rc = ORC_OK; break; }
  }
  double nu = (tau - 0.5) / 3.0;
  double mean_u = sum / (double)(N - 2 * plane);
  out[0] = nu * mean_u * (double)(nx - 1) / ((rho_in - rho_out) / 3.0);
  out[1] = mean_u;
  out[2] = (double)n;
  out[3] = rel;
  free(ux);
  free(prev);
  return rc;
}

/* ======================================================================
 * 7. BGK diffusion (Sec. 3.2, Eq. 10): g_i^eq = a_i C, C = sum g_i, one
 *    relaxation time per node from the local pore size (Eq. 12, supplied as
 *    omega = 1/tau_g), on D3Q7 (a_0 = 1/4, a_1..6 = 1/8, c_s^2 = 1/4; order
 *    rest, +x, -x, +y, -y, +z, -z) or the paper's D3Q19 (Eq. 2 velocities,
 *    Eq. 3 weights, c_s^2 = 1/3).  Bounce-back at walls; periodic y, z; fixed
 *    concentration at the half links x = -1/2 (C_in) and x = nx - 1/2 (C_out)
 *    by anti-bounce-back of every population whose link crosses the face.
 * ====================================================================== */
/* The diffusion lattice: D3Q7 (rest, +x, -x, +y, -y, +z, -z; a_0 = 1/4,
 * a_1..6 = 1/8; c_s^2 = 1/4) or the paper's D3Q19 (the velocities and
 * weights of Eqs. 2-3 in the order of orc_velocities19: 1/3, 1/18, 1/36;
 * c_s^2 = 1/3).  The BGK relaxation, bounce-back and anti-bounce-back rules
 * below are the same for both. */
typedef struct {
  int q;
  int e[19][3];
  int opp[19];
  double w[19];
} orc_dlat;

static int orc_dlat_make(int q, orc_dlat *L) {
  static const int E7[7][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
  static const int OPP7[7] = {0, 2, 1, 4, 3, 6, 5};
  L->q = q;
  if (q == 7) {
    for (int i = 0; i < 7; ++i) {
      for (int d = 0; d < 3; ++d) L->e[i][d] = E7[i][d];
      L->opp[i] = OPP7[i];
      L->w[i] = i == 0 ? 0.25 : 0.125;
    }
    return ORC_OK;
  }
  if (q == 19) {
    int e[57];
    orc_velocities19(e);
    for (int i = 0; i < 19; ++i) {
      for (int d = 0; d < 3; ++d) L->e[i][d] = e[3 * i + d];
      L->opp[i] = orc_opp19(i);
      L->w[i] = orc_w19(i);
    }
    return ORC_OK;
  }
  return ORC_EINVAL;
}

/* Eq. 12: tau_g = (d / d_ref)(tau_ref - 1/2) + 1/2 */
double orc_tau_knudsen(double d_nm, double d_ref_nm, double tau_ref) {
  return (d_nm / d_ref_nm) * (tau_ref - 0.5) + 0.5;
}

int orc_diffq_init(int q, const uint8_t *node, int nx, int ny, int nz, double cin, double cout, double *g) {
  orc_dlat L;
  if (orc_dlat_make(q, &L)) return ORC_EINVAL;
  int64_t N = (int64_t)nx * ny * nz;
  for (int64_t v = 0; v < N; ++v) {
    int x = (int)(v / ((int64_t)ny * nz));
    double c = cin + (cout - cin) * (((double)x + 0.5) / (double)nx);
    for (int i = 0; i < q; ++i) g[(int64_t)i * N + v] = node[v] ? L.w[i] * c : 0.0;
  }
  return ORC_OK;
}

int orc_diffq_step(int q, const uint8_t *node, int nx, int ny, int nz, const double *omega, double cin,
                   double cout, double *g) {
  orc_dlat L;
  if (orc_dlat_make(q, &L)) return ORC_EINVAL;
  int64_t N = (int64_t)nx * ny * nz;
  double *gs = (double *)malloc(sizeof(double) * (size_t)q * (size_t)N);
  if (!gs) return ORC_ENOMEM;
  for (int64_t v = 0; v < N; ++v) {
    if (!node[v]) continue;
    double C = 0.0;
    for (int i = 0; i < q; ++i) C += g[(int64_t)i * N + v];
    for (int i = 0; i < q; ++i) {
      double gi = g[(int64_t)i * N + v];
      gs[(int64_t)i * N + v] = gi - omega[v] * (gi - L.w[i] * C);
    }
  }
  for (int64_t v = 0; v < N; ++v) {
    if (!node[v]) continue;
    int x = (int)(v / ((int64_t)ny * nz)), y = (int)((v / nz) % ny), z = (int)(v % nz);
    for (int i = 0; i < q; ++i) {
      int sx = x - L.e[i][0];
      double val;
      if (sx < 0)
        val = -gs[(int64_t)L.opp[i] * N + v] + 2.0 * L.w[i] * cin;
      else if (sx >= nx)
        val = -gs[(int64_t)L.opp[i] * N + v] + 2.0 * L.w[i] * cout;
      else {
        int64_t src = vidx(sx, wrap(y - L.e[i][1], ny), wrap(z - L.e[i][2], nz), ny, nz);
        val = node[src] ? gs[(int64_t)i * N + src] : gs[(int64_t)L.opp[i] * N + v];
      }
      g[(int64_t)i * N + v] = val;
    }
  }
  free(gs);
  return ORC_OK;
}

/* C = sum g_i; diffusive flux J_x = (1 - omega/2) sum_i e_ix g_i */
int orc_diffq_fields(int q, const uint8_t *node, int nx, int ny, int nz, const double *omega, const double *g,
                     double *C, double *Jx) {
  orc_dlat L;
  if (orc_dlat_make(q, &L)) return ORC_EINVAL;
  int64_t N = (int64_t)nx * ny * nz;
  for (int64_t v = 0; v < N; ++v) {
    double c = 0.0, j = 0.0;
    if (node[v]) {
      for (int i = 0; i < q; ++i) {
        c += g[(int64_t)i * N + v];
        j += L.e[i][0] * g[(int64_t)i * N + v];
      }
      j *= (1.0 - 0.5 * omega[v]);
    }
    if (C) C[v] = c;
    if (Jx) Jx[v] = j;
  }
  return ORC_OK;
}

/* Solve to the steady state.  Every K steps both the concentration field
 * (sum|dC| / sum|C|) and the total flux (|d sum J_x| / |sum J_x|) must have
 * changed by less than tol: the concentration alone can sit at its final
 * profile while the flux is still relaxing.  Eq. 14 with the volume-averaged
 * flux: D_eff,L = (sum J_x / N) * nx / (C_in - C_out).
 * out[0] D_eff,L, out[1] sum J_x, out[2] steps, out[3] last relative change
 * (the larger of the two), out[4] sum C. */
int orc_diffq_solve(int q, const uint8_t *node, int nx, int ny, int nz, const double *omega, double cin,
                    double cout, double tol, int K, int64_t max_steps, double *g, double *out) {
  if (q != 7 && q != 19) return ORC_EINVAL;
  int64_t N = (int64_t)nx * ny * nz;
  double *C = (double *)malloc(sizeof(double) * (size_t)N);
  double *J = (double *)malloc(sizeof(double) * (size_t)N);
  double *prev = (double *)malloc(sizeof(double) * (size_t)N);
  if (!C || !J || !prev) { free(C); free(J); free(prev); return ORC_ENOMEM; }
  orc_diffq_init(q, node, nx, ny, nz, cin, cout, g);
  orc_diffq_fields(q, node, nx, ny, nz, omega, g, prev, J);
  double sj_prev = 0.0;
  for (int64_t v = 0; v < N; ++v)
    if (node[v]) sj_prev += J[v];
  int64_t n = 0;
  double rel = 1.0, sj = 0.0, sc = 0.0;
  int rc = ORC_ENOTCONVERGED;
  while (n < max_steps) {
    for (int k = 0; k < K && n < max_steps; ++k, ++n) {
      int r = orc_diffq_step(q, node, nx, ny, nz, omega, cin, cout, g);
      if (r) { free(C); free(J); free(prev); return r; }
    }
    orc_diffq_fields(q, node, nx, ny, nz, omega, g, C, J);
    double dc = 0.0, ac = 0.0;
    sj = 0.0;
    sc = 0.0;
    for (int64_t v = 0; v < N; ++v) {
      if (!node[v]) continue;
      dc += fabs(C[v] - prev[v]);
      ac += fabs(C[v]);
      sj += J[v];
      sc += C[v];
      prev[v] = C[v];
    }
    rel = ac > 0.0 ? dc / ac : 0.0;
    double relj = sj != 0.0 ? fabs(sj - sj_prev) / fabs(sj) : 0.0;
    if (relj > rel) rel = relj;
    sj_prev = sj;
    if (rel < tol) { rc = ORC_OK; break; }
  }
  out[0] = (sj / (double)N) * (double)nx / (cin - cout);
  out[1] = sj;
  out[2] = (double)n;
  out[3] = rel;
  out[4] = sc;
  free(C);
  free(J);
  free(prev);
  return rc;
}

/* The D3Q7 entry points (the lattice of the benchmark workloads). */
void orc_diff_init(const uint8_t *node, int nx, int ny, int nz, double cin, double cout, double *g) {
  orc_diffq_init(7, node, nx, ny, nz, cin, cout, g);
}
int orc_diff_step(const uint8_t *node, int nx, int ny, int nz, const double *omega, double cin, double cout,
                  double *g) {
  return orc_diffq_step(7, node, nx, ny, nz, omega, cin, cout, g);
}
void orc_diff_fields(const uint8_t *node, int nx, int ny, int nz, const double *omega, const double *g,
                     double *C, double *Jx) {
  orc_diffq_fields(7, node, nx, ny, nz, omega, g, C, Jx);
}
int orc_diff_solve(const uint8_t *node, int nx, int ny, int nz, const double *omega, double cin, double cout,
                   double tol, int K, int64_t max_steps, double *g, double *out) {
  return orc_diffq_solve(7, node, nx, ny, nz, omega, cin, cout, tol, K, max_steps, g, out);
}
