// multilevel.cu -- a two-level warm start for the diffusion solves.
//
// Not in the paper (it starts every solve from rest / the linear profile):
// the slowest modes of a diffusion solve are the structure-scale ones, and a
// solve on a copy of the structure coarsened 2x per axis (8x fewer nodes,
// ~4x fewer steps for the same diffusive time) resolves them for about 1/32
// of the fine solve's work.  Its concentration, carried to the fine nodes,
// is the fine solve's initial state; the fine LB then iterates from it to the
// same convergence test, so the result is the fine method's.
//
// Coarsening: coarse voxel (X, Y, Z) covers the fine voxels 2X..2X+1 (and so
// on, clipped at an odd edge); it is a node when at least half of the fine
// voxels it covers are nodes, and its pore size is the mean of theirs.
// Prolongation: a fine node takes the concentration of the coarse voxel
// that covers it when that is a coarse node, else the linear inlet-outlet
// profile C_lin(x); optionally as the departure from C_lin (an input of the
// warm-start network) and plus a per-voxel correction (the network's
// output), so that the network refines the coarse solution.
#include "common.cuh"

namespace om {
namespace {

__global__ void coarsen2(const uint8_t* __restrict__ nodes, const float* __restrict__ d_nm, int nx, int ny, int nz,
                         int cx, int cy, int cz, uint8_t* __restrict__ nodes_c, float* __restrict__ d_c) {
  const int64_t nc = (int64_t)cx * cy * cz;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nc; k += (int64_t)gridDim.x * blockDim.x) {
    const int X = (int)(k / ((int64_t)cy * cz));
    const int Y = (int)((k / cz) % cy);
    const int Z = (int)(k % cz);
    int cover = 0, count = 0;
    double sum = 0.0;
    for (int dx = 0; dx < 2; ++dx)
      for (int dy = 0; dy < 2; ++dy)
        for (int dz = 0; dz < 2; ++dz) {
          const int x = 2 * X + dx, y = 2 * Y + dy, z = 2 * Z + dz;
          if (x >= nx || y >= ny || z >= nz) continue;
          ++cover;
          const int64_t v = ((int64_t)x * ny + y) * nz + z;
          if (nodes[v]) {
            ++count;
            if (d_nm) sum += (double)d_nm[v];
          }
        }
    nodes_c[k] = 2 * count >= cover ? 1 : 0;
    if (d_c) d_c[k] = count > 0 ? (float)(sum / count) : 0.0f;
  }
}

__global__ void prolong2(const double* __restrict__ g_c, int q, const uint8_t* __restrict__ nodes_c, int cx, int cy,
                         int cz, int nx, int ny, int nz, double c_in, double c_out, const float* __restrict__ corr,
                         int64_t corr_stride, int departure, float* __restrict__ c) {
  const int64_t n = (int64_t)nx * ny * nz, nc = (int64_t)cx * cy * cz;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(v / ((int64_t)ny * nz));
    const int y = (int)((v / nz) % ny);
    const int z = (int)(v % nz);
    const int64_t k = ((int64_t)(x / 2) * cy + y / 2) * cz + z / 2;
    const double clin = c_in + (c_out - c_in) * ((double)x + 0.5) / (double)nx;  // C_lin(x)
    double val = clin;
    if (nodes_c[k]) {
      double s = 0.0;
      for (int i = 0; i < q; ++i) s += g_c[(int64_t)i * nc + k];
      val = s;
    }
    if (departure) val -= clin;
    if (corr) val += (double)corr[v * corr_stride];
    c[v] = (float)val;
  }
}

// fine u_x from the coarse flow populations: scale * (sum_i e_ix f_i + g/2)
// at the covering coarse voxel where it is a node, else 0 (Guo's half-force
// velocity, Sec. 3.1)
__global__ void prolong2_ux(const double* __restrict__ f_c, const uint8_t* __restrict__ nodes_c, int cx, int cy,
                            int cz, int nx, int ny, int nz, double half_g, double scale, float* __restrict__ u) {
  const int64_t n = (int64_t)nx * ny * nz, nc = (int64_t)cx * cy * cz;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(v / ((int64_t)ny * nz));
    const int y = (int)((v / nz) % ny);
    const int z = (int)(v % nz);
    const int64_t k = ((int64_t)(x / 2) * cy + y / 2) * cz + z / 2;
    double val = 0.0;
    if (nodes_c[k]) {
      double jx = 0.0;
      for (int i = 1; i < 19; ++i)
        if (q19_e(i, 0)) jx += q19_e(i, 0) > 0 ? f_c[(int64_t)i * nc + k] : -f_c[(int64_t)i * nc + k];
      val = scale * (jx + half_g);
    }
    u[v] = (float)val;
  }
}

om_domain coarse_domain(const om_domain& d) {
  om_domain c = d;
  c.nx = (d.nx + 1) / 2;
  c.ny = (d.ny + 1) / 2;
  c.nz = (d.nz + 1) / 2;
  c.dx_nm = 2.0 * d.dx_nm;
  return c;
}

unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16); }

}  // namespace
}  // namespace om

using namespace om;

extern "C" om_status om_coarse_domain(om_domain d, om_domain* dc) {
  if (!dc) return fail(OM_EINVAL, "om_coarse_domain: null pointer");
  OM_TRY(check_domain(d));
  *dc = coarse_domain(d);
  return OM_OK;
}

extern "C" om_status om_coarsen2_dev(const uint8_t* nodes_dev, const float* d_nm_dev, om_domain d,
                                     uint8_t* nodes_c_dev, float* d_c_dev, void* stream) {
  if (!nodes_dev || !nodes_c_dev || (!d_nm_dev) != (!d_c_dev))
    return fail(OM_EINVAL, "om_coarsen2_dev: null pointer (pore sizes need both arrays or neither)");
  OM_TRY(check_domain(d));
  const om_domain c = coarse_domain(d);
  const int64_t nc = voxels(c);
  coarsen2<<<grid_for(nc), 256, 0, as_stream(stream)>>>(nodes_dev, d_nm_dev, d.nx, d.ny, d.nz, c.nx, c.ny, c.nz,
                                                       nodes_c_dev, d_c_dev);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

extern "C" om_status om_prolong2_dev(const double* g_c_dev, int32_t q, const uint8_t* nodes_c_dev, om_domain d,
                                     double c_in, double c_out, const float* corr_dev, int64_t corr_stride,
                                     int32_t departure, float* c_dev, void* stream) {
  if (!g_c_dev || !nodes_c_dev || !c_dev || q < 1 || q > 27 || (corr_dev && corr_stride < 1))
    return fail(OM_EINVAL, "om_prolong2_dev: bad argument");
  OM_TRY(check_domain(d));
  const om_domain c = coarse_domain(d);
  prolong2<<<grid_for(voxels(d)), 256, 0, as_stream(stream)>>>(g_c_dev, q, nodes_c_dev, c.nx, c.ny, c.nz, d.nx, d.ny,
                                                              d.nz, c_in, c_out, corr_dev, corr_stride, departure,
                                                              c_dev);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

extern "C" om_status om_prolong2_ux_dev(const double* f_c_dev, const uint8_t* nodes_c_dev, om_domain d,
                                        double body_force_c, double scale, float* ux_dev, void* stream) {
  if (!f_c_dev || !nodes_c_dev || !ux_dev) return fail(OM_EINVAL, "om_prolong2_ux_dev: null pointer");
  OM_TRY(check_domain(d));
  const om_domain c = coarse_domain(d);
  prolong2_ux<<<grid_for(voxels(d)), 256, 0, as_stream(stream)>>>(f_c_dev, nodes_c_dev, c.nx, c.ny, c.nz, d.nx, d.ny,
                                                                 d.nz, 0.5 * body_force_c, scale, ux_dev);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}
