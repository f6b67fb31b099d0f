// poresize.cu -- local pore size on the GPU.
//
// CHORD13 (Sec. 4.1): for each pore voxel and each of the 13 line
// directions (3 axes, 6 face diagonals, 4 body diagonals) count the cells of
// the all-pore line through it; lines wrap in y and z, stop at the x faces,
// and a closed all-pore loop counts each of its cells once.  The pore size
// is the mean of the 13 lengths, a count along a diagonal weighing sqrt(2)
// or sqrt(3) cells.
//
// MIS: r2(c), the squared distance from pore voxel c to the nearest solid
// voxel (periodic y, z; nothing solid beyond the x faces), by three separable
// 1-D minimisations; then every pore voxel v takes the largest r2(c) over
// centres c with |v - c|^2 < r2(c) and d = dx (2 sqrt(r2) - 1).
//
// Counts and distances are integers; the final diameters are fixed
// sequences of IEEE double operations (no fused multiply-add) rounded once
// to float.
#include "common.cuh"

namespace om {
namespace {

__constant__ int8_t c_dir13[13][3] = {{1, 0, 0},  {0, 1, 0},  {0, 0, 1},   {1, 1, 0},  {1, -1, 0},
                                      {1, 0, 1},  {1, 0, -1}, {0, 1, 1},   {0, 1, -1}, {1, 1, 1},
                                      {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};

// cells along +-e from (x,y,z), stopping at solid or the x faces; *closed is
// set when the walk comes back to its start (an all-pore loop)
__device__ int walk(const uint8_t* __restrict__ m, int nx, int ny, int nz, int x, int y, int z, int ex,
                    int ey, int ez, bool* closed) {
  int n = 0, cx = x, cy = y, cz = z;
  *closed = false;
  for (;;) {
    cx += ex;
    if (cx < 0 || cx >= nx) return n;
    cy += ey;
    cy = cy < 0 ? cy + ny : (cy >= ny ? cy - ny : cy);
    cz += ez;
    cz = cz < 0 ? cz + nz : (cz >= nz ? cz - nz : cz);
    if (cx == x && cy == y && cz == z) {
      *closed = true;
      return n;
    }
    if (!m[((int64_t)cx * ny + cy) * nz + cz]) return n;
    ++n;
  }
}

__global__ void chord13_kernel(const uint8_t* __restrict__ m, int nx, int ny, int nz, double dx,
                               double sq2, double sq3, float* d_nm, int32_t* witness) {
  const int64_t N = (int64_t)nx * ny * nz;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    if (!m[v]) {
      d_nm[v] = 0.f;
      if (witness)
        for (int k = 0; k < 13; ++k) witness[k * N + v] = 0;
      continue;
    }
    const int x = (int)(v / ((int64_t)ny * nz));
    const int y = (int)((v / nz) % ny), z = (int)(v % nz);
    long long s[3] = {0, 0, 0};
    for (int k = 0; k < 13; ++k) {
      const int ex = c_dir13[k][0], ey = c_dir13[k][1], ez = c_dir13[k][2];
      bool closed;
      int n = 1 + walk(m, nx, ny, nz, x, y, z, ex, ey, ez, &closed);
      if (!closed) n += walk(m, nx, ny, nz, x, y, z, -ex, -ey, -ez, &closed);
      if (witness) witness[k * N + v] = n;
      s[k < 3 ? 0 : (k < 9 ? 1 : 2)] += n;
    }
    double acc = __dadd_rn(__dadd_rn((double)s[0], __dmul_rn(sq2, (double)s[1])), __dmul_rn(sq3, (double)s[2]));
    acc = __ddiv_rn(acc, 13.0);
    d_nm[v] = (float)__dmul_rn(acc, dx);
  }
}

constexpr int kFar = 0x3fffffff;  // "no solid on this line": larger than any squared distance

// pass 1 (z, periodic): squared distance to the nearest solid in the z line
__global__ void edt_z(const uint8_t* __restrict__ m, int nx, int ny, int nz, int* g) {
  const int64_t N = (int64_t)nx * ny * nz;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    const int z = (int)(v % nz);
    const int64_t base = v - z;
    int best = kFar;
    for (int zz = 0; zz < nz; ++zz)
      if (!m[base + zz]) {
        int dz = abs(z - zz);
        dz = min(dz, nz - dz);
        best = min(best, dz * dz);
      }
    g[v] = best;
  }
}

// pass 2 (y, periodic): min over y' of g(y') + dy^2
__global__ void edt_y(const int* __restrict__ g, int nx, int ny, int nz, int* h) {
  const int64_t N = (int64_t)nx * ny * nz;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    const int z = (int)(v % nz), y = (int)((v / nz) % ny);
    const int64_t base = v - (int64_t)y * nz;
    int best = kFar;
    for (int yy = 0; yy < ny; ++yy) {
      const int a = g[base + (int64_t)yy * nz];
      if (a >= kFar) continue;
      int dy = abs(y - yy);
      dy = min(dy, ny - dy);
      best = min(best, a + dy * dy);
    }
    h[v] = best;
    (void)z;
  }
}

// pass 3 (x, bounded): min over x' of h(x') + dx^2; pore voxels only
__global__ void edt_x(const uint8_t* __restrict__ m, const int* __restrict__ h, int nx, int ny, int nz,
                      int* r2, int* maxr2) {
  const int64_t N = (int64_t)nx * ny * nz;
  const int64_t plane = (int64_t)ny * nz;
  int local = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    if (!m[v]) {
      r2[v] = 0;
      continue;
    }
    const int x = (int)(v / plane);
    const int64_t rem = v - (int64_t)x * plane;
    int best = kFar;
    for (int xx = 0; xx < nx; ++xx) {
      const int a = h[(int64_t)xx * plane + rem];
      if (a >= kFar) continue;
      best = min(best, a + (x - xx) * (x - xx));
    }
    r2[v] = best;
    local = max(local, best);
  }
  for (int o = 16; o > 0; o >>= 1) local = max(local, __shfl_down_sync(0xffffffffu, local, o));
  if ((threadIdx.x & 31) == 0) atomicMax(maxr2, local);
}

// largest inscribed ball holding each pore voxel
__global__ void mis_gather(const uint8_t* __restrict__ m, const int* __restrict__ r2, int nx, int ny, int nz,
                           int R, double dx, float* d_nm) {
  const int64_t N = (int64_t)nx * ny * nz;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    if (!m[v]) {
      d_nm[v] = 0.f;
      continue;
    }
    const int x = (int)(v / ((int64_t)ny * nz));
    const int y = (int)((v / nz) % ny), z = (int)(v % nz);
    int best = 0;
    const int Ry = min(R, ny / 2), Rz = min(R, nz / 2);
    for (int cx = max(0, x - R); cx <= min(nx - 1, x + R); ++cx) {
      const int ddx = (cx - x) * (cx - x);
      for (int oy = -Ry; oy <= Ry - ((ny & 1) == 0 && Ry == ny / 2 ? 1 : 0); ++oy) {
        int cy = y + oy;
        cy = cy < 0 ? cy + ny : (cy >= ny ? cy - ny : cy);
        int dy = abs(oy);
        dy = min(dy, ny - dy);
        const int dxy = ddx + dy * dy;
        const int64_t rowb = ((int64_t)cx * ny + cy) * nz;
        for (int oz = -Rz; oz <= Rz - ((nz & 1) == 0 && Rz == nz / 2 ? 1 : 0); ++oz) {
          int cz = z + oz;
          cz = cz < 0 ? cz + nz : (cz >= nz ? cz - nz : cz);
          int dz = abs(oz);
          dz = min(dz, nz - dz);
          const int rc = r2[rowb + cz];
          if (rc > best && dxy + dz * dz < rc) best = rc;
        }
      }
    }
    const double val = __dsub_rn(__dmul_rn(2.0, sqrt((double)best)), 1.0);
    d_nm[v] = (float)__dmul_rn(val, dx);
  }
}

__global__ void any_solid(const uint8_t* m, int64_t N, int* flag) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    if (!m[v]) {
      *flag = 1;
      return;
    }
}

om_status pore_impl(const uint8_t* m, const om_domain& d, int mode, float* d_nm, int32_t* witness,
                    cudaStream_t s) {
  OM_TRY(check_domain(d));
  if (!m || !d_nm) return fail(OM_EINVAL, "local_pore_diameter: null pointer");
  const int64_t N = voxels(d);
  if (mode == OM_PORE_CHORD13) {
    chord13_kernel<<<4 * 1216, 128, 0, s>>>(m, d.nx, d.ny, d.nz, d.dx_nm, std::sqrt(2.0), std::sqrt(3.0), d_nm,
                                            witness);
    OM_CUDA(cudaGetLastError());
    return OM_OK;
  }
  if (mode != OM_PORE_MIS) return fail(OM_EINVAL, "local_pore_diameter: unknown mode");
  DevBuf<int> g, h, r2own, mx;
  OM_TRY(g.alloc(N));
  OM_TRY(h.alloc(N));
  OM_TRY(mx.alloc(2));
  int* r2 = witness;
  if (!r2) {
    OM_TRY(r2own.alloc(N));
    r2 = r2own.p;
  }
  OM_CUDA(cudaMemsetAsync(mx.p, 0, 2 * sizeof(int), s));
  any_solid<<<1216, 256, 0, s>>>(m, N, mx.p + 1);
  edt_z<<<1216, 256, 0, s>>>(m, d.nx, d.ny, d.nz, g.p);
  edt_y<<<1216, 256, 0, s>>>(g.p, d.nx, d.ny, d.nz, h.p);
  edt_x<<<1216, 256, 0, s>>>(m, h.p, d.nx, d.ny, d.nz, r2, mx.p);
  OM_CUDA(cudaGetLastError());
  int hm[2];
  OM_CUDA(cudaMemcpyAsync(hm, mx.p, sizeof hm, cudaMemcpyDeviceToHost, s));
  OM_CUDA(cudaStreamSynchronize(s));
  if (!hm[1]) return fail(OM_EINVAL, "local_pore_diameter (MIS): the mask has no solid voxel");
  int R = 0;
  while ((int64_t)R * R < hm[0]) ++R;  // ball radius bound: |v - c| < sqrt(r2) <= R
  mis_gather<<<1216, 256, 0, s>>>(m, r2, d.nx, d.ny, d.nz, R, d.dx_nm, d_nm);
  OM_CUDA(cudaGetLastError());
  OM_CUDA(cudaStreamSynchronize(s));
  return OM_OK;
}

}  // namespace
}  // namespace om

using namespace om;

extern "C" om_status om_local_pore_diameter_dev(const uint8_t* mask_dev, om_domain d, int32_t mode,
                                                float* d_nm_dev, int32_t* witness_dev, void* stream) {
  return pore_impl(mask_dev, d, mode, d_nm_dev, witness_dev, as_stream(stream));
}

extern "C" om_status om_local_pore_diameter(const uint8_t* mask, om_domain d, int32_t mode, float* d_nm,
                                            int32_t* witness) {
  if (!mask || !d_nm) return fail(OM_EINVAL, "om_local_pore_diameter: null pointer");
  OM_TRY(check_domain(d));
  const int64_t N = voxels(d);
  const int64_t nw = mode == OM_PORE_CHORD13 ? 13 * N : N;
  cudaStream_t s;
  OM_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  DevBuf<uint8_t> m;
  DevBuf<float> dd;
  DevBuf<int32_t> w;
  om_status st = m.alloc(N);
  if (st == OM_OK) st = dd.alloc(N);
  if (st == OM_OK && witness) st = w.alloc(nw);
  if (st == OM_OK) {
    cudaError_t e = cudaMemcpyAsync(m.p, mask, N, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) st = cuda_fail(e, "copy-in", __FILE__, __LINE__);
  }
  if (st == OM_OK) st = pore_impl(m.p, d, mode, dd.p, witness ? w.p : nullptr, s);
  if (st == OM_OK) {
    cudaError_t e = cudaMemcpyAsync(d_nm, dd.p, N * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && witness) e = cudaMemcpyAsync(witness, w.p, nw * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "copy-out", __FILE__, __LINE__);
  }
  cudaStreamDestroy(s);
  return st;
}
