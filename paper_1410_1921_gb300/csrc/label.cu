// label.cu -- connected-phase labelling (Sec. 4.1) on the GPU.
//
// Pore voxels are joined with their 18 neighbours (the D3Q19 links; y and z
// periodic, x not) by a lock-free union-find: a root is only ever linked
// below a smaller index, so every component ends as a tree rooted at its
// smallest voxel index, the canonical label.  Runs of pore voxels along z
// start as single trees, and two runs that touch along several voxels are
// joined once, at the lowest voxel of their overlap.  Transport voxels belong to a
// component with voxels on both x faces.
#include <algorithm>

#include "common.cuh"

namespace om {
namespace {

__device__ __forceinline__ int uf_find(volatile int* par, int x) {
  int p = par[x];
  while (p != x) {
    const int gp = par[p];
    if (gp != p) par[x] = gp;  // path halving: only ever points further up
    x = p;
    p = gp;
  }
  return x;
}

__device__ __forceinline__ void uf_union(int* par, int a, int b) {
  for (;;) {
    a = uf_find(par, a);
    b = uf_find(par, b);
    if (a == b) return;
    if (a < b) {
      const int t = a;
      a = b;
      b = t;
    }
    const int old = atomicCAS(par + a, a, b);  // link the larger root below the smaller
    if (old == a) return;
    a = old;
  }
}

// Runs of pore voxels along z (not wrapping at z = 0) start as one tree
// each: every voxel points at the first voxel of its run, which is its own
// root and the run's smallest index.  One thread per (x, y) column.
__global__ void uf_init_runs(const uint8_t* mask, int64_t ncol, int nz, int* par) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncol; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t base = c * nz;
    int head = -1;
    for (int z = 0; z < nz; ++z) {
      const int64_t v = base + z;
      if (!mask[v]) {
        par[v] = -1;
        head = -1;
        continue;
      }
      if (head < 0) head = (int)v;
      par[v] = head;
    }
  }
}

// The forward half of the 18 neighbour offsets (the other half is the same
// pairs seen from the other voxel).  Voxel v is joined to its neighbour u =
// v + o unless the pair one step lower in z, (v - 1, u - 1), is a pore pair
// inside the same two runs: that pair already joins the two runs.  So each
// overlap of two runs issues one union, at its lowest voxel.  One block row
// of threads per (x, y) column, threads along z: no 64-bit index division.
__global__ void uf_link_runs(const uint8_t* mask, int nx, int ny, int nz, int* par) {
  constexpr int8_t H[9][3] = {{1, 0, 0}, {1, 1, 0}, {1, -1, 0}, {1, 0, 1}, {1, 0, -1},
                              {0, 1, 0}, {0, 1, 1}, {0, 1, -1}, {0, 0, 1}};
  const int64_t ncol = (int64_t)nx * ny;
  for (int64_t c = blockIdx.x; c < ncol; c += gridDim.x) {
    const int x = (int)(c / ny), y = (int)(c - (int64_t)x * ny);
    const int64_t base = c * nz;
    for (int z = threadIdx.x; z < nz; z += blockDim.x) {
      const int64_t v = base + z;
      if (!mask[v]) continue;
      const bool below = z > 0 && mask[v - 1];  // v - 1 in the same run
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const int xx = x + H[k][0];
        if (xx >= nx) continue;
        int yy = y + H[k][1], zz = z + H[k][2];
        yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
        zz = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
        const int64_t u = ((int64_t)xx * ny + yy) * nz + zz;
        if (!mask[u]) continue;
        if (k == 8 && zz > 0) continue;              // z + 1 without wrap: the same run
        if (below && zz > 0 && mask[u - 1]) continue;  // (v-1, u-1) joins these runs
        uf_union(par, (int)v, (int)u);
      }
    }
  }
}

// Root without path compression.  The flatten pass must not compress: a
// compressing walk could overwrite a root another thread has just stored
// with an intermediate ancestor it read earlier.
__device__ __forceinline__ int uf_root(const volatile int* par, int x) {
  int p = par[x];
  while (p != x) {
    x = p;
    p = par[x];
  }
  return x;
}

__global__ void uf_flatten(int* par, int64_t N) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    if (par[v] >= 0) par[v] = uf_root(par, (int)v);
}

__global__ void mark_faces(const int* lab, int nx, int ny, int nz, uint8_t* touch) {
  const int64_t plane = (int64_t)ny * nz;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += (int64_t)gridDim.x * blockDim.x) {
    // flag bytes are set through their aligned 32-bit word: bit 0 inlet, bit 1 outlet
    const int a = lab[i];
    if (a >= 0) atomicOr((unsigned int*)(touch + (a & ~3)), 1u << (8 * (a & 3)));
    const int b = lab[(int64_t)(nx - 1) * plane + i];
    if (b >= 0) atomicOr((unsigned int*)(touch + (b & ~3)), 2u << (8 * (b & 3)));
  }
}

__global__ void transport_from_labels(const int* lab, const uint8_t* touch, int64_t N, uint8_t* tr,
                                      unsigned long long* counts) {
  unsigned long long np = 0, nt = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    const int a = lab[v];
    const bool t = a >= 0 && touch[a] == 3;
    if (tr) tr[v] = t ? 1 : 0;
    np += a >= 0;
    nt += t;
  }
  for (int o = 16; o > 0; o >>= 1) {
    np += __shfl_down_sync(0xffffffffu, np, o);
    nt += __shfl_down_sync(0xffffffffu, nt, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(counts, np);
    atomicAdd(counts + 1, nt);
  }
}

}  // namespace

void launch_union_find(const uint8_t* mask_dev, const om_domain& d, int* labels_dev, cudaStream_t s);

// labels (int32 N) and transport flags on the device; counts of pore and
// transport voxels returned through the host pointers when non-null.
om_status label_impl(const uint8_t* mask_dev, const om_domain& d, int* labels_dev, uint8_t* transport_dev,
                     int64_t* npore, int64_t* ntrans, cudaStream_t s) {
  const int64_t N = voxels(d);
  if (N >= (int64_t)0x7fffffff) return fail(OM_EINVAL, "labelling needs fewer than 2^31 voxels");
  // mark_faces sets flag bytes through 32-bit words: pad to a multiple of 4
  DevBuf<uint8_t> touch;
  DevBuf<unsigned long long> cnt;
  OM_TRY(touch.alloc((N + 3) / 4 * 4));
  OM_TRY(cnt.alloc(2));
  OM_CUDA(cudaMemsetAsync(touch.p, 0, (N + 3) / 4 * 4, s));
  OM_CUDA(cudaMemsetAsync(cnt.p, 0, 2 * sizeof(unsigned long long), s));
  launch_union_find(mask_dev, d, labels_dev, s);
  mark_faces<<<152, 256, 0, s>>>(labels_dev, d.nx, d.ny, d.nz, touch.p);
  transport_from_labels<<<1216, 256, 0, s>>>(labels_dev, touch.p, N, transport_dev, cnt.p);
  OM_CUDA(cudaGetLastError());
  unsigned long long h[2];
  OM_CUDA(cudaMemcpyAsync(h, cnt.p, sizeof h, cudaMemcpyDeviceToHost, s));
  OM_CUDA(cudaStreamSynchronize(s));
  if (npore) *npore = (int64_t)h[0];
  if (ntrans) *ntrans = (int64_t)h[1];
  return OM_OK;
}

// Union-find labelling alone (labels_dev: int32 N, written), for callers
// that bring their own flag storage.
void launch_union_find(const uint8_t* mask_dev, const om_domain& d, int* labels_dev, cudaStream_t s) {
  const int64_t N = voxels(d), ncol = (int64_t)d.nx * d.ny;
  const int zt = d.nz >= 128 ? 128 : (d.nz >= 64 ? 64 : 32);  // threads along z per column
  uf_init_runs<<<(unsigned)std::min<int64_t>((ncol + 255) / 256, 4864), 256, 0, s>>>(mask_dev, ncol, d.nz,
                                                                                     labels_dev);
  uf_link_runs<<<(unsigned)std::min<int64_t>(ncol, 152 * 64), zt, 0, s>>>(mask_dev, d.nx, d.ny, d.nz, labels_dev);
  uf_flatten<<<1216, 256, 0, s>>>(labels_dev, N);
}

}  // namespace om

using namespace om;

extern "C" om_status om_label_connectivity_dev(const uint8_t* mask_dev, om_domain d, int32_t* labels_dev,
                                               uint8_t* transport_dev, double* connectivity_out,
                                               void* stream) {
  if (!mask_dev) return fail(OM_EINVAL, "om_label_connectivity_dev: null mask");
  OM_TRY(check_domain(d));
  cudaStream_t s = as_stream(stream);
  DevBuf<int> lab;
  int* lp = labels_dev;
  if (!lp) {
    OM_TRY(lab.alloc(voxels(d)));
    lp = lab.p;
  }
  int64_t np = 0, nt = 0;
  OM_TRY(label_impl(mask_dev, d, lp, transport_dev, &np, &nt, s));
  if (connectivity_out) *connectivity_out = np > 0 ? (double)nt / (double)np : 0.0;
  return OM_OK;
}

extern "C" om_status om_label_connectivity(const uint8_t* mask, om_domain d, int32_t* labels,
                                           uint8_t* transport, double* connectivity_out) {
  if (!mask) return fail(OM_EINVAL, "om_label_connectivity: null mask");
  OM_TRY(check_domain(d));
  const int64_t N = voxels(d);
  cudaStream_t s;
  OM_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  DevBuf<uint8_t> m, tr;
  DevBuf<int> lab;
  om_status st = m.alloc(N);
  if (st == OM_OK) st = tr.alloc(N);
  if (st == OM_OK) st = lab.alloc(N);
  if (st == OM_OK) {
    cudaError_t e = cudaMemcpyAsync(m.p, mask, N, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) st = cuda_fail(e, "copy-in", __FILE__, __LINE__);
  }
  int64_t np = 0, nt = 0;
  if (st == OM_OK) st = label_impl(m.p, d, lab.p, tr.p, &np, &nt, s);
  if (st == OM_OK) {
    cudaError_t e = cudaSuccess;
    if (labels) e = cudaMemcpyAsync(labels, lab.p, N * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && transport) e = cudaMemcpyAsync(transport, tr.p, N, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "copy-out", __FILE__, __LINE__);
    if (connectivity_out) *connectivity_out = np > 0 ? (double)nt / (double)np : 0.0;
  }
  cudaStreamDestroy(s);
  return st;
}
