// label.cu -- connected-phase labelling (Sec. 4.1) on the GPU.
//
// Pore voxels are joined with their 18 neighbours (the D3Q19 links; y and z
// periodic, x not) by a lock-free union-find: a root is only ever linked
// below a smaller index, so every component ends as a tree rooted at its
// smallest voxel index, the canonical label.  Transport voxels belong to a
// component with voxels on both x faces.
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

__global__ void uf_init(const uint8_t* mask, int64_t N, int* par) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    par[v] = mask[v] ? (int)v : -1;
}

// the forward half of the 18 neighbour offsets; the other half is the same
// pairs seen from the other voxel
__global__ void uf_link(const uint8_t* mask, int nx, int ny, int nz, int* par) {
  constexpr int8_t H[9][3] = {{1, 0, 0}, {1, 1, 0}, {1, -1, 0}, {1, 0, 1}, {1, 0, -1},
                              {0, 1, 0}, {0, 1, 1}, {0, 1, -1}, {0, 0, 1}};
  const int64_t N = (int64_t)nx * ny * nz;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    if (!mask[v]) continue;
    const int x = (int)(v / ((int64_t)ny * nz));
    const int y = (int)((v / nz) % ny), z = (int)(v % nz);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int xx = x + H[k][0];
      if (xx >= nx) continue;
      int yy = y + H[k][1], zz = z + H[k][2];
      yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
      zz = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
      const int64_t u = ((int64_t)xx * ny + yy) * nz + zz;
      if (mask[u]) uf_union(par, (int)v, (int)u);
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
  uf_init<<<1216, 256, 0, s>>>(mask_dev, N, labels_dev);
  uf_link<<<1216, 256, 0, s>>>(mask_dev, d.nx, d.ny, d.nz, labels_dev);
  uf_flatten<<<1216, 256, 0, s>>>(labels_dev, N);
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
  const int64_t N = voxels(d);
  uf_init<<<1216, 256, 0, s>>>(mask_dev, N, labels_dev);
  uf_link<<<1216, 256, 0, s>>>(mask_dev, d.nx, d.ny, d.nz, labels_dev);
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
