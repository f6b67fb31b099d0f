// nodeset.cu -- the fluid-node layout of the LB sweeps.
//
// Lattice nodes (transport voxels) are numbered in lexicographic voxel order
// and their populations stored densely by that number, so no solid voxel
// occupies memory or bandwidth.  A neighbour's node number is not stored:
// each (x, y) column keeps, per 32 voxels in z, a bit map of nodes and the
// number of nodes that precede the word, and
//     node(x, y, z) = rank[w] + popc(bits[w] & ((1 << (z & 31)) - 1)),
//     w = column word of z,
// plus the node numbers of the voxel just below the word's first and just
// above its last (periodic in z), so that z - 1, z, z + 1 of any column come
// from one 16-byte word without branches.  16 bytes per 32 voxels (the whole
// map sits in L2) instead of an 18-entry neighbour table per node.
#include "common.cuh"

namespace om {

__global__ void ns_bits(const uint8_t* nodes, int ny, int nz, int W, int64_t ncol, uint32_t* bits,
                        uint32_t* cnt) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // word index
  if (k >= ncol * W) return;
  int64_t c = k / W;
  int w = (int)(k - c * W);
  const uint8_t* p = nodes + c * nz;
  uint32_t b = 0;
  int z0 = w * 32;
  int z1 = min(nz, z0 + 32);
  for (int z = z0; z < z1; ++z) b |= (p[z] ? 1u : 0u) << (z - z0);
  bits[k] = b;
  cnt[k] = __popc(b);
}

// node number of voxel z of the column whose first word is k0, or kNoNode
__device__ __forceinline__ uint32_t ns_node(const uint32_t* bits, const uint32_t* rank, int64_t k0, int z) {
  const int64_t k = k0 + (z >> 5);
  const uint32_t bit = 1u << (z & 31);
  return (bits[k] & bit) ? rank[k] + __popc(bits[k] & (bit - 1u)) : kNoNode;
}

__global__ void ns_fill(const uint32_t* bits, const uint32_t* rank, int ny, int nz, int W,
                        int64_t nwords, uint4* col, uint32_t* coord, int64_t* vox) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nwords) return;
  uint32_t b = bits[k], r = rank[k];
  int64_t c = k / W;
  int w = (int)(k - c * W);
  const int zprev = w == 0 ? nz - 1 : 32 * w - 1;      // below the word's first voxel
  const int znext = 32 * w + 32 >= nz ? 0 : 32 * w + 32;  // above its last (nz - 1 in the last word)
  col[k] = make_uint4(b, r, ns_node(bits, rank, c * W, zprev), ns_node(bits, rank, c * W, znext));
  int x = (int)(c / ny), y = (int)(c - (int64_t)x * ny);
  while (b) {
    int bit = __ffs(b) - 1;
    b &= b - 1;
    int z = w * 32 + bit;
    coord[r] = pack_xyz(x, y, z);
    vox[r] = c * nz + z;
    ++r;
  }
}

// Links of the flow lattice across the periodic x boundary: node voxels
// (nx-1, y, z) whose neighbour (0, y + dy, z + dz), |dy| + |dz| <= 1, along
// one of the five velocities with e_x = +1, is a node voxel (y, z periodic).
// Without any, the x wrap is a wall for the flow and its steady net flux is
// zero.
__global__ void ns_wrap_links(const uint8_t* nodes, int nx, int ny, int nz, unsigned long long* count) {
  const int64_t plane = (int64_t)ny * nz;
  const uint8_t* last = nodes + (int64_t)(nx - 1) * plane;
  unsigned long long c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += (int64_t)gridDim.x * blockDim.x) {
    if (!last[i]) continue;
    const int y = (int)(i / nz), z = (int)(i - (int64_t)y * nz);
    const int yp = y + 1 == ny ? 0 : y + 1, ym = y == 0 ? ny - 1 : y - 1;
    const int zp = z + 1 == nz ? 0 : z + 1, zm = z == 0 ? nz - 1 : z - 1;
    c += nodes[(int64_t)y * nz + z] != 0;
    c += nodes[(int64_t)yp * nz + z] != 0;
    c += nodes[(int64_t)ym * nz + z] != 0;
    c += nodes[(int64_t)y * nz + zp] != 0;
    c += nodes[(int64_t)y * nz + zm] != 0;
  }
  if (c) atomicAdd(count, c);
}

}  // namespace om

using namespace om;

extern "C" om_status om_nodeset_create(const uint8_t* nodes_dev, om_domain d, void* stream,
                                       om_nodeset** out) {
  if (!nodes_dev || !out) return fail(OM_EINVAL, "om_nodeset_create: null pointer");
  OM_TRY(check_domain(d));
  cudaStream_t s = as_stream(stream);
  const int W = (d.nz + 31) / 32;
  const int64_t ncol = (int64_t)d.nx * d.ny;
  const int64_t nw = ncol * W;
  DevBuf<uint32_t> bits, cnt, rank;
  DevBuf<uint64_t> total;
  DevBuf<unsigned long long> wrap;
  OM_TRY(bits.alloc(nw));
  OM_TRY(cnt.alloc(nw));
  OM_TRY(rank.alloc(nw));
  OM_TRY(total.alloc(1));
  OM_TRY(wrap.alloc(1));
  OM_CUDA(cudaMemsetAsync(wrap.p, 0, sizeof(unsigned long long), s));
  ns_bits<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(nodes_dev, d.ny, d.nz, W, ncol, bits.p, cnt.p);
  ns_wrap_links<<<152, 256, 0, s>>>(nodes_dev, d.nx, d.ny, d.nz, wrap.p);
  OM_CUDA(cudaGetLastError());
  OM_TRY(exclusive_scan_u32(cnt.p, rank.p, nw, total.p, s));
  uint64_t nf = 0;
  unsigned long long nwrap = 0;
  OM_CUDA(cudaMemcpyAsync(&nf, total.p, sizeof nf, cudaMemcpyDeviceToHost, s));
  OM_CUDA(cudaMemcpyAsync(&nwrap, wrap.p, sizeof nwrap, cudaMemcpyDeviceToHost, s));
  OM_CUDA(cudaStreamSynchronize(s));

  om_nodeset* ns = new om_nodeset();
  ns->dom = d;
  ns->W = W;
  ns->N = voxels(d);
  ns->nf = (int64_t)nf;
  ns->pitch = ((int64_t)nf + 63) / 64 * 64;
  ns->wrap_links = (int64_t)nwrap;
  DevBuf<uint4> col;
  DevBuf<uint32_t> coord;
  DevBuf<int64_t> vox;
  om_status st = col.alloc(nw);
  if (st == OM_OK) st = coord.alloc(nf);
  if (st == OM_OK) st = vox.alloc(nf);
  if (st != OM_OK) {
    delete ns;
    return st;
  }
  ns_fill<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(bits.p, rank.p, d.ny, d.nz, W, nw, col.p,
                                                      coord.p, vox.p);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    delete ns;
    return cuda_fail(e, "om_nodeset_create fill", __FILE__, __LINE__);
  }
  ns->col = col.take();
  ns->coord = coord.take();
  ns->vox = vox.take();
  *out = ns;
  return OM_OK;
}

extern "C" om_status om_nodeset_count(const om_nodeset* ns, int64_t* n_nodes) {
  if (!ns || !n_nodes) return fail(OM_EINVAL, "om_nodeset_count: null pointer");
  *n_nodes = ns->nf;
  return OM_OK;
}

extern "C" om_status om_nodeset_voxels(const om_nodeset* ns, int64_t* voxel_dev, void* stream) {
  if (!ns || !voxel_dev) return fail(OM_EINVAL, "om_nodeset_voxels: null pointer");
  if (ns->nf > 0)
    OM_CUDA(cudaMemcpyAsync(voxel_dev, ns->vox, sizeof(int64_t) * ns->nf, cudaMemcpyDeviceToDevice,
                            as_stream(stream)));
  return OM_OK;
}

extern "C" om_status om_nodeset_destroy(om_nodeset* ns) {
  if (!ns) return OM_OK;
  cudaFree(ns->col);
  cudaFree(ns->coord);
  cudaFree(ns->vox);
  delete ns;
  return OM_OK;
}
