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
#include "lattice.cuh"

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

// R_c(z) (nodes before voxel (x, y, z)) and whether that voxel is a node
__device__ __forceinline__ void ns_rank_bit(const uint4* col, int ny, int W, int x, int y, int z, uint32_t& r,
                                            uint32_t& bit) {
  const uint4 w = col[((int64_t)x * ny + y) * W + (z >> 5)];
  r = w.y + __popc(w.x & ((1u << (z & 31)) - 1u));
  bit = (w.x >> (z & 31)) & 1u;
}

// The neighbour records of lattice.cuh for every node, and a 0/1 "slow" flag
// per node (a face of the box, or a box beyond the record fields: !fit).
__global__ void ns_records(const uint4* col, const uint32_t* coord, int64_t nf, int nx, int ny, int nz, int W,
                           int fit, uint2* rec7, uint2* rec19, uint32_t* slow) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nf) return;
  int x, y, z;
  unpack_xyz(coord[n], x, y, z);
  if (!fit || x == 0 || x == nx - 1 || y == 0 || y == ny - 1 || z == 0 || z == nz - 1) {
    rec7[n] = make_uint2(kRecSlow, 0u);
    rec19[n] = make_uint2(0u, 0u);
    slow[n] = 1u;
    return;
  }
  const uint32_t nn = (uint32_t)n;
  uint32_t rxp, bxp, rxm, bxm, ryp, byp, rym, bym, r;
  ns_rank_bit(col, ny, W, x + 1, y, z, rxp, bxp);
  ns_rank_bit(col, ny, W, x - 1, y, z, rxm, bxm);
  ns_rank_bit(col, ny, W, x, y + 1, z, ryp, byp);
  ns_rank_bit(col, ny, W, x, y - 1, z, rym, bym);
  uint32_t szp, szm;
  ns_rank_bit(col, ny, W, x, y, z + 1, r, szp);
  ns_rank_bit(col, ny, W, x, y, z - 1, r, szm);
  uint2 a;
  a.x = (rxp - nn - 1u) | ((ryp - nn - 1u) << 19) | (bxp << 29) | (byp << 30) | (szp << 31);
  a.y = (nn - rxm) | ((nn - rym) << 19) | (bxm << 29) | (bym << 30) | (szm << 31);
  uint32_t r1, b1, r2, b2, r3, b3, r4, b4;
  ns_rank_bit(col, ny, W, x + 1, y + 1, z, r1, b1);
  ns_rank_bit(col, ny, W, x + 1, y - 1, z, r2, b2);
  ns_rank_bit(col, ny, W, x - 1, y + 1, z, r3, b3);
  ns_rank_bit(col, ny, W, x - 1, y - 1, z, r4, b4);
  uint32_t zb[8];
  ns_rank_bit(col, ny, W, x + 1, y, z - 1, r, zb[0]);
  ns_rank_bit(col, ny, W, x + 1, y, z + 1, r, zb[1]);
  ns_rank_bit(col, ny, W, x - 1, y, z - 1, r, zb[2]);
  ns_rank_bit(col, ny, W, x - 1, y, z + 1, r, zb[3]);
  ns_rank_bit(col, ny, W, x, y + 1, z - 1, r, zb[4]);
  ns_rank_bit(col, ny, W, x, y + 1, z + 1, r, zb[5]);
  ns_rank_bit(col, ny, W, x, y - 1, z - 1, r, zb[6]);
  ns_rank_bit(col, ny, W, x, y - 1, z + 1, r, zb[7]);
  uint2 q;
  q.x = (r1 - rxp) | ((rxp - r2) << 10) | ((r3 - rxm) << 20) | (b1 << 30) | (b2 << 31);
  q.y = (rxm - r4) | (b3 << 10) | (b4 << 11);
  for (int k = 0; k < 8; ++k) q.y |= zb[k] << (12 + k);
  rec7[n] = a;
  rec19[n] = q;
  slow[n] = 0u;
}

__global__ void ns_slow_list(const uint32_t* flag, const uint32_t* pos, int64_t nf, uint32_t* list) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n < nf && flag[n]) list[pos[n]] = (uint32_t)n;
}

}  // namespace om

using namespace om;

namespace {
// The neighbour records and the list of slow nodes (see lattice.cuh).
om_status build_records(om_nodeset* ns, cudaStream_t s) {
  const om_domain& d = ns->dom;
  const int64_t nf = ns->nf;
  const int fit = d.nz <= kRecMaxNz && (int64_t)d.ny * d.nz <= kRecMaxPlane;
  DevBuf<uint2> r7, r19;
  DevBuf<uint32_t> flag, pos, list;
  DevBuf<uint64_t> total;
  OM_TRY(r7.alloc(nf));
  OM_TRY(r19.alloc(nf));
  OM_TRY(flag.alloc(nf));
  OM_TRY(pos.alloc(nf));
  OM_TRY(total.alloc(1));
  const unsigned nb = (unsigned)((nf + 255) / 256);
  ns_records<<<nb, 256, 0, s>>>(ns->col, ns->coord, nf, d.nx, d.ny, d.nz, ns->W, fit, r7.p, r19.p, flag.p);
  OM_CUDA(cudaGetLastError());
  OM_TRY(exclusive_scan_u32(flag.p, pos.p, nf, total.p, s));
  uint64_t nslow = 0;
  OM_CUDA(cudaMemcpyAsync(&nslow, total.p, sizeof nslow, cudaMemcpyDeviceToHost, s));
  OM_CUDA(cudaStreamSynchronize(s));
  OM_TRY(list.alloc(nslow));
  ns_slow_list<<<nb, 256, 0, s>>>(flag.p, pos.p, nf, list.p);
  OM_CUDA(cudaGetLastError());
  OM_CUDA(cudaStreamSynchronize(s));
  ns->rec7 = fit ? r7.take() : nullptr;
  ns->rec19 = fit ? r19.take() : nullptr;
  ns->slow = list.take();
  ns->n_slow = (int64_t)nslow;
  return OM_OK;
}
}  // namespace

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
  if (nf > 0) {
    om_status rs = build_records(ns, s);
    if (rs != OM_OK) {
      om_nodeset_destroy(ns);
      return rs;
    }
  }
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
  cudaFree(ns->rec7);
  cudaFree(ns->rec19);
  cudaFree(ns->slow);
  delete ns;
  return OM_OK;
}
