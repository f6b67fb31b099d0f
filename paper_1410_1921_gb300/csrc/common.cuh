// common.cuh -- shared definitions of the CUDA library behind include/om.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/om.h"

namespace om {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
om_status fail(om_status st, const std::string& msg);
om_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define OM_CUDA(call)                                                        \
  do {                                                                       \
    cudaError_t _e = (call);                                                 \
    if (_e != cudaSuccess) return ::om::cuda_fail(_e, #call, __FILE__, __LINE__); \
  } while (0)

#define OM_TRY(call)                \
  do {                              \
    om_status _s = (call);          \
    if (_s != OM_OK) return _s;     \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

om_status check_domain(const om_domain& d);
inline int64_t voxels(const om_domain& d) { return (int64_t)d.nx * d.ny * d.nz; }

// Device buffer owned by a host scope; freed on destruction.
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  om_status alloc(size_t count) {
    release();
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      (void)cudaGetLastError();
      return fail(OM_ENOMEM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) +
                                 " bytes failed: " + cudaGetErrorString(e));
    }
    n = count;
    return OM_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  T* take() {
    T* q = p;
    p = nullptr;
    n = 0;
    return q;
  }
};

// ------------------------------------------------------------------ lattices
// D3Q19 in the population order of the transformation matrix of App. A:
// rest, +-x, +-y, +-z, then (+-1,+-1,0), (+-1,0,+-1), (0,+-1,+-1) with the
// sign pattern (+,+), (-,+), (+,-), (-,-).
__host__ __device__ constexpr int q19_e(int i, int a) {
  constexpr int8_t E[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                               {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, 1, 0}, {1, -1, 0},
                               {-1, -1, 0}, {1, 0, 1},  {-1, 0, 1}, {1, 0, -1}, {-1, 0, -1},
                               {0, 1, 1},  {0, -1, 1},  {0, 1, -1}, {0, -1, -1}};
  return E[i][a];
}
__host__ __device__ constexpr int q19_opp(int i) {
  constexpr int8_t O[19] = {0, 2, 1, 4, 3, 6, 5, 10, 9, 8, 7, 14, 13, 12, 11, 18, 17, 16, 15};
  return O[i];
}
__host__ __device__ constexpr double q19_w(int i) {
  return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// D3Q7: rest, +x, -x, +y, -y, +z, -z; weights 1/4 and 1/8 (c_s^2 = 1/4).
__host__ __device__ constexpr int q7_e(int i, int a) {
  constexpr int8_t E[7][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
  return E[i][a];
}
__host__ __device__ constexpr int q7_opp(int i) {
  constexpr int8_t O[7] = {0, 2, 1, 4, 3, 6, 5};
  return O[i];
}
__host__ __device__ constexpr double q7_w(int i) { return i == 0 ? 0.25 : 0.125; }

constexpr uint32_t kNoNode = 0xFFFFFFFFu;

// packed node coordinates: x in bits 22..31, y in 11..21, z in 0..10
__host__ __device__ inline uint32_t pack_xyz(int x, int y, int z) {
  return ((uint32_t)x << 22) | ((uint32_t)y << 11) | (uint32_t)z;
}
__host__ __device__ inline void unpack_xyz(uint32_t c, int& x, int& y, int& z) {
  x = (int)(c >> 22);
  y = (int)((c >> 11) & 2047u);
  z = (int)(c & 2047u);
}

// ------------------------------------------------------------------ misc
constexpr int kObsBlocks = 1216;  // 8 x 152 SMs: fixed grid of reductions
constexpr int kObsThreads = 256;

// Blocks of `threads` threads of `kernel` (with `smem` bytes of dynamic
// shared memory) that fit on the device at once (SMs x resident blocks per
// SM), capped at nb: the grid of a kernel whose threads stride over their
// work.  Cached per kernel, launch shape and device.
unsigned resident_blocks(const void* kernel, int threads, size_t smem);
template <class K>
inline unsigned resident_grid(K kernel, unsigned nb, int threads = 256, size_t smem = 0) {
  const unsigned r = resident_blocks((const void*)kernel, threads, smem);
  return nb < r ? nb : r;
}

// Launch variants the autotuner chose, remembered for the life of the
// process per (solver kind, precision, device, octave of the node count):
// the first solver of a class times the variants, later ones reuse the choice.
enum { kTuneFlow = 0, kTuneDiff7 = 1, kTuneDiff19 = 2, kTuneFlowReb = 3 };
bool tuned_lookup(int kind, int prec, int64_t nf, int var[2]);
void tuned_store(int kind, int prec, int64_t nf, const int var[2]);

om_status exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint64_t* total_dev,
                             cudaStream_t s);
// sum the per-block partials [nblk][nval] in fixed order into out[nval]
void launch_finalize(const double* partials, int nblk, int nval, double* out, cudaStream_t s);

}  // namespace om

// The opaque node set of include/om.h.
struct om_nodeset {
  om_domain dom;
  int W = 0;            // 32-voxel words per (x, y) column
  int64_t N = 0;        // voxels
  int64_t nf = 0;       // nodes
  int64_t pitch = 0;    // population array stride (nodes, padded to 64)
  // [nx*ny*W]: {node bits, nodes before this word, node number of the voxel
  // below the word's first and above its last (periodic in z; kNoNode if none)}
  uint4* col = nullptr;
  uint32_t* coord = nullptr;  // [nf] packed x, y, z
  int64_t* vox = nullptr;     // [nf] voxel index
  int64_t wrap_links = 0;     // D3Q19 links from node voxels at x = nx-1 to node voxels at x = 0
  // Neighbour records (lattice.cuh, "neighbour records"): per node the
  // D3Q7 part rec7[n] and the rest of the D3Q19 neighbourhood rec19[n], from
  // which an odd sweep derives its neighbours' node numbers without the
  // column map; nodes on a face of the box (where neighbours wrap or an x
  // face is crossed) carry the "slow" mark and are listed in slow[n_slow]
  // (ascending), updated through the column map instead.  rec7 == nullptr
  // when the box is too large for the record fields (then no sweep uses them).
  uint2* rec7 = nullptr;
  uint2* rec19 = nullptr;
  uint32_t* slow = nullptr;
  int64_t n_slow = 0;
};
