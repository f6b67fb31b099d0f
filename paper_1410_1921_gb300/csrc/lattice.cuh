// lattice.cuh -- storage traits and neighbour lookups shared by the D3Q19
// flow and D3Q7 diffusion sweeps.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace om {

// Population storage.  Values are stored as deviations from a reference
// state (w_i for flow, a_i C_lin(x) for diffusion).  Reduced-precision
// storage also multiplies by a power-of-two scale (`up` on store, `down` on
// load) so the deviations sit in the normal range of the format.
template <class T>
struct Stg;

template <>
struct Stg<double> {
  using C = double;
  __device__ __forceinline__ static C ld(const double* p, C) { return *p; }
  __device__ __forceinline__ static void st(double* p, C v, C) { *p = v; }
};
template <>
struct Stg<float> {
  using C = float;
  __device__ __forceinline__ static C ld(const float* p, C) { return *p; }
  __device__ __forceinline__ static void st(float* p, C v, C) { *p = v; }
};
template <>
struct Stg<__half> {
  using C = float;
  __device__ __forceinline__ static C ld(const __half* p, C down) { return __half2float(*p) * down; }
  __device__ __forceinline__ static void st(__half* p, C v, C up) { *p = __float2half_rn(v * up); }
};
template <>
struct Stg<__nv_bfloat16> {
  using C = float;
  __device__ __forceinline__ static C ld(const __nv_bfloat16* p, C down) {
    return __bfloat162float(*p) * down;
  }
  __device__ __forceinline__ static void st(__nv_bfloat16* p, C v, C up) {
    *p = __float2bfloat16_rn(v * up);
  }
};

// Two consecutive nodes' values of one population as one vector access (the
// even sweeps that update two nodes per thread): the same conversions and
// rounding as Stg<T>::ld / st, element by element.  p must be 2-element
// aligned (an even node number in a slot array of even pitch).
template <class T>
struct Pair;
template <>
struct Pair<double> {
  __device__ __forceinline__ static void ld(const double* p, double, double& a, double& b) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    a = v.x;
    b = v.y;
  }
  __device__ __forceinline__ static void st(double* p, double a, double b, double) {
    *reinterpret_cast<double2*>(p) = make_double2(a, b);
  }
};
template <>
struct Pair<float> {
  __device__ __forceinline__ static void ld(const float* p, float, float& a, float& b) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    a = v.x;
    b = v.y;
  }
  __device__ __forceinline__ static void st(float* p, float a, float b, float) {
    *reinterpret_cast<float2*>(p) = make_float2(a, b);
  }
};
template <>
struct Pair<__half> {
  __device__ __forceinline__ static void ld(const __half* p, float down, float& a, float& b) {
    const float2 v = __half22float2(*reinterpret_cast<const __half2*>(p));
    a = v.x * down;
    b = v.y * down;
  }
  __device__ __forceinline__ static void st(__half* p, float a, float b, float up) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a * up, b * up);
  }
};
template <>
struct Pair<__nv_bfloat16> {
  __device__ __forceinline__ static void ld(const __nv_bfloat16* p, float down, float& a, float& b) {
    const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
    a = v.x * down;
    b = v.y * down;
  }
  __device__ __forceinline__ static void st(__nv_bfloat16* p, float a, float b, float up) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a * up, b * up);
  }
};

// Storage S rebased on a per-node reference (the flow's rebased mode): the
// same bits in memory as S; the type only selects the kernels that apply the
// reference (kFlowRebased in flow_core.cuh).
template <class S>
struct Reb {
  using base = S;
  S v;
};
// the storage type without the rebased tag
template <class T>
struct Plain {
  using type = T;
};
template <class S>
struct Plain<Reb<S>> {
  using type = S;
};
template <class S>
struct Stg<Reb<S>> {
  using C = typename Stg<S>::C;
  __device__ __forceinline__ static C ld(const Reb<S>* p, C down) { return Stg<S>::ld(&p->v, down); }
  __device__ __forceinline__ static void st(Reb<S>* p, C v, C up) { Stg<S>::st(&p->v, v, up); }
};
template <class S>
struct Pair<Reb<S>> {
  using C = typename Stg<S>::C;
  __device__ __forceinline__ static void ld(const Reb<S>* p, C down, C& a, C& b) {
    Pair<S>::ld(reinterpret_cast<const S*>(p), down, a, b);
  }
  __device__ __forceinline__ static void st(Reb<S>* p, C a, C b, C up) {
    Pair<S>::st(reinterpret_cast<S*>(p), a, b, up);
  }
};

// Node number of voxel (x, y, z) from its column's bit map, or kNoNode.
// Column-map indices fit 32 bits (nx*ny*W <= 1024*2048*64).
__device__ __forceinline__ uint32_t node_at(const uint4* __restrict__ col, int ny, int W, int x,
                                            int y, int z) {
  const uint32_t k = ((uint32_t)x * (uint32_t)ny + (uint32_t)y) * (uint32_t)W + ((uint32_t)z >> 5);
  const uint2 b = __ldg(reinterpret_cast<const uint2*>(col + k));
  const uint32_t bit = 1u << (z & 31);
  return (b.x & bit) ? b.y + __popc(b.x & (bit - 1u)) : kNoNode;
}

// Where z sits in its 32-voxel column word, worked out once per node and
// shared by the lookups in all neighbour columns: first / last say that
// z - 1 / z + 1 (periodic in z) lies outside the word, where the word's own
// prev / next fields give its node number.
struct ZPos {
  uint32_t w;      // word index within the column
  uint32_t zb;     // bit of z within the word
  uint32_t below;  // bits of the word below z
  bool first, last;
};

__device__ __forceinline__ ZPos zpos(int z, int nz) {
  ZPos p;
  p.w = (uint32_t)z >> 5;
  p.zb = (uint32_t)z & 31u;
  p.below = (1u << p.zb) - 1u;
  p.first = p.zb == 0;
  p.last = p.zb == 31 || z == nz - 1;
  return p;
}

// Node numbers of the voxels z - 1, z, z + 1 (periodic) of one (x, y) column
// from one 16-byte word: a popcount gives z's rank, its neighbours inside
// the word are one rank away, and the word's prev / next fields hold the
// node numbers across the word edge and the periodic wrap.  Branch-free.
__device__ __forceinline__ void column3(const uint4* __restrict__ col, uint32_t base, const ZPos& p,
                                        uint32_t& rm, uint32_t& r0, uint32_t& rp) {
  const uint4 w = __ldg(col + base + p.w);
  const uint32_t rank0 = w.y + __popc(w.x & p.below);
  const uint32_t b0 = (w.x >> p.zb) & 1u;
  const uint32_t bp = ((w.x >> p.zb) >> 1) & 1u;  // z + 1 inside the word
  const uint32_t bm = ((w.x << 1) >> p.zb) & 1u;  // z - 1 inside the word
  r0 = b0 ? rank0 : kNoNode;
  rp = p.last ? w.w : (bp ? rank0 + b0 : kNoNode);
  rm = p.first ? w.z : (bm ? rank0 - 1u : kNoNode);
}

__device__ __forceinline__ uint32_t column1(const uint4* __restrict__ col, uint32_t base, const ZPos& p) {
  const uint2 w = __ldg(reinterpret_cast<const uint2*>(col + base + p.w));
  return ((w.x >> p.zb) & 1u) ? w.y + __popc(w.x & p.below) : kNoNode;
}

// nb[i] = node number of x + e_i for the D3Q19 velocities (kNoNode off the
// node set) of the node with packed coordinates c; periodic y, z, and x when
// px (else no neighbour beyond the x faces).
__device__ __forceinline__ void q19_neighbours(const uint4* __restrict__ col, int nx, int ny, int nz, int W,
                                               int px, uint32_t c, uint32_t (&nb)[19]) {
  int x, y, z;
  unpack_xyz(c, x, y, z);
  const int xp = x + 1 == nx ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
  const bool hp = px || x + 1 < nx, hm = px || x > 0;
  const int yp = y + 1 == ny ? 0 : y + 1, ym = y == 0 ? ny - 1 : y - 1;
  const ZPos p = zpos(z, nz);
  const uint32_t uy = (uint32_t)ny, uW = (uint32_t)W;
  auto base = [&](int xx, int yy) { return ((uint32_t)xx * uy + (uint32_t)yy) * uW; };
  uint32_t self;
  column3(col, base(x, y), p, nb[6], self, nb[5]);
  if (hp) {
    column3(col, base(xp, y), p, nb[13], nb[1], nb[11]);
    nb[7] = column1(col, base(xp, yp), p);
    nb[9] = column1(col, base(xp, ym), p);
  } else {
    nb[13] = nb[1] = nb[11] = nb[7] = nb[9] = kNoNode;
  }
  if (hm) {
    column3(col, base(xm, y), p, nb[14], nb[2], nb[12]);
    nb[8] = column1(col, base(xm, yp), p);
    nb[10] = column1(col, base(xm, ym), p);
  } else {
    nb[14] = nb[2] = nb[12] = nb[8] = nb[10] = kNoNode;
  }
  column3(col, base(x, yp), p, nb[17], nb[3], nb[15]);
  column3(col, base(x, ym), p, nb[18], nb[4], nb[16]);
  (void)self;
}

// Neighbour records.  For a node n at (x, y, z) away from every face of the
// box, R_c(z) = the number of nodes that precede voxel (c, z) in voxel order
// (its node number if it is a node) differs from n by a bounded amount for
// each of the eight columns c = (x +- 1, y), (x, y +- 1), (x +- 1, y +- 1),
// and the neighbours at z +- 1 of a column are R_c(z) + [voxel (c, z) is a
// node] and R_c(z) - 1.  Two 8-byte words per node hold those differences and
// the node bits of the 18 neighbour voxels, so an odd sweep gets every
// neighbour's node number from its own coalesced record with integer adds:
//   rec7.x : [0,19) R(x+1,y) - n - 1 (all ones: "slow" node), [19,29)
//            R(x,y+1) - n - 1, bit 29 (x+1,y,z), 30 (x,y+1,z), 31 (x,y,z+1)
//   rec7.y : [0,19) n - R(x-1,y), [19,29) n - R(x,y-1), bit 29 (x-1,y,z),
//            30 (x,y-1,z), 31 (x,y,z-1)
//   rec19.x: [0,10) R(x+1,y+1) - R(x+1,y), [10,20) R(x+1,y) - R(x+1,y-1),
//            [20,30) R(x-1,y+1) - R(x-1,y), bit 30 (x+1,y+1,z), 31 (x+1,y-1,z)
//   rec19.y: [0,10) R(x-1,y) - R(x-1,y-1), bit 10 (x-1,y+1,z),
//            11 (x-1,y-1,z), 12/13 (x+1,y,z-+1), 14/15 (x-1,y,z-+1),
//            16/17 (x,y+1,z-+1), 18/19 (x,y-1,z-+1)
// The fields bound the box: nz <= kRecMaxNz, ny nz <= kRecMaxPlane.  Nodes on
// a face (x, y or z = 0 or the last; their neighbours wrap or cross an x
// face) are "slow": their sweeps use the column map.  The differences are
// invariant under a shift of all node numbers, so a batch, whose node
// numbers are offset per structure, uses the records as they are.
constexpr uint32_t kRecSlow = 0x7FFFFu;
constexpr int kRecMaxNz = 1023;
constexpr int64_t kRecMaxPlane = 0x7FFFF;

__device__ __forceinline__ bool rec_slow(uint2 r7) { return (r7.x & kRecSlow) == kRecSlow; }

// nb[1..6] of a node that is not slow (nb[0] untouched)
template <int Q>
__device__ __forceinline__ void rec_axis(uint2 r, uint32_t n, uint32_t (&nb)[Q]) {
  const uint32_t ap = n + (r.x & 0x7FFFFu) + 1u, am = n - (r.y & 0x7FFFFu);
  const uint32_t bp = n + ((r.x >> 19) & 0x3FFu) + 1u, bm = n - ((r.y >> 19) & 0x3FFu);
  nb[1] = (r.x >> 29) & 1u ? ap : kNoNode;
  nb[2] = (r.y >> 29) & 1u ? am : kNoNode;
  nb[3] = (r.x >> 30) & 1u ? bp : kNoNode;
  nb[4] = (r.y >> 30) & 1u ? bm : kNoNode;
  nb[5] = (r.x >> 31) ? n + 1u : kNoNode;
  nb[6] = (r.y >> 31) ? n - 1u : kNoNode;
}

// the D3Q19 neighbours nb[1..18] of a node that is not slow
__device__ __forceinline__ void rec_neighbours19(uint2 r, uint2 q, uint32_t n, uint32_t (&nb)[19]) {
  rec_axis<19>(r, n, nb);
  const uint32_t ap = n + (r.x & 0x7FFFFu) + 1u, am = n - (r.y & 0x7FFFFu);
  const uint32_t bp = n + ((r.x >> 19) & 0x3FFu) + 1u, bm = n - ((r.y >> 19) & 0x3FFu);
  const uint32_t a0 = (r.x >> 29) & 1u, am0 = (r.y >> 29) & 1u, b0 = (r.x >> 30) & 1u, bm0 = (r.y >> 30) & 1u;
  const uint32_t e1 = q.x & 0x3FFu, e2 = (q.x >> 10) & 0x3FFu, e3 = (q.x >> 20) & 0x3FFu, e4 = q.y & 0x3FFu;
  nb[7] = (q.x >> 30) & 1u ? ap + e1 : kNoNode;   // (1, 1, 0)
  nb[8] = (q.y >> 10) & 1u ? am + e3 : kNoNode;   // (-1, 1, 0)
  nb[9] = (q.x >> 31) ? ap - e2 : kNoNode;        // (1, -1, 0)
  nb[10] = (q.y >> 11) & 1u ? am - e4 : kNoNode;  // (-1, -1, 0)
  nb[11] = (q.y >> 13) & 1u ? ap + a0 : kNoNode;  // (1, 0, 1)
  nb[12] = (q.y >> 15) & 1u ? am + am0 : kNoNode; // (-1, 0, 1)
  nb[13] = (q.y >> 12) & 1u ? ap - 1u : kNoNode;  // (1, 0, -1)
  nb[14] = (q.y >> 14) & 1u ? am - 1u : kNoNode;  // (-1, 0, -1)
  nb[15] = (q.y >> 17) & 1u ? bp + b0 : kNoNode;  // (0, 1, 1)
  nb[16] = (q.y >> 19) & 1u ? bm + bm0 : kNoNode; // (0, -1, 1)
  nb[17] = (q.y >> 16) & 1u ? bp - 1u : kNoNode;  // (0, 1, -1)
  nb[18] = (q.y >> 18) & 1u ? bm - 1u : kNoNode;  // (0, -1, -1)
}

// Ask L1 for the column-map words the neighbour lookup of the node with
// packed coordinates c will read (z's 32-voxel word of the columns (x + dx,
// y + dy): all nine for D3Q19, the five with |dx| + |dy| <= 1 for D3Q7), so
// that a node's lookup finds them on chip when its turn comes.  No register
// holds the result; x wraps only when px.
template <int Q>
__device__ __forceinline__ void prefetch_columns(const uint4* col, int nx, int ny, int W, int px, uint32_t c) {
  int x, y, z;
  unpack_xyz(c, x, y, z);
  const uint32_t w = (uint32_t)z >> 5;
#pragma unroll
  for (int dx = -1; dx <= 1; ++dx) {
    int xx = x + dx;
    if (xx < 0 || xx >= nx) {
      if (!px) continue;
      xx = xx < 0 ? xx + nx : xx - nx;
    }
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      if (Q == 7 && dx != 0 && dy != 0) continue;
      const int yy = y + dy < 0 ? y + dy + ny : (y + dy >= ny ? y + dy - ny : y + dy);
      const uint4* p = col + ((uint32_t)xx * (uint32_t)ny + (uint32_t)yy) * (uint32_t)W + w;
      asm volatile("prefetch.global.L1 [%0];" ::"l"(__cvta_generic_to_global(p)));  // in bounds: xx, yy, w valid
    }
  }
}

// Diffusion lattices: D3Q7 (rest, +-x, +-y, +-z; a = 1/4, 1/8; c_s^2 = 1/4)
// and the paper's D3Q19 (the flow's velocity set and weights, c_s^2 = 1/3).
struct D3Q7 {
  static constexpr int Q = 7;
  static constexpr double cs2 = 0.25;
  __host__ __device__ static constexpr int e(int i, int d) { return q7_e(i, d); }
  __host__ __device__ static constexpr int opp(int i) { return q7_opp(i); }
  __host__ __device__ static constexpr double w(int i) { return q7_w(i); }
};
struct D3Q19 {
  static constexpr int Q = 19;
  static constexpr double cs2 = 1.0 / 3.0;
  __host__ __device__ static constexpr int e(int i, int d) { return q19_e(i, d); }
  __host__ __device__ static constexpr int opp(int i) { return q19_opp(i); }
  __host__ __device__ static constexpr double w(int i) { return q19_w(i); }
};

// Warm-start fields come from outside the solver (a network's output).  A
// non-finite value falls back to the cold start; a velocity is kept inside
// the low-Mach range the lattice is stable in; a concentration inside
// [min(c_in, c_out), max(c_in, c_out)], where the steady state lies (maximum
// principle: no sources, Dirichlet ends, no-flux walls).
__device__ __forceinline__ double warm_velocity(double u) {
  return isfinite(u) ? fmin(fmax(u, -0.1), 0.1) : 0.0;
}
__device__ __forceinline__ double warm_concentration(double c, double clin, double cin, double cout) {
  return isfinite(c) ? fmin(fmax(c, fmin(cin, cout)), fmax(cin, cout)) : clin;
}

// Fixed-grid block reduction of NV doubles into partials[blockIdx.x][NV].
template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&v)[NV], double* partials) {
  __shared__ double sm[NV][kObsThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sm[k][wid] = x;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double acc = 0.0;
    for (int w = 0; w < kObsThreads / 32; ++w) acc += sm[threadIdx.x][w];
    partials[(int64_t)blockIdx.x * NV + threadIdx.x] = acc;
  }
}

}  // namespace om

namespace om {
// Block reduction of NV doubles written to out[0..NV) (any block size that
// is a multiple of 32, at most 1024).  Ends with a barrier, so a block may
// call it again in a loop.
template <int NV>
__device__ __forceinline__ void block_reduce_write(double (&v)[NV], double* out) {
  __shared__ double sm[NV][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sm[k][wid] = x;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double acc = 0.0;
    for (int w = 0; w < nw; ++w) acc += sm[threadIdx.x][w];
    out[threadIdx.x] = acc;
  }
  __syncthreads();
}
}  // namespace om
