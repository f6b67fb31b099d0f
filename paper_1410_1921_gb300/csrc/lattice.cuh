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

// Node number of voxel (x, y, z) from its column's bit map, or kNoNode.
// Column-map indices fit 32 bits (nx*ny*W <= 1024*2048*64).
__device__ __forceinline__ uint32_t node_at(const uint2* __restrict__ col, int ny, int W, int x,
                                            int y, int z) {
  const uint32_t k = ((uint32_t)x * (uint32_t)ny + (uint32_t)y) * (uint32_t)W + ((uint32_t)z >> 5);
  const uint2 b = __ldg(col + k);
  const uint32_t bit = 1u << (z & 31);
  return (b.x & bit) ? b.y + __popc(b.x & (bit - 1u)) : kNoNode;
}

// Node numbers of the voxels z-1, z, z+1 of one (x, y) column.  The three
// usually share one 32-voxel word of the column map, so one load and a
// popcount serve all of them; a neighbour across a word edge or the periodic
// wrap takes its own word.
__device__ __forceinline__ void column3(const uint2* __restrict__ col, uint32_t base, int z, int zp, int zm,
                                        uint32_t& rm, uint32_t& r0, uint32_t& rp) {
  const int zb = z & 31;
  const uint2 w = __ldg(col + base + ((uint32_t)z >> 5));
  const uint32_t b0 = (w.x >> zb) & 1u;
  const uint32_t rank0 = w.y + __popc(w.x & ((1u << zb) - 1u));
  r0 = b0 ? rank0 : kNoNode;
  if (zb != 31 && zp == z + 1) {
    rp = ((w.x >> (zb + 1)) & 1u) ? rank0 + b0 : kNoNode;
  } else {
    const uint2 v = __ldg(col + base + ((uint32_t)zp >> 5));
    const uint32_t bit = 1u << (zp & 31);
    rp = (v.x & bit) ? v.y + __popc(v.x & (bit - 1u)) : kNoNode;
  }
  if (zb != 0 && zm == z - 1) {
    rm = ((w.x >> (zb - 1)) & 1u) ? rank0 - 1u : kNoNode;
  } else {
    const uint2 v = __ldg(col + base + ((uint32_t)zm >> 5));
    const uint32_t bit = 1u << (zm & 31);
    rm = (v.x & bit) ? v.y + __popc(v.x & (bit - 1u)) : kNoNode;
  }
}

__device__ __forceinline__ uint32_t column1(const uint2* __restrict__ col, uint32_t base, int z) {
  const uint2 w = __ldg(col + base + ((uint32_t)z >> 5));
  const uint32_t bit = 1u << (z & 31);
  return (w.x & bit) ? w.y + __popc(w.x & (bit - 1u)) : kNoNode;
}

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
