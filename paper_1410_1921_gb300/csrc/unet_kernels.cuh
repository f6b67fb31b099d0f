// unet_kernels.cuh -- kernels of the learned warm start (a 3-D U-Net that
// predicts the steady velocity and concentration fields from the structure).
//
// Activations are BF16 in NDHWC layout (channels last, a multiple of 16 per
// tensor); weights are kept in FP32 (master copy for Adam) and converted to
// BF16 operand layouts before each pass.  The 3x3x3 convolutions are
// implicit GEMMs on the tensor cores (mma.sync m16n8k16 BF16 -> FP32):
//   forward  Y[v][n] = sum_k sum_c X[v + o_k][c] WT[k][n][c]
//   data grad: the forward kernel on dY with WT[k][ci][co] = W[26-k][ci][co]
//   weight grad dW[k][ci][co] = sum_v X[v + o_k][ci] dY[v][co]
// with o_k = (k/9 - 1, k/3 % 3 - 1, k % 3 - 1) over (z, y, x) and zero
// padding at the box faces.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace om {
namespace nn {

typedef __nv_bfloat16 bf16;

struct Grid {
  int B, D, H, W;
  __host__ __device__ int64_t voxels() const { return (int64_t)B * D * H * W; }
};

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// neighbour voxel of v at offset k, or -1 outside the box
__device__ __forceinline__ int64_t nbr_voxel(const Grid& g, int b, int z, int y, int x, int k) {
  const int zz = z + k / 9 - 1, yy = y + (k / 3) % 3 - 1, xx = x + k % 3 - 1;
  if (zz < 0 || zz >= g.D || yy < 0 || yy >= g.H || xx < 0 || xx >= g.W) return -1;
  return (((int64_t)b * g.D + zz) * g.H + yy) * g.W + xx;
}

// ------------------------------------------------------------------ forward / data-grad convolution
struct ConvArgs {
  const bf16* x1;  // first input: channels [o1, o1 + c1) of rows of ld1 elements
  int c1, ld1, o1;
  const bf16* x2;  // second input (concatenated after the first), c2 = 0 if none
  int c2, ld2, o2;
  const bf16* wt;     // [27][N][c1 + c2]
  const float* bias;  // [N] or null
  int N;
  bf16* y;  // output rows of ldy elements, channels [oy, oy + N)
  int ldy, oy;
  float* yf;  // optional FP32 copy of the output, rows of N
  int relu;
  Grid g;
};

constexpr int kConvBM = 64;   // voxels per CTA
constexpr int kApad = 24;     // smem row pitch (bf16) of the A tile: 48 B, conflict-free fragments

template <int BN>
__global__ void __launch_bounds__(128) conv3d_igemm(ConvArgs a) {
  __shared__ __align__(16) bf16 As[2][kConvBM][kApad];
  __shared__ __align__(16) bf16 Bs[2][BN][kApad];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = lane >> 2, tig = lane & 3;
  const int64_t V = a.g.voxels();
  const int64_t v0 = (int64_t)blockIdx.x * kConvBM;
  const int n0 = blockIdx.y * BN;
  const int K = a.c1 + a.c2, nc = K / 16, nstage = 27 * nc;
  // the A row this thread loads, and its coordinates
  const int arow = tid >> 1, ahalf = tid & 1;
  const int64_t av = v0 + arow;
  int ab = 0, az = 0, ay = 0, ax = 0;
  if (av < V) {
    int64_t r = av;
    ax = (int)(r % a.g.W); r /= a.g.W;
    ay = (int)(r % a.g.H); r /= a.g.H;
    az = (int)(r % a.g.D);
    ab = (int)(r / a.g.D);
  }
  auto load_stage = [&](int s, int buf) {
    const int k = s / nc, c = s % nc;
    // A: 64 rows x 16 channels, two 16-byte halves per row
    const int64_t nv = av < V ? nbr_voxel(a.g, ab, az, ay, ax, k) : -1;
    bf16* dst = &As[buf][arow][ahalf * 8];
    if (nv >= 0) {
      const int ch = c * 16 + ahalf * 8;
      const bf16* src = ch < a.c1 ? a.x1 + nv * a.ld1 + a.o1 + ch : a.x2 + nv * a.ld2 + a.o2 + (ch - a.c1);
      cp_async16(dst, src);
    } else {
      *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);
    }
    // B: BN output rows x 16 channels
    for (int q = tid; q < BN * 2; q += 128) {
      const int row = q >> 1, h = q & 1;
      const bf16* src = a.wt + ((int64_t)k * a.N + n0 + row) * K + c * 16 + h * 8;
      cp_async16(&Bs[buf][row][h * 8], src);
    }
    cp_async_commit();
  };
  float acc[BN / 8][4];
#pragma unroll
  for (int j = 0; j < BN / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  load_stage(0, 0);
  for (int s = 0; s < nstage; ++s) {
    const int buf = s & 1;
    cp_async_wait_all();
    __syncthreads();
    if (s + 1 < nstage) load_stage(s + 1, buf ^ 1);
    const int r0 = warp * 16 + grp;
    uint32_t af[4];
    af[0] = *reinterpret_cast<const uint32_t*>(&As[buf][r0][tig * 2]);
    af[1] = *reinterpret_cast<const uint32_t*>(&As[buf][r0 + 8][tig * 2]);
    af[2] = *reinterpret_cast<const uint32_t*>(&As[buf][r0][tig * 2 + 8]);
    af[3] = *reinterpret_cast<const uint32_t*>(&As[buf][r0 + 8][tig * 2 + 8]);
#pragma unroll
    for (int j = 0; j < BN / 8; ++j) {
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&Bs[buf][j * 8 + grp][tig * 2]);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&Bs[buf][j * 8 + grp][tig * 2 + 8]);
      mma_bf16_16816(acc[j], af, b0, b1);
    }
    __syncthreads();
  }
  // epilogue: bias, ReLU, BF16 (and FP32) store
#pragma unroll
  for (int j = 0; j < BN / 8; ++j) {
    const int col = n0 + j * 8 + tig * 2;
    const float bb0 = a.bias ? a.bias[col] : 0.f, bb1 = a.bias ? a.bias[col + 1] : 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t v = v0 + warp * 16 + grp + h * 8;
      if (v >= V) continue;
      float y0 = acc[j][2 * h] + bb0, y1 = acc[j][2 * h + 1] + bb1;
      if (a.relu) {
        y0 = fmaxf(y0, 0.f);
        y1 = fmaxf(y1, 0.f);
      }
      if (a.y) {
        __nv_bfloat162 p = __floats2bfloat162_rn(y0, y1);
        *reinterpret_cast<__nv_bfloat162*>(a.y + v * a.ldy + a.oy + col) = p;
      }
      if (a.yf) {
        a.yf[v * a.N + col] = y0;
        a.yf[v * a.N + col + 1] = y1;
      }
    }
  }
}

// ------------------------------------------------------------------ weight-gradient convolution
struct WgradArgs {
  const bf16* x1;  // layer input (as in ConvArgs)
  int c1, ld1, o1;
  const bf16* x2;
  int c2, ld2, o2;
  const bf16* dy;  // gradient at the pre-activation, rows of N
  int N;
  float* dw;  // [27][c1 + c2][N], accumulated with atomics
  Grid g;
  int chunk;  // voxels per CTA
};

// CTA: one offset k (blockIdx.y), a chunk of voxels (blockIdx.x), a tile of
// MT input channels x NT output channels (blockIdx.z); warps split the MT
// rows into 16-row slices.
template <int MT, int NT>
__global__ void __launch_bounds__(MT * 2) conv3d_wgrad(WgradArgs a) {
  constexpr int NW = MT / 16;
  __shared__ __align__(16) bf16 Xs[16][MT + 8];
  __shared__ __align__(16) bf16 Ys[16][NT + 8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = lane >> 2, tig = lane & 3;
  const int K = a.c1 + a.c2;
  const int k = blockIdx.y;
  const int ntile_n = a.N / NT;
  const int ci0 = (blockIdx.z / ntile_n) * MT, co0 = (blockIdx.z % ntile_n) * NT;
  const int64_t V = a.g.voxels();
  const int64_t vbeg = (int64_t)blockIdx.x * a.chunk;
  const int64_t vend = min(V, vbeg + a.chunk);
  float acc[NT / 8][4];
#pragma unroll
  for (int j = 0; j < NT / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  for (int64_t vb = vbeg; vb < vend; vb += 16) {
    // stage 16 voxels x MT input channels (shifted by o_k) and x NT gradient channels
    for (int q = tid; q < 16 * (MT / 8); q += NW * 32) {
      const int r = q / (MT / 8), cc = (q % (MT / 8)) * 8;
      const int64_t v = vb + r;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (v < vend) {
        int64_t t = v;
        const int x = (int)(t % a.g.W); t /= a.g.W;
        const int y = (int)(t % a.g.H); t /= a.g.H;
        const int z = (int)(t % a.g.D);
        const int b = (int)(t / a.g.D);
        const int64_t nv = nbr_voxel(a.g, b, z, y, x, k);
        const int ch = ci0 + cc;
        if (nv >= 0)
          val = *reinterpret_cast<const uint4*>(ch < a.c1 ? a.x1 + nv * a.ld1 + a.o1 + ch
                                                          : a.x2 + nv * a.ld2 + a.o2 + (ch - a.c1));
      }
      *reinterpret_cast<uint4*>(&Xs[r][cc]) = val;
    }
    for (int q = tid; q < 16 * (NT / 8); q += NW * 32) {
      const int r = q / (NT / 8), cc = (q % (NT / 8)) * 8;
      const int64_t v = vb + r;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (v < vend) val = *reinterpret_cast<const uint4*>(a.dy + v * a.N + co0 + cc);
      *reinterpret_cast<uint4*>(&Ys[r][cc]) = val;
    }
    __syncthreads();
    // A (m = input channel, k = voxel), B (k = voxel, n = output channel)
    const int m0 = warp * 16 + grp;
    uint32_t af[4];
    af[0] = pack_bf16(Xs[tig * 2][m0], Xs[tig * 2 + 1][m0]);
    af[1] = pack_bf16(Xs[tig * 2][m0 + 8], Xs[tig * 2 + 1][m0 + 8]);
    af[2] = pack_bf16(Xs[tig * 2 + 8][m0], Xs[tig * 2 + 9][m0]);
    af[3] = pack_bf16(Xs[tig * 2 + 8][m0 + 8], Xs[tig * 2 + 9][m0 + 8]);
#pragma unroll
    for (int j = 0; j < NT / 8; ++j) {
      const int n = j * 8 + grp;
      const uint32_t b0 = pack_bf16(Ys[tig * 2][n], Ys[tig * 2 + 1][n]);
      const uint32_t b1 = pack_bf16(Ys[tig * 2 + 8][n], Ys[tig * 2 + 9][n]);
      mma_bf16_16816(acc[j], af, b0, b1);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < NT / 8; ++j) {
    const int co = co0 + j * 8 + tig * 2;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int ci = ci0 + warp * 16 + grp + h * 8;
      float* p = a.dw + ((int64_t)k * K + ci) * a.N + co;
      atomicAdd(p, acc[j][2 * h]);
      atomicAdd(p + 1, acc[j][2 * h + 1]);
    }
  }
}

}  // namespace nn
}  // namespace om
