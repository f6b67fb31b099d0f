// unet_tc.cuh -- the 3x3x3 convolutions of the learned warm start's U-Net (it
// predicts the steady velocity and concentration fields from the structure)
// on the 5th-generation tensor cores: tcgen05.mma with the accumulator in
// tensor memory, operands staged in shared memory by TMA.
//
// Activations are BF16 in NDHWC layout (channels last); weights are kept in
// FP32 (master copy for Adam) and converted to BF16 operand layouts before
// each pass.  With o_k = (k/9 - 1, k/3 % 3 - 1, k % 3 - 1) over (z, y, x) and
// zero padding at the box faces:
//   forward    Y[v][n] = sum_k sum_c X[v + o_k][c] WT[k][n][c]
//   data grad  the forward kernels on dY with WT[k][ci][co] = W[26-k][ci][co]
//   weight grad  dW[k][ci][co] = sum_v X[v + o_k][ci] dY[v][co]
// Kernels: conv3d_tc (below), conv3d_tc_res (the forward with resident
// weights, for narrow inputs), conv3d_wgrad_tc and conv3d_wgrad_tc32 (the
// weight gradient; the second for at most 32 output channels).
//
// conv3d_tc: implicit GEMM  Y[v][n] = sum_k sum_c X[v + o_k][c] WT[k][n][c]  with a CTA
// tile of M = 128 voxels (a box of 8 x 8 x 2 voxels in x, y, z) and all N
// output channels (16..256).  For each of the 27 offsets o_k and each
// 64-channel chunk of each input, TMA copies
//   A: the voxel box shifted by o_k, 64 channels -- a 5-D box {64, 8, 8, 2, 1}
//      of the NDHWC activation tensor (channels, x, y, z, batch); the box's
//      part outside the grid (and channels past the input's count) is
//      filled with zeros by the copy itself, which is the convolution's
//      zero padding at the box faces;
//   B: 64 columns of the N weight rows of offset k, a 2-D box {64, N} of
//      WT[27 N][K];
// both K-major with the 128-byte swizzle, into one of three stages.  One
// thread (warp 0) issues the copies, another (warp 1) per stage four MMAs of
// K = 16 (cta_group::1, kind::f16: BF16 x BF16 -> FP32, M = 128)
// accumulating in TMEM; tcgen05.commit frees a stage when its MMAs have
// read it.  The epilogue reads the accumulator with tcgen05.ld (warp w owns
// TMEM lanes = tile rows 32w..32w+31), adds the bias, applies ReLU and
// stores BF16 (and an FP32 copy) for the rows inside the grid.
//
// Every wait on an mbarrier is bounded; a wait that runs out stops both
// issuing threads, sets the error word, lets what was issued finish (again
// bounded), frees the CTA's TMEM and returns without writing.
#pragma once

#include <cuda.h>  // CUtensorMap (the type only; the encoder is fetched through the runtime)

#include <cuda_bf16.h>

#include "common.cuh"

namespace om {
namespace nn {

typedef __nv_bfloat16 bf16;

struct Grid {
  int B, D, H, W;
  __host__ __device__ int64_t voxels() const { return (int64_t)B * D * H * W; }
};

constexpr int kTcM = 128;            // voxels per CTA tile (8 x 8 x 2 box)
constexpr int kTcKc = 64;            // channels per stage (128 bytes of BF16: one swizzle span)
constexpr int kTcStages = 3;
constexpr int kTcThreads = 128;
constexpr uint32_t kTcATile = kTcM * kTcKc * 2;  // 16 KB
constexpr unsigned long long kTcSpin = 1ull << 26;  // try_wait rounds before giving up
// the resident-weight form's tile (8 x 16 voxels at one z) and its halo box
constexpr int kTcTx = 8, kTcTy = 16;
constexpr int kTcHx = kTcTx + 2, kTcHy = kTcTy + 2, kTcHz = 3;
constexpr int kTcHRows = kTcHx * kTcHy * kTcHz;  // 540 rows

struct TcConvArgs {
  int c1, c2;         // channels of the two inputs (c2 = 0: one input)
  int N;              // output channels (multiple of 16, <= 256)
  const float* bias;  // [N] or null
  bf16* y;            // output rows of ldy elements, channels [oy, oy + N)
  int ldy, oy;
  float* yf;          // optional FP32 copy, rows of N
  int relu;
  Grid g;
  int tx, ty, tz;     // tiles along x, y, z (8, 8, 2 voxels each; the resident form: 8, 16, 1)
  int nhalo, nacc;    // the resident form's halo buffers and TMEM accumulators (2..4 each)
  int nw, n0;         // the resident form: weight rows per offset in WT, and this launch's first
  int* err;           // set when a wait ran out
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// bounded wait for the phase with the given parity to complete; false if it
// ran out or (checked every 1024 rounds) another thread set *stop
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int* stop = nullptr) {
  for (unsigned long long i = 0; i < kTcSpin; ++i) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (stop && (i & 1023) == 1023 && *stop) return false;
  }
  return false;
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            int c4, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile with the
// 128-byte swizzle: rows of 128 bytes (64 BF16), 8-row atoms 1024 bytes
// apart (stride byte offset), the leading byte offset unused for this
// layout (encoded 1), descriptor version 1, layout type 2 (128-byte
// swizzle).  The tile starts 1024-byte aligned; the k-th 16-element slice
// of the 64 starts 32 k bytes further.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B BF16 (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 in
// bits 17-22, M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__global__ void __launch_bounds__(kTcThreads) conv3d_tc(const __grid_constant__ CUtensorMap map1,
                                                        const __grid_constant__ CUtensorMap map2,
                                                        const __grid_constant__ CUtensorMap mapw, TcConvArgs a) {
  extern __shared__ uint8_t tc_smem_raw[];
  // stages 1024-byte aligned: [A 16 KB][B N x 128 B] x kTcStages, then the barriers
  const uint32_t raw = smem_u32(tc_smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = tc_smem_raw + (base - raw);
  const uint32_t btile = (uint32_t)a.N * 128u;
  const uint32_t stage_bytes = kTcATile + btile;
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + kTcStages * stage_bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kTcStages + 1);
  __shared__ volatile int stop;         // a wait ran out: issue nothing more
  __shared__ int n_issued, n_consumed;  // copies issued / waited for by the MMA thread
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8u * kTcStages, done = full0 + 16u * kTcStages;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // tile coordinates
  int t = blockIdx.x;
  const int bx = t % a.tx;
  t /= a.tx;
  const int by = t % a.ty;
  t /= a.ty;
  const int bz = t % a.tz;
  const int bb = t / a.tz;
  const int x0 = bx * 8, y0 = by * 8, z0 = bz * 2;

  const uint32_t ncols = a.N <= 32 ? 32u : (a.N <= 64 ? 64u : (a.N <= 128 ? 128u : 256u));
  if (tid == 0) {
    stop = 0;
    n_issued = 0;
    n_consumed = 0;
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(full0 + 8u * s, 1);
      mbar_init(empty0 + 8u * s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int n1 = (a.c1 + kTcKc - 1) / kTcKc, n2 = (a.c2 + kTcKc - 1) / kTcKc;
  const int per_k = n1 + n2, nsteps = 27 * per_k;
  if (tid == 0) {
    // producer: step s = (offset k, chunk j) into stage s % kTcStages once
    // the MMAs of step s - kTcStages have read that stage
    int s = 0;
    for (; s < nsteps; ++s) {
      const int st = s % kTcStages;
      if (s >= kTcStages && !mbar_wait(empty0 + 8u * st, (uint32_t)(s / kTcStages - 1) & 1u, &stop)) break;
      if (stop) break;
      const int k = s / per_k, j = s % per_k;
      const int dz = k / 9 - 1, dy = (k / 3) % 3 - 1, dx = k % 3 - 1;
      const uint32_t sa = base + (uint32_t)st * stage_bytes, sb = sa + kTcATile;
      const uint32_t fb = full0 + 8u * st;
      mbar_expect_tx(fb, kTcATile + btile);
      int cw;  // column of WT's K dimension
      if (j < n1) {
        tma_load_5d(sa, &map1, j * kTcKc, x0 + dx, y0 + dy, z0 + dz, bb, fb);
        cw = j * kTcKc;
      } else {
        tma_load_5d(sa, &map2, (j - n1) * kTcKc, x0 + dx, y0 + dy, z0 + dz, bb, fb);
        cw = a.c1 + (j - n1) * kTcKc;
      }
      tma_load_2d(sb, &mapw, cw, k * a.N, fb);
    }
    n_issued = s;
    if (s < nsteps) stop = 1;
  } else if (tid == 32) {
    // MMA issue: four K = 16 slices per stage, accumulating in TMEM
    const uint32_t idesc = tc_idesc(kTcM, a.N);
    int s = 0;
    for (; s < nsteps; ++s) {
      const int st = s % kTcStages;
      if (!mbar_wait(full0 + 8u * st, (uint32_t)(s / kTcStages) & 1u, &stop)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = base + (uint32_t)st * stage_bytes, sb = sa + kTcATile;
#pragma unroll
      for (int kk = 0; kk < kTcKc / 16; ++kk) {
        const uint64_t ad = sw128_desc(sa + 32u * kk), bd = sw128_desc(sb + 32u * kk);
        const uint32_t acc = (s > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       empty0 + 8u * st)
                   : "memory");
    }
    n_consumed = s;
    if (s < nsteps) stop = 1;
    // `done` fires when every MMA issued above has completed
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(done)
                 : "memory");
  }
  const bool fin = mbar_wait(done, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // one decision for the whole CTA (the epilogue's TMEM loads are warp-collective)
  const bool failed = __syncthreads_or(!fin || stop) != 0;
  if (failed && tid == 0) {
    atomicExch(a.err, 1);
    // copies still in flight land in their stages: wait for them (bounded)
    for (int s = n_consumed; s < n_issued; ++s)
      (void)mbar_wait(full0 + 8u * (s % kTcStages), (uint32_t)(s / kTcStages) & 1u);
  }

  // epilogue: warp w reads TMEM lanes 32w..32w+31 = tile rows
  if (!failed) {
    const int r = warp * 32 + lane;
    const int xx = x0 + (r & 7), yy = y0 + ((r >> 3) & 7), zz = z0 + (r >> 6);
    const bool inside = xx < a.g.W && yy < a.g.H && zz < a.g.D;
    const int64_t v = inside ? (((int64_t)bb * a.g.D + zz) * a.g.H + yy) * a.g.W + xx : 0;
    for (int c0 = 0; c0 < a.N; c0 += 16) {
      uint32_t q[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15}, [%16];"
          : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
            "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (!inside) continue;
      float f[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        f[i] = __uint_as_float(q[i]) + (a.bias ? a.bias[c0 + i] : 0.f);
        if (a.relu) f[i] = fmaxf(f[i], 0.f);
      }
      if (a.y) {
        uint32_t p[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
          p[i] = *reinterpret_cast<const uint32_t*>(&h);
        }
        uint4* dst = reinterpret_cast<uint4*>(a.y + v * a.ldy + a.oy + c0);
        dst[0] = make_uint4(p[0], p[1], p[2], p[3]);
        dst[1] = make_uint4(p[4], p[5], p[6], p[7]);
      }
      if (a.yf) {
        float4* dst = reinterpret_cast<float4*>(a.yf + v * a.N + c0);
#pragma unroll
        for (int i = 0; i < 4; ++i) dst[i] = make_float4(f[4 * i], f[4 * i + 1], f[4 * i + 2], f[4 * i + 3]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// ------------------------------------------------------------------ resident-weight form
// For a single input of at most 32 channels and at most 64 output channels
// (the finest level's convolutions, which carry most of the voxels) the
// whole operand WT[27][N][32] fits in shared memory next to two halo
// buffers: a persistent CTA per SM loads the weights once and then walks its
// tiles (8 x 16 voxels at one z).  Per tile TMA copies the halo -- 10 x 18 x
// 3 voxels of 32 channels, rows of 64 bytes with the 64-byte swizzle -- and
// the 27 filter offsets read it through shifted descriptors (the swizzle is
// applied to the absolute shared-memory address, so a view shifted by whole
// rows inside the TMA-written box is consistent).  Warp 0 issues the copies,
// warp 1 the MMAs (2 per offset, K = 16) into one of two TMEM accumulators,
// warps 2-5 drain the other accumulator (bias, ReLU, BF16 store) while the
// next tile accumulates.  Channels past the input's count are the copy's
// zero fill.  nhalo halo buffers and nacc accumulators (2..4 each, as the
// shared memory and TMEM allow) keep that many tiles in flight.  Waits are
// bounded as in conv3d_tc.
constexpr int kTrThreads = 192;
constexpr uint32_t kTrHBox = (uint32_t)kTcHRows * 64u;        // 34560 bytes
constexpr uint32_t kTrHalo = (kTrHBox + 1023u) / 1024u * 1024u;  // 34816

__device__ __forceinline__ uint64_t sw64_desc(uint32_t addr, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

__global__ void __launch_bounds__(kTrThreads) conv3d_tc_res(const __grid_constant__ CUtensorMap map1,
                                                            const __grid_constant__ CUtensorMap mapw, TcConvArgs a) {
  extern __shared__ uint8_t tc_smem_raw[];
  // [halo x nhalo][weights 27 x N rows x 64 B][barriers][TMEM address], 1024-byte aligned
  const uint32_t raw = smem_u32(tc_smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = tc_smem_raw + (base - raw);
  const int NH = a.nhalo, NA = a.nacc;
  const uint32_t wbox = (uint32_t)a.N * 64u, wres = base + (uint32_t)NH * kTrHalo;
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + (size_t)NH * kTrHalo + 27 * (size_t)wbox);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 18);
  const uint32_t b0 = smem_u32(bars);
  const uint32_t wfull = b0, hfull0 = b0 + 8u, hempty0 = b0 + 40u, afull0 = b0 + 72u, aempty0 = b0 + 104u,
                 done = b0 + 136u;
  __shared__ volatile int stop;
  __shared__ int h_issued, h_used;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = a.g.B * a.g.D * a.ty * a.tx;
  uint32_t ncols = 32u;  // NA accumulators of N columns, a power of two
  while (ncols < (uint32_t)(NA * a.N)) ncols <<= 1;

  if (tid == 0) {
    stop = 0;
    h_issued = h_used = 0;
    mbar_init(wfull, 1);
    for (int i = 0; i < 4; ++i) {
      mbar_init(hfull0 + 8u * i, 1);
      mbar_init(hempty0 + 8u * i, 1);
      mbar_init(afull0 + 8u * i, 1);
      mbar_init(aempty0 + 8u * i, 4);  // one arrival per epilogue warp
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  auto tile_xyz = [&](int t, int& x0, int& y0, int& z0, int& bb) {
    x0 = (t % a.tx) * kTcTx;
    t /= a.tx;
    y0 = (t % a.ty) * kTcTy;
    t /= a.ty;
    z0 = t % a.g.D;
    bb = t / a.g.D;
  };

  if (tid == 0) {
    // producer: the weights once, then each tile's halo into the buffer its
    // tile two back has released
    mbar_expect_tx(wfull, 27u * wbox);
    for (int k = 0; k < 27; ++k) tma_load_2d(wres + (uint32_t)k * wbox, &mapw, 0, k * a.nw + a.n0, wfull);
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int hb = i % NH;
      if (i >= NH && !mbar_wait(hempty0 + 8u * hb, (uint32_t)(i / NH - 1) & 1u, &stop)) break;
      if (stop) break;
      int x0, y0, z0, bb;
      tile_xyz(t, x0, y0, z0, bb);
      mbar_expect_tx(hfull0 + 8u * hb, kTrHBox);
      tma_load_5d(base + (uint32_t)hb * kTrHalo, &map1, 0, x0 - 1, y0 - 1, z0 - 1, bb, hfull0 + 8u * hb);
      h_issued = i + 1;
    }
    if (blockIdx.x + (int64_t)h_issued * gridDim.x < ntiles) stop = 1;
  } else if (tid == 32) {
    // MMA issue
    const uint32_t idesc = tc_idesc(kTcM, a.N);
    bool ok = mbar_wait(wfull, 0, &stop);
    int i = 0;
    for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x, ++i) {
      const int hb = i % NH, ab = i % NA;
      if (i >= NA && !mbar_wait(aempty0 + 8u * ab, (uint32_t)(i / NA - 1) & 1u, &stop)) break;
      if (!mbar_wait(hfull0 + 8u * hb, (uint32_t)(i / NH) & 1u, &stop)) break;
      h_used = i + 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t hbase = base + (uint32_t)hb * kTrHalo, acc_addr = tmem + (uint32_t)(ab * a.N);
      // descriptors of offset k, slice kk: the start-address field (address / 16)
      // of the first ones advanced by the offset's row shift and the slice's 32 bytes
      const uint64_t ad0 = sw64_desc(hbase, kTcHx * 64u), bd0 = sw64_desc(wres, 512u);
      const uint64_t bstep = wbox >> 4;
#pragma unroll
      for (int k = 0; k < 27; ++k) {
        constexpr uint32_t kRow = 64u / 16u;  // a halo row in units of 16 bytes
        const uint32_t shift = (uint32_t)((((k / 9) * kTcHy) + (k / 3) % 3) * kTcHx + k % 3) * kRow;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const uint64_t ad = ad0 + shift + 2u * kk;
          const uint64_t bd = bd0 + (uint64_t)k * bstep + 2u * kk;
          const uint32_t acc = (k > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(acc_addr),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       hempty0 + 8u * hb)
                   : "memory");
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       afull0 + 8u * ab)
                   : "memory");
    }
    if (!ok || blockIdx.x + (int64_t)h_used * gridDim.x < ntiles) stop = 1;
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(done)
                 : "memory");
  } else if (warp >= 2) {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = tile rows
    const int q = warp & 3, r = q * 32 + lane;
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int ab = i % NA;
      if (!mbar_wait(afull0 + 8u * ab, (uint32_t)(i / NA) & 1u, &stop)) {
        if (lane == 0) stop = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int x0, y0, z0, bb;
      tile_xyz(t, x0, y0, z0, bb);
      const int xx = x0 + (r & 7), yy = y0 + (r >> 3);
      const bool inside = xx < a.g.W && yy < a.g.H;
      const int64_t v = inside ? (((int64_t)bb * a.g.D + z0) * a.g.H + yy) * a.g.W + xx : 0;
      for (int c0 = 0; c0 < a.N; c0 += 16) {
        uint32_t qv[16];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * a.N + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(qv[0]), "=r"(qv[1]), "=r"(qv[2]), "=r"(qv[3]), "=r"(qv[4]), "=r"(qv[5]), "=r"(qv[6]),
              "=r"(qv[7]), "=r"(qv[8]), "=r"(qv[9]), "=r"(qv[10]), "=r"(qv[11]), "=r"(qv[12]), "=r"(qv[13]),
              "=r"(qv[14]), "=r"(qv[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (!inside) continue;
        float f[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          f[j] = __uint_as_float(qv[j]) + (a.bias ? a.bias[c0 + j] : 0.f);
          if (a.relu) f[j] = fmaxf(f[j], 0.f);
        }
        if (a.y) {
          uint32_t p[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
            p[j] = *reinterpret_cast<const uint32_t*>(&h);
          }
          uint4* dst = reinterpret_cast<uint4*>(a.y + v * a.ldy + a.oy + c0);
          dst[0] = make_uint4(p[0], p[1], p[2], p[3]);
          dst[1] = make_uint4(p[4], p[5], p[6], p[7]);
        }
        if (a.yf) {
          float4* dst = reinterpret_cast<float4*>(a.yf + v * a.N + c0);
#pragma unroll
          for (int j = 0; j < 4; ++j) dst[j] = make_float4(f[4 * j], f[4 * j + 1], f[4 * j + 2], f[4 * j + 3]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(aempty0 + 8u * ab) : "memory");
    }
  }
  const bool fin = mbar_wait(done, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool failed = __syncthreads_or(!fin || stop) != 0;
  if (failed && tid == 0) {
    atomicExch(a.err, 1);
    (void)mbar_wait(wfull, 0);  // the weight copies, if they never landed
    for (int i = h_used; i < h_issued; ++i) (void)mbar_wait(hfull0 + 8u * (i % NH), (uint32_t)(i / NH) & 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// ------------------------------------------------------------------ weight gradient
// dW[k][ci][co] = sum over voxels v of X[v + o_k][ci] dY[v][co], read in
// place: no transposed copies.  Both operands are "MN-major" (channels
// contiguous, voxels along K) views of TMA copies with the 64-byte swizzle:
// A of the input's halo (rows of 32 channels, as conv3d_tc_res loads it), B
// of the 8 x 16-voxel tile of dY (one 32-channel atom per 8 KB).  An MN atom
// of A is 32 channels; its four atoms sit one halo row (64 bytes) apart, so
// one MMA's 128 rows of D are the channels of the offsets dx = -1, 0, +1 (and
// a fourth, discarded).  A K-group of 8 voxels is one x row of the tile (10
// halo rows apart in A, 8 in B); one K = 16 MMA covers two y rows.  A CTA
// takes one 32-channel chunk of the input, a group of (dz, dy) pairs (all
// nine when 9 x N columns fit TMEM; the host launches it with the three of
// one dz, for more than 32 output channels) and up to 128 output channels, keeps one TMEM accumulator per pair over every gridDim.x-th
// tile and adds them to dW with FP32 atomics (four columns each) at the end.
// Waits are bounded as in conv3d_tc.
struct TcWgradArgs {
  int c1, c2;     // input channels of the two concatenated parts
  int nch1;       // 32-channel chunks of the first part
  int N, Nm;      // output channels, and the MMA's N (min(N, 128) rounded up to 32)
  int npart;      // parts of Nm output channels (N / 128 rounded up)
  int npair;      // (dz, dy) pairs per CTA: 9, or 3 (one dz, a one-plane halo)
  int nstage;     // pipeline stages
  float* dw;      // [27][c1 + c2][N], accumulated
  Grid g;
  int tx, ty;     // tiles along x (8) and y (16); one z plane per tile
  int vec4;       // dw 16-byte aligned: add four columns per atomic
  int* err;
};

constexpr uint32_t kWgPlane = (uint32_t)(kTcHx * kTcHy) * 64u;  // 11520: one z plane of the halo
constexpr uint32_t kWgAtom = 128u * 64u;                         // 8192: 32 channels of the dY tile

__host__ __device__ constexpr uint32_t wg_halo_bytes(int npair) { return npair == 9 ? kTrHalo : 12288u; }
__host__ __device__ constexpr uint32_t wg_stage_bytes(int npair, int Nm) {
  return wg_halo_bytes(npair) + (uint32_t)(Nm / 32) * kWgAtom;
}

// MN-major shared-memory descriptor, 64-byte swizzle: MN atoms of 32
// elements `lbo` bytes apart, K-groups of 8 rows (64 bytes each) `sbo` apart
__device__ __forceinline__ uint64_t mn_sw64_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

__global__ void __launch_bounds__(kTcThreads) conv3d_wgrad_tc(const __grid_constant__ CUtensorMap xm1,
                                                              const __grid_constant__ CUtensorMap xm2,
                                                              const __grid_constant__ CUtensorMap dym, TcWgradArgs a) {
  extern __shared__ uint8_t tc_smem_raw[];
  // [halo + dY atoms] x nstage (1024-byte aligned), then the barriers and the TMEM address
  const uint32_t raw = smem_u32(tc_smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = tc_smem_raw + (base - raw);
  const int S = a.nstage;
  const uint32_t hbytes = wg_halo_bytes(a.npair), stage_bytes = wg_stage_bytes(a.npair, a.Nm);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + (size_t)S * stage_bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8u * S, done = full0 + 16u * S;
  __shared__ volatile int stop;
  __shared__ int n_issued, n_used;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = a.g.B * a.g.D * a.ty * a.tx;
  // this CTA's input chunk and (dz, dy) group
  const int ngroup = 9 / a.npair;
  const int part = (int)blockIdx.y % a.npart, n0 = part * a.Nm;
  const int chunk = (int)blockIdx.y / a.npart / ngroup, grp = (int)blockIdx.y / a.npart % ngroup;
  const bool second = chunk >= a.nch1;
  const int ch0 = second ? (chunk - a.nch1) * 32 : chunk * 32;            // channel coordinate in its part
  const int cnt = min(32, (second ? a.c2 : a.c1) - ch0);                  // real channels of the chunk
  const int row0 = second ? a.c1 + ch0 : ch0;                             // its first row of dW
  const int pair0 = grp * a.npair;                                        // first (dz, dy) pair: dz * 3 + dy
  const CUtensorMap* xm = second ? &xm2 : &xm1;
  const uint32_t tx_bytes = (a.npair == 9 ? 3u : 1u) * kWgPlane + (uint32_t)(a.Nm / 32) * kWgAtom;
  uint32_t ncols = 32u;
  while (ncols < (uint32_t)(a.npair * a.Nm)) ncols <<= 1;
  int mytiles = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) ++mytiles;

  if (tid == 0) {
    stop = 0;
    n_issued = n_used = 0;
    for (int i = 0; i < S; ++i) {
      mbar_init(full0 + 8u * i, 1);
      mbar_init(empty0 + 8u * i, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (tid == 0) {
    // producer: per tile the input halo (three planes, or plane z + dz) and the dY atoms
    int i = 0;
    for (; i < mytiles; ++i) {
      const int st = i % S;
      if (i >= S && !mbar_wait(empty0 + 8u * st, (uint32_t)(i / S - 1) & 1u, &stop)) break;
      if (stop) break;
      int t = blockIdx.x + i * gridDim.x;
      const int x0 = (t % a.tx) * kTcTx;
      t /= a.tx;
      const int y0 = (t % a.ty) * kTcTy;
      t /= a.ty;
      const int z0 = t % a.g.D, bb = t / a.g.D;
      const uint32_t sa = base + (uint32_t)st * stage_bytes, fb = full0 + 8u * st;
      mbar_expect_tx(fb, tx_bytes);
      tma_load_5d(sa, xm, ch0, x0 - 1, y0 - 1, a.npair == 9 ? z0 - 1 : z0 + grp - 1, bb, fb);
      for (int j = 0; j < a.Nm / 32; ++j)
        tma_load_5d(sa + hbytes + (uint32_t)j * kWgAtom, &dym, n0 + 32 * j, x0, y0, z0, bb, fb);
      n_issued = i + 1;
    }
    if (i < mytiles) stop = 1;
  } else if (tid == 32) {
    // MMA issue: per pair and two y rows, A = halo rows (plane, y + dy, x + dx) for dx = 0..3
    const uint32_t idesc = tc_idesc(kTcM, a.Nm) | (1u << 15) | (1u << 16);
    int i = 0;
    for (; i < mytiles; ++i) {
      const int st = i % S;
      if (!mbar_wait(full0 + 8u * st, (uint32_t)(i / S) & 1u, &stop)) break;
      n_used = i + 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = base + (uint32_t)st * stage_bytes;
      const uint64_t ad0 = mn_sw64_desc(sa, 64u, kTcHx * 64u), bd0 = mn_sw64_desc(sa + hbytes, kWgAtom, 512u);
      for (int p = 0; p < a.npair; ++p) {
        const int pr = pair0 + p, dz = pr / 3, dy = pr % 3;
        const uint32_t row = (uint32_t)((a.npair == 9 ? dz * kTcHy : 0) + dy) * kTcHx;  // first halo row
        const uint32_t acc_addr = tmem + (uint32_t)(p * a.Nm);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const uint64_t ad = ad0 + (row + (uint32_t)kk * 2u * kTcHx) * 4u;  // 64-byte rows in units of 16 bytes
          const uint64_t bd = bd0 + (uint32_t)kk * 64u;                      // 1024 bytes: two rows of 8 voxels
          const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(acc_addr),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       empty0 + 8u * st)
                   : "memory");
    }
    if (i < mytiles) stop = 1;
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(done)
                 : "memory");
  }
  const bool fin = mbar_wait(done, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool failed = __syncthreads_or(!fin || stop) != 0;
  if (failed && tid == 0) {
    atomicExch(a.err, 1);
    for (int j = n_used; j < n_issued; ++j) (void)mbar_wait(full0 + 8u * (j % S), (uint32_t)(j / S) & 1u);
  }
  // epilogue: warp w < 3 holds TMEM lanes 32 w .. + 31 = offset dx = w - 1, channel ch0 + lane
  if (!failed && mytiles > 0 && warp < 3) {
    for (int p = 0; p < a.npair; ++p) {
      const int k = (pair0 + p) * 3 + warp;
      float* dst = a.dw + ((int64_t)k * (a.c1 + a.c2) + row0 + lane) * a.N + n0;
      for (int c0 = 0; c0 < a.Nm && n0 + c0 < a.N; c0 += 16) {
        uint32_t q[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(p * a.Nm + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
              "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (lane >= cnt) continue;
        if (a.vec4) {
#pragma unroll
          for (int j = 0; j < 16; j += 4)
            atomicAdd(reinterpret_cast<float4*>(dst + c0 + j),
                      make_float4(__uint_as_float(q[j]), __uint_as_float(q[j + 1]), __uint_as_float(q[j + 2]),
                                  __uint_as_float(q[j + 3])));
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) atomicAdd(dst + c0 + j, __uint_as_float(q[j]));
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// Weight gradient for at most 32 output channels: the roles swapped, so that
// one MMA is 128 x 96 x 16 instead of 128 x 32 x 16.  A = dY from a copy of
// the tile's rows y0 - 2 .. y0 + 15 (box {32, 8, 18, 1, 1}); its four 32-channel
// atoms are those rows shifted by a = 0..3 in y (one tile row, 512 bytes,
// apart).  B = the input's rows y0 - 1 .. y0 + 14 of planes z0 - 1 .. z0 + 1
// (box {32, 10, 16, 3, 1}); its three atoms are shifted by b = 0..2 in x (one
// halo row apart).  For the dY voxel u the product pairs dY[u] with
// X[u + (b - 1, 1 - a, dz)]: D row (a, co), column (b, ci) of the accumulator
// of plane dz is the gradient of offset (dz, dy = 1 - a, dx = b - 1), and
// a = 3 is discarded.  Tile row j sums u over y0 - 2 + a + [0, 16); one more
// tile row (j = ty) with only its first two rows closes the gap this leaves
// at the far face for a < 2.  A CTA takes one 32-channel input chunk and all
// 27 offsets (3 accumulators of 96 columns).
constexpr uint32_t kWnB = 3u * 160u * 64u;  // 30720: B, three planes of 16 x 10 rows
constexpr uint32_t kWnA = 10240u;           // A: 18 x 8 rows (9216 bytes) and the discarded atom's overrun
constexpr uint32_t kWnStage = kWnB + kWnA;
constexpr uint32_t kWnTx = kWnB + 144u * 64u;

__global__ void __launch_bounds__(kTcThreads) conv3d_wgrad_tc32(const __grid_constant__ CUtensorMap xm1,
                                                                const __grid_constant__ CUtensorMap xm2,
                                                                const __grid_constant__ CUtensorMap dym, TcWgradArgs a) {
  extern __shared__ uint8_t tc_smem_raw[];
  const uint32_t raw = smem_u32(tc_smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = tc_smem_raw + (base - raw);
  const int S = a.nstage;
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + (size_t)S * kWnStage);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8u * S, done = full0 + 16u * S;
  __shared__ volatile int stop;
  __shared__ int n_issued, n_used;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tyx = a.ty + 1;  // tile rows, the last one two rows high
  const int ntiles = a.g.B * a.g.D * tyx * a.tx;
  const int chunk = (int)blockIdx.y;
  const bool second = chunk >= a.nch1;
  const int ch0 = second ? (chunk - a.nch1) * 32 : chunk * 32;
  const int cnt = min(32, (second ? a.c2 : a.c1) - ch0);
  const int row0 = second ? a.c1 + ch0 : ch0;
  const CUtensorMap* xm = second ? &xm2 : &xm1;
  constexpr uint32_t ncols = 512u;  // 3 x 96
  int mytiles = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) ++mytiles;

  if (tid == 0) {
    stop = 0;
    n_issued = n_used = 0;
    for (int i = 0; i < S; ++i) {
      mbar_init(full0 + 8u * i, 1);
      mbar_init(empty0 + 8u * i, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (tid == 0) {
    int i = 0;
    for (; i < mytiles; ++i) {
      const int st = i % S;
      if (i >= S && !mbar_wait(empty0 + 8u * st, (uint32_t)(i / S - 1) & 1u, &stop)) break;
      if (stop) break;
      int t = blockIdx.x + i * gridDim.x;
      const int x0 = (t % a.tx) * kTcTx;
      t /= a.tx;
      const int y0 = (t % tyx) * kTcTy;
      t /= tyx;
      const int z0 = t % a.g.D, bb = t / a.g.D;
      const uint32_t sa = base + (uint32_t)st * kWnStage, fb = full0 + 8u * st;
      mbar_expect_tx(fb, kWnTx);
      tma_load_5d(sa, xm, ch0, x0 - 1, y0 - 1, z0 - 1, bb, fb);
      tma_load_5d(sa + kWnB, &dym, 0, x0, y0 - 2, z0, bb, fb);
      n_issued = i + 1;
    }
    if (i < mytiles) stop = 1;
  } else if (tid == 32) {
    const uint32_t idesc = tc_idesc(kTcM, 96) | (1u << 15) | (1u << 16);
    int i = 0;
    for (; i < mytiles; ++i) {
      const int st = i % S;
      if (!mbar_wait(full0 + 8u * st, (uint32_t)(i / S) & 1u, &stop)) break;
      n_used = i + 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int yt = (blockIdx.x + i * gridDim.x) / a.tx % tyx;
      const int nk = yt == a.ty ? 1 : 8;  // the last tile row: its first two rows only
      const uint32_t sa = base + (uint32_t)st * kWnStage;
      // A: dY, atoms one tile row (512 bytes) apart, K-groups one tile row apart;
      // B: the planes, atoms one halo row (64 bytes) apart, K-groups 10 rows apart
      const uint64_t ad0 = mn_sw64_desc(sa + kWnB, 512u, 512u), bd0 = mn_sw64_desc(sa, 64u, kTcHx * 64u);
      for (int dz = 0; dz < 3; ++dz) {
        const uint32_t acc_addr = tmem + (uint32_t)(dz * 96);
        for (int kk = 0; kk < nk; ++kk) {
          const uint64_t ad = ad0 + (uint32_t)kk * 64u;                                    // 1024 bytes
          const uint64_t bd = bd0 + ((uint32_t)dz * 160u + (uint32_t)kk * 2u * kTcHx) * 4u;  // 64-byte rows
          const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(acc_addr),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       empty0 + 8u * st)
                   : "memory");
    }
    if (i < mytiles) stop = 1;
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(done)
                 : "memory");
  }
  const bool fin = mbar_wait(done, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool failed = __syncthreads_or(!fin || stop) != 0;
  if (failed && tid == 0) {
    atomicExch(a.err, 1);
    for (int j = n_used; j < n_issued; ++j) (void)mbar_wait(full0 + 8u * (j % S), (uint32_t)(j / S) & 1u);
  }
  // epilogue: warp w < 3 holds TMEM lanes 32 w .. + 31 = dy = 1 - w, output channel lane;
  // columns dz * 96 + b * 32 + ci
  if (!failed && mytiles > 0 && warp < 3) {
    const bool live = lane < a.N;
    for (int dz = 0; dz < 3; ++dz)
      for (int b = 0; b < 3; ++b) {
        const int k = dz * 9 + (2 - warp) * 3 + b;
        float* dst = a.dw + ((int64_t)k * (a.c1 + a.c2) + row0) * a.N + lane;
        for (int c0 = 0; c0 < 32; c0 += 16) {
          uint32_t q[16];
          const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(dz * 96 + b * 32 + c0);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
              "%14, %15}, [%16];"
              : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
                "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]),
                "=r"(q[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (!live) continue;
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c0 + j < cnt) atomicAdd(dst + (int64_t)(c0 + j) * a.N, __uint_as_float(q[j]));
        }
      }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

}  // namespace nn
}  // namespace om
