// unet.cu -- the learned warm start: a 3-D U-Net that maps the structure
// (pore mask, local pore size) to the steady fields the LB solves produce
// (velocity u_x, concentration C), trained on the GPU by this file's own
// forward and backward passes; the LB then iterates from the prediction to
// the same convergence test, so the plain solve stays the judge of the
// result.
//
// Network (levels L, channels c_0..c_{L-1}): per encoder level two 3x3x3
// convolutions with ReLU, 2x average pooling between levels; per decoder
// level nearest 2x upsampling, the skip tensor concatenated (read as a second
// conv input, never materialised) and two 3x3x3 convolutions with ReLU; a
// 1x1 head without activation.  Masked mean-squared error; Adam.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "unet_tc.cuh"

namespace om {
namespace nn {
namespace {

constexpr int kT = 256;
inline unsigned blocks(int64_t n, int t = kT) { return (unsigned)std::min<int64_t>((n + t - 1) / t, 1 << 20); }

__global__ void pack_input(const float* x, int cin, int64_t V, bf16* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V * 16; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / 16;
    const int c = (int)(i % 16);
    out[i] = __float2bfloat16_rn(c < cin ? x[v * cin + c] : 0.f);
  }
}

// fine grid gf -> coarse grid (gf / 2)
__global__ void avgpool2(const bf16* in, Grid gf, int C, bf16* out) {
  const Grid gc{gf.B, gf.D / 2, gf.H / 2, gf.W / 2};
  const int64_t n = gc.voxels() * C;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    int64_t r = i / C;
    const int x = (int)(r % gc.W); r /= gc.W;
    const int y = (int)(r % gc.H); r /= gc.H;
    const int z = (int)(r % gc.D);
    const int b = (int)(r / gc.D);
    float s = 0.f;
    for (int q = 0; q < 8; ++q) {
      const int64_t vf = (((int64_t)b * gf.D + 2 * z + (q >> 2)) * gf.H + 2 * y + ((q >> 1) & 1)) * gf.W + 2 * x + (q & 1);
      s += __bfloat162float(in[vf * C + c]);
    }
    out[i] = __float2bfloat16_rn(0.125f * s);
  }
}

// The element-wise kernels below move 8 channels (one 16-byte vector of
// BF16) per thread: every channel count and row offset of the network is a
// multiple of 16.
union V8 {
  uint4 u;
  __nv_bfloat16 h[8];
};

__device__ __forceinline__ void fine_xyzb(int64_t v, const Grid& g, int& x, int& y, int& z, int& b) {
  x = (int)(v % g.W);
  v /= g.W;
  y = (int)(v % g.H);
  v /= g.H;
  z = (int)(v % g.D);
  b = (int)(v / g.D);
}

__device__ __forceinline__ int64_t coarse_of(const Grid& gf, int x, int y, int z, int b) {
  return (((int64_t)b * (gf.D / 2) + z / 2) * (gf.H / 2) + y / 2) * (gf.W / 2) + x / 2;
}

// d(fine) = d(coarse parent) / 8
__global__ void avgpool2_bwd(const bf16* dout, Grid gf, int C, bf16* din) {
  const int C8 = C / 8;
  const int64_t n = gf.voxels() * C8;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c8 = (int)(i % C8);
    const int64_t v = i / C8;
    int x, y, z, b;
    fine_xyzb(v, gf, x, y, z, b);
    V8 a, o;
    a.u = *reinterpret_cast<const uint4*>(dout + coarse_of(gf, x, y, z, b) * C + 8 * c8);
#pragma unroll
    for (int j = 0; j < 8; ++j) o.h[j] = __float2bfloat16_rn(0.125f * __bfloat162float(a.h[j]));
    *reinterpret_cast<uint4*>(din + v * C + 8 * c8) = o.u;
  }
}

// nearest 2x: coarse [V_c x C] -> fine rows of ldo, channels [oo, oo + C)
__global__ void upsample2(const bf16* in, Grid gf, int C, bf16* out, int ldo, int oo) {
  const int C8 = C / 8;
  const int64_t n = gf.voxels() * C8;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c8 = (int)(i % C8);
    const int64_t v = i / C8;
    int x, y, z, b;
    fine_xyzb(v, gf, x, y, z, b);
    *reinterpret_cast<uint4*>(out + v * ldo + oo + 8 * c8) =
        *reinterpret_cast<const uint4*>(in + coarse_of(gf, x, y, z, b) * C + 8 * c8);
  }
}

// d(coarse) = sum of the 8 fine children, read from rows of ldi at offset oi
__global__ void upsample2_bwd(const bf16* dfine, int ldi, int oi, Grid gf, int C, bf16* dcoarse) {
  const Grid gc{gf.B, gf.D / 2, gf.H / 2, gf.W / 2};
  const int C8 = C / 8;
  const int64_t n = gc.voxels() * C8;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c8 = (int)(i % C8);
    const int64_t vcoarse = i / C8;
    int x, y, z, b;
    fine_xyzb(vcoarse, gc, x, y, z, b);
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int q = 0; q < 8; ++q) {
      const int64_t vf = (((int64_t)b * gf.D + 2 * z + (q >> 2)) * gf.H + 2 * y + ((q >> 1) & 1)) * gf.W + 2 * x + (q & 1);
      V8 a;
      a.u = *reinterpret_cast<const uint4*>(dfine + vf * ldi + oi + 8 * c8);
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] += __bfloat162float(a.h[j]);
    }
    V8 o;
#pragma unroll
    for (int j = 0; j < 8; ++j) o.h[j] = __float2bfloat16_rn(acc[j]);
    *reinterpret_cast<uint4*>(dcoarse + vcoarse * C + 8 * c8) = o.u;
  }
}

// gradient at the pre-activation: g * [y > 0]; g read from rows of ldg at og
__global__ void relu_bwd(const bf16* g, int ldg, int og, const bf16* y, int N, int64_t V, bf16* out) {
  const int N8 = N / 8;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V * N8; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / N8;
    const int c8 = (int)(i % N8);
    V8 yy, gg, o;
    yy.u = *reinterpret_cast<const uint4*>(y + v * N + 8 * c8);
    gg.u = *reinterpret_cast<const uint4*>(g + v * ldg + og + 8 * c8);
#pragma unroll
    for (int j = 0; j < 8; ++j) o.h[j] = __bfloat162float(yy.h[j]) > 0.f ? gg.h[j] : __float2bfloat16_rn(0.f);
    *reinterpret_cast<uint4*>(out + v * N + 8 * c8) = o.u;
  }
}

// a[i] += b (rows of ldb at ob), BF16; 8 channels per thread
__global__ void add_into(bf16* a, int N, int64_t V, const bf16* b, int ldb, int ob) {
  const int N8 = N / 8;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V * N8; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / N8;
    const int c8 = (int)(i % N8);
    V8 x, y;
    x.u = *reinterpret_cast<const uint4*>(a + v * N + 8 * c8);
    y.u = *reinterpret_cast<const uint4*>(b + v * ldb + ob + 8 * c8);
#pragma unroll
    for (int j = 0; j < 8; ++j) x.h[j] = __float2bfloat16_rn(__bfloat162float(x.h[j]) + __bfloat162float(y.h[j]));
    *reinterpret_cast<uint4*>(a + v * N + 8 * c8) = x.u;
  }
}

// db[c] += sum_v g[v][c]: thread t of a block sums channel t % N over the
// block's voxels t / N, t / N + lanes, ... (coalesced rows), then the lanes
// of a channel are reduced in shared memory and added to db
__global__ void bias_grad(const bf16* g, int N, int64_t V, float* db) {
  extern __shared__ float sh[];
  const int lanes = blockDim.x / N, c = threadIdx.x % N, lane = threadIdx.x / N;
  float acc = 0.f;
  if (lane < lanes)
    for (int64_t v = (int64_t)blockIdx.x * lanes + lane; v < V; v += (int64_t)gridDim.x * lanes)
      acc += __bfloat162float(g[v * N + c]);
  sh[threadIdx.x] = lane < lanes ? acc : 0.f;
  __syncthreads();
  if (threadIdx.x < N) {
    float t = 0.f;
    for (int l = 0; l < lanes; ++l) t += sh[l * N + threadIdx.x];
    atomicAdd(&db[threadIdx.x], t);
  }
}

// 1x1 head: y[v][o] = b[o] + sum_c x[v][c] w[c][o]  (FP32 out); a thread per voxel reads its row
// of C channels as 16-byte vectors
__global__ void head_fwd(const bf16* x, int C, const float* w, const float* b, int O, int64_t V, float* y) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    const uint4* row = reinterpret_cast<const uint4*>(x + v * C);
    for (int o = 0; o < O; ++o) {
      float acc = b[o];
      for (int c8 = 0; c8 < C / 8; ++c8) {
        V8 q;
        q.u = row[c8];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc += __bfloat162float(q.h[j]) * w[(8 * c8 + j) * O + o];
      }
      y[v * O + o] = acc;
    }
  }
}

// the mask's nonzero count, added to *cnt (a double: exact below 2^53)
__global__ void mask_count(const uint8_t* m, int64_t V, double* cnt) {
  unsigned long long k = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x)
    k += m[v] != 0;
  for (int o = 16; o > 0; o >>= 1) k += __shfl_down_sync(0xffffffffu, k, o);
  if ((threadIdx.x & 31) == 0 && k) atomicAdd(cnt, (double)k);
}

// masked MSE: loss = sum m (y - t)^2 * scale, dy = 2 m (y - t) * scale, scale = 1 / (count O)
// with the mask's count read from *cnt
__global__ void mse_grad(const float* y, const float* t, const uint8_t* m, int O, int64_t V, const double* cnt,
                         float* dy, double* loss) {
  const int64_t nk = (int64_t)*cnt;
  const float scale = nk > 0 ? 1.f / (float)(nk * O) : 0.f;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V * O; i += (int64_t)gridDim.x * blockDim.x) {
    const float keep = m[i / O] ? 1.f : 0.f;
    const float d = (y[i] - t[i]) * keep;
    dy[i] = 2.f * d * scale;
    acc += (double)d * d * scale;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// head backward: dw[c][o] += sum_v x[v][c] dy[v][o]; db[o] += sum_v dy; dx[v][c] = sum_o dy w[c][o]
__global__ void head_bwd_dx(const float* dy, const float* w, int C, int O, int64_t V, bf16* dx) {
  const int C8 = C / 8;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V * C8; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / C8;
    const int c0 = (int)(i % C8) * 8;
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int o = 0; o < O; ++o) {
      const float d = dy[v * O + o];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] += d * w[(c0 + j) * O + o];
    }
    V8 q;
#pragma unroll
    for (int j = 0; j < 8; ++j) q.h[j] = __float2bfloat16_rn(acc[j]);
    *reinterpret_cast<uint4*>(dx + v * C + c0) = q.u;
  }
}
// dw[c][o] and db[o] for o in [o0, o0 + 4): thread t of a block takes channel t % C of the
// voxels t / C, t / C + lanes, ... (coalesced rows); the lanes are reduced in shared memory
__global__ void head_bwd_dw(const bf16* x, const float* dy, int C, int O, int o0, int64_t V, float* dw, float* db) {
  extern __shared__ float sh[];  // [8][blockDim.x]
  const int lanes = blockDim.x / C, c = threadIdx.x % C, lane = threadIdx.x / C;
  const int no = min(4, O - o0);
  float aw[4] = {0, 0, 0, 0}, ab[4] = {0, 0, 0, 0};
  if (lane < lanes)
    for (int64_t v = (int64_t)blockIdx.x * lanes + lane; v < V; v += (int64_t)gridDim.x * lanes) {
      const float xv = __bfloat162float(x[v * C + c]);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j < no) {
          const float d = dy[v * O + o0 + j];
          aw[j] += xv * d;
          ab[j] += d;
        }
    }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    sh[j * blockDim.x + threadIdx.x] = lane < lanes ? aw[j] : 0.f;
    sh[(4 + j) * blockDim.x + threadIdx.x] = lane < lanes ? ab[j] : 0.f;
  }
  __syncthreads();
  if ((int)threadIdx.x < C) {
    for (int j = 0; j < no; ++j) {
      float tw = 0.f, tb = 0.f;
      for (int l = 0; l < lanes; ++l) {
        tw += sh[j * blockDim.x + l * C + threadIdx.x];
        tb += sh[(4 + j) * blockDim.x + l * C + threadIdx.x];
      }
      atomicAdd(&dw[threadIdx.x * O + o0 + j], tw);
      if (threadIdx.x == 0) atomicAdd(&db[o0 + j], tb);
    }
  }
}

// FP32 master W[27][K][N] -> forward operand WT[27][N][K] (BF16)
__global__ void weights_fwd(const float* W, int K, int N, bf16* WT) {
  const int64_t n = 27LL * K * N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(i / ((int64_t)K * N));
    const int r = (int)(i % ((int64_t)K * N));
    const int ci = r / N, co = r % N;
    WT[((int64_t)k * N + co) * K + ci] = __float2bfloat16_rn(W[i]);
  }
}
// data-gradient operand WD[27][K][N] = W[26 - k][K][N] (BF16): the forward
// kernel with inputs dY (N channels) and output channels K
__global__ void weights_dgrad(const float* W, int K, int N, bf16* WD) {
  const int64_t n = 27LL * K * N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(i / ((int64_t)K * N));
    const int64_t r = i % ((int64_t)K * N);
    WD[i] = __float2bfloat16_rn(W[(int64_t)(26 - k) * K * N + r]);
  }
}

__global__ void adam_step(float* w, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                          float eps, float bc1, float bc2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

// ------------------------------------------------------------------ host side
struct Conv {
  int cin1, cin2, cout;
  int64_t w_off, b_off;  // into the flat parameter vector
  bf16* wt = nullptr;    // forward operand
  bf16* wd = nullptr;    // data-gradient operand
};

template <class T>
struct Buf {
  T* p = nullptr;
  size_t n = 0;
  om_status ensure(size_t count) {
    if (count <= n) return OM_OK;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    if (cudaMalloc((void**)&p, sizeof(T) * std::max<size_t>(count, 1)) != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(OM_ENOMEM, "U-Net: device allocation failed");
    }
    n = count;
    return OM_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

}  // namespace
}  // namespace nn
}  // namespace om

using namespace om;
using namespace om::nn;

struct om_unet {
  int in_ch = 0, out_ch = 0, L = 0;
  std::vector<int> ch;
  std::vector<Conv> enc1, enc2, dec1, dec2;  // per level (dec: levels 0..L-2)
  int64_t head_w = 0, head_b = 0, nparam = 0;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 master, grad, Adam moments
  int64_t step = 0;
  Grid grid{0, 0, 0, 0};
  // activations per level
  Buf<bf16> x0;
  std::vector<Buf<bf16>> in, a, s, u, b, h;
  Buf<float> out, dout;
  // gradients (scratch)
  std::vector<Buf<bf16>> d1, d2, dcat, ds;
  Buf<double> loss;
  Buf<int> tc_err;  // set by a tensor-core convolution whose wait ran out
};

namespace {

// ------------------------------------------------------------------ tensor-core convolutions (unet_tc.cuh)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, fetched through the runtime (nothing links libcuda)
om_status tensor_map_encoder(EncodeTiledFn* out) {
  static std::mutex mu;
  static EncodeTiledFn fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    OM_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) return fail(OM_ECUDA, "U-Net: cuTensorMapEncodeTiled unavailable");
    fn = (EncodeTiledFn)p;
  }
  *out = fn;
  return OM_OK;
}

// 5-D map of an NDHWC activation tensor: rows of ld BF16, c channels from o,
// zero fill; box by mode: 0 = {64 channels, 8 x, 8 y, 2 z, 1 batch} with the
// 128-byte swizzle, and with the 64-byte swizzle 1 = the {32, 10, 18, 3, 1}
// halo, 2 = its one-plane form {32, 10, 18, 1, 1}, 3 = the 8 x 16 tile
// {32, 8, 16, 1, 1}, 4 = {32, 10, 16, 3, 1}, 5 = {32, 8, 18, 1, 1}
om_status activation_map(CUtensorMap* m, const bf16* x, int c, int ld, int o, const Grid& g, int mode = 0) {
  const bool halo = mode != 0;
  EncodeTiledFn enc;
  OM_TRY(tensor_map_encoder(&enc));
  const cuuint64_t row = (cuuint64_t)ld * 2;
  cuuint64_t dims[5] = {(cuuint64_t)c, (cuuint64_t)g.W, (cuuint64_t)g.H, (cuuint64_t)g.D, (cuuint64_t)g.B};
  cuuint64_t strides[4] = {row, row * g.W, row * g.W * g.H, row * g.W * g.H * g.D};
  cuuint32_t box[5] = {(cuuint32_t)kTcKc, 8, 8, 2, 1};
  if (mode == 1 || mode == 2) box[0] = 32, box[1] = kTcHx, box[2] = kTcHy, box[3] = mode == 1 ? kTcHz : 1;
  if (mode == 3) box[0] = 32, box[1] = kTcTx, box[2] = kTcTy, box[3] = 1;
  if (mode == 4) box[0] = 32, box[1] = kTcHx, box[2] = kTcTy, box[3] = 3;
  if (mode == 5) box[0] = 32, box[1] = kTcTx, box[2] = kTcTy + 2, box[3] = 1;
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void*)(x + o), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, halo ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(OM_ECUDA, "U-Net: activation tensor map rejected (" + std::to_string((int)r) + ")");
  return OM_OK;
}

// 2-D map of the operand WT[27 N][K]: box {64 columns, N rows}, 128-byte
// swizzle (narrow = true: {32 columns, rows (default N) rows}, 64-byte swizzle)
om_status weight_map(CUtensorMap* m, const bf16* wt, int K, int N, bool narrow = false, int rows = 0) {
  EncodeTiledFn enc;
  OM_TRY(tensor_map_encoder(&enc));
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)27 * N};
  cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  cuuint32_t box[2] = {narrow ? 32u : (cuuint32_t)kTcKc, (cuuint32_t)(rows > 0 ? rows : N)};
  cuuint32_t es[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)wt, dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, narrow ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(OM_ECUDA, "U-Net: weight tensor map rejected (" + std::to_string((int)r) + ")");
  return OM_OK;
}

// stages + 1 KB alignment slack + barriers and the TMEM address slot
size_t tc_smem_bytes(int N) { return 1024 + (size_t)kTcStages * (kTcATile + (size_t)N * 128) + 8 * (2 * kTcStages + 1) + 16; }

// Y (rows of ldy, channels [oy, oy + N)) = conv of concat(x1, x2) with WT[27][N][c1 + c2]
om_status conv_tc(const om_unet* U, const bf16* x1, int c1, int ld1, int o1, const bf16* x2, int c2, int ld2, int o2,
                  const bf16* wt, int N, const float* bias, bf16* y, int ldy, int oy, float* yf, int relu, const Grid& g,
                  cudaStream_t s) {
  if (N % 16 || N < 16 || N > 256 || c1 < 8 || (c1 % 8) || (c2 % 8) || (ld1 % 8) || (o1 % 8) || (ldy % 8) || (oy % 8))
    return fail(OM_EINVAL, "U-Net: convolution shape outside the tensor-core kernel's layout");
  CUtensorMap m1, m2, mw;
  if (c2 == 0 && c1 <= 32 && (N <= 64 || !yf)) {
    // resident weights: one persistent CTA per SM (conv3d_tc_res); wider outputs in parts
    // of at most 64 channels (multiples of 16), one launch each
    OM_TRY(activation_map(&m1, x1, c1, ld1, o1, g, 1));
    const int nparts = (N + 63) / 64, width = ((N + nparts - 1) / nparts + 15) / 16 * 16;
    int dev = 0, sms = 0;
    OM_CUDA(cudaGetDevice(&dev));
    OM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    for (int n0 = 0; n0 < N; n0 += width) {
      const int np = std::min(width, N - n0);
      OM_TRY(weight_map(&mw, wt, c1, N, true, np));
      TcConvArgs a{};
      a.c1 = c1, a.c2 = 0, a.N = np, a.bias = bias ? bias + n0 : nullptr, a.y = y, a.ldy = ldy, a.oy = oy + n0;
      a.yf = yf, a.relu = relu, a.g = g, a.nw = N, a.n0 = n0;
      a.tx = (g.W + kTcTx - 1) / kTcTx, a.ty = (g.H + kTcTy - 1) / kTcTy;
      a.err = U->tc_err.p;
      const int64_t tiles = (int64_t)g.B * g.D * a.ty * a.tx;
      // as many halo buffers (2..4) as 227 KB of shared memory hold next to the weights, and
      // as many accumulators (2..4) as 256 TMEM columns
      auto smem_for = [&](int nh) { return 1024 + (size_t)nh * kTrHalo + 27 * (size_t)np * 64 + 8 * 18 + 16; };
      a.nhalo = 4;
      while (a.nhalo > 2 && smem_for(a.nhalo) > 227 * 1024) --a.nhalo;
      a.nacc = std::min(4, 256 / np);
      const size_t smem = smem_for(a.nhalo);
      OM_CUDA(cudaFuncSetAttribute(conv3d_tc_res, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      conv3d_tc_res<<<(unsigned)std::min<int64_t>(tiles, sms), kTrThreads, smem, s>>>(m1, mw, a);
      OM_CUDA(cudaGetLastError());
    }
    return OM_OK;
  }
  OM_TRY(activation_map(&m1, x1, c1, ld1, o1, g));
  if (c2 > 0) {
    if ((ld2 % 8) || (o2 % 8)) return fail(OM_EINVAL, "U-Net: second input not 16-byte aligned");
    OM_TRY(activation_map(&m2, x2, c2, ld2, o2, g));
  } else {
    m2 = m1;
  }
  OM_TRY(weight_map(&mw, wt, c1 + c2, N));
  TcConvArgs a{};
  a.c1 = c1, a.c2 = c2, a.N = N, a.bias = bias, a.y = y, a.ldy = ldy, a.oy = oy, a.yf = yf, a.relu = relu, a.g = g;
  a.tx = (g.W + 7) / 8, a.ty = (g.H + 7) / 8, a.tz = (g.D + 1) / 2;
  a.err = U->tc_err.p;
  OM_CUDA(cudaFuncSetAttribute(conv3d_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes(N)));
  const unsigned grid = (unsigned)((int64_t)g.B * a.tz * a.ty * a.tx);
  conv3d_tc<<<grid, kTcThreads, tc_smem_bytes(N), s>>>(m1, m2, mw, a);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

// a tensor-core convolution gave up a wait: report (synchronises)
om_status check_tc(const om_unet* U, cudaStream_t s) {
  int h = 0;
  OM_CUDA(cudaMemcpyAsync(&h, U->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  OM_CUDA(cudaStreamSynchronize(s));
  if (h) return fail(OM_ETIMEOUT, "U-Net: a tensor-core convolution's wait ran out");
  return OM_OK;
}

om_status conv_forward(const om_unet* U, const Conv& c, const bf16* x1, int ld1, int o1, const bf16* x2, int ld2, int o2,
                       bf16* y, const Grid& g, cudaStream_t s) {
  return conv_tc(U, x1, c.cin1, ld1, o1, x2, c.cin2, ld2, o2, c.wt, c.cout, U->w + c.b_off, y, c.cout, 0, nullptr, 1, g,
                 s);
}

// dX (rows of cin1 + cin2) = data gradient of conv c for the pre-activation gradient dyp: the
// forward convolution of dyp with the flipped, transposed weights WD[27][cin][cout]
om_status conv_dgrad(const om_unet* U, const Conv& c, const bf16* dyp, bf16* dx, const Grid& g, cudaStream_t s) {
  const int N = c.cin1 + c.cin2;
  return conv_tc(U, dyp, c.cout, c.cout, 0, nullptr, 0, 0, 0, c.wd, N, nullptr, dx, N, 0, nullptr, 0, g, s);
}

// dW += the weight gradient on tcgen05: conv3d_wgrad_tc32 for at most 32 output channels
// (one CTA per input chunk of 32 channels), else conv3d_wgrad_tc (one CTA per chunk, dz and
// part of 128 output channels); gridDim.x of them over the tiles
om_status wgrad_tc(om_unet* U, const Conv& c, const bf16* x1, int ld1, int o1, const bf16* x2, int ld2, int o2,
                   const bf16* dyp, const Grid& g, cudaStream_t s) {
  TcWgradArgs a{};
  a.c1 = c.cin1, a.c2 = c.cin2, a.nch1 = (c.cin1 + 31) / 32;
  const int nch2 = (c.cin2 + 31) / 32;
  a.N = c.cout, a.Nm = (std::min(c.cout, 128) + 31) / 32 * 32;
  a.npart = (c.cout + 127) / 128;
  a.dw = U->g + c.w_off;
  a.g = g;
  a.tx = (g.W + kTcTx - 1) / kTcTx, a.ty = (g.H + kTcTy - 1) / kTcTy;
  a.vec4 = reinterpret_cast<uintptr_t>(a.dw) % 16 == 0;
  a.err = U->tc_err.p;
  int dev = 0, sms = 0;
  OM_CUDA(cudaGetDevice(&dev));
  OM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (a.Nm == 32) {
    // at most 32 output channels: the swapped form (conv3d_wgrad_tc32), all 27 offsets per CTA
    CUtensorMap m1, m2, md;
    OM_TRY(activation_map(&m1, x1, c.cin1, ld1, o1, g, 4));
    if (c.cin2 > 0) OM_TRY(activation_map(&m2, x2, c.cin2, ld2, o2, g, 4));
    else m2 = m1;
    OM_TRY(activation_map(&md, dyp, c.cout, c.cout, 0, g, 5));
    a.nstage = (int)std::min<size_t>(4, (227 * 1024 - 2048) / kWnStage);
    const size_t smem = 1024 + (size_t)a.nstage * kWnStage + 8 * (2 * a.nstage + 1) + 16;
    const int gy = a.nch1 + nch2;
    const int64_t ntiles = (int64_t)g.B * g.D * (a.ty + 1) * a.tx;
    const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ntiles, sms / gy));
    OM_CUDA(cudaFuncSetAttribute(conv3d_wgrad_tc32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    conv3d_wgrad_tc32<<<dim3(gx, (unsigned)gy), kTcThreads, smem, s>>>(m1, m2, md, a);
    OM_CUDA(cudaGetLastError());
    return OM_OK;
  }
  // wider outputs: conv3d_wgrad_tc, the three (dz, dy) pairs of one dz per CTA
  a.npair = 3;
  const int hmode = 2;
  CUtensorMap m1, m2, md;
  OM_TRY(activation_map(&m1, x1, c.cin1, ld1, o1, g, hmode));
  if (c.cin2 > 0) OM_TRY(activation_map(&m2, x2, c.cin2, ld2, o2, g, hmode));
  else m2 = m1;
  OM_TRY(activation_map(&md, dyp, c.cout, c.cout, 0, g, 3));
  const size_t stage = wg_stage_bytes(a.npair, a.Nm);
  a.nstage = (int)std::min<size_t>(4, (227 * 1024 - 2048) / stage);
  const size_t smem = 1024 + (size_t)a.nstage * stage + 8 * (2 * a.nstage + 1) + 16;
  const int gy = (a.nch1 + nch2) * (9 / a.npair) * a.npart;
  const int64_t ntiles = (int64_t)g.B * g.D * a.ty * a.tx;
  // one CTA per SM fits (shared memory); at most one wave, or the last CTAs run as a second
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ntiles, sms / gy));
  OM_CUDA(cudaFuncSetAttribute(conv3d_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  conv3d_wgrad_tc<<<dim3(gx, (unsigned)gy), kTcThreads, smem, s>>>(m1, m2, md, a);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

// dW += the weight gradient of conv c, db += its bias gradient, for the pre-activation gradient dyp
om_status conv_wgrad(om_unet* U, const Conv& c, const bf16* x1, int ld1, int o1, const bf16* x2, int ld2, int o2,
                     const bf16* dyp, const Grid& g, cudaStream_t s) {
  if (c.cout % 16 || c.cout > 256 || c.cin1 % 8 || c.cin2 % 8 || ld1 % 8 || o1 % 8 ||
      (c.cin2 > 0 && (ld2 % 8 || o2 % 8)))
    return fail(OM_EINVAL, "U-Net: weight-gradient shape outside the tensor-core kernel's layout");
  OM_TRY(wgrad_tc(U, c, x1, ld1, o1, x2, ld2, o2, dyp, g, s));
  bias_grad<<<std::min<int64_t>(blocks(g.voxels() * c.cout), 1216), kT, kT * sizeof(float), s>>>(
      dyp, c.cout, g.voxels(), U->g + c.b_off);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

Grid level_grid(const Grid& g, int l) { return Grid{g.B, g.D >> l, g.H >> l, g.W >> l}; }

om_status prepare(om_unet* U, const Grid& g) {
  if (g.B == U->grid.B && g.D == U->grid.D && g.H == U->grid.H && g.W == U->grid.W) return OM_OK;
  const int L = U->L;
  for (int l = 0; l < L; ++l) {
    const int64_t V = level_grid(g, l).voxels();
    const int cprev = l == 0 ? 16 : U->ch[l - 1];
    const int cnext = l + 1 < L ? U->ch[l + 1] : 0;
    const int c = U->ch[l];
    if (l > 0) OM_TRY(U->in[l].ensure(V * cprev));
    OM_TRY(U->a[l].ensure(V * c));
    OM_TRY(U->s[l].ensure(V * c));
    if (l + 1 < L) {
      OM_TRY(U->u[l].ensure(V * cnext));
      OM_TRY(U->b[l].ensure(V * c));
      OM_TRY(U->h[l].ensure(V * c));
      OM_TRY(U->dcat[l].ensure(V * (cnext + c)));
    }
    const int64_t wmax = std::max((int64_t)c, std::max((int64_t)cprev, (int64_t)(cnext + c)));
    OM_TRY(U->d1[l].ensure(V * wmax));
    OM_TRY(U->d2[l].ensure(V * wmax));
    OM_TRY(U->ds[l].ensure(V * c));
  }
  OM_TRY(U->x0.ensure(g.voxels() * 16));
  OM_TRY(U->out.ensure(g.voxels() * U->out_ch));
  OM_TRY(U->dout.ensure(g.voxels() * U->out_ch));
  U->grid = g;
  return OM_OK;
}

om_status refresh_operands(om_unet* U, cudaStream_t s) {
  auto conv = [&](Conv& c) {
    const int K = c.cin1 + c.cin2;
    weights_fwd<<<blocks(27LL * K * c.cout), kT, 0, s>>>(U->w + c.w_off, K, c.cout, c.wt);
    weights_dgrad<<<blocks(27LL * K * c.cout), kT, 0, s>>>(U->w + c.w_off, K, c.cout, c.wd);
  };
  for (int l = 0; l < U->L; ++l) {
    conv(U->enc1[l]);
    conv(U->enc2[l]);
    if (l + 1 < U->L) {
      conv(U->dec1[l]);
      conv(U->dec2[l]);
    }
  }
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

om_status forward(om_unet* U, const float* x, const Grid& g, cudaStream_t s) {
  OM_TRY(prepare(U, g));
  OM_TRY(refresh_operands(U, s));
  const int L = U->L;
  pack_input<<<blocks(g.voxels() * 16), kT, 0, s>>>(x, U->in_ch, g.voxels(), U->x0.p);
  for (int l = 0; l < L; ++l) {
    const Grid gl = level_grid(g, l);
    const bf16* in = l == 0 ? U->x0.p : U->in[l].p;
    const int cin = l == 0 ? 16 : U->ch[l - 1];
    if (l > 0) avgpool2<<<blocks(gl.voxels() * cin), kT, 0, s>>>(U->s[l - 1].p, level_grid(g, l - 1), cin, U->in[l].p);
    OM_TRY(conv_forward(U, U->enc1[l], in, cin, 0, nullptr, 0, 0, U->a[l].p, gl, s));
    OM_TRY(conv_forward(U, U->enc2[l], U->a[l].p, U->ch[l], 0, nullptr, 0, 0, U->s[l].p, gl, s));
  }
  for (int l = L - 2; l >= 0; --l) {
    const Grid gl = level_grid(g, l);
    const bf16* below = l + 1 == L - 1 ? U->s[L - 1].p : U->h[l + 1].p;
    const int cb = U->ch[l + 1];
    upsample2<<<blocks(gl.voxels() * cb / 8), kT, 0, s>>>(below, gl, cb, U->u[l].p, cb, 0);
    OM_TRY(conv_forward(U, U->dec1[l], U->u[l].p, cb, 0, U->s[l].p, U->ch[l], 0, U->b[l].p, gl, s));
    OM_TRY(conv_forward(U, U->dec2[l], U->b[l].p, U->ch[l], 0, nullptr, 0, 0, U->h[l].p, gl, s));
  }
  const bf16* top = L > 1 ? U->h[0].p : U->s[0].p;
  head_fwd<<<blocks(g.voxels()), kT, 0, s>>>(top, U->ch[0], U->w + U->head_w, U->w + U->head_b, U->out_ch,
                                                         g.voxels(), U->out.p);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

// gradients of the masked MSE w.r.t. every parameter, into U->g
om_status backward(om_unet* U, const float* t, const uint8_t* mk, const Grid& g, double* loss_out, cudaStream_t s) {
  const int L = U->L;
  const int64_t V = g.voxels();
  OM_CUDA(cudaMemsetAsync(U->g, 0, sizeof(float) * U->nparam, s));
  OM_TRY(U->loss.ensure(2));
  OM_CUDA(cudaMemsetAsync(U->loss.p, 0, 2 * sizeof(double), s));
  // masked mean over pore voxels and output channels: the count in loss[1]
  mask_count<<<std::min<unsigned>(blocks(V), 1216), kT, 0, s>>>(mk, V, U->loss.p + 1);
  mse_grad<<<std::min<unsigned>(blocks(V * U->out_ch), 1216), kT, 0, s>>>(U->out.p, t, mk, U->out_ch, V, U->loss.p + 1,
                                                                           U->dout.p, U->loss.p);
  // head
  const int c0 = U->ch[0];
  const bf16* top = L > 1 ? U->h[0].p : U->s[0].p;
  for (int o0 = 0; o0 < U->out_ch; o0 += 4)
    head_bwd_dw<<<1216, kT, 8 * kT * sizeof(float), s>>>(top, U->dout.p, c0, U->out_ch, o0, V, U->g + U->head_w,
                                                         U->g + U->head_b);
  head_bwd_dx<<<blocks(V * c0 / 8), kT, 0, s>>>(U->dout.p, U->w + U->head_w, c0, U->out_ch, V, U->d1[0].p);
  // decoder, top level down: d1[l] holds the gradient of the level's output h_l
  for (int l = 0; l + 1 < L; ++l) {
    const Grid gl = level_grid(g, l);
    const int64_t Vl = gl.voxels();
    const int c = U->ch[l], cb = U->ch[l + 1];
    // h_l = relu(conv(b_l))
    relu_bwd<<<blocks(Vl * c / 8), kT, 0, s>>>(U->d1[l].p, c, 0, U->h[l].p, c, Vl, U->d2[l].p);
    OM_TRY(conv_wgrad(U, U->dec2[l], U->b[l].p, c, 0, nullptr, 0, 0, U->d2[l].p, gl, s));
    OM_TRY(conv_dgrad(U, U->dec2[l], U->d2[l].p, U->d1[l].p, gl, s));
    // b_l = relu(conv(concat(u_l, s_l)))
    relu_bwd<<<blocks(Vl * c / 8), kT, 0, s>>>(U->d1[l].p, c, 0, U->b[l].p, c, Vl, U->d2[l].p);
    OM_TRY(conv_wgrad(U, U->dec1[l], U->u[l].p, cb, 0, U->s[l].p, c, 0, U->d2[l].p, gl, s));
    OM_TRY(conv_dgrad(U, U->dec1[l], U->d2[l].p, U->dcat[l].p, gl, s));
    // u_l = up(h_{l+1}) (or s_{L-1} at the bottom): gradient of the level below
    upsample2_bwd<<<blocks(level_grid(g, l + 1).voxels() * cb / 8), kT, 0, s>>>(U->dcat[l].p, cb + c, 0, gl, cb,
                                                                            U->d1[l + 1].p);
  }
  // encoder, bottom level up: ds[l] = gradient of s_l
  for (int l = L - 1; l >= 0; --l) {
    const Grid gl = level_grid(g, l);
    const int64_t Vl = gl.voxels();
    const int c = U->ch[l];
    const int cin = l == 0 ? 16 : U->ch[l - 1];
    // s_l receives: from the level below (pooling) and from the decoder's skip
    if (l == L - 1) {
      OM_CUDA(cudaMemcpyAsync(U->ds[l].p, U->d1[l].p, sizeof(bf16) * Vl * c, cudaMemcpyDeviceToDevice, s));
    } else {
      avgpool2_bwd<<<blocks(Vl * c / 8), kT, 0, s>>>(U->d2[l + 1].p, gl, c, U->ds[l].p);
      add_into<<<blocks(Vl * c / 8), kT, 0, s>>>(U->ds[l].p, c, Vl, U->dcat[l].p, U->ch[l + 1] + c, U->ch[l + 1]);
    }
    // s_l = relu(conv(a_l))
    relu_bwd<<<blocks(Vl * c / 8), kT, 0, s>>>(U->ds[l].p, c, 0, U->s[l].p, c, Vl, U->d1[l].p);
    OM_TRY(conv_wgrad(U, U->enc2[l], U->a[l].p, c, 0, nullptr, 0, 0, U->d1[l].p, gl, s));
    OM_TRY(conv_dgrad(U, U->enc2[l], U->d1[l].p, U->d2[l].p, gl, s));
    // a_l = relu(conv(in_l))
    relu_bwd<<<blocks(Vl * c / 8), kT, 0, s>>>(U->d2[l].p, c, 0, U->a[l].p, c, Vl, U->d1[l].p);
    const bf16* in = l == 0 ? U->x0.p : U->in[l].p;
    OM_TRY(conv_wgrad(U, U->enc1[l], in, cin, 0, nullptr, 0, 0, U->d1[l].p, gl, s));
    // d2[l] = gradient of in_l (pooled s_{l-1}); not needed at the input
    if (l > 0) OM_TRY(conv_dgrad(U, U->enc1[l], U->d1[l].p, U->d2[l].p, gl, s));
  }
  double h = 0.0;
  OM_CUDA(cudaMemcpyAsync(&h, U->loss.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  OM_TRY(check_tc(U, s));
  if (loss_out) *loss_out = h;
  return OM_OK;
}

uint64_t splitmix(uint64_t& st) {
  st += 0x9E3779B97F4A7C15ULL;
  uint64_t z = st;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

om_status check_grid(const om_unet* U, const Grid& g) {
  const int q = 1 << (U->L - 1);
  if (g.B <= 0 || g.D <= 0 || g.H <= 0 || g.W <= 0 || g.D % q || g.H % q || g.W % q)
    return fail(OM_EINVAL, "U-Net: box edges must be positive multiples of 2^(levels-1)");
  return OM_OK;
}

}  // namespace

extern "C" om_status om_unet_destroy(om_unet* U) {
  if (!U) return OM_OK;
  auto drop = [](std::vector<Buf<bf16>>& v) {
    for (auto& b : v) b.release();
  };
  drop(U->in), drop(U->a), drop(U->s), drop(U->u), drop(U->b), drop(U->h);
  drop(U->d1), drop(U->d2), drop(U->dcat), drop(U->ds);
  U->x0.release(), U->out.release(), U->dout.release(), U->loss.release(), U->tc_err.release();
  for (auto* v : {&U->enc1, &U->enc2, &U->dec1, &U->dec2})
    for (auto& c : *v) {
      cudaFree(c.wt);
      cudaFree(c.wd);
    }
  cudaFree(U->w), cudaFree(U->g), cudaFree(U->m), cudaFree(U->v);
  delete U;
  return OM_OK;
}

extern "C" om_status om_unet_create(int32_t in_ch, int32_t out_ch, int32_t levels, const int32_t* ch, uint64_t seed,
                                    om_unet** out) {
  if (!out || !ch || in_ch < 1 || in_ch > 16 || out_ch < 1 || levels < 1 || levels > 6)
    return fail(OM_EINVAL, "om_unet_create: 1..16 inputs, >= 1 output, 1..6 levels");
  for (int l = 0; l < levels; ++l)
    if (ch[l] < 16 || ch[l] % 16 || ch[l] > 256) return fail(OM_EINVAL, "om_unet_create: channels must be multiples of 16 up to 256");
  om_unet* U = new om_unet();
  U->in_ch = in_ch, U->out_ch = out_ch, U->L = levels;
  U->ch.assign(ch, ch + levels);
  int64_t off = 0;
  auto add = [&](int c1, int c2, int co) {
    Conv c;
    c.cin1 = c1, c.cin2 = c2, c.cout = co;
    c.w_off = off;
    off += 27LL * (c1 + c2) * co;
    c.b_off = off;
    off += co;
    return c;
  };
  for (int l = 0; l < levels; ++l) {
    U->enc1.push_back(add(l == 0 ? 16 : ch[l - 1], 0, ch[l]));
    U->enc2.push_back(add(ch[l], 0, ch[l]));
  }
  U->dec1.resize(std::max(0, levels - 1));
  U->dec2.resize(std::max(0, levels - 1));
  for (int l = levels - 2; l >= 0; --l) {
    U->dec1[l] = add(ch[l + 1], ch[l], ch[l]);
    U->dec2[l] = add(ch[l], 0, ch[l]);
  }
  U->head_w = off;
  off += (int64_t)ch[0] * out_ch;
  U->head_b = off;
  off += out_ch;
  U->nparam = off;
  const int L = levels;
  U->in.resize(L), U->a.resize(L), U->s.resize(L), U->u.resize(L), U->b.resize(L), U->h.resize(L);
  U->d1.resize(L), U->d2.resize(L), U->dcat.resize(L), U->ds.resize(L);
  // He-uniform initial weights from a SplitMix64 stream, zero biases
  std::vector<float> w((size_t)off, 0.f);
  uint64_t st = seed;
  auto init = [&](const Conv& c, int fan_in) {
    const double bound = std::sqrt(6.0 / fan_in);
    for (int64_t i = 0; i < 27LL * (c.cin1 + c.cin2) * c.cout; ++i)
      w[(size_t)(c.w_off + i)] = (float)(bound * (2.0 * ((double)(splitmix(st) >> 11) * 0x1.0p-53) - 1.0));
  };
  for (int l = 0; l < L; ++l) {
    init(U->enc1[l], 27 * (l == 0 ? in_ch : ch[l - 1]));
    init(U->enc2[l], 27 * ch[l]);
  }
  for (int l = L - 2; l >= 0; --l) {
    init(U->dec1[l], 27 * (ch[l + 1] + ch[l]));
    init(U->dec2[l], 27 * ch[l]);
  }
  // the 1x1 head starts at zero: the network's first output is 0 (the cold
  // start) and the first Adam steps cannot blow the decoder's ReLUs up (with
  // a He-initialised head the first outputs are O(10) and training stalls
  // in a state that predicts a constant)
  auto dal = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      (void)cudaGetLastError();
      *p = nullptr;
      return false;
    }
    return true;
  };
  bool ok = dal((void**)&U->w, sizeof(float) * off) && dal((void**)&U->g, sizeof(float) * off) &&
            dal((void**)&U->m, sizeof(float) * off) && dal((void**)&U->v, sizeof(float) * off);
  for (auto* v : {&U->enc1, &U->enc2, &U->dec1, &U->dec2})
    for (auto& c : *v) {
      const size_t n = 27ull * (c.cin1 + c.cin2) * c.cout;
      ok = ok && dal((void**)&c.wt, n * sizeof(bf16)) && dal((void**)&c.wd, n * sizeof(bf16));
    }
  ok = ok && U->tc_err.ensure(1) == OM_OK;
  if (!ok) {
    om_unet_destroy(U);
    return fail(OM_ENOMEM, "om_unet_create: device allocation failed");
  }
  if (cudaMemcpy(U->w, w.data(), sizeof(float) * off, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(U->tc_err.p, 0, sizeof(int)) != cudaSuccess ||
      cudaMemset(U->m, 0, sizeof(float) * off) != cudaSuccess || cudaMemset(U->v, 0, sizeof(float) * off) != cudaSuccess) {
    om_unet_destroy(U);
    return fail(OM_ECUDA, "om_unet_create: initialisation failed");
  }
  *out = U;
  return OM_OK;
}

extern "C" om_status om_unet_param_count(const om_unet* U, int64_t* n) {
  if (!U || !n) return fail(OM_EINVAL, "om_unet_param_count: null pointer");
  *n = U->nparam;
  return OM_OK;
}

extern "C" om_status om_unet_get_params(const om_unet* U, float* dst_dev, void* stream) {
  if (!U || !dst_dev) return fail(OM_EINVAL, "om_unet_get_params: null pointer");
  OM_CUDA(cudaMemcpyAsync(dst_dev, U->w, sizeof(float) * U->nparam, cudaMemcpyDeviceToDevice, as_stream(stream)));
  return OM_OK;
}

extern "C" om_status om_unet_set_params(om_unet* U, const float* src_dev, void* stream) {
  if (!U || !src_dev) return fail(OM_EINVAL, "om_unet_set_params: null pointer");
  OM_CUDA(cudaMemcpyAsync(U->w, src_dev, sizeof(float) * U->nparam, cudaMemcpyDeviceToDevice, as_stream(stream)));
  return OM_OK;
}

extern "C" om_status om_unet_get_grads(const om_unet* U, float* dst_dev, void* stream) {
  if (!U || !dst_dev) return fail(OM_EINVAL, "om_unet_get_grads: null pointer");
  OM_CUDA(cudaMemcpyAsync(dst_dev, U->g, sizeof(float) * U->nparam, cudaMemcpyDeviceToDevice, as_stream(stream)));
  return OM_OK;
}

extern "C" om_status om_unet_forward(om_unet* U, const float* x, int32_t B, int32_t D, int32_t H, int32_t W, float* y,
                                     void* stream) {
  if (!U || !x || !y) return fail(OM_EINVAL, "om_unet_forward: null pointer");
  const Grid g{B, D, H, W};
  OM_TRY(check_grid(U, g));
  cudaStream_t s = as_stream(stream);
  OM_TRY(forward(U, x, g, s));
  OM_CUDA(cudaMemcpyAsync(y, U->out.p, sizeof(float) * g.voxels() * U->out_ch, cudaMemcpyDeviceToDevice, s));
  return check_tc(U, s);
}

extern "C" om_status om_unet_backward(om_unet* U, const float* x, const float* t, const uint8_t* m, int32_t B,
                                      int32_t D, int32_t H, int32_t W, double* loss_out, void* stream) {
  if (!U || !x || !t || !m) return fail(OM_EINVAL, "om_unet_backward: null pointer");
  const Grid g{B, D, H, W};
  OM_TRY(check_grid(U, g));
  cudaStream_t s = as_stream(stream);
  OM_TRY(forward(U, x, g, s));
  return backward(U, t, m, g, loss_out, s);
}

namespace om {
namespace nn {
__global__ void pack_structure(const uint8_t* mask, const float* d, int64_t n, float ds, float* x) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    x[2 * v] = mask[v] ? 1.f : 0.f;
    x[2 * v + 1] = d[v] * ds;
  }
}

__global__ void pack_structure3(const uint8_t* mask, const float* d, const float* e, int64_t n, float ds, float* x) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    x[3 * v] = mask[v] ? 1.f : 0.f;
    x[3 * v + 1] = d[v] * ds;
    x[3 * v + 2] = e[v];
  }
}
}  // namespace nn
}  // namespace om

extern "C" om_status om_unet_pack_structure(const uint8_t* mask_dev, const float* d_nm_dev, int64_t n, double d_scale,
                                           float* x_dev, void* stream) {
  if (!mask_dev || !d_nm_dev || !x_dev || n < 0) return fail(OM_EINVAL, "om_unet_pack_structure: bad argument");
  if (n == 0) return OM_OK;
  om::nn::pack_structure<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1 << 20), 256, 0, as_stream(stream)>>>(
      mask_dev, d_nm_dev, n, (float)d_scale, x_dev);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

extern "C" om_status om_unet_pack_structure3(const uint8_t* mask_dev, const float* d_nm_dev, double d_scale,
                                            const float* extra_dev, int64_t n, float* x_dev, void* stream) {
  if (!mask_dev || !d_nm_dev || !extra_dev || !x_dev || n < 0)
    return fail(OM_EINVAL, "om_unet_pack_structure3: bad argument");
  if (n == 0) return OM_OK;
  om::nn::pack_structure3<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1 << 20), 256, 0, as_stream(stream)>>>(
      mask_dev, d_nm_dev, extra_dev, n, (float)d_scale, x_dev);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

extern "C" om_status om_unet_train_step(om_unet* U, const float* x, const float* t, const uint8_t* m, int32_t B,
                                        int32_t D, int32_t H, int32_t W, float lr, double* loss_out, void* stream) {
  OM_TRY(om_unet_backward(U, x, t, m, B, D, H, W, loss_out, stream));
  cudaStream_t s = as_stream(stream);
  ++U->step;
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.f - std::pow(b1, (float)U->step), bc2 = 1.f - std::pow(b2, (float)U->step);
  adam_step<<<blocks(U->nparam), kT, 0, s>>>(U->w, U->g, U->m, U->v, U->nparam, lr, b1, b2, 1e-8f, bc1, bc2);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}
