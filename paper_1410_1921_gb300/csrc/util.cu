// util.cu -- error state, domain checks, device scan and fixed-order
// reductions shared by the kernels of the library.
#include <cstdio>

#include "common.cuh"

#include <map>
#include <mutex>
#include <tuple>

namespace om {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

om_status fail(om_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

om_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof buf, "%s failed at %s:%d: %s", what, file, line, cudaGetErrorString(e));
  g_err = buf;
  return e == cudaErrorMemoryAllocation ? OM_ENOMEM : OM_ECUDA;
}

om_status check_domain(const om_domain& d) {
  if (d.nx <= 0 || d.ny <= 0 || d.nz <= 0) return fail(OM_EINVAL, "domain sizes must be positive");
  if (d.nx > 1024 || d.ny > 2048 || d.nz > 2048)
    return fail(OM_EINVAL, "domain limits: nx <= 1024, ny <= 2048, nz <= 2048");
  if (!(d.dx_nm > 0.0)) return fail(OM_EINVAL, "dx_nm must be positive");
  if (voxels(d) >= (int64_t)0xFFFFFFFFll) return fail(OM_EINVAL, "domain has too many voxels");
  return OM_OK;
}

// ------------------------------------------------------------------ scan
// Exclusive prefix sum of uint32 in three passes: per-block totals, a scan of
// the totals (recursively), and a per-block scan that adds the block offset.
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;  // per thread
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ inline uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_sums, uint32_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_sums[lane] = w;  // inclusive scan of the warp totals
  }
  __syncthreads();
  uint32_t base = wid > 0 ? warp_sums[wid - 1] : 0u;
  if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
  return base + x - v;
}

__global__ void scan_tile_sums(const uint32_t* in, int64_t n, uint32_t* sums) {
  __shared__ uint32_t ws[32];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
    if (i < n) s += in[i];
  }
  uint32_t tot;
  block_exclusive_scan(s, ws, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void scan_tile_apply(const uint32_t* in, uint32_t* out, int64_t n, const uint32_t* offs,
                                uint64_t* total_dev) {
  __shared__ uint32_t ws[32];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
    v[k] = i < n ? in[i] : 0u;
    s += v[k];
  }
  uint32_t tot;
  uint32_t ex = block_exclusive_scan(s, ws, &tot) + (offs ? offs[blockIdx.x] : 0u);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
    if (i < n) out[i] = ex;
    ex += v[k];
  }
  if (total_dev && blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1)
    *total_dev = (uint64_t)ex;
}

om_status exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint64_t* total_dev,
                             cudaStream_t s) {
  if (n <= 0) {
    if (total_dev) OM_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(uint64_t), s));
    return OM_OK;
  }
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 1) {
    scan_tile_apply<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, total_dev);
    OM_CUDA(cudaGetLastError());
    return OM_OK;
  }
  DevBuf<uint32_t> sums, offs;
  OM_TRY(sums.alloc(tiles));
  OM_TRY(offs.alloc(tiles));
  scan_tile_sums<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums.p);
  OM_CUDA(cudaGetLastError());
  OM_TRY(exclusive_scan_u32(sums.p, offs.p, tiles, nullptr, s));
  scan_tile_apply<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, offs.p, total_dev);
  OM_CUDA(cudaGetLastError());
  // the buffers are freed by cudaFree, which waits for the stream's work
  return OM_OK;
}

// ------------------------------------------------------------------ reductions
__global__ void finalize_partials(const double* partials, int nblk, int nval, double* out) {
  // one block; value k summed by the block in a fixed order
  __shared__ double sm[256];
  for (int k = 0; k < nval; ++k) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += partials[(int64_t)b * nval + k];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = sm[0];
    __syncthreads();
  }
}

// ------------------------------------------------------------------ tuning cache
namespace {
struct TuneKey {
  int kind, prec, dev, octave;
  bool operator<(const TuneKey& o) const {
    if (kind != o.kind) return kind < o.kind;
    if (prec != o.prec) return prec < o.prec;
    if (dev != o.dev) return dev < o.dev;
    return octave < o.octave;
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune;

TuneKey tune_key(int kind, int prec, int64_t nf) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  int oct = 0;
  while (oct < 62 && (int64_t(1) << (oct + 1)) <= nf) ++oct;
  return TuneKey{kind, prec, dev, oct};
}
}  // namespace

bool tuned_lookup(int kind, int prec, int64_t nf, int var[2]) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(tune_key(kind, prec, nf));
  if (it == g_tune.end()) return false;
  var[0] = it->second.first;
  var[1] = it->second.second;
  return true;
}

void tuned_store(int kind, int prec, int64_t nf, const int var[2]) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[tune_key(kind, prec, nf)] = {var[0], var[1]};
}

unsigned resident_blocks(const void* kernel, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t, int>, unsigned> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  const auto key = std::make_tuple(kernel, threads, smem, dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
  const unsigned r = sms * per > 0 ? (unsigned)(sms * per) : 1u;
  cache[key] = r;
  return r;
}

void launch_finalize(const double* partials, int nblk, int nval, double* out, cudaStream_t s) {
  finalize_partials<<<1, 256, 0, s>>>(partials, nblk, nval, out);
}

}  // namespace om

extern "C" const char* om_last_error(void) { return om::g_err.c_str(); }

extern "C" const char* om_version(void) { return "om-gb300 0.1 (sm_103a)"; }
