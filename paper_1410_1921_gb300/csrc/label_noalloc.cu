// label_noalloc.cu -- om_label_connectivity_noalloc: the connected-phase
// labelling of om_label_connectivity_dev for callers that cannot allocate
// device memory.
//
// Who needs it: a host process whose device memory is already owned by
// another allocator (a framework's caching pool that has reserved most of
// the GPU), or a long-running service that fixes its memory plan at start-up
// and must not take the implicit device-wide synchronisation and failure
// modes of cudaMalloc / cudaFree in its steady state.  Those callers still
// own every input and output buffer; what they cannot provide is the
// labelling's scratch (the per-component inlet/outlet flags and two
// counters).
//
// Scratch: g_label_scratch below, a file-scope device array.  Every GPU that
// loads this library holds it (4 MiB + 256 B) until the process exits.  It
// bounds the problem size to kNoAllocMaxVoxels = 2^24 voxels (256^3): two
// flag bits per voxel, packed 16 to a 32-bit word.  Larger boxes are
// rejected with OM_EINVAL.
//
// Host code cannot use the array's name as a device address (in host code
// it names a host-side stand-in), so the first call on each device, with
// that device current, asks the runtime for the address with
// cudaGetSymbolAddress and keeps it, together with the unique id of the
// CUDA context that was current.  A later call under another context (the
// device was reset and its primary context recreated, or the caller made a
// context of its own current) looks the address up again for that context.
// That first call on a device (or in a new context) should come before any
// stream capture on it.  Device code below still names the array only
// through the pointer it is given.
//
// Every call shares the one array and leaves its contents behind: each call
// clears the flag words and counters it uses before its kernels run.  Calls
// whose work overlaps on the GPU (on different streams, or from different
// host threads) race on the array; serialise them.
#include <cuda.h>  // driver types only: the two driver calls are fetched through the runtime

#include <mutex>

#include "common.cuh"

namespace om {
void launch_union_find(const uint8_t* mask_dev, const om_domain& d, int* labels_dev, cudaStream_t s);

namespace {

constexpr int64_t kNoAllocMaxVoxels = int64_t(1) << 24;
constexpr size_t kFlagBytes = (size_t)(kNoAllocMaxVoxels / 16) * sizeof(uint32_t);  // 4 MiB
constexpr size_t kScratchBytes = kFlagBytes + 256;                                  // + counters
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_label_scratch[kScratchBytes];

std::mutex g_scratch_mu;
struct ScratchSlot {
  unsigned long long ctx_id;  // unique id of the context the address belongs to
  void* addr;
};
ScratchSlot g_scratch[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// unique id of the context current on this thread (0 if none is current);
// the driver functions come through the runtime, so nothing links libcuda
om_status current_context_id(unsigned long long* id) {
  if (!g_ctx_get_current || !g_ctx_get_id) {
    void* a = nullptr;
    void* b = nullptr;
    cudaDriverEntryPointQueryResult qa{}, qb{};
    OM_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa));
    OM_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb));
    if (qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
      return fail(OM_ECUDA, "om_label_connectivity_noalloc: driver context queries unavailable");
    g_ctx_get_current = (CtxGetCurrentFn)a;
    g_ctx_get_id = (CtxGetIdFn)b;
  }
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return fail(OM_ECUDA, "cuCtxGetCurrent failed");
  *id = 0;
  if (ctx && g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return fail(OM_ECUDA, "cuCtxGetId failed");
  return OM_OK;
}

// device address of g_label_scratch on the current device, looked up once
// per device and context
om_status scratch_address(void** out) {
  int dev = 0;
  OM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(OM_EINVAL, "om_label_connectivity_noalloc: device ordinal too large");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  unsigned long long id = 0;
  OM_TRY(current_context_id(&id));
  if (id == 0 || !g_scratch[dev].addr || g_scratch[dev].ctx_id != id) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_label_scratch);  // makes the device's context current if none is
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_label_scratch)", __FILE__, __LINE__);
    OM_TRY(current_context_id(&id));
    g_scratch[dev] = ScratchSlot{id, p};
  }
  *out = g_scratch[dev].addr;
  return OM_OK;
}

// two bits per component root in packed words: bit 0 inlet, bit 1 outlet
__global__ void mark_faces_packed(const int* lab, int nx, int ny, int nz, uint32_t* flags) {
  const int64_t plane = (int64_t)ny * nz;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += (int64_t)gridDim.x * blockDim.x) {
    const int a = lab[i];
    if (a >= 0) atomicOr(flags + (a >> 4), 1u << (2 * (a & 15)));
    const int b = lab[(int64_t)(nx - 1) * plane + i];
    if (b >= 0) atomicOr(flags + (b >> 4), 2u << (2 * (b & 15)));
  }
}

__global__ void transport_from_packed(const int* lab, const uint32_t* flags, int64_t N, uint8_t* tr,
                                      unsigned long long* counts) {
  unsigned long long np = 0, nt = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    const int a = lab[v];
    const bool t = a >= 0 && ((flags[a >> 4] >> (2 * (a & 15))) & 3u) == 3u;
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
}  // namespace om

using namespace om;

extern "C" om_status om_label_connectivity_noalloc(const uint8_t* mask_dev, om_domain d, int32_t* labels_dev,
                                                   uint8_t* transport_dev, double* connectivity_out,
                                                   void* stream) {
  if (!mask_dev || !labels_dev) return fail(OM_EINVAL, "om_label_connectivity_noalloc: mask and labels are required");
  OM_TRY(check_domain(d));
  const int64_t N = voxels(d);
  if (N > kNoAllocMaxVoxels)
    return fail(OM_EINVAL, "om_label_connectivity_noalloc: " + std::to_string(N) +
                               " voxels exceed the static scratch limit of 2^24 (16777216) voxels");
  cudaStream_t s = as_stream(stream);
  void* base = nullptr;
  OM_TRY(scratch_address(&base));
  uint32_t* flags = (uint32_t*)base;
  unsigned long long* counts = (unsigned long long*)((unsigned char*)base + kFlagBytes);
  // the array keeps the previous call's contents: clear what this call reads
  OM_CUDA(cudaMemsetAsync(flags, 0, (size_t)((N + 15) / 16) * sizeof(uint32_t), s));
  OM_CUDA(cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), s));
  launch_union_find(mask_dev, d, labels_dev, s);
  mark_faces_packed<<<152, 256, 0, s>>>(labels_dev, d.nx, d.ny, d.nz, flags);
  transport_from_packed<<<1216, 256, 0, s>>>(labels_dev, flags, N, transport_dev, counts);
  OM_CUDA(cudaGetLastError());
  unsigned long long h[2] = {0, 0};
  OM_CUDA(cudaMemcpyAsync(h, counts, sizeof h, cudaMemcpyDeviceToHost, s));
  OM_CUDA(cudaStreamSynchronize(s));
  if (connectivity_out) *connectivity_out = h[0] > 0 ? (double)h[1] / (double)h[0] : 0.0;
  return OM_OK;
}
