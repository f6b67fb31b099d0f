// dense.cu -- the dense population layout (om_flow_params.layout,
// om_diff_params.layout = OM_LAYOUT_DENSE), an alternative to the
// fluid-node-only storage of the node set (nodeset.cu) for structures whose
// pores fill most of the box.
//
// Populations are stored for every voxel v = (x ny + y) nz + z of the box,
// one array per population (SoA, pitch P >= N).  A thread updates one voxel
// and leaves at once when the voxel is not a node (a solid or an isolated
// pore voxel): a warp is 32 voxels consecutive in z, so a node's neighbours
// in +-y and +-x are 32 consecutive voxels of another column, at an offset
// fixed by the direction -- the addresses need no lookup, only the node mask
// byte of each neighbour (bounce-back where it is 0).  The update of a node
// is the sparse sweeps' own (flow_node_nb / diff_node_nb on the node's
// voxel index): the same collision, streaming, bounce-back, Dirichlet
// half-links and rebased references, so both layouts give the same bits per
// node and step.  What the layout trades: no neighbour lookup (the sparse odd
// sweeps' dependent column-map loads) and aligned coalesced neighbour rows,
// against moving the non-node voxels' lanes through every launch (a warp
// whose 32 voxels are all solid costs one load of the mask).  Solves: the
// flow with the body force (periodic in x, y, z), FP64 or FP32 (rebased for
// its last decades as om_flow_solve does); the D3Q7 diffusion, FP64 or FP32
// (rebased storage, extrapolated restarts as om_diff_solve does).  The
// loops, tests and results are those of om_flow_solve / om_diff_solve.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "diff_core.cuh"
#include "flow_core.cuh"

namespace om {
namespace {

struct DenseBox {
  int nx, ny, nz;
  uint32_t N;
  const uint8_t* node;  // 1 where the voxel is a lattice node (the transport set)
};

__device__ __forceinline__ void dense_xyz(const DenseBox& b, uint32_t v, int& x, int& y, int& z) {
  z = (int)(v % (uint32_t)b.nz);
  const uint32_t r = v / (uint32_t)b.nz;
  y = (int)(r % (uint32_t)b.ny);
  x = (int)(r / (uint32_t)b.ny);
}

__device__ __forceinline__ uint32_t dense_voxel(const DenseBox& b, int x, int y, int z) {
  return ((uint32_t)x * (uint32_t)b.ny + (uint32_t)y) * (uint32_t)b.nz + (uint32_t)z;
}

__device__ __forceinline__ int wrap(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

// nb[i] = voxel of x + e_i (every axis periodic: the body-force flow), or
// kNoNode where that voxel is not a node; the 3 x 3 row bases of the
// neighbourhood are formed once
__device__ __forceinline__ void dense_nb19(const DenseBox& b, int x, int y, int z, uint32_t (&nb)[19]) {
  const uint32_t X[3] = {(uint32_t)wrap(x - 1, b.nx), (uint32_t)x, (uint32_t)wrap(x + 1, b.nx)};
  const uint32_t Y[3] = {(uint32_t)wrap(y - 1, b.ny), (uint32_t)y, (uint32_t)wrap(y + 1, b.ny)};
  const uint32_t Z[3] = {(uint32_t)wrap(z - 1, b.nz), (uint32_t)z, (uint32_t)wrap(z + 1, b.nz)};
  uint32_t row[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) row[i][j] = (X[i] * (uint32_t)b.ny + Y[j]) * (uint32_t)b.nz;
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const uint32_t w = row[q19_e(i, 0) + 1][q19_e(i, 1) + 1] + Z[q19_e(i, 2) + 1];
    nb[i] = __ldg(b.node + w) ? w : kNoNode;
  }
}

// the same for the D3Q7 diffusion: y, z periodic, nothing beyond the x faces
// (those links are the Dirichlet half links)
__device__ __forceinline__ void dense_nb7(const DenseBox& b, int x, int y, int z, uint32_t (&nb)[7]) {
  nb[0] = dense_voxel(b, x, y, z);
#pragma unroll
  for (int i = 1; i < 7; ++i) {
    const int xx = x + D3Q7::e(i, 0);
    if (xx < 0 || xx >= b.nx) {
      nb[i] = kNoNode;
      continue;
    }
    const uint32_t w = dense_voxel(b, xx, wrap(y + D3Q7::e(i, 1), b.ny), wrap(z + D3Q7::e(i, 2), b.nz));
    nb[i] = __ldg(b.node + w) ? w : kNoNode;
  }
}

template <class T, bool ODD>
__global__ void __launch_bounds__(256) dense_flow_sweep(FlowArgs<T> a, DenseBox b) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= b.N || !__ldg(b.node + v)) return;
  uint32_t nb[19];
  if (ODD) {
    int x, y, z;
    dense_xyz(b, v, x, y, z);
    dense_nb19(b, x, y, z, nb);
  }
  flow_node_nb<T, ODD>(a, v, nb);
}

// even steps two consecutive voxels per thread: both nodes move as vectors
// of two (flow_pair_even), else each node alone
template <class T>
__global__ void __launch_bounds__(256) dense_flow_pair(FlowArgs<T> a, DenseBox b) {
  const uint32_t v = 2u * (blockIdx.x * blockDim.x + threadIdx.x);
  if (v >= b.N) return;
  const bool n0 = __ldg(b.node + v), n1 = v + 1 < b.N && __ldg(b.node + v + 1);
  uint32_t nb[19];
  if (n0 && n1) {
    flow_pair_even<T>(a, v);
  } else {
    if (n0) flow_node_nb<T, false>(a, v, nb);
    if (n1) flow_node_nb<T, false>(a, v + 1, nb);
  }
}

template <class T>
__global__ void __launch_bounds__(256) dense_diff_pair(DiffArgs<T> a, DenseBox b) {
  const uint32_t v = 2u * (blockIdx.x * blockDim.x + threadIdx.x);
  if (v >= b.N) return;
  const bool n0 = __ldg(b.node + v), n1 = v + 1 < b.N && __ldg(b.node + v + 1);
  uint32_t nb[7];
  if (n0 && n1) {
    diff_pair_even<T, D3Q7>(a, v);
  } else {
    // the even update does not depend on x
    if (n0) diff_node_nb<T, D3Q7, false>(a, v, 0, nb);
    if (n1) diff_node_nb<T, D3Q7, false>(a, v + 1, 0, nb);
  }
}

template <class T, bool ODD>
__global__ void __launch_bounds__(256) dense_diff_sweep(DiffArgs<T> a, DenseBox b) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= b.N || !__ldg(b.node + v)) return;
  int x, y, z;
  dense_xyz(b, v, x, y, z);
  uint32_t nb[7];
  if (ODD) dense_nb7(b, x, y, z, nb);
  diff_node_nb<T, D3Q7, ODD>(a, v, x, nb);
}

// Observables at an even time, as the sparse observe kernels: flow sum u_x,
// sum |u_x - prev|, sum |u_x|, sum rho - 1; diffusion sum J_x, sum |C - prev|,
// sum |C|, sum C, sum D_L.  prev <- the field (dprev <- its change).
template <class T>
__global__ void __launch_bounds__(kObsThreads) dense_flow_observe(FlowArgs<T> a, DenseBox b, double* prev,
                                                                  double* partials) {
  using C = typename Stg<T>::C;
  double acc[4] = {0, 0, 0, 0};
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < b.N; v += gridDim.x * blockDim.x) {
    if (!b.node[v]) continue;
    uint32_t nb[19];
    C f[19];
    flow_load<T, false>(a, v, nb, f);
    double rho = 0, jx = 0;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
      rho += (double)f[i];
      jx += (double)q19_e(i, 0) * (double)f[i];
    }
    const double ux = jx + 0.5 * (double)a.g;
    acc[3] += rho + flow_ref(a, v);
    acc[0] += ux;
    acc[1] += fabs(ux - prev[v]);
    acc[2] += fabs(ux);
    prev[v] = ux;
  }
  block_reduce_store<4>(acc, partials);
}

template <class T>
__global__ void __launch_bounds__(kObsThreads) dense_diff_observe(DiffArgs<T> a, DenseBox b, double* prev,
                                                                  double* partials, double* dprev) {
  using C = typename Stg<T>::C;
  double acc[5] = {0, 0, 0, 0, 0};
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < b.N; v += gridDim.x * blockDim.x) {
    if (!b.node[v]) continue;
    int x, y, z;
    dense_xyz(b, v, x, y, z);
    uint32_t nb[7];
    C g[7];
    diff_load<T, D3Q7, false>(a, v, nb, x, g);
    double dev = 0, ex = 0;
#pragma unroll
    for (int i = 0; i < 7; ++i) {
      dev += (double)g[i];
      if (D3Q7::e(i, 0)) ex += D3Q7::e(i, 0) > 0 ? (double)g[i] : -(double)g[i];
    }
    const double c = dev + diff_ref(a, v, x);
    const double om = (double)a.omega[v];
    acc[0] += (1.0 - 0.5 * om) * ex;
    acc[1] += fabs(c - prev[v]);
    acc[2] += fabs(c);
    acc[3] += c;
    acc[4] += D3Q7::cs2 * (1.0 / om - 0.5);
    if (dprev) dprev[v] = c - prev[v];
    prev[v] = c;
  }
  block_reduce_store<5>(acc, partials);
}

// fields at an even time (float N, 0 off the nodes): u_x as om_flow_get_velocity, C as om_diff_get_fields
template <class T>
__global__ void dense_flow_ux(FlowArgs<T> a, DenseBox b, float* ux) {
  using C = typename Stg<T>::C;
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= b.N) return;
  if (!b.node[v]) {
    ux[v] = 0.f;
    return;
  }
  uint32_t nb[19];
  C f[19];
  flow_load<T, false>(a, v, nb, f);
  double jx = 0;
#pragma unroll
  for (int i = 0; i < 19; ++i) jx += (double)q19_e(i, 0) * (double)f[i];
  ux[v] = (float)(jx + 0.5 * (double)a.g);
}

template <class T>
__global__ void dense_diff_c(DiffArgs<T> a, DenseBox b, float* c) {
  using C = typename Stg<T>::C;
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= b.N) return;
  if (!b.node[v]) {
    c[v] = 0.f;
    return;
  }
  int x, y, z;
  dense_xyz(b, v, x, y, z);
  uint32_t nb[7];
  C g[7];
  diff_load<T, D3Q7, false>(a, v, nb, x, g);
  double dev = 0;
#pragma unroll
  for (int i = 0; i < 7; ++i) dev += (double)g[i];
  c[v] = (float)(dev + diff_ref(a, v, x));
}

// the flow's rebased mode: every node's reference moved to its density (even time)
template <class T>
__global__ void dense_flow_rebase(FlowArgs<T> a, DenseBox b) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < b.N && b.node[v]) flow_rebase_node<T>(a, v);
}

// the diffusion's per-window rebase, its initial linear profile (as the
// sparse solver's import of the linear profile) and extrapolated restart
template <class T>
__global__ void dense_diff_rebase(DiffArgs<T> a, DenseBox b) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < b.N && b.node[v]) diff_rebase_node<T>(a, v);
}

template <class T>
__global__ void dense_diff_linear(DiffArgs<T> a, DenseBox b) {
  using S = Stg<T>;
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= b.N || !b.node[v]) return;
  int x, y, z;
  dense_xyz(b, v, x, y, z);
  const double clin = a.cin + (double)a.s * ((double)x + 0.5);
  double ref = clin;
  if constexpr (kRebased<T>) {
    a.cr[v] = (float)ref;
    ref = (double)a.cr[v];
  }
#pragma unroll
  for (int i = 0; i < 7; ++i) S::st(a.q[i] + v, (typename S::C)(D3Q7::w(i) * clin - D3Q7::w(i) * ref), a.up);
}

template <class T>
__global__ void dense_diff_extrapolate(DiffArgs<T> a, DenseBox b, double* prev, const double* dprev, double f) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= b.N || !b.node[v]) return;
  const double dc = f * dprev[v];
  prev[v] += dc;
  if constexpr (kRebased<T>) {
    a.cr[v] = (float)((double)a.cr[v] + dc);
  } else {
    using S = Stg<T>;
#pragma unroll
    for (int i = 0; i < 7; ++i) S::st(a.q[i] + v, S::ld(a.q[i] + v, a.down) + (typename S::C)(D3Q7::w(i) * dc), a.up);
  }
}

// Eq. 12 per node voxel (as the sparse solver's diff_omega)
template <class C>
__global__ void dense_omega(DenseBox b, const float* d_nm, double d_ref, double tau_ref, C* omega, int* bad) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= b.N) return;
  if (!b.node[v]) {
    omega[v] = C(1);
    return;
  }
  const double tau = ((double)d_nm[v] / d_ref) * (tau_ref - 0.5) + 0.5;
  if (!(tau > 0.5)) atomicExch(bad, 1);
  omega[v] = (C)(1.0 / tau);
}

inline unsigned nblocks(uint32_t n) { return (n + 255) / 256; }

// device storage of one dense solve
struct DenseState {
  DenseBox b{};
  uint32_t P = 0;
  DevBuf<uint8_t> pop;  // q arrays of P values each
  DevBuf<float> ref;    // per-voxel reference (rebased storage)
  DevBuf<double> prev, dprev, partials, obs;
  DevBuf<uint8_t> omega;
  double host_obs[5] = {0, 0, 0, 0, 0};
};

template <class T>
FlowArgs<T> dense_flow_args(const DenseState& d, const om_flow_params& p) {
  FlowArgs<T> a{};
  for (int i = 0; i < 19; ++i) a.s[i] = (T*)d.pop.p + (size_t)i * d.P;
  a.P = d.P;
  a.nf = d.b.N;
  a.nx = d.b.nx, a.ny = d.b.ny, a.nz = d.b.nz;
  const double tau = p.tau;
  a.wp = (typename Stg<T>::C)(1.0 / tau);
  a.wm = (typename Stg<T>::C)(8.0 * (2.0 * tau - 1.0) / (8.0 * tau - 1.0));
  a.g = (typename Stg<T>::C)p.body_force;
  a.up = 1;
  a.down = 1;
  a.rr = d.ref.p;
  return a;
}

template <class T>
DiffArgs<T> dense_diff_args(const DenseState& d, const om_diff_params& p) {
  DiffArgs<T> a{};
  for (int i = 0; i < 7; ++i) a.q[i] = (T*)d.pop.p + (size_t)i * d.P;
  a.nf = d.b.N;
  a.omega = (const typename Stg<T>::C*)d.omega.p;
  a.nx = d.b.nx, a.ny = d.b.ny, a.nz = d.b.nz;
  a.s = (typename Stg<T>::C)((p.c_out - p.c_in) / (double)d.b.nx);
  a.up = 1;
  a.down = 1;
  a.cin = p.c_in;
  a.cout = p.c_out;
  a.cr = d.ref.p;
  return a;
}

template <int NV>
om_status finish_observe(DenseState& d, cudaStream_t s) {
  launch_finalize(d.partials.p, kObsBlocks, NV, d.obs.p, s);
  OM_CUDA(cudaGetLastError());
  OM_CUDA(cudaMemcpyAsync(d.host_obs, d.obs.p, NV * sizeof(double), cudaMemcpyDeviceToHost, s));
  OM_CUDA(cudaStreamSynchronize(s));
  return OM_OK;
}

om_status dense_alloc(DenseState& d, const uint8_t* node, const om_domain& dom, int q, int prec, bool ref,
                      bool dprev, cudaStream_t s) {
  const int64_t N = voxels(dom);
  if (19 * ((N + 63) / 64 * 64) > (int64_t)UINT32_MAX)
    return fail(OM_EINVAL, "dense layout: more than 226 M voxels (slot offsets are 32-bit)");
  d.b = DenseBox{dom.nx, dom.ny, dom.nz, (uint32_t)N, node};
  d.P = (uint32_t)((N + 63) / 64 * 64);
  const size_t sz = prec == OM_F64 ? 8 : 4;
  OM_TRY(d.pop.alloc((size_t)q * d.P * sz));
  OM_CUDA(cudaMemsetAsync(d.pop.p, 0, (size_t)q * d.P * sz, s));
  if (ref) {
    OM_TRY(d.ref.alloc(d.P));
    OM_CUDA(cudaMemsetAsync(d.ref.p, 0, sizeof(float) * d.P, s));
  }
  OM_TRY(d.prev.alloc(d.P));
  OM_CUDA(cudaMemsetAsync(d.prev.p, 0, sizeof(double) * d.P, s));
  if (dprev) OM_TRY(d.dprev.alloc(d.P));
  OM_TRY(d.partials.alloc((size_t)kObsBlocks * 5));
  OM_TRY(d.obs.alloc(5));
  return OM_OK;
}

// K steps from an even time (K even), then the flow's per-window rebase in its rebased mode
template <class T>
void dense_flow_window(const DenseState& d, const om_flow_params& p, int64_t K, cudaStream_t s) {
  const FlowArgs<T> a = dense_flow_args<T>(d, p);
  for (int64_t k = 0; k < K; ++k) {
    if (k & 1) dense_flow_sweep<T, true><<<nblocks(d.b.N), 256, 0, s>>>(a, d.b);
    else dense_flow_pair<T><<<nblocks((d.b.N + 1) / 2), 256, 0, s>>>(a, d.b);
  }
  if (kFlowRebased<T>) dense_flow_rebase<T><<<nblocks(d.b.N), 256, 0, s>>>(a, d.b);
}

template <class T>
om_status dense_flow_obs(DenseState& d, const om_flow_params& p, cudaStream_t s) {
  dense_flow_observe<T><<<kObsBlocks, kObsThreads, 0, s>>>(dense_flow_args<T>(d, p), d.b, d.prev.p, d.partials.p);
  return finish_observe<4>(d, s);
}

// om_flow_solve's loop on the dense layout; S the storage format
template <class S>
om_status dense_flow_solve_t(const uint8_t* node, const om_domain& dom, int64_t nf, const om_flow_params& p,
                             double* k_lattice, om_run_info* info, float* ux, double* pair_ms, cudaStream_t s) {
  DenseState d;
  const bool can_rebase = std::is_same_v<S, float>;
  OM_TRY(dense_alloc(d, node, dom, 19, p.precision, can_rebase, false, s));
  if (pair_ms) {  // timing of one even + odd pair (after a warm-up pair) for the layout choice
    cudaEvent_t e0, e1;
    OM_CUDA(cudaEventCreate(&e0));
    OM_CUDA(cudaEventCreate(&e1));
    dense_flow_window<S>(d, p, 2, s);
    OM_CUDA(cudaEventRecord(e0, s));
    dense_flow_window<S>(d, p, 2, s);
    OM_CUDA(cudaEventRecord(e1, s));
    OM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    OM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *pair_ms = ms;
    return OM_OK;
  }
  bool reb = false;
  auto window = [&](int64_t K) {
    if constexpr (std::is_same_v<S, float>) {
      if (reb) return dense_flow_window<Reb<float>>(d, p, K, s);
    }
    dense_flow_window<S>(d, p, K, s);
  };
  auto observe = [&]() -> om_status {
    if constexpr (std::is_same_v<S, float>) {
      if (reb) return dense_flow_obs<Reb<float>>(d, p, s);
    }
    return dense_flow_obs<S>(d, p, s);
  };
  cudaEvent_t e0, e1;
  OM_CUDA(cudaEventCreate(&e0));
  OM_CUDA(cudaEventCreate(&e1));
  OM_TRY(observe());
  OM_CUDA(cudaEventRecord(e0, s));
  int64_t t = 0;
  om_status rc = OM_ENOTCONVERGED;
  double rel = 1.0;
  bool diverged = false;
  const double* o = d.host_obs;
  while (t < p.max_steps) {
    const int64_t k = std::min<int64_t>(p.check_every, p.max_steps - t);
    window(k);
    t += k;
    OM_CUDA(cudaGetLastError());
    OM_TRY(observe());
    if (!std::isfinite(o[0]) || !std::isfinite(o[2])) {
      diverged = true;
      break;
    }
    rel = o[2] > 0.0 ? o[1] / o[2] : 0.0;
    if (rel < p.conv_tol) {
      rc = OM_OK;
      break;
    }
    if constexpr (std::is_same_v<S, float>) {
      if (!reb && rel < kRebaseBelow) {  // the rebased mode for the last decades (om_flow_solve)
        OM_CUDA(cudaMemsetAsync(d.ref.p, 0, sizeof(float) * d.P, s));
        dense_flow_rebase<Reb<float>><<<nblocks(d.b.N), 256, 0, s>>>(dense_flow_args<Reb<float>>(d, p), d.b);
        reb = true;
      }
    }
  }
  OM_CUDA(cudaEventRecord(e1, s));
  OM_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  OM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double nu = (p.tau - 0.5) / 3.0;
  if (k_lattice) *k_lattice = nu * (o[0] / (double)d.b.N) / p.body_force;
  if (info) {
    info->steps = t;
    info->n_nodes = nf;
    info->rel_change = rel;
    info->mass = o[3];
    info->seconds = ms * 1e-3;
    info->mlups = ms > 0 ? (double)nf * (double)t / (ms * 1e-3) / 1e6 : 0.0;
  }
  if (ux) {
    if constexpr (std::is_same_v<S, float>) {
      if (reb) dense_flow_ux<Reb<float>><<<nblocks(d.b.N), 256, 0, s>>>(dense_flow_args<Reb<float>>(d, p), d.b, ux);
      else dense_flow_ux<S><<<nblocks(d.b.N), 256, 0, s>>>(dense_flow_args<S>(d, p), d.b, ux);
    } else {
      dense_flow_ux<S><<<nblocks(d.b.N), 256, 0, s>>>(dense_flow_args<S>(d, p), d.b, ux);
    }
    OM_CUDA(cudaGetLastError());
  }
  if (diverged) set_error("dense flow solve: the populations diverged (non-finite velocity sums)");
  else if (rc != OM_OK) set_error("dense flow solve: step cap reached before convergence");
  return rc;
}

template <class T>
void dense_diff_window(const DenseState& d, const om_diff_params& p, int64_t K, cudaStream_t s) {
  const DiffArgs<T> a = dense_diff_args<T>(d, p);
  for (int64_t k = 0; k < K; ++k) {
    if (k & 1) dense_diff_sweep<T, true><<<nblocks(d.b.N), 256, 0, s>>>(a, d.b);
    else dense_diff_pair<T><<<nblocks((d.b.N + 1) / 2), 256, 0, s>>>(a, d.b);
  }
  if (kRebased<T>) dense_diff_rebase<T><<<nblocks(d.b.N), 256, 0, s>>>(a, d.b);
}

// om_diff_solve's loop on the dense layout (D3Q7)
template <class T>
om_status dense_diff_solve_t(const uint8_t* node, const float* d_nm, const om_domain& dom, int64_t nf,
                             const om_diff_params& p, double* D_lattice, double* DL_sum, om_run_info* info, float* c,
                             double* pair_ms, cudaStream_t s) {
  using C = typename Stg<T>::C;
  DenseState d;
  OM_TRY(dense_alloc(d, node, dom, 7, p.precision, kRebased<T>, p.accel == OM_ACCEL_EXTRAPOLATE, s));
  OM_TRY(d.omega.alloc(sizeof(C) * d.P));
  DevBuf<int> bad;
  OM_TRY(bad.alloc(1));
  OM_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
  dense_omega<C><<<nblocks(d.b.N), 256, 0, s>>>(d.b, d_nm, p.d_ref_nm, p.tau_ref, (C*)d.omega.p, bad.p);
  int hb = 0;
  OM_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  OM_CUDA(cudaStreamSynchronize(s));
  if (hb) return fail(OM_EINVAL, "dense diffusion: a node has a pore size <= 0");
  const DiffArgs<T> a = dense_diff_args<T>(d, p);
  dense_diff_linear<T><<<nblocks(d.b.N), 256, 0, s>>>(a, d.b);
  OM_CUDA(cudaGetLastError());
  if (pair_ms) {
    cudaEvent_t e0, e1;
    OM_CUDA(cudaEventCreate(&e0));
    OM_CUDA(cudaEventCreate(&e1));
    dense_diff_window<T>(d, p, 2, s);
    OM_CUDA(cudaEventRecord(e0, s));
    dense_diff_window<T>(d, p, 2, s);
    OM_CUDA(cudaEventRecord(e1, s));
    OM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    OM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *pair_ms = ms;
    return OM_OK;
  }
  auto observe = [&]() -> om_status {
    dense_diff_observe<T><<<kObsBlocks, kObsThreads, 0, s>>>(a, d.b, d.prev.p, d.partials.p, d.dprev.p);
    return finish_observe<5>(d, s);
  };
  cudaEvent_t e0, e1;
  OM_CUDA(cudaEventCreate(&e0));
  OM_CUDA(cudaEventCreate(&e1));
  const double* o = d.host_obs;
  OM_TRY(observe());
  double sj_prev = o[0];
  OM_CUDA(cudaEventRecord(e0, s));
  int64_t t = 0;
  om_status rc = OM_ENOTCONVERGED;
  double rel = 1.0;
  bool diverged = false;
  ExtrapolationTrack track;
  while (t < p.max_steps) {
    const int64_t k = std::min<int64_t>(p.check_every, p.max_steps - t);
    dense_diff_window<T>(d, p, k, s);
    t += k;
    OM_CUDA(cudaGetLastError());
    OM_TRY(observe());
    if (!std::isfinite(o[0]) || !std::isfinite(o[2])) {
      diverged = true;
      break;
    }
    rel = o[2] > 0.0 ? o[1] / o[2] : 0.0;
    const double relj = o[0] != 0.0 ? std::fabs(o[0] - sj_prev) / std::fabs(o[0]) : 0.0;
    rel = std::max(rel, relj);
    sj_prev = o[0];
    if (rel < p.conv_tol) {
      rc = OM_OK;
      break;
    }
    if (d.dprev.p) {
      const double f = track.observe(o[1]);
      if (f > 0.0)
        dense_diff_extrapolate<T><<<nblocks(d.b.N), 256, 0, s>>>(a, d.b, d.prev.p, d.dprev.p, std::min(f, 1e3));
    }
  }
  OM_CUDA(cudaEventRecord(e1, s));
  OM_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  OM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (D_lattice) *D_lattice = (o[0] / (double)d.b.N) * (double)dom.nx / (p.c_in - p.c_out);
  if (DL_sum) *DL_sum = o[4];
  if (info) {
    info->steps = t;
    info->n_nodes = nf;
    info->rel_change = rel;
    info->mass = o[3];
    info->seconds = ms * 1e-3;
    info->mlups = ms > 0 ? (double)nf * (double)t / (ms * 1e-3) / 1e6 : 0.0;
  }
  if (c) {
    dense_diff_c<T><<<nblocks(d.b.N), 256, 0, s>>>(a, d.b, c);
    OM_CUDA(cudaGetLastError());
  }
  if (diverged) set_error("dense diffusion solve: the populations diverged (non-finite concentration sums)");
  else if (rc != OM_OK) set_error("dense diffusion solve: step cap reached before convergence");
  return rc;
}

}  // namespace

bool dense_flow_supported(const om_flow_params& p) {
  return (p.precision == OM_F64 || p.precision == OM_F32) && p.drive == OM_DRIVE_FORCE;
}
bool dense_diff_supported(const om_diff_params& p) {
  return (p.precision == OM_F64 || p.precision == OM_F32) && p.lattice == 7;
}

om_status dense_flow_solve(const uint8_t* node_dev, const om_domain& dom, int64_t nf, const om_flow_params& p,
                           double* k_lattice, om_run_info* info, float* ux_dev, double* pair_ms, cudaStream_t s) {
  if (!dense_flow_supported(p)) return fail(OM_EINVAL, "dense layout: FP64 or FP32 flow with the body force only");
  if (p.check_every <= 0 || (p.check_every & 1))
    return fail(OM_EINVAL, "dense flow solve: check_every must be a positive even number");
  if (p.precision == OM_F64) return dense_flow_solve_t<double>(node_dev, dom, nf, p, k_lattice, info, ux_dev, pair_ms, s);
  return dense_flow_solve_t<float>(node_dev, dom, nf, p, k_lattice, info, ux_dev, pair_ms, s);
}

om_status dense_diff_solve(const uint8_t* node_dev, const float* d_nm_dev, const om_domain& dom, int64_t nf,
                           const om_diff_params& p, double* D_lattice, double* DL_sum, om_run_info* info, float* c_dev,
                           double* pair_ms, cudaStream_t s) {
  if (!dense_diff_supported(p)) return fail(OM_EINVAL, "dense layout: FP64 or FP32 D3Q7 diffusion only");
  if (p.check_every <= 0 || (p.check_every & 1))
    return fail(OM_EINVAL, "dense diffusion solve: check_every must be a positive even number");
  if (p.precision == OM_F64)
    return dense_diff_solve_t<double>(node_dev, d_nm_dev, dom, nf, p, D_lattice, DL_sum, info, c_dev, pair_ms, s);
  return dense_diff_solve_t<float>(node_dev, d_nm_dev, dom, nf, p, D_lattice, DL_sum, info, c_dev, pair_ms, s);
}

}  // namespace om
