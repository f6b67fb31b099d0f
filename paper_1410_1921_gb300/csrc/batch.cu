// batch.cu -- many reconstructed structures of uneven size solved together.
//
// All structures of a batch share one population arena per model: structure
// k owns the global node numbers [off_k, off_k + nf_k), and its column map is
// rebased so neighbour lookups return global numbers directly.  A work list of
// 256-node tiles (structure, first local node) drives persistent kernels: a
// fixed grid of CTAs strides over the list, so one launch advances every
// active structure by one LB step whatever their sizes, and a converged
// structure simply leaves the list.  A check window of K steps is captured
// once into a CUDA graph and replayed; the work list and its length live in
// device memory, so retiring structures never invalidates the graph.
//
// Per-structure observables come from per-tile FP64 partial sums reduced in
// tile order (deterministic).  Launch shapes (residency cap, CTAs per SM) are
// picked per parity by timing them on the batch itself.
#include <algorithm>
#include <array>
#include <cstddef>
#include <cmath>
#include <vector>

#include "diff_core.cuh"
#include "flow_core.cuh"

namespace om {

struct BatchItem {
  const uint4* col;       // rebased column map (global node numbers)
  const uint32_t* coord;  // structure-local packed coordinates
  uint32_t off, nf;
  int nx, ny, nz, W;
  double slope;  // diffusion: (c_out - c_in) / nx
};

constexpr int kTile = 256;

__global__ void rebase_columns(uint4* col, int64_t nw, uint32_t off) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nw; k += (int64_t)gridDim.x * blockDim.x) {
    uint4 w = col[k];
    w.y += off;
    if (w.z != kNoNode) w.z += off;
    if (w.w != kNoNode) w.w += off;
    col[k] = w;
  }
}

// ------------------------------------------------------------------ sweeps
// A sweep launch covers one group of items.  The whole group travels in the
// kernel parameters (the constant bank, like the arguments of the
// single-structure sweeps): its items' geometry and the first tile of each
// item within the group, so a block finds its tile's item by a binary
// search over at most kGroupItems constant-bank entries -- no work-list load
// and no dependent global read before the node's own loads.
constexpr int kGroupItems = 32;

struct GroupItem {
  const uint4* col;       // rebased column map (global node numbers)
  const uint32_t* coord;  // structure-local packed coordinates
  uint32_t off, nf;
  int nx, ny, nz, W;
  double slope;  // diffusion: (c_out - c_in) / nx
};

struct GroupDesc {
  GroupItem it[kGroupItems];
  int tile0[kGroupItems + 1];  // first tile of item k within the group; tile0[n] = tiles
  int n;                       // items
};

// item of tile w of the group (tile0[k] <= w < tile0[k + 1]); warp-uniform
__device__ __forceinline__ int group_item(const GroupDesc& g, int w) {
  int lo = 0, hi = g.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (g.tile0[mid] <= w) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// one step of the nodes of tile w of group g
template <class T, bool ODD>
__device__ __forceinline__ void flow_group_tile(const FlowArgs<T>& a, const GroupDesc& g, int w) {
  const int k = group_item(g, w);
  const GroupItem& it = g.it[k];
  const uint32_t ln = (uint32_t)(w - g.tile0[k]) * kTile + threadIdx.x;
  if (ln >= it.nf) return;
  if (ODD) {
    FlowArgs<T> b = a;
    b.col = it.col;
    b.coord = it.coord;
    b.nx = it.nx;
    b.ny = it.ny;
    b.nz = it.nz;
    b.W = it.W;
    flow_node<T, true>(b, it.off + ln, ln);
  } else {
    flow_node<T, false>(a, it.off + ln, ln);
  }
}

template <class T, bool ODD>
__device__ __forceinline__ void diff_group_tile(const DiffArgs<T>& a, const GroupDesc& g, int w) {
  const int k = group_item(g, w);
  const GroupItem& it = g.it[k];
  const uint32_t ln = (uint32_t)(w - g.tile0[k]) * kTile + threadIdx.x;
  if (ln >= it.nf) return;
  DiffArgs<T> b = a;
  b.nx = it.nx;
  b.s = (typename Stg<T>::C)it.slope;
  if (ODD) {
    b.col = it.col;
    b.coord = it.coord;
    b.ny = it.ny;
    b.nz = it.nz;
    b.W = it.W;
  }
  diff_node<T, ODD>(b, it.off + ln, ln);
}

template <class T, bool ODD, int MINB>
__global__ void __launch_bounds__(kTile, MINB) flow_batch_sweep(FlowArgs<T> a, const __grid_constant__ GroupDesc g) {
  const int nw = g.tile0[g.n];
  for (int w = blockIdx.x; w < nw; w += gridDim.x) flow_group_tile<T, ODD>(a, g, w);
}

template <class T, bool ODD, int MINB>
__global__ void __launch_bounds__(kTile, MINB) diff_batch_sweep(DiffArgs<T> a, const __grid_constant__ GroupDesc g) {
  const int nw = g.tile0[g.n];
  for (int w = blockIdx.x; w < nw; w += gridDim.x) diff_group_tile<T, ODD>(a, g, w);
}

// ------------------------------------------------------------------ persistent windows
// A window of K steps of one group in a single cooperative launch (all its
// blocks co-resident): the blocks stride over the group's tiles for a step,
// meet at a grid barrier, and go on to the next step.  The barrier waits are
// bounded: a block that waits more than `limit` polls (about 100 ns each)
// records OM_ETIMEOUT in the barrier's status word and returns, and every
// other block leaves at its next wait once it sees the status, so the
// launch always ends and the host reads the status instead of a hang.
struct GridBar {
  unsigned count;  // arrivals at the current barrier
  unsigned gen;    // barriers completed (only ever incremented)
  int status;      // OM_OK, or OM_ETIMEOUT once a wait gave up
  int pad;
};

constexpr unsigned long long kBarrierPolls = 20000000ull;  // ~2 s of polling

// Barrier of `expected` blocks; false when a wait gave up (the caller
// returns).
__device__ __forceinline__ bool grid_barrier(GridBar* bar, unsigned expected, unsigned long long limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int good = 1;
    volatile unsigned* gen = &bar->gen;
    volatile int* status = &bar->status;
    const unsigned g0 = *gen;
    __threadfence();  // this block's stores of the step before its arrival
    if (atomicAdd(&bar->count, 1u) == expected - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      unsigned long long polls = 0;
      while (*gen == g0) {
        if (*status != OM_OK || ++polls > limit) {
          atomicCAS(&bar->status, OM_OK, OM_ETIMEOUT);
          good = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();  // the other blocks' stores before this block reads
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

template <class T, int MINB>
__global__ void __launch_bounds__(kTile, MINB) flow_batch_window(FlowArgs<T> a, const __grid_constant__ GroupDesc g,
                                                                 int odd0, int K, GridBar* bar) {
  const int nw = g.tile0[g.n];
  for (int k = 0; k < K; ++k) {
    if ((odd0 + k) & 1) {
      for (int w = blockIdx.x; w < nw; w += gridDim.x) flow_group_tile<T, true>(a, g, w);
    } else {
      for (int w = blockIdx.x; w < nw; w += gridDim.x) flow_group_tile<T, false>(a, g, w);
    }
    if (k + 1 < K && !grid_barrier(bar, gridDim.x, kBarrierPolls)) return;
  }
}

template <class T, int MINB>
__global__ void __launch_bounds__(kTile, MINB) diff_batch_window(DiffArgs<T> a, const __grid_constant__ GroupDesc g,
                                                                 int odd0, int K, GridBar* bar) {
  const int nw = g.tile0[g.n];
  for (int k = 0; k < K; ++k) {
    if ((odd0 + k) & 1) {
      for (int w = blockIdx.x; w < nw; w += gridDim.x) diff_group_tile<T, true>(a, g, w);
    } else {
      for (int w = blockIdx.x; w < nw; w += gridDim.x) diff_group_tile<T, false>(a, g, w);
    }
    if (k + 1 < K && !grid_barrier(bar, gridDim.x, kBarrierPolls)) return;
  }
}

// Self-test of the bounded barrier: `rounds` barriers among the launch's
// blocks, expecting `extra` more blocks than the launch has (extra > 0: a
// barrier that can never complete, so every wait runs out).
__global__ void barrier_selftest(GridBar* bar, int rounds, unsigned extra, unsigned long long limit) {
  for (int r = 0; r < rounds; ++r)
    if (!grid_barrier(bar, gridDim.x + extra, limit)) return;
}

// An item large enough to fill the GPU alone (a "solo" group) runs the
// single-structure sweep body: its geometry is in the scalar arguments, its
// nodes are [off, off + nf) of the arena, one thread per node.
template <class T, bool ODD, int MINB>
__global__ void __launch_bounds__(kTile, MINB) flow_solo_sweep(FlowArgs<T> a, uint32_t off) {
  const uint32_t ln = blockIdx.x * blockDim.x + threadIdx.x;
  if (ln >= a.nf) return;
  flow_node<T, ODD>(a, off + ln, ln);
}

// The same item with the single-structure solver's fastest forms (launch
// variant 2): odd steps on a resident grid whose threads stride over the
// item's nodes, the next node's coordinates loaded ahead; even steps two
// consecutive nodes per thread with 8-byte loads and stores (pairs from the
// first even node number; a node before it is a single -- never the case
// for a solo item, whose arena offset is a multiple of 32).
template <class T>
__global__ void __launch_bounds__(kTile) flow_solo_strided(FlowArgs<T> a, uint32_t off) {
  const uint32_t stride = gridDim.x * blockDim.x;
  uint32_t ln = blockIdx.x * blockDim.x + threadIdx.x;
  if (ln >= a.nf) return;
  uint32_t c = __ldg(a.coord + ln);
  for (;;) {
    const uint64_t nn = (uint64_t)ln + stride;
    const bool more = nn < a.nf;
    const uint32_t cn = more ? __ldg(a.coord + nn) : 0u;
    flow_node_at<T, true>(a, off + ln, c);
    if (!more) break;
    ln = (uint32_t)nn;
    c = cn;
  }
}

template <class T>
__global__ void __launch_bounds__(kTile) flow_solo_pair(FlowArgs<T> a, uint32_t off) {
  const uint32_t head = off & 1u;
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (head && t == 0) flow_node_at<T, false>(a, off, 0u);
  const uint32_t ln = head + 2 * t;
  if (ln >= a.nf) return;
  if (ln + 1 == a.nf) flow_node_at<T, false>(a, off + ln, 0u);
  else flow_pair_even<T>(a, off + ln);
}

template <class T, bool ODD, int MINB>
__global__ void __launch_bounds__(kTile, MINB) diff_solo_sweep(DiffArgs<T> a, uint32_t off) {
  const uint32_t ln = blockIdx.x * blockDim.x + threadIdx.x;
  if (ln >= a.nf) return;
  diff_node<T, ODD>(a, off + ln, ln);
}

// ------------------------------------------------------------------ observables
// partials[w][NV] for every tile w of the work list
template <class T, bool ODD>
__global__ void __launch_bounds__(kTile) flow_batch_observe(FlowArgs<T> a, const BatchItem* items, const uint2* work,
                                                            const int* nwork, double* prev, double* partials) {
  using C = typename Stg<T>::C;
  const int nw = *nwork;
  for (int w = blockIdx.x; w < nw; w += gridDim.x) {
    const uint2 t = work[w];
    const BatchItem& it = items[t.x];
    const uint32_t ln = t.y + threadIdx.x;
    double acc[4] = {0, 0, 0, 0};
    if (ln < it.nf) {
      FlowArgs<T> b = a;
      b.col = it.col;
      b.coord = it.coord;
      b.nx = it.nx;
      b.ny = it.ny;
      b.nz = it.nz;
      b.W = it.W;
      const uint32_t n = it.off + ln;
      uint32_t nb[19];
      if (ODD) flow_neighbours(b, b.coord[ln], nb);
      C f[19];
      flow_load<T, ODD>(b, n, nb, f);
      double rho = 0, jx = 0;
#pragma unroll
      for (int i = 0; i < 19; ++i) {
        rho += (double)f[i];
        jx += (double)q19_e(i, 0) * (double)f[i];
      }
      const double ux = jx + 0.5 * (double)a.g;
      acc[0] = ux;
      acc[1] = fabs(ux - prev[n]);
      acc[2] = fabs(ux);
      acc[3] = rho + flow_ref(a, n);
      prev[n] = ux;
    }
    block_reduce_write<4>(acc, partials + (int64_t)w * 4);
  }
}

template <class T, bool ODD>
__global__ void __launch_bounds__(kTile) diff_batch_observe(DiffArgs<T> a, const BatchItem* items, const uint2* work,
                                                            const int* nwork, double* prev, double* partials,
                                                            double* dprev) {
  using C = typename Stg<T>::C;
  const int nw = *nwork;
  for (int w = blockIdx.x; w < nw; w += gridDim.x) {
    const uint2 t = work[w];
    const BatchItem& it = items[t.x];
    const uint32_t ln = t.y + threadIdx.x;
    double acc[5] = {0, 0, 0, 0, 0};
    if (ln < it.nf) {
      DiffArgs<T> b = a;
      b.col = it.col;
      b.coord = it.coord;
      b.nx = it.nx;
      b.ny = it.ny;
      b.nz = it.nz;
      b.W = it.W;
      b.s = (typename Stg<T>::C)it.slope;
      const uint32_t n = it.off + ln;
      uint32_t nb[7];
      int x, y, z;
      unpack_xyz(b.coord[ln], x, y, z);
      if (ODD) diff_neighbours(b, b.coord[ln], nb, x);
      C g[7];
      diff_load<T, D3Q7, ODD>(b, n, nb, x, g);
      double dev = 0;
#pragma unroll
      for (int i = 0; i < 7; ++i) dev += (double)g[i];
      const double c = dev + diff_ref(b, n, x);
      const double om = (double)b.omega[n];
      acc[0] = (1.0 - 0.5 * om) * ((double)g[1] - (double)g[2]);
      acc[1] = fabs(c - prev[n]);
      acc[2] = fabs(c);
      acc[3] = c;
      acc[4] = 0.25 * (1.0 / om - 0.5);
      if (dprev) dprev[n] = c - prev[n];
      prev[n] = c;
    }
    block_reduce_write<5>(acc, partials + (int64_t)w * 5);
  }
}

// Extrapolated restart of one item (om_diff_params.accel; see
// diff_extrapolate in diff.cu): nodes [off, off + nf) move by f dC.
template <class T>
__global__ void diff_batch_extrapolate(DiffArgs<T> a, uint32_t off, uint32_t nf, double* prev, const double* dprev,
                                       double f) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf) return;
  const uint32_t n = off + k;
  const double dc = f * dprev[n];
  prev[n] += dc;
  if constexpr (kRebased<T>) {
    a.cr[n] = (float)((double)a.cr[n] + dc);
  } else {
    using S = Stg<T>;
#pragma unroll
    for (int i = 0; i < 7; ++i) S::st(a.q[i] + n, S::ld(a.q[i] + n, a.down) + (typename S::C)(q7_w(i) * dc), a.up);
  }
}

// out[k][NV] = sum of partials over the tiles [range[k].x, range[k].y), in order
template <int NV>
__global__ void batch_finalize(const double* partials, const int2* range, double* out) {
  const int2 r = range[blockIdx.x];
  __shared__ double sm[256];
  for (int k = 0; k < NV; ++k) {
    double acc = 0.0;
    for (int w = r.x + threadIdx.x; w < r.y; w += blockDim.x) acc += partials[(int64_t)w * NV + k];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[(int64_t)blockIdx.x * NV + k] = sm[0];
    __syncthreads();
  }
}

// ------------------------------------------------------------------ set-up and exchange
template <class C>
__global__ void batch_omega(const int64_t* vox, const float* d_nm, uint32_t nf, double d_ref, double tau_ref, C* omega,
                            int* bad) {
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nf) return;
  const double tau = ((double)d_nm[vox[n]] / d_ref) * (tau_ref - 0.5) + 0.5;  // Eq. 12
  if (!(tau > 0.5)) atomicExch(bad, 1);
  omega[n] = (C)(1.0 / tau);
}

// an item's populations (dense, FP64) and/or its field (dense, float: the
// flow's u_x = sum_i e_ix f_i + g/2, as om_flow_get_velocity; the
// diffusion's C = sum_i g_i, as om_diff_get_fields)
template <class T, bool ODD>
__global__ void flow_batch_export(FlowArgs<T> a, uint32_t off, const int64_t* vox, int64_t N, double* out,
                                  float* ux) {
  using C = typename Stg<T>::C;
  const uint32_t ln = blockIdx.x * blockDim.x + threadIdx.x;
  if (ln >= a.nf) return;
  uint32_t nb[19];
  if (ODD) flow_neighbours(a, a.coord[ln], nb);
  C f[19];
  flow_load<T, ODD>(a, off + ln, nb, f);
  const int64_t v = vox[ln];
  if (out) {
    const double r1 = 1.0 + flow_ref(a, off + ln);
#pragma unroll
    for (int i = 0; i < 19; ++i) out[i * N + v] = (double)f[i] + q19_w(i) * r1;
  }
  if (ux) {
    double jx = 0.0;
#pragma unroll
    for (int i = 0; i < 19; ++i) jx += (double)q19_e(i, 0) * (double)f[i];
    ux[v] = (float)(jx + 0.5 * (double)a.g);
  }
}

template <class T, bool ODD>
__global__ void diff_batch_export(DiffArgs<T> a, uint32_t off, const int64_t* vox, int64_t N, double* out,
                                  float* c) {
  using C = typename Stg<T>::C;
  const uint32_t ln = blockIdx.x * blockDim.x + threadIdx.x;
  if (ln >= a.nf) return;
  uint32_t nb[7];
  int x, y, z;
  unpack_xyz(a.coord[ln], x, y, z);
  if (ODD) diff_neighbours(a, a.coord[ln], nb, x);
  C g[7];
  diff_load<T, D3Q7, ODD>(a, off + ln, nb, x, g);
  const int64_t v = vox[ln];
  const double cref = diff_ref(a, off + ln, x);
  double dev = 0.0;
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    dev += (double)g[i];
    if (out) out[i * N + v] = (double)g[i] + q7_w(i) * cref;
  }
  if (c) c[v] = (float)(dev + cref);
}

template <class T>
__global__ void flow_batch_import(FlowArgs<T> a, uint32_t off, const int64_t* vox, int64_t N, const double* in) {
  const uint32_t ln = blockIdx.x * blockDim.x + threadIdx.x;
  if (ln >= a.nf) return;
  const int64_t v = vox[ln];
  if constexpr (kFlowRebased<T>) a.rr[off + ln] = 0.f;
#pragma unroll
  for (int i = 0; i < 19; ++i)
    Stg<T>::st(a.s[i] + off + ln, (typename Stg<T>::C)(in[i * N + v] - q19_w(i)), a.up);
}

template <class T>
__global__ void diff_batch_import(DiffArgs<T> a, uint32_t off, const int64_t* vox, int64_t N, const double* in) {
  const uint32_t ln = blockIdx.x * blockDim.x + threadIdx.x;
  if (ln >= a.nf) return;
  const int64_t v = vox[ln];
  int x, y, z;
  unpack_xyz(a.coord[ln], x, y, z);
  double cref = a.cin + (double)a.s * ((double)x + 0.5);
  if constexpr (kRebased<T>) {
    cref = 0.0;
    for (int i = 0; i < 7; ++i) cref += in[i * N + v];
    a.cr[off + ln] = (float)cref;
    cref = (double)a.cr[off + ln];
  }
#pragma unroll
  for (int i = 0; i < 7; ++i)
    Stg<T>::st(a.q[i] + off + ln, (typename Stg<T>::C)(in[i * N + v] - q7_w(i) * cref), a.up);
}

// warm start of one structure: flow f = f_eq(1, (scale * field, 0, 0));
// diffusion g = a_i C with C = field (+ C_lin(x) when from_linear)
template <class T>
__global__ void flow_batch_init(FlowArgs<T> a, uint32_t off, const int64_t* vox, const float* field, int64_t stride,
                                double scale) {
  const uint32_t ln = blockIdx.x * blockDim.x + threadIdx.x;
  if (ln >= a.nf) return;
  const double u = warm_velocity(scale * (double)field[vox[ln] * stride]);
  if constexpr (kFlowRebased<T>) a.rr[off + ln] = 0.f;
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const double eu = (double)q19_e(i, 0) * u;
    Stg<T>::st(a.s[i] + off + ln, (typename Stg<T>::C)(q19_w(i) * (3.0 * eu + 4.5 * eu * eu - 1.5 * u * u)), a.up);
  }
}

template <class T>
__global__ void diff_batch_init(DiffArgs<T> a, uint32_t off, const int64_t* vox, const float* field, int64_t stride,
                                int from_linear) {
  const uint32_t ln = blockIdx.x * blockDim.x + threadIdx.x;
  if (ln >= a.nf) return;
  int x, y, z;
  unpack_xyz(a.coord[ln], x, y, z);
  const double clin = a.cin + (double)a.s * ((double)x + 0.5);
  const double cv =
      warm_concentration((double)field[vox[ln] * stride] + (from_linear ? clin : 0.0), clin, a.cin, a.cout);
  double dc = cv - clin;
  if constexpr (kRebased<T>) {
    a.cr[off + ln] = (float)cv;
    dc = 0.0;
  }
#pragma unroll
  for (int i = 0; i < 7; ++i) Stg<T>::st(a.q[i] + off + ln, (typename Stg<T>::C)(q7_w(i) * dc), a.up);
}

// 16-bit diffusion: reference of every node of every structure set to C_lin(x)
__global__ void batch_cr_linear(const BatchItem* items, const uint2* work, const int* nwork, double cin, float* cr) {
  const int nw = *nwork;
  for (int w = blockIdx.x; w < nw; w += gridDim.x) {
    const uint2 t = work[w];
    const BatchItem& it = items[t.x];
    const uint32_t ln = t.y + threadIdx.x;
    if (ln >= it.nf) continue;
    int x, y, z;
    unpack_xyz(it.coord[ln], x, y, z);
    cr[it.off + ln] = (float)(cin + it.slope * ((double)x + 0.5));
  }
}

template <class T>
__global__ void batch_rebase(DiffArgs<T> a) {
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < a.nf) diff_rebase_node<T>(a, n);
}

// the flow's rebased mode, per structure: every node of a group's items
// (once per check window), or of one item (when it enters the mode)
template <class T>
__global__ void batch_flow_rebase_group(FlowArgs<T> a, const __grid_constant__ GroupDesc g) {
  const int nw = g.tile0[g.n];
  for (int w = blockIdx.x; w < nw; w += gridDim.x) {
    const int k = group_item(g, w);
    const uint32_t ln = (uint32_t)(w - g.tile0[k]) * kTile + threadIdx.x;
    if (ln < g.it[k].nf) flow_rebase_node<T>(a, g.it[k].off + ln);
  }
}

template <class T>
__global__ void batch_flow_rebase_range(FlowArgs<T> a, uint32_t off, uint32_t nf) {
  const uint32_t ln = blockIdx.x * blockDim.x + threadIdx.x;
  if (ln < nf) flow_rebase_node<T>(a, off + ln);
}

}  // namespace om

using namespace om;

namespace {

size_t stg_bytes(int prec) { return prec == OM_F64 ? 8 : (prec == OM_F32 ? 4 : 2); }

// One model's state inside a batch.
struct Model {
  bool on = false;
  int prec = OM_F32;
  int q = 0;             // populations per node
  void* pop = nullptr;   // arena [q][pitch]
  void* omega = nullptr; // diffusion only, compute type, [pitch]
  float* cr = nullptr;   // rebased storage: per-node reference concentration (diffusion) or density (flow)
  // flow with cr: the items in the rebased mode (their sweeps take Reb<S>;
  // every other item keeps cr = 0 on its nodes and takes the plain S sweeps)
  std::vector<char> reb;
  double* prev = nullptr;
  double* dprev = nullptr;  // diffusion with OM_ACCEL_EXTRAPOLATE: each node's change over the last window
  int64_t t = 0;
  double up = 1.0;
  int var[2] = {0, 0};   // launch variant per parity
  int grid[2] = {152, 152};
  // check windows: 0 = replay of the captured per-step launches, 1 = one
  // persistent cooperative launch per group (grid-barrier steps); -1 = not
  // chosen yet (the first windows time both)
  int mode = -1;
  float trial_ms[2] = {-1.f, -1.f};  // time of the window timed in each mode
  cudaGraphExec_t exec = nullptr;
  int graph_k = 0;
  int graph_layout = -1;  // work-list layout the graph was captured for
};

}  // namespace

struct om_batch {
  int n = 0;
  std::vector<om_domain> dom;
  std::vector<om_nodeset*> ns;
  std::vector<BatchItem> items_h;
  BatchItem* items = nullptr;
  uint32_t total = 0;   // nodes
  int64_t pitch = 0;
  uint2* work = nullptr;      // device work list
  int* nwork = nullptr;       // device count
  uint2* work_h = nullptr;    // pinned staging
  int2* range = nullptr;      // device per-active-item tile ranges
  int2* range_h = nullptr;    // pinned
  int* nwork_h = nullptr;     // pinned
  // the work list in groups of items whose populations fit in L2 together
  // (at most kGroupItems each): group g holds the tiles work[gstart[g] ..
  // gstart[g] + gcnt_h[g]); its sweeps take the descriptor gdesc[g]
  int* gcnt_h = nullptr;      // pinned, [n]
  std::vector<int> gstart;
  std::vector<GroupDesc> gdesc;
  std::vector<int> gsolo;     // item of a solo group (one large item), else -1
  std::vector<char> greb;     // flow: the group's items are in the rebased mode
  // items of >= kSoloNodes nodes: their arena offset is a multiple of 32, and
  // they keep a copy of their column map in local node numbers (col_local)
  // for the single-structure sweeps (flow launch variant 3), whose tuned
  // variants svar[item][2 * rebased + odd] are picked at creation
  std::vector<uint4*> col_local;
  std::vector<std::array<int, 4>> svar;
  std::vector<std::array<int, 2>> dvar;  // the same for the diffusion (diffusion launch variant 3)
  int ngroups = 0;
  int layout = 0;             // bumped whenever the work list is rebuilt
  int layout_model = -1;      // the model whose footprint sized the groups
  int max_tiles = 0;
  double* partials = nullptr; // [max_tiles][5]
  double* obs = nullptr;      // [n][5]
  double* obs_h = nullptr;    // pinned [n][5]
  om_flow_params fp{};
  om_diff_params dp{};
  Model m[2];
  cudaStream_t cap = nullptr;  // capture stream
  int sms = 152;
  GridBar* bar = nullptr;      // grid barrier of the persistent windows
  int* bar_h = nullptr;        // pinned copy of its status
};

namespace {

// L2 budget of a group: the populations (and per-node fields) of the items
// of one group stay on chip across the steps of a check window, as a single
// small structure's do when it is solved alone.
constexpr double kGroupBytes = 80e6;

// bytes per node a sweep of the model touches (populations, omega for the
// diffusion, the reference of rebased storage, packed coordinates)
double node_bytes(const om_batch* b, int model) {
  const Model& m = b->m[model];
  double per = (double)m.q * stg_bytes(m.prec) + 4.0 + (m.cr ? 4.0 : 0.0);
  if (model == 1) per += m.prec == OM_F64 ? 8.0 : 4.0;
  return per;
}

// Items with at least this many nodes fill the GPU alone: they form a group
// of their own and run the single-structure sweep body.
constexpr uint32_t kSoloNodes = 1u << 19;

// Work list of all tiles of the items flagged active, ordered by group
// (consecutive small items packed while their footprint fits kGroupBytes;
// every large item alone); ranges per active item; the layout counter
// moves on.
int build_work(om_batch* b, const std::vector<int>& active, int model) {
  const double per = node_bytes(b, model);
  int w = 0;
  b->gstart.clear();
  b->ngroups = 0;
  double fill = 0.0;
  b->gdesc.clear();
  b->gsolo.clear();
  b->greb.clear();
  int in_group = 0;
  // the flow's items in the plain mode first, then those in the rebased mode
  const std::vector<char>& reb = b->m[0].reb;
  const bool two = model == 0 && !reb.empty();
  for (int pass = 0; pass < (two ? 2 : 1); ++pass)
  for (size_t a = 0; a < active.size(); ++a) {
    const int k = active[a];
    const char mode = two ? reb[k] : 0;
    if (mode != pass) continue;
    const BatchItem& bi = b->items_h[k];
    const double bytes = per * (double)bi.nf;
    const bool solo = bi.nf >= kSoloNodes;
    if (b->ngroups == 0 || solo || b->gsolo.back() >= 0 || in_group == kGroupItems || b->greb.back() != mode ||
        (fill > 0.0 && fill + bytes > kGroupBytes)) {
      b->gstart.push_back(w);
      b->gcnt_h[b->ngroups] = 0;
      b->gdesc.push_back(GroupDesc{});
      b->gsolo.push_back(solo ? k : -1);
      b->greb.push_back(mode);
      ++b->ngroups;
      fill = 0.0;
      in_group = 0;
    }
    fill += bytes;
    GroupDesc& gd = b->gdesc.back();
    gd.it[in_group] = GroupItem{bi.col, bi.coord, bi.off, bi.nf, bi.nx, bi.ny, bi.nz, bi.W, bi.slope};
    gd.tile0[in_group] = w - b->gstart.back();
    gd.n = in_group + 1;
    const int w0 = w;
    for (uint32_t s = 0; s < bi.nf; s += kTile) b->work_h[w++] = make_uint2((unsigned)k, s);
    ++in_group;
    b->gcnt_h[b->ngroups - 1] += w - w0;
    gd.tile0[in_group] = w - b->gstart.back();
    b->range_h[a] = make_int2(w0, w);
  }
  *b->nwork_h = w;
  ++b->layout;
  b->layout_model = model;
  return w;
}

om_status upload_work(om_batch* b, int nw, int nact, cudaStream_t s) {
  if (nw > 0) OM_CUDA(cudaMemcpyAsync(b->work, b->work_h, sizeof(uint2) * nw, cudaMemcpyHostToDevice, s));
  if (nact > 0) OM_CUDA(cudaMemcpyAsync(b->range, b->range_h, sizeof(int2) * nact, cudaMemcpyHostToDevice, s));
  OM_CUDA(cudaMemcpyAsync(b->nwork, b->nwork_h, sizeof(int), cudaMemcpyHostToDevice, s));
  return OM_OK;
}

template <class T>
FlowArgs<T> bflow_args(const om_batch* b) {
  FlowArgs<T> a{};
  const Model& m = b->m[0];
  for (int i = 0; i < 19; ++i) a.s[i] = (T*)m.pop + (size_t)i * b->pitch;
  a.P = (uint32_t)b->pitch;
  a.nf = b->total;
  const double tau = b->fp.tau;
  a.wp = (typename Stg<T>::C)(1.0 / tau);
  a.wm = (typename Stg<T>::C)(8.0 * (2.0 * tau - 1.0) / (8.0 * tau - 1.0));
  a.g = (typename Stg<T>::C)b->fp.body_force;
  a.up = (typename Stg<T>::C)m.up;
  a.down = (typename Stg<T>::C)(1.0 / m.up);
  a.rr = m.cr;
  return a;
}

template <class T>
DiffArgs<T> bdiff_args(const om_batch* b) {
  DiffArgs<T> a{};
  const Model& m = b->m[1];
  for (int i = 0; i < 7; ++i) a.q[i] = (T*)m.pop + (size_t)i * b->pitch;
  a.nf = b->total;
  a.omega = (const typename Stg<T>::C*)m.omega;
  a.up = (typename Stg<T>::C)m.up;
  a.down = (typename Stg<T>::C)(1.0 / m.up);
  a.cin = b->dp.c_in;
  a.cout = b->dp.c_out;
  a.cr = m.cr;
  return a;
}

// the single-structure solver's view of solo item k: its slice of the arena
// (pointers shifted by its offset, the slot pitch the arena's), its local
// column map, coordinates and neighbour records
template <class T>
FlowArgs<T> solo_args(const om_batch* b, int k) {
  FlowArgs<T> a = bflow_args<T>(b);
  const BatchItem& it = b->items_h[k];
  const om_nodeset* ns = b->ns[k];
  for (int i = 0; i < 19; ++i) a.s[i] += it.off;
  a.nf = it.nf;
  a.col = b->col_local[k];
  a.coord = it.coord;
  a.rec7 = ns->rec7;
  a.rec19 = ns->rec19;
  a.slow = ns->slow;
  a.nslow = (uint32_t)ns->n_slow;
  if (a.rr) a.rr += it.off;
  a.nx = it.nx;
  a.ny = it.ny;
  a.nz = it.nz;
  a.W = it.W;
  return a;
}

template <class T, int MINB>
void launch_flow_t(const om_batch* b, bool odd, int grid, int g, int form, cudaStream_t s) {
  FlowArgs<T> a = bflow_args<T>(b);
  const int solo = b->gsolo[g];
  if (solo >= 0 && form == 3 && b->col_local[solo]) {
    flow_sweep_variant<T>(odd, b->svar[solo][2 * (int)kFlowRebased<T> + (int)odd], solo_args<T>(b, solo), s);
    return;
  }
  const bool fast = form >= 2;
  if (solo >= 0) {
    const BatchItem& it = b->items_h[solo];
    a.nf = it.nf;
    a.col = it.col;
    a.coord = it.coord;
    a.nx = it.nx;
    a.ny = it.ny;
    a.nz = it.nz;
    a.W = it.W;
    const unsigned nb = (it.nf + kTile - 1) / kTile;
    if (fast) {
      if (odd) {
        flow_solo_strided<T><<<(unsigned)std::max(1, std::min<int>(grid, (int)nb)), kTile, 0, s>>>(a, it.off);
      } else {
        const uint32_t pairs = (it.nf - (it.off & 1u) + 1) / 2;
        flow_solo_pair<T><<<std::max(1u, (pairs + kTile - 1) / kTile), kTile, 0, s>>>(a, it.off);
      }
      return;
    }
    if (odd) flow_solo_sweep<T, true, MINB><<<nb, kTile, 0, s>>>(a, it.off);
    else flow_solo_sweep<T, false, MINB><<<nb, kTile, 0, s>>>(a, it.off);
    return;
  }
  if (odd) flow_batch_sweep<T, true, MINB><<<grid, kTile, 0, s>>>(a, b->gdesc[g]);
  else flow_batch_sweep<T, false, MINB><<<grid, kTile, 0, s>>>(a, b->gdesc[g]);
}

// the flow's sweeps of group g: rebased storage T = Reb<S> only for a group
// in the rebased mode, the plain S sweeps (cr = 0 on its nodes) otherwise
template <class T, int MINB>
void launch_flow(const om_batch* b, bool odd, int grid, int g, int form, cudaStream_t s) {
  if constexpr (kFlowRebased<T>) {
    if (!b->greb[g]) return launch_flow_t<typename T::base, MINB>(b, odd, grid, g, form, s);
  }
  launch_flow_t<T, MINB>(b, odd, grid, g, form, s);
}

// the single-structure solver's view of solo item k (as solo_args)
template <class T>
DiffArgs<T> solo_dargs(const om_batch* b, int k) {
  DiffArgs<T> a = bdiff_args<T>(b);
  const BatchItem& it = b->items_h[k];
  const om_nodeset* ns = b->ns[k];
  for (int i = 0; i < 7; ++i) a.q[i] += it.off;
  a.omega += it.off;
  if (a.cr) a.cr += it.off;
  a.nf = it.nf;
  a.col = b->col_local[k];
  a.coord = it.coord;
  a.rec7 = ns->rec7;
  a.rec19 = ns->rec19;
  a.slow = ns->slow;
  a.nslow = (uint32_t)ns->n_slow;
  a.nx = it.nx;
  a.ny = it.ny;
  a.nz = it.nz;
  a.W = it.W;
  a.s = (typename Stg<T>::C)it.slope;
  return a;
}

template <class T, int MINB>
void launch_diff(const om_batch* b, bool odd, int grid, int g, int form, cudaStream_t s) {
  DiffArgs<T> a = bdiff_args<T>(b);
  const int solo = b->gsolo[g];
  // (the diffusion is never stored as Reb<S>: the batch's dispatch
  // instantiates that type for both models, only the flow runs it)
  if constexpr (!kFlowRebased<T>) {
    if (solo >= 0 && form == 3 && b->col_local[solo]) {
      diff_sweep_variant<T>(odd, b->dvar[solo][(int)odd], solo_dargs<T>(b, solo), s);
      return;
    }
  }
  if (solo >= 0) {
    const BatchItem& it = b->items_h[solo];
    a.nf = it.nf;
    a.col = it.col;
    a.coord = it.coord;
    a.nx = it.nx;
    a.ny = it.ny;
    a.nz = it.nz;
    a.W = it.W;
    a.s = (typename Stg<T>::C)it.slope;
    const unsigned nb = (it.nf + kTile - 1) / kTile;
    if (odd) diff_solo_sweep<T, true, MINB><<<nb, kTile, 0, s>>>(a, it.off);
    else diff_solo_sweep<T, false, MINB><<<nb, kTile, 0, s>>>(a, it.off);
    return;
  }
  if (odd) diff_batch_sweep<T, true, MINB><<<grid, kTile, 0, s>>>(a, b->gdesc[g]);
  else diff_batch_sweep<T, false, MINB><<<grid, kTile, 0, s>>>(a, b->gdesc[g]);
}

// variant 0: no residency hint; variant 1: capped for 4 (flow; 3 in FP64) / 8
// (diffusion) CTAs per SM; variant 2 (flow): as 1, with the solo groups in
// the single-structure solver's fastest forms (flow_solo_strided / _pair);
// variant 3 (flow): as 1, with each solo group in the single-structure
// solver's own sweeps, the variants tuned for its size
// one step of group g
template <class T>
void launch_step(const om_batch* b, int model, bool odd, int variant, int grid, int g, cudaStream_t s) {
  if (model == 0) {
    if (variant == 0) launch_flow<T, 0>(b, odd, grid, g, 0, s);
    else launch_flow<T, (sizeof(T) == 8 ? 3 : 4)>(b, odd, grid, g, variant, s);
  } else {
    if (variant == 0) launch_diff<T, 0>(b, odd, grid, g, 0, s);
    else launch_diff<T, 8>(b, odd, grid, g, variant, s);
  }
}

// n steps of every item, group after group (each group's n steps run while
// its populations sit in L2); launches onto s in that order
template <class T>
void launch_steps_grouped(const om_batch* b, int model, int64_t t0, int64_t n, cudaStream_t s) {
  const Model& m = b->m[model];
  for (int g = 0; g < b->ngroups; ++g) {
    const int tiles = b->gcnt_h[g];
    if (tiles == 0) continue;
    for (int64_t k = 0; k < n; ++k) {
      const bool odd = (t0 + k) & 1;
      const int grid = m.grid[odd] > 0 ? std::min(m.grid[odd], tiles) : tiles;  // 0: one CTA per tile
      launch_step<T>(b, model, odd, m.var[odd], grid, g, s);
    }
  }
}

template <class T>
om_status capture_t(om_batch* b, int model, int K);

// whether the current device takes cooperative launches
inline bool cooperative_ok() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) return false;
  return v != 0;
}

// Largest grid of the window kernel of a model whose blocks are all
// resident at once (the cooperative-launch limit).
template <class T>
int window_grid(const om_batch* b, int model) {
  static int cache[2] = {0, 0};
  if (cache[model] <= 0) {
    int per = 0;
    if (model == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, flow_batch_window<T, 0>, kTile, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, diff_batch_window<T, 0>, kTile, 0);
    cache[model] = std::max(1, per) * b->sms;
  }
  return cache[model];
}

// K steps (from time t0) of every group, each group in one persistent
// cooperative launch.  The barrier's status is cleared once per window (a
// timeout in one group stays visible, and the later groups' waits then give
// up at once); its counters before every launch.
template <class T>
om_status launch_window_persistent(om_batch* b, int model, int64_t t0, int K, cudaStream_t s) {
  const int cap = window_grid<T>(b, model);
  int odd0 = (int)(t0 & 1);
  OM_CUDA(cudaMemsetAsync(b->bar, 0, sizeof(GridBar), s));
  for (int g = 0; g < b->ngroups; ++g) {
    const int tiles = b->gcnt_h[g];
    if (tiles == 0) continue;
    unsigned grid = (unsigned)std::min(tiles, cap);
    OM_CUDA(cudaMemsetAsync(b->bar, 0, offsetof(GridBar, status), s));
    GridBar* bar = b->bar;
    if (model == 0) {
      if constexpr (kFlowRebased<T>) {
        if (!b->greb[g]) {
          using S = typename T::base;
          grid = (unsigned)std::min(tiles, window_grid<S>(b, model));
          FlowArgs<S> a = bflow_args<S>(b);
          void* args[] = {&a, &b->gdesc[g], &odd0, &K, &bar};
          OM_CUDA(cudaLaunchCooperativeKernel((const void*)flow_batch_window<S, 0>, dim3(grid), dim3(kTile), args, 0,
                                              s));
          continue;
        }
      }
      FlowArgs<T> a = bflow_args<T>(b);
      void* args[] = {&a, &b->gdesc[g], &odd0, &K, &bar};
      OM_CUDA(cudaLaunchCooperativeKernel((const void*)flow_batch_window<T, 0>, dim3(grid), dim3(kTile), args, 0, s));
    } else {
      DiffArgs<T> a = bdiff_args<T>(b);
      void* args[] = {&a, &b->gdesc[g], &odd0, &K, &bar};
      OM_CUDA(cudaLaunchCooperativeKernel((const void*)diff_batch_window<T, 0>, dim3(grid), dim3(kTile), args, 0, s));
    }
  }
  return OM_OK;
}

// one check window of K steps from an even time: mode 0 replays the
// captured per-step launches, mode 1 runs each group as one persistent
// launch and queues a copy of the barrier status to the host (read after the
// caller's next synchronisation)
template <class T>
om_status window_t(om_batch* b, int model, int K, int mode, cudaStream_t s) {
  Model& m = b->m[model];
  if (mode == 1) {
    OM_TRY(launch_window_persistent<T>(b, model, m.t, K, s));
    OM_CUDA(cudaMemcpyAsync(b->bar_h, &b->bar->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  } else {
    OM_TRY(capture_t<T>(b, model, K));
    OM_CUDA(cudaGraphLaunch(m.exec, s));
  }
  m.t += K;
  if (model == 1 && m.cr) batch_rebase<T><<<(b->total + 255) / 256, 256, 0, s>>>(bdiff_args<T>(b));
  if (model == 0 && m.cr)
    for (int g = 0; g < b->ngroups; ++g)
      if (b->greb[g] && b->gcnt_h[g] > 0)
        batch_flow_rebase_group<T><<<std::min(b->gcnt_h[g], b->sms * 8), kTile, 0, s>>>(bflow_args<T>(b), b->gdesc[g]);
  return OM_OK;
}

// Advance n steps: whole check windows from even times replay the captured
// window graph (and, for rebased diffusion storage, move the reference after
// it, as a solve does); anything else is launched step by step.
template <class T>
om_status steps_t(om_batch* b, int model, int64_t n, cudaStream_t s) {
  Model& m = b->m[model];
  if (b->layout_model != model) {  // groups sized for this model's footprint, every item
    std::vector<int> all;
    for (int k = 0; k < b->n; ++k)
      if (b->items_h[k].nf > 0) all.push_back(k);
    const int nw = build_work(b, all, model);
    OM_TRY(upload_work(b, nw, (int)all.size(), s));
  }
  const int K = model == 0 ? b->fp.check_every : b->dp.check_every;
  while (n > 0) {
    if (K >= 2 && !(K & 1) && !(m.t & 1) && n >= K) {
      OM_TRY(window_t<T>(b, model, K, 0, s));
      n -= K;
      continue;
    }
    launch_steps_grouped<T>(b, model, m.t, 1, s);
    ++m.t;
    --n;
  }
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

template <class T>
om_status observe_t(om_batch* b, int model, int nact, cudaStream_t s) {
  Model& m = b->m[model];
  const int grid = b->sms * 4;
  const int nv = model == 0 ? 4 : 5;
  if (model == 0) {
    FlowArgs<T> a = bflow_args<T>(b);
    if (m.t & 1) flow_batch_observe<T, true><<<grid, kTile, 0, s>>>(a, b->items, b->work, b->nwork, m.prev, b->partials);
    else flow_batch_observe<T, false><<<grid, kTile, 0, s>>>(a, b->items, b->work, b->nwork, m.prev, b->partials);
    if (nact > 0) batch_finalize<4><<<nact, 256, 0, s>>>(b->partials, b->range, b->obs);
  } else {
    DiffArgs<T> a = bdiff_args<T>(b);
    if (m.t & 1)
      diff_batch_observe<T, true><<<grid, kTile, 0, s>>>(a, b->items, b->work, b->nwork, m.prev, b->partials, m.dprev);
    else
      diff_batch_observe<T, false><<<grid, kTile, 0, s>>>(a, b->items, b->work, b->nwork, m.prev, b->partials, m.dprev);
    if (nact > 0) batch_finalize<5><<<nact, 256, 0, s>>>(b->partials, b->range, b->obs);
  }
  OM_CUDA(cudaGetLastError());
  if (nact > 0)
    OM_CUDA(cudaMemcpyAsync(b->obs_h, b->obs, sizeof(double) * nv * nact, cudaMemcpyDeviceToHost, s));
  OM_CUDA(cudaStreamSynchronize(s));
  return OM_OK;
}

// the single-structure variants of every solo item, in both storage modes
// of the flow (the populations change: the caller restores the state)
template <class T>
om_status tune_solo_t(om_batch* b, cudaStream_t s) {
  using S = typename Plain<T>::type;
  for (int k = 0; k < b->n; ++k) {
    if (!b->col_local[k]) continue;
    int V[2] = {0, 0};
    OM_TRY(flow_tuned_variants<S>(solo_args<S>(b, k), b->m[0].prec, V, s, nullptr));
    b->svar[k][0] = V[0], b->svar[k][1] = V[1];
    if constexpr (kFlowRebased<T>) {
      OM_TRY(flow_tuned_variants<T>(solo_args<T>(b, k), b->m[0].prec, V, s, nullptr));
      b->svar[k][2] = V[0], b->svar[k][3] = V[1];
    }
  }
  return OM_OK;
}

template <class T>
om_status tune_solo_diff_t(om_batch* b, cudaStream_t s) {
  if constexpr (kFlowRebased<T>) {
    return fail(OM_EINVAL, "om_batch: rebased storage is the flow's");
  } else {
    for (int k = 0; k < b->n; ++k) {
      if (!b->col_local[k]) continue;
      int V[2] = {0, 0};
      OM_TRY(diff_tuned_variants<T>(solo_dargs<T>(b, k), b->m[1].prec, V, s));
      b->dvar[k][0] = V[0], b->dvar[k][1] = V[1];
    }
    return OM_OK;
  }
}

// Autotuner: for each parity, time (variant, CTAs per SM) shapes over 6
// steps after a warm-up step and keep the fastest.  Steps run from the
// initial state, which the caller restores afterwards.
template <class T>
om_status tune_t(om_batch* b, int model, cudaStream_t s) {
  Model& m = b->m[model];
  if (b->total == 0) return OM_OK;
  // {variant, CTAs per SM}; 0 CTAs per SM: one CTA per 256-node tile, the
  // hardware scheduler balancing the tiles, instead of a resident grid
  // (flow only) {2, 3}: solo groups in the batch's forms of the single-
  // structure sweeps, odd steps on 3 resident CTAs per SM; {3, .}: solo
  // groups in the single-structure solver's own sweeps, their variants
  // tuned per item (by size class) first
  // (diffusion: {3, 0}, {3, 8} likewise, no variant 2)
  const int shapes[10][2] = {{0, 0}, {1, 0}, {0, 2}, {0, 4}, {1, 4}, {1, 8}, {2, 3}, {2, 4}, {3, 0}, {3, 4}};
  const int dshapes[8][2] = {{0, 0}, {1, 0}, {0, 2}, {0, 4}, {1, 4}, {1, 8}, {3, 0}, {3, 8}};
  const int nshapes = model == 0 ? 10 : 8;
  if (model == 0) OM_TRY(tune_solo_t<T>(b, s));
  else OM_TRY(tune_solo_diff_t<T>(b, s));
  cudaEvent_t ev[3];
  for (auto& e : ev) OM_CUDA(cudaEventCreate(&e));
  float best[2] = {1e30f, 1e30f};
  for (int si = 0; si < nshapes; ++si) {
    const int* sh = model == 0 ? shapes[si] : dshapes[si];
    const int grid = sh[1] * b->sms;  // 0: one CTA per tile
    float tot[2] = {0.f, 0.f};
    for (int r = 0; r < 7; ++r) {
      OM_CUDA(cudaEventRecord(ev[0], s));
      for (int gi = 0; gi < b->ngroups; ++gi)
        launch_step<T>(b, model, false, sh[0], grid > 0 ? std::min(grid, b->gcnt_h[gi]) : b->gcnt_h[gi], gi, s);
      OM_CUDA(cudaEventRecord(ev[1], s));
      for (int gi = 0; gi < b->ngroups; ++gi)
        launch_step<T>(b, model, true, sh[0], grid > 0 ? std::min(grid, b->gcnt_h[gi]) : b->gcnt_h[gi], gi, s);
      OM_CUDA(cudaEventRecord(ev[2], s));
      OM_CUDA(cudaEventSynchronize(ev[2]));
      if (r == 0) continue;
      float a0 = 0.f, a1 = 0.f;
      OM_CUDA(cudaEventElapsedTime(&a0, ev[0], ev[1]));
      OM_CUDA(cudaEventElapsedTime(&a1, ev[1], ev[2]));
      tot[0] += a0;
      tot[1] += a1;
    }
    for (int p = 0; p < 2; ++p)
      if (tot[p] < best[p]) {
        best[p] = tot[p];
        m.var[p] = sh[0];
        m.grid[p] = grid;
      }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

// capture K steps (K even, starting from an even time) into a graph
template <class T>
om_status capture_t(om_batch* b, int model, int K) {
  Model& m = b->m[model];
  if (m.exec && m.graph_k == K && m.graph_layout == b->layout) return OM_OK;
  if (m.exec) {
    cudaGraphExecDestroy(m.exec);
    m.exec = nullptr;
  }
  cudaGraph_t g = nullptr;
  OM_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  launch_steps_grouped<T>(b, model, 0, K, b->cap);
  cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  e = cudaGraphInstantiate(&m.exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
  m.graph_k = K;
  m.graph_layout = b->layout;
  return OM_OK;
}

template <class T>
om_status init_state_t(om_batch* b, int model, cudaStream_t s) {
  Model& m = b->m[model];
  OM_CUDA(cudaMemsetAsync(m.pop, 0, (size_t)m.q * b->pitch * stg_bytes(m.prec), s));  // rest / linear profile
  if (m.cr && model == 1) batch_cr_linear<<<b->sms * 4, kTile, 0, s>>>(b->items, b->work, b->nwork, b->dp.c_in, m.cr);
  if (m.cr && model == 0) {
    OM_CUDA(cudaMemsetAsync(m.cr, 0, sizeof(float) * b->pitch, s));  // rest density
    // as om_flow_solve: 16-bit storage rebased from the start, single
    // precision from the last decades of each item's convergence
    m.reb.assign(b->n, m.prec == OM_F32 ? 0 : 1);
    b->layout_model = -1;  // groups follow the modes
  }
  OM_CUDA(cudaGetLastError());
  m.t = 0;
  return OM_OK;
}

template <class T>
om_status solve_t(om_batch* b, int model, double* result, double* aux, om_run_info* info, int32_t* status,
                  cudaStream_t s) {
  Model& m = b->m[model];
  const int K = model == 0 ? b->fp.check_every : b->dp.check_every;
  const int64_t max_steps = model == 0 ? b->fp.max_steps : b->dp.max_steps;
  const double tol = model == 0 ? b->fp.conv_tol : b->dp.conv_tol;
  const int nv = model == 0 ? 4 : 5;
  if (K <= 0 || (K & 1)) return fail(OM_EINVAL, "om_batch_solve: check_every must be a positive even number");
  if (m.t & 1) return fail(OM_EINVAL, "om_batch_solve: the batch must be at an even time");
  std::vector<int> active;
  for (int k = 0; k < b->n; ++k) {
    if (status) status[k] = OM_ENOPERC;
    if (info) info[k] = om_run_info{};
    if (result) result[k] = 0.0;
    if (aux) aux[k] = 0.0;
    // flow: no lattice link across the periodic x boundary means zero flux
    if (b->items_h[k].nf > 0 && (model == 1 || b->ns[k]->wrap_links > 0)) active.push_back(k);
  }
  std::vector<double> sj_prev(b->n, 0.0);
  std::vector<ExtrapolationTrack> track(b->n);
  int nw = build_work(b, active, model);
  OM_TRY(upload_work(b, nw, (int)active.size(), s));
  OM_TRY(observe_t<T>(b, model, (int)active.size(), s));  // reference state
  for (size_t a = 0; a < active.size(); ++a) sj_prev[active[a]] = b->obs_h[a * nv + 0];
  cudaEvent_t e0, e1, w0, w1;
  OM_CUDA(cudaEventCreate(&e0));
  OM_CUDA(cudaEventCreate(&e1));
  OM_CUDA(cudaEventCreate(&w0));
  OM_CUDA(cudaEventCreate(&w1));
  OM_CUDA(cudaEventRecord(e0, s));
  const int64_t t0 = m.t;
  int64_t updates = 0;
  while (!active.empty() && m.t - t0 < max_steps) {
    const int64_t k = std::min<int64_t>(K, max_steps - (m.t - t0));
    // a whole window: in the model's mode, or, until both modes have been
    // timed on a window of this solve, the one not timed yet
    int mode = -1;
    if (k == K) {
      if (m.mode < 0 && !cooperative_ok()) m.mode = 0;  // no cooperative launches here: graphs only
      mode = m.mode >= 0 ? m.mode : (m.trial_ms[0] < 0.f ? 0 : 1);
      *b->bar_h = OM_OK;
      if (mode == 0) OM_TRY(capture_t<T>(b, model, K));  // host work outside the timed window
      OM_CUDA(cudaEventRecord(w0, s));
      OM_TRY(window_t<T>(b, model, K, mode, s));
      OM_CUDA(cudaEventRecord(w1, s));
    } else {
      OM_TRY(steps_t<T>(b, model, k, s));
    }
    for (int a : active) updates += (int64_t)b->items_h[a].nf * k;
    OM_TRY(observe_t<T>(b, model, (int)active.size(), s));  // synchronises
    if (mode == 1 && *b->bar_h != OM_OK) {
      for (cudaEvent_t e : {e0, e1, w0, w1}) cudaEventDestroy(e);
      return fail(OM_ETIMEOUT, "om_batch_solve: a grid-barrier wait of a persistent window gave up");
    }
    if (mode >= 0 && m.mode < 0) {
      float ms = 0.f;
      OM_CUDA(cudaEventElapsedTime(&ms, w0, w1));
      m.trial_ms[mode] = ms;
      if (m.trial_ms[0] >= 0.f && m.trial_ms[1] >= 0.f) m.mode = m.trial_ms[1] < m.trial_ms[0] ? 1 : 0;
    }
    std::vector<int> keep;
    bool switched = false;
    for (size_t a = 0; a < active.size(); ++a) {
      const int it = active[a];
      const double* o = b->obs_h + a * nv;
      const BatchItem& bi = b->items_h[it];
      const double N = (double)b->dom[it].nx * b->dom[it].ny * b->dom[it].nz;
      double rel = o[2] > 0.0 ? o[1] / o[2] : 0.0;
      if (model == 1) {  // the diffusion: the net flux sum J_x too
        const double relj = o[0] != 0.0 ? std::fabs(o[0] - sj_prev[it]) / std::fabs(o[0]) : 0.0;
        rel = std::max(rel, relj);
        sj_prev[it] = o[0];
      }
      if (result) {
        if (model == 0) result[it] = ((b->fp.tau - 0.5) / 3.0) * (o[0] / N) / b->fp.body_force;
        else result[it] = (o[0] / N) * (double)bi.nx / (b->dp.c_in - b->dp.c_out);
      }
      if (aux) aux[it] = model == 0 ? o[3] : o[4] / (double)bi.nf;
      if (info) {
        info[it].steps = m.t - t0;
        info[it].n_nodes = bi.nf;
        info[it].rel_change = rel;
        info[it].mass = o[3];
      }
      const bool done = rel < tol;
      // non-finite sums: the item diverged; it leaves the batch unconverged
      const bool diverged = !std::isfinite(o[0]) || !std::isfinite(o[2]);
      if (status) status[it] = done && !diverged ? OM_OK : OM_ENOTCONVERGED;
      if (!done && !diverged) keep.push_back(it);
      // the flow: an item enters the rebased mode for its last decades, as
      // om_flow_solve does (its group changes: the work list is rebuilt)
      if (!done && !diverged && model == 0 && !m.reb.empty() && !m.reb[it] && rel < kRebaseBelow) {
        if constexpr (kFlowRebased<T>)
          batch_flow_rebase_range<T><<<(bi.nf + 255) / 256, 256, 0, s>>>(bflow_args<T>(b), bi.off, bi.nf);
        OM_CUDA(cudaGetLastError());
        m.reb[it] = 1;
        switched = true;
      }
      if (!done && !diverged && model == 1 && m.dprev) {
        const double f = track[it].observe(o[1]);
        if (f > 0.0) {
          diff_batch_extrapolate<T><<<(bi.nf + 255) / 256, 256, 0, s>>>(bdiff_args<T>(b), bi.off, bi.nf, m.prev,
                                                                         m.dprev, std::min(f, 1e3));
          OM_CUDA(cudaGetLastError());
        }
      }
    }
    if (keep.size() != active.size() || switched) {
      active.swap(keep);
      nw = build_work(b, active, model);
      OM_TRY(upload_work(b, nw, (int)active.size(), s));
    }
  }
  OM_CUDA(cudaEventRecord(e1, s));
  OM_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  OM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(w0);
  cudaEventDestroy(w1);
  if (info)
    for (int k = 0; k < b->n; ++k) {
      info[k].seconds = ms * 1e-3;
      info[k].mlups = ms > 0 ? (double)updates / (ms * 1e-3) / 1e6 : 0.0;
    }
  // leave the full work list in place for later steps
  std::vector<int> all;
  for (int k = 0; k < b->n; ++k)
    if (b->items_h[k].nf > 0) all.push_back(k);
  nw = build_work(b, all, model);
  OM_TRY(upload_work(b, nw, (int)all.size(), s));
  OM_CUDA(cudaStreamSynchronize(s));
  return OM_OK;
}

// The storage type of a model: the flow's single- and half-precision
// populations are handled as rebased storage (Reb<S>, flow_core.cuh) --
// exact for every item, since an item not in the rebased mode keeps its
// reference cr = 0 -- and the sweeps of the groups whose items are not in
// that mode take the plain S (launch_flow).  The diffusion's storage is
// rebased by its own scheme.
#define OM_BATCH_DISPATCH(prec, fn, ...)                                      \
  switch (prec) {                                                             \
    case OM_F64: return fn<double>(__VA_ARGS__);                              \
    case OM_F32: return model == 0 ? fn<Reb<float>>(__VA_ARGS__) : fn<float>(__VA_ARGS__); \
    case OM_F16DEV: return model == 0 ? fn<Reb<__half>>(__VA_ARGS__) : fn<__half>(__VA_ARGS__); \
    case OM_BF16DEV:                                                          \
      return model == 0 ? fn<Reb<__nv_bfloat16>>(__VA_ARGS__) : fn<__nv_bfloat16>(__VA_ARGS__); \
    default: return fail(OM_EINVAL, "unknown precision");                     \
  }

om_status dispatch_tune(om_batch* b, int model, cudaStream_t s) { OM_BATCH_DISPATCH(b->m[model].prec, tune_t, b, model, s); }
om_status dispatch_tune_solo(om_batch* b, int model, cudaStream_t s) {
  if (model == 0) {
    OM_BATCH_DISPATCH(b->m[0].prec, tune_solo_t, b, s);
  }
  OM_BATCH_DISPATCH(b->m[1].prec, tune_solo_diff_t, b, s);
}
om_status dispatch_init(om_batch* b, int model, cudaStream_t s) { OM_BATCH_DISPATCH(b->m[model].prec, init_state_t, b, model, s); }

}  // namespace

extern "C" om_status om_batch_destroy(om_batch* b) {
  if (!b) return OM_OK;
  for (auto* ns : b->ns) om_nodeset_destroy(ns);
  for (auto* c : b->col_local) cudaFree(c);
  for (auto& m : b->m) {
    if (m.exec) cudaGraphExecDestroy(m.exec);
    cudaFree(m.pop);
    cudaFree(m.omega);
    cudaFree(m.cr);
    cudaFree(m.prev);
    cudaFree(m.dprev);
  }
  cudaFree(b->items);
  cudaFree(b->work);
  cudaFree(b->nwork);
  cudaFree(b->range);
  cudaFree(b->partials);
  cudaFree(b->obs);
  cudaFree(b->bar);
  if (b->bar_h) cudaFreeHost(b->bar_h);
  if (b->work_h) cudaFreeHost(b->work_h);
  if (b->range_h) cudaFreeHost(b->range_h);
  if (b->nwork_h) cudaFreeHost(b->nwork_h);
  if (b->gcnt_h) cudaFreeHost(b->gcnt_h);
  if (b->obs_h) cudaFreeHost(b->obs_h);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return OM_OK;
}

extern "C" om_status om_batch_create(int32_t n, const om_domain* doms, const uint8_t* const* nodes_dev,
                                     const float* const* d_nm_dev, const om_flow_params* fp,
                                     const om_diff_params* dp, void* stream, om_batch** out) {
  if (n <= 0 || !doms || !nodes_dev || !out || (!fp && !dp)) return fail(OM_EINVAL, "om_batch_create: bad arguments");
  if (dp && !d_nm_dev) return fail(OM_EINVAL, "om_batch_create: diffusion needs pore sizes");
  if (dp && dp->lattice != 7) return fail(OM_EINVAL, "om_batch_create: batches take the D3Q7 diffusion lattice");
  if (dp && dp->accel != OM_ACCEL_NONE && dp->accel != OM_ACCEL_EXTRAPOLATE)
    return fail(OM_EINVAL, "om_batch_create: unknown accel");
  if (fp && !(fp->tau > 0.5)) return fail(OM_EINVAL, "om_batch_create: tau must exceed 1/2");
  if ((fp && fp->layout == OM_LAYOUT_DENSE) || (dp && dp->layout == OM_LAYOUT_DENSE))
    return fail(OM_EINVAL, "om_batch_create: batches use the sparse layout");
  if (fp && fp->drive != OM_DRIVE_FORCE) return fail(OM_EINVAL, "om_batch_create: batches take the body-force drive");
  if (dp && (!(dp->d_ref_nm > 0.0) || !(dp->tau_ref > 0.5) || !(dp->c_in != dp->c_out)))
    return fail(OM_EINVAL, "om_batch_create: need d_ref > 0, tau_ref > 1/2, c_in != c_out");
  for (const auto* p : {fp ? &fp->precision : nullptr, dp ? &dp->precision : nullptr})
    if (p && (*p < OM_F64 || *p > OM_BF16DEV)) return fail(OM_EINVAL, "om_batch_create: unknown precision");
  cudaStream_t s = as_stream(stream);
  om_batch* b = new om_batch();
  auto bail = [&](om_status st) {
    om_batch_destroy(b);
    return st;
  };
  b->n = n;
  if (fp) b->fp = *fp;
  if (dp) b->dp = *dp;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  // node sets, offsets, rebased column maps
  uint64_t total = 0;
  int tiles = 0;
  for (int k = 0; k < n; ++k) {
    om_nodeset* ns = nullptr;
    om_status st = om_nodeset_create(nodes_dev[k], doms[k], stream, &ns);
    if (st != OM_OK) return bail(st);
    b->ns.push_back(ns);
    b->dom.push_back(doms[k]);
    BatchItem it{};
    it.col = ns->col;
    it.coord = ns->coord;
    uint4* local = nullptr;
    if ((uint32_t)ns->nf >= kSoloNodes) {
      total = (total + 31) / 32 * 32;
      const size_t bytes = sizeof(uint4) * (size_t)doms[k].nx * doms[k].ny * ns->W;
      if (cudaMalloc((void**)&local, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        return bail(fail(OM_ENOMEM, "om_batch_create: device allocation failed"));
      }
      b->col_local.push_back(local);  // owned by the batch from here on
      if (cudaMemcpyAsync(local, ns->col, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return bail(fail(OM_ECUDA, "om_batch_create: column map copy failed"));
    } else {
      b->col_local.push_back(nullptr);
    }
    b->svar.push_back({0, 0, 0, 0});
    b->dvar.push_back({0, 0});
    it.off = (uint32_t)total;
    it.nf = (uint32_t)ns->nf;
    it.nx = doms[k].nx;
    it.ny = doms[k].ny;
    it.nz = doms[k].nz;
    it.W = ns->W;
    it.slope = dp ? (dp->c_out - dp->c_in) / (double)doms[k].nx : 0.0;
    const int64_t nw = (int64_t)doms[k].nx * doms[k].ny * ns->W;
    if (total > 0) rebase_columns<<<(unsigned)std::min<int64_t>((nw + 255) / 256, 4096), 256, 0, s>>>(ns->col, nw, it.off);
    total += (uint64_t)ns->nf;
    tiles += (int)((ns->nf + kTile - 1) / kTile);
    b->items_h.push_back(it);
  }
  b->pitch = ((int64_t)total + 63) / 64 * 64;
  if (19 * b->pitch > (int64_t)UINT32_MAX)
    return bail(fail(OM_EINVAL, "om_batch_create: more than 226 M nodes (slot offsets are 32-bit)"));
  b->total = (uint32_t)total;
  b->max_tiles = std::max(1, tiles);
  auto dalloc = [&](void** p, size_t bytes) -> om_status {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      (void)cudaGetLastError();
      *p = nullptr;
      return fail(OM_ENOMEM, "om_batch_create: device allocation failed");
    }
    return OM_OK;
  };
  auto halloc = [&](void** p, size_t bytes) -> om_status {
    if (cudaMallocHost(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      (void)cudaGetLastError();
      *p = nullptr;
      return fail(OM_ENOMEM, "om_batch_create: pinned allocation failed");
    }
    return OM_OK;
  };
  om_status st = OM_OK;
  if ((st = dalloc((void**)&b->items, sizeof(BatchItem) * n)) != OM_OK) return bail(st);
  if ((st = dalloc((void**)&b->work, sizeof(uint2) * b->max_tiles)) != OM_OK) return bail(st);
  if ((st = dalloc((void**)&b->nwork, sizeof(int))) != OM_OK) return bail(st);
  if ((st = dalloc((void**)&b->range, sizeof(int2) * n)) != OM_OK) return bail(st);
  if ((st = dalloc((void**)&b->partials, sizeof(double) * 5 * b->max_tiles)) != OM_OK) return bail(st);
  if ((st = dalloc((void**)&b->obs, sizeof(double) * 5 * n)) != OM_OK) return bail(st);
  if ((st = halloc((void**)&b->work_h, sizeof(uint2) * b->max_tiles)) != OM_OK) return bail(st);
  if ((st = halloc((void**)&b->range_h, sizeof(int2) * n)) != OM_OK) return bail(st);
  if ((st = halloc((void**)&b->nwork_h, sizeof(int))) != OM_OK) return bail(st);
  if ((st = halloc((void**)&b->gcnt_h, sizeof(int) * n)) != OM_OK) return bail(st);
  if ((st = halloc((void**)&b->obs_h, sizeof(double) * 5 * n)) != OM_OK) return bail(st);
  if ((st = dalloc((void**)&b->bar, sizeof(GridBar))) != OM_OK) return bail(st);
  if ((st = halloc((void**)&b->bar_h, sizeof(int))) != OM_OK) return bail(st);
  *b->bar_h = OM_OK;
  if (cudaMemcpyAsync(b->items, b->items_h.data(), sizeof(BatchItem) * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return bail(fail(OM_ECUDA, "om_batch_create: copy of the item table failed"));
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(OM_ECUDA, "om_batch_create: stream creation failed"));
  // models
  for (int model = 0; model < 2; ++model) {
    const bool on = model == 0 ? fp != nullptr : dp != nullptr;
    if (!on) continue;
    Model& m = b->m[model];
    m.on = true;
    m.prec = model == 0 ? fp->precision : dp->precision;
    m.q = model == 0 ? 19 : 7;
    m.up = m.prec == OM_F16DEV ? (model == 0 ? 1024.0 : 64.0) : 1.0;
    if ((st = dalloc(&m.pop, (size_t)m.q * b->pitch * stg_bytes(m.prec))) != OM_OK) return bail(st);
    if ((st = dalloc((void**)&m.prev, sizeof(double) * b->pitch)) != OM_OK) return bail(st);
    if (model == 0 && stg_bytes(m.prec) <= 4 && (st = dalloc((void**)&m.cr, sizeof(float) * b->pitch)) != OM_OK)
      return bail(st);
    if (m.cr) cudaMemsetAsync(m.cr, 0, sizeof(float) * b->pitch, s);
    if (model == 1 && dp->accel == OM_ACCEL_EXTRAPOLATE &&
        (st = dalloc((void**)&m.dprev, sizeof(double) * b->pitch)) != OM_OK)
      return bail(st);
    if (model == 1) {
      const size_t cb = m.prec == OM_F64 ? 8 : 4;
      if ((st = dalloc(&m.omega, cb * b->pitch)) != OM_OK) return bail(st);
      cudaMemsetAsync(m.omega, 0, cb * b->pitch, s);  // the arena's gaps before aligned items
      if (stg_bytes(m.prec) <= 4 && (st = dalloc((void**)&m.cr, sizeof(float) * b->pitch)) != OM_OK) return bail(st);
      if (m.cr) cudaMemsetAsync(m.cr, 0, sizeof(float) * b->pitch, s);
      int* bad = nullptr;
      if ((st = dalloc((void**)&bad, sizeof(int))) != OM_OK) return bail(st);
      cudaMemsetAsync(bad, 0, sizeof(int), s);
      for (int k = 0; k < n; ++k) {
        const BatchItem& it = b->items_h[k];
        if (it.nf == 0) continue;
        const unsigned g = (it.nf + 255) / 256;
        if (m.prec == OM_F64)
          batch_omega<double><<<g, 256, 0, s>>>(b->ns[k]->vox, d_nm_dev[k], it.nf, dp->d_ref_nm, dp->tau_ref,
                                                (double*)m.omega + it.off, bad);
        else
          batch_omega<float><<<g, 256, 0, s>>>(b->ns[k]->vox, d_nm_dev[k], it.nf, dp->d_ref_nm, dp->tau_ref,
                                               (float*)m.omega + it.off, bad);
      }
      int hb = 0;
      cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
      cudaStreamSynchronize(s);
      cudaFree(bad);
      if (hb) return bail(fail(OM_EINVAL, "om_batch_create: a node has a pore size <= 0"));
    }
    // full work list, tune the launch shapes from the initial state, restore it
    std::vector<int> all;
    for (int k = 0; k < n; ++k)
      if (b->items_h[k].nf > 0) all.push_back(k);
    int nw = build_work(b, all, model);
    if ((st = upload_work(b, nw, (int)all.size(), s)) != OM_OK) return bail(st);
    if ((st = dispatch_init(b, model, s)) != OM_OK) return bail(st);
    if (model == 0) {  // the flow's groups follow the modes its items start in
      nw = build_work(b, all, model);
      if ((st = upload_work(b, nw, (int)all.size(), s)) != OM_OK) return bail(st);
    }
    const int variant = model == 0 ? fp->variant : dp->variant;
    if (variant < 0) {
      if ((st = dispatch_tune(b, model, s)) != OM_OK) return bail(st);
      if ((st = dispatch_init(b, model, s)) != OM_OK) return bail(st);
    } else {
      m.var[0] = m.var[1] = std::min(variant, 3);
      if (m.var[0] == 2 && model == 1) m.var[0] = m.var[1] = 1;
      if (m.var[0] == 3) {
        if ((st = dispatch_tune_solo(b, model, s)) != OM_OK) return bail(st);
        if ((st = dispatch_init(b, model, s)) != OM_OK) return bail(st);
      }
      m.grid[0] = m.grid[1] = 4 * b->sms;
    }
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "om_batch_create", __FILE__, __LINE__));
  *out = b;
  return OM_OK;
}

extern "C" om_status om_batch_step(om_batch* b, int32_t model, int64_t nsteps, void* stream) {
  if (!b || model < 0 || model > 1 || !b->m[model].on || nsteps < 0) return fail(OM_EINVAL, "om_batch_step: bad arguments");
  OM_BATCH_DISPATCH(b->m[model].prec, steps_t, b, model, nsteps, as_stream(stream));
}

extern "C" om_status om_batch_set_window_mode(om_batch* b, int32_t model, int32_t mode) {
  if (!b || model < 0 || model > 1 || !b->m[model].on || mode < -1 || mode > 1)
    return fail(OM_EINVAL, "om_batch_set_window_mode: bad arguments");
  Model& m = b->m[model];
  m.mode = mode;
  m.trial_ms[0] = m.trial_ms[1] = -1.f;
  return OM_OK;
}

extern "C" om_status om_barrier_selftest(int32_t blocks, int32_t rounds, int32_t extra, int64_t max_polls,
                                         int32_t* status, void* stream) {
  if (blocks <= 0 || rounds < 0 || extra < 0 || max_polls <= 0 || !status)
    return fail(OM_EINVAL, "om_barrier_selftest: bad arguments");
  int dev = 0, sms = 0, per = 0;
  OM_CUDA(cudaGetDevice(&dev));
  OM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  OM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, barrier_selftest, kTile, 0));
  if ((int64_t)blocks > (int64_t)per * sms)
    return fail(OM_EINVAL, "om_barrier_selftest: more blocks than can be resident at once");
  cudaStream_t s = as_stream(stream);
  GridBar* bar = nullptr;
  if (cudaMalloc((void**)&bar, sizeof(GridBar)) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(OM_ENOMEM, "om_barrier_selftest: device allocation failed");
  }
  unsigned ex = (unsigned)extra;
  unsigned long long lim = (unsigned long long)max_polls;
  void* args[] = {&bar, &rounds, &ex, &lim};
  int st = OM_OK;
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBar), s);
  if (e == cudaSuccess)
    e = cudaLaunchCooperativeKernel((const void*)barrier_selftest, dim3(blocks), dim3(kTile), args, 0, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, &bar->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(bar);
  if (e != cudaSuccess) return cuda_fail(e, "om_barrier_selftest", __FILE__, __LINE__);
  *status = st;
  return OM_OK;
}

extern "C" om_status om_batch_solve(om_batch* b, int32_t model, double* result, double* aux, om_run_info* info,
                                    int32_t* status, void* stream) {
  if (!b || model < 0 || model > 1 || !b->m[model].on) return fail(OM_EINVAL, "om_batch_solve: bad arguments");
  OM_BATCH_DISPATCH(b->m[model].prec, solve_t, b, model, result, aux, info, status, as_stream(stream));
}

namespace {
template <class T>
om_status exchange_t(om_batch* b, int model, int item, double* out, const double* in, cudaStream_t s,
                     float* field = nullptr) {
  const BatchItem& it = b->items_h[item];
  const om_nodeset* ns = b->ns[item];
  const int64_t N = ns->N;
  const Model& m = b->m[model];
  if (out) OM_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * m.q * N, s));
  if (field) OM_CUDA(cudaMemsetAsync(field, 0, sizeof(float) * N, s));
  if (it.nf == 0) return OM_OK;
  const unsigned g = (it.nf + 255) / 256;
  if (model == 0) {
    FlowArgs<T> a = bflow_args<T>(b);
    a.nf = it.nf;
    a.col = it.col;
    a.coord = it.coord;
    a.nx = it.nx;
    a.ny = it.ny;
    a.nz = it.nz;
    a.W = it.W;
    if (in) flow_batch_import<T><<<g, 256, 0, s>>>(a, it.off, ns->vox, N, in);
    else if (m.t & 1) flow_batch_export<T, true><<<g, 256, 0, s>>>(a, it.off, ns->vox, N, out, field);
    else flow_batch_export<T, false><<<g, 256, 0, s>>>(a, it.off, ns->vox, N, out, field);
  } else {
    DiffArgs<T> a = bdiff_args<T>(b);
    a.nf = it.nf;
    a.col = it.col;
    a.coord = it.coord;
    a.nx = it.nx;
    a.ny = it.ny;
    a.nz = it.nz;
    a.W = it.W;
    a.s = (typename Stg<T>::C)it.slope;
    if (in) diff_batch_import<T><<<g, 256, 0, s>>>(a, it.off, ns->vox, N, in);
    else if (m.t & 1) diff_batch_export<T, true><<<g, 256, 0, s>>>(a, it.off, ns->vox, N, out, field);
    else diff_batch_export<T, false><<<g, 256, 0, s>>>(a, it.off, ns->vox, N, out, field);
  }
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}
}  // namespace

extern "C" om_status om_batch_get_populations(om_batch* b, int32_t model, int32_t item, double* dense_dev,
                                              void* stream) {
  if (!b || model < 0 || model > 1 || !b->m[model].on || item < 0 || item >= b->n || !dense_dev)
    return fail(OM_EINVAL, "om_batch_get_populations: bad arguments");
  OM_BATCH_DISPATCH(b->m[model].prec, exchange_t, b, model, item, dense_dev, nullptr, as_stream(stream));
}

extern "C" om_status om_batch_get_field(om_batch* b, int32_t model, int32_t item, float* field_dev, void* stream) {
  if (!b || model < 0 || model > 1 || !b->m[model].on || item < 0 || item >= b->n || !field_dev)
    return fail(OM_EINVAL, "om_batch_get_field: bad arguments");
  OM_BATCH_DISPATCH(b->m[model].prec, exchange_t, b, model, item, nullptr, nullptr, as_stream(stream), field_dev);
}

extern "C" om_status om_batch_set_populations(om_batch* b, int32_t model, int32_t item, const double* dense_dev,
                                              void* stream) {
  if (!b || model < 0 || model > 1 || !b->m[model].on || item < 0 || item >= b->n || !dense_dev)
    return fail(OM_EINVAL, "om_batch_set_populations: bad arguments");
  if (b->m[model].t & 1) return fail(OM_EINVAL, "om_batch_set_populations: the batch must be at an even time");
  OM_BATCH_DISPATCH(b->m[model].prec, exchange_t, b, model, item, nullptr, dense_dev, as_stream(stream));
}

namespace {
template <class T>
om_status init_item_t(om_batch* b, int model, int item, const float* field, int64_t stride, double scale,
                      int from_linear, cudaStream_t s) {
  const BatchItem& it = b->items_h[item];
  if (it.nf == 0) return OM_OK;
  const unsigned g = (it.nf + 255) / 256;
  if (model == 0) {
    FlowArgs<T> a = bflow_args<T>(b);
    a.nf = it.nf;
    flow_batch_init<T><<<g, 256, 0, s>>>(a, it.off, b->ns[item]->vox, field, stride, scale);
  } else {
    DiffArgs<T> a = bdiff_args<T>(b);
    a.nf = it.nf;
    a.coord = it.coord;
    a.s = (typename Stg<T>::C)it.slope;
    diff_batch_init<T><<<g, 256, 0, s>>>(a, it.off, b->ns[item]->vox, field, stride, from_linear);
  }
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}
}  // namespace

extern "C" om_status om_batch_init_fields(om_batch* b, int32_t model, int32_t item, const float* field_dev,
                                          int64_t stride, double scale, int32_t from_linear, void* stream) {
  if (!b || model < 0 || model > 1 || !b->m[model].on || item < 0 || item >= b->n || !field_dev || stride < 1)
    return fail(OM_EINVAL, "om_batch_init_fields: bad arguments");
  if (b->m[model].t & 1) return fail(OM_EINVAL, "om_batch_init_fields: the batch must be at an even time");
  OM_BATCH_DISPATCH(b->m[model].prec, init_item_t, b, model, item, field_dev, stride, scale, from_linear,
                    as_stream(stream));
}

extern "C" om_status om_batch_reset(om_batch* b, int32_t model, void* stream) {
  if (!b || model < 0 || model > 1 || !b->m[model].on) return fail(OM_EINVAL, "om_batch_reset: bad arguments");
  return dispatch_init(b, model, as_stream(stream));
}
