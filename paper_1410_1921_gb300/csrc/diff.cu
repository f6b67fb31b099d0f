// diff.cu -- BGK Knudsen-diffusion sweep (Sec. 3.2, Eqs. 10-12) in the AA
// pattern on the fluid-node layout of nodeset.cu, on D3Q7 (a = {1/4, 1/8 x
// 6}, c_s^2 = 1/4) or the paper's D3Q19 (Eq. 2-3 velocities and weights,
// c_s^2 = 1/3), chosen by om_diff_params.lattice.
//
// g*_i = g_i - omega(x) (g_i - a_i C), C = sum g_i, with omega = 1/tau_g
// from the local pore size by Eq. 12.  Populations are
// stored as deviations from a reference equilibrium a_i C_ref: in FP64 the
// linear profile C_lin(x) between the two fixed concentrations (the odd step
// adds the jump a_i s e_ix, s = dC_lin/dx, when a population changes cell);
// in FP32 and 16-bit storage a per-node concentration moved to the node's
// current C once per check window (see diff_core.cuh), the odd step adding
// a_i (C_ref(source) - C_ref(target)).
//
// Boundaries: bounce-back at walls and missing neighbours (no flux), periodic
// y and z, and fixed concentration on the half links x = -1/2 (c_in) and
// x = nx - 1/2 (c_out) by anti-bounce-back,
//     g_i(x_b, t+1) = -g*_opp(i)(x_b, t) + 2 a_i C_w.
#include <algorithm>
#include <cmath>

#include "solvers.cuh"

namespace om {

// Launch variants for the autotuner of om_diff_create (identical
// arithmetic): 0 = one thread per node, registers as the compiler wants;
// 1 = capped for 8 resident blocks; 2, 3 = the same on a resident grid whose
// threads stride over nodes, loading the next node's coordinates before
// updating the current one (the flow sweep's variants 2 and 3); 4 = variant
// 2 two nodes deep with the next node's column-map words prefetched into L1
// (the flow sweep's variant 5); 5 = even steps two consecutive nodes per
// thread with vector loads and stores (the flow sweep's variant 6), odd
// steps as variant 0; 6, 7, 8 = odd steps from the neighbour records with
// the slow nodes in the same grid (the flow sweep's variants 7, 8, 9: one
// thread per node, capped, and a resident grid loading the next node's
// records ahead), even steps as variant 5.  Without records 6-8 run as 5.
constexpr int kDiffVariants = 9;

template <class T, class L, bool ODD, int MINB>
__global__ void __launch_bounds__(256, MINB) diff_sweep(DiffArgs<T, L> a) {
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.nf) return;
  diff_node<T, ODD>(a, n, n);
}

template <class T, class L, bool ODD, int MINB>
__global__ void __launch_bounds__(256, MINB) diff_sweep_strided(DiffArgs<T, L> a) {
  const uint32_t stride = gridDim.x * blockDim.x;
  uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.nf) return;
  uint32_t c = ODD ? __ldg(a.coord + n) : 0u;
  for (;;) {
    const uint64_t nn = (uint64_t)n + stride;
    const bool more = nn < a.nf;
    uint32_t cn = 0u;
    if (ODD && more) cn = __ldg(a.coord + nn);
    diff_node_at<T, L, ODD>(a, n, c);
    if (!more) break;
    n = (uint32_t)nn;
    c = cn;
  }
}

template <class T, class L, bool ODD, int MINB>
__global__ void __launch_bounds__(256, MINB) diff_sweep_pipelined(DiffArgs<T, L> a) {
  const uint32_t stride = gridDim.x * blockDim.x;
  uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.nf) return;
  if (!ODD) {
    for (; n < a.nf; n += stride) diff_node_at<T, L, false>(a, n, 0u);
    return;
  }
  uint32_t c0 = __ldg(a.coord + n);
  uint32_t c1 = (uint64_t)n + stride < a.nf ? __ldg(a.coord + n + stride) : 0u;
  for (;;) {
    const uint64_t nn = (uint64_t)n + stride, nn2 = nn + stride;
    const uint32_t c2 = nn2 < a.nf ? __ldg(a.coord + nn2) : 0u;
    if (nn < a.nf) prefetch_columns<L::Q>(a.col, a.nx, a.ny, a.W, 0, c1);
    diff_node_at<T, L, true>(a, n, c0);
    if (nn >= a.nf) break;
    n = (uint32_t)nn;
    c0 = c1;
    c1 = c2;
  }
}

template <class T, class L, int MINB>
__global__ void __launch_bounds__(256, MINB) diff_sweep_rec(DiffArgs<T, L> a) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.nf + a.nslow) return;
  uint2 r, q;
  diff_rec_load<L>(a.rec7, a.rec19, t, a.nf, r, q);
  diff_odd_rec<T, L>(a, t, r, q);
}

template <class T, class L>
__global__ void __launch_bounds__(256) diff_sweep_rec_strided(DiffArgs<T, L> a) {
  const uint32_t stride = gridDim.x * blockDim.x, total = a.nf + a.nslow;
  uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  uint2 r, q;
  diff_rec_load<L>(a.rec7, a.rec19, t, a.nf, r, q);
  for (;;) {
    const uint64_t tn = (uint64_t)t + stride;
    uint2 rn, qn;
    diff_rec_load<L>(a.rec7, a.rec19, tn < a.nf ? (uint32_t)tn : a.nf, a.nf, rn, qn);
    diff_odd_rec<T, L>(a, t, r, q);
    if (tn >= total) break;
    t = (uint32_t)tn;
    r = rn;
    q = qn;
  }
}

template <class T, class L>
__global__ void __launch_bounds__(256) diff_sweep_pair(DiffArgs<T, L> a) {
  const uint32_t n = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (n >= a.nf) return;
  if (n + 1 == a.nf) diff_node_at<T, L, false>(a, n, 0u);
  else diff_pair_even<T, L>(a, n);
}

// Observables: sum J_x, sum |C - prev|, sum |C|, sum C, sum D_L; prev <- C.
template <class T, class L, bool ODD>
__global__ void __launch_bounds__(kObsThreads) diff_observe(DiffArgs<T, L> a, double* prev,
                                                            double* partials, double* dprev) {
  using C = typename Stg<T>::C;
  double acc[5] = {0, 0, 0, 0, 0};
  for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < a.nf; n += gridDim.x * blockDim.x) {
    uint32_t nb[L::Q];
    int x, y, z;
    unpack_xyz(a.coord[n], x, y, z);
    if (ODD) diff_neighbours(a, a.coord[n], nb, x);
    C g[L::Q];
    diff_load<T, L, ODD>(a, n, nb, x, g);
    double dev = 0, ex = 0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      dev += (double)g[i];
      if (L::e(i, 0)) ex += L::e(i, 0) > 0 ? (double)g[i] : -(double)g[i];
    }
    const double c = dev + diff_ref(a, n, x);
    const double om = (double)a.omega[n];
    const double jx = (1.0 - 0.5 * om) * ex;
    acc[0] += jx;
    acc[1] += fabs(c - prev[n]);
    acc[2] += fabs(c);
    acc[3] += c;
    acc[4] += L::cs2 * (1.0 / om - 0.5);
    if (dprev) dprev[n] = c - prev[n];
    prev[n] = c;
  }
  block_reduce_store<5>(acc, partials);
}

// Extrapolated restart (om_diff_params.accel): node n's concentration
// moves by f dC(n); the stored non-equilibrium parts stay.  Rebased storage
// moves the node's reference (every population of the node shifts by a_i
// times it, in either parity's slots); FP64 storage shifts each slot by
// a_i f dC (the weights are symmetric, so slot i and slot opposite(i) take
// the same shift).  prev follows, so the next window's change is measured
// from the new state.
template <class T, class L>
__global__ void diff_extrapolate(DiffArgs<T, L> a, double* prev, const double* dprev, double f) {
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.nf) return;
  const double dc = f * dprev[n];
  prev[n] += dc;
  if constexpr (kRebased<T>) {
    a.cr[n] = (float)((double)a.cr[n] + dc);
  } else {
    using S = Stg<T>;
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
      S::st(a.q[i] + n, S::ld(a.q[i] + n, a.down) + (typename S::C)(L::w(i) * dc), a.up);
  }
}

template <class T, class L, bool ODD>
__global__ void diff_export(DiffArgs<T, L> a, const int64_t* vox, int64_t N, double* gdense,
                            float* cdense, float* jdense) {
  using C = typename Stg<T>::C;
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.nf) return;
  uint32_t nb[L::Q];
  int x, y, z;
  unpack_xyz(a.coord[n], x, y, z);
  if (ODD) diff_neighbours(a, a.coord[n], nb, x);
  C g[L::Q];
  diff_load<T, L, ODD>(a, n, nb, x, g);
  const int64_t v = vox[n];
  const double cref = diff_ref(a, n, x);
  double dev = 0, ex = 0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    dev += (double)g[i];
    if (L::e(i, 0)) ex += L::e(i, 0) > 0 ? (double)g[i] : -(double)g[i];
    if (gdense) gdense[i * N + v] = (double)g[i] + L::w(i) * cref;
  }
  if (cdense) cdense[v] = (float)(dev + cref);
  if (jdense) jdense[v] = (float)((1.0 - 0.5 * (double)a.omega[n]) * ex);
}

// populations from the dense layout (linear != 0: the linear profile a_i C_lin);
// 16-bit storage takes the node's C as its reference
template <class T, class L>
__global__ void diff_import(DiffArgs<T, L> a, const int64_t* vox, int64_t N, const double* gdense,
                            int linear) {
  using S = Stg<T>;
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.nf) return;
  const int64_t v = vox[n];
  int x, y, z;
  unpack_xyz(a.coord[n], x, y, z);
  const double clin = a.cin + (double)a.s * ((double)x + 0.5);
  double ref = clin;
  if constexpr (kRebased<T>) {
    if (!linear) {
      ref = 0.0;
      for (int i = 0; i < L::Q; ++i) ref += gdense[i * N + v];
    }
    a.cr[n] = (float)ref;
    ref = (double)a.cr[n];
  }
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const double g = linear ? L::w(i) * clin : gdense[i * N + v];
    S::st(a.q[i] + n, (typename S::C)(g - L::w(i) * ref), a.up);
  }
}

// warm start: g_i = a_i C (deviation a_i (C - C_lin(x))) in the even layout
template <class T, class L>
__global__ void diff_init_c(DiffArgs<T, L> a, const int64_t* vox, const float* c, int64_t stride, int from_linear) {
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.nf) return;
  int x, y, z;
  unpack_xyz(a.coord[n], x, y, z);
  const double clin = a.cin + (double)a.s * ((double)x + 0.5);
  const double cv = warm_concentration((double)c[vox[n] * stride] + (from_linear ? clin : 0.0), clin, a.cin, a.cout);
  double dc;
  if constexpr (kRebased<T>) {
    a.cr[n] = (float)cv;
    dc = 0.0;
  } else {
    dc = cv - clin;
  }
#pragma unroll
  for (int i = 0; i < L::Q; ++i) Stg<T>::st(a.q[i] + n, (typename Stg<T>::C)(L::w(i) * dc), a.up);
}

template <class T, class L>
__global__ void diff_rebase(DiffArgs<T, L> a) {
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.nf) return;
  diff_rebase_node<T>(a, n);
}

template <class T>
__global__ void diff_omega(const int64_t* vox, const float* d_nm, int64_t nf, double d_ref,
                           double tau_ref, typename Stg<T>::C* omega, int* bad) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nf) return;
  // Eq. 12: tau_g = (d / d_ref)(tau_ref - 1/2) + 1/2
  const double tau = ((double)d_nm[vox[n]] / d_ref) * (tau_ref - 0.5) + 0.5;
  if (!(tau > 0.5)) atomicExch(bad, 1);
  omega[n] = (typename Stg<T>::C)(1.0 / tau);
}

}  // namespace om

using namespace om;


namespace {


inline unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// residency cap of variants 1 and 3: 8 blocks of 256 on D3Q7, 4 on D3Q19
template <class L>
constexpr int kDiffMinBlocks = L::Q == 7 ? 8 : 4;

template <class T, class L, bool ODD>
void launch_sweep_p(int variant, unsigned nb, cudaStream_t s, const DiffArgs<T, L>& a) {
  constexpr int M = kDiffMinBlocks<L>;
  switch (variant) {
    case 1: diff_sweep<T, L, ODD, M><<<nb, 256, 0, s>>>(a); break;
    case 2: {
      auto k = diff_sweep_strided<T, L, ODD, 0>;
      k<<<resident_grid(k, nb), 256, 0, s>>>(a);
      break;
    }
    case 3: {
      auto k = diff_sweep_strided<T, L, ODD, M>;
      k<<<resident_grid(k, nb), 256, 0, s>>>(a);
      break;
    }
    case 4: {
      auto k = diff_sweep_pipelined<T, L, ODD, 0>;
      k<<<resident_grid(k, nb), 256, 0, s>>>(a);
      break;
    }
    case 6:
    case 7:
    case 8:
      if (ODD && a.rec7) {
        const unsigned nbr = blocks_for((int64_t)a.nf + a.nslow);
        if (variant == 6) diff_sweep_rec<T, L, 0><<<nbr, 256, 0, s>>>(a);
        else if (variant == 7) diff_sweep_rec<T, L, M><<<nbr, 256, 0, s>>>(a);
        else {
          auto k = diff_sweep_rec_strided<T, L>;
          k<<<resident_grid(k, nbr), 256, 0, s>>>(a);
        }
        break;
      }
      [[fallthrough]];
    case 5:
      if (!ODD) {
        diff_sweep_pair<T, L><<<blocks_for((a.nf + 1) / 2), 256, 0, s>>>(a);
        break;
      }
      [[fallthrough]];
    default: diff_sweep<T, L, ODD, 0><<<nb, 256, 0, s>>>(a); break;
  }
}

template <class T, class L>
void launch_sweep(bool odd, int variant, unsigned nb, cudaStream_t s, const DiffArgs<T, L>& a) {
  if (odd) launch_sweep_p<T, L, true>(variant, nb, s, a);
  else launch_sweep_p<T, L, false>(variant, nb, s, a);
}

}  // namespace

namespace om {

template <class T>
void diff_sweep_variant(bool odd, int variant, const DiffArgs<T, D3Q7>& a, cudaStream_t s) {
  launch_sweep<T, D3Q7>(odd, variant, blocks_for(a.nf), s, a);
}

// Time each launch variant of both sweeps on a (6 even/odd pairs after a
// warm-up pair; the populations change) and keep the fastest per parity,
// unless a node set of the same size class was tuned before in this process.
template <class T, class L>
om_status diff_tuned_variants_l(const DiffArgs<T, L>& a, int precision, int V[2], cudaStream_t s) {
  const int kind = L::Q == 19 ? kTuneDiff19 : kTuneDiff7;
  if (a.nf == 0 || tuned_lookup(kind, precision, a.nf, V)) return OM_OK;
  const unsigned nb = blocks_for(a.nf);
  cudaEvent_t ev[3];
  for (auto& e : ev) OM_CUDA(cudaEventCreate(&e));
  float best[2] = {1e30f, 1e30f};
  for (int v = 0; v < kDiffVariants; ++v) {
    float tot[2] = {0.f, 0.f};
    for (int r = 0; r < 7; ++r) {
      OM_CUDA(cudaEventRecord(ev[0], s));
      launch_sweep<T, L>(false, v, nb, s, a);
      OM_CUDA(cudaEventRecord(ev[1], s));
      launch_sweep<T, L>(true, v, nb, s, a);
      OM_CUDA(cudaEventRecord(ev[2], s));
      OM_CUDA(cudaEventSynchronize(ev[2]));
      if (r == 0) continue;
      float m0 = 0.f, m1 = 0.f;
      OM_CUDA(cudaEventElapsedTime(&m0, ev[0], ev[1]));
      OM_CUDA(cudaEventElapsedTime(&m1, ev[1], ev[2]));
      tot[0] += m0;
      tot[1] += m1;
    }
    for (int p = 0; p < 2; ++p)
      if (tot[p] < best[p]) {
        best[p] = tot[p];
        V[p] = v;
      }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  tuned_store(kind, precision, a.nf, V);
  return OM_OK;
}

template <class T>
om_status diff_tuned_variants(const DiffArgs<T, D3Q7>& a, int precision, int V[2], cudaStream_t s) {
  return diff_tuned_variants_l<T, D3Q7>(a, precision, V, s);
}

#define OM_DIFF_SWEEP_API(T)                                                                      \
  template void diff_sweep_variant<T>(bool, int, const DiffArgs<T, D3Q7>&, cudaStream_t);        \
  template om_status diff_tuned_variants<T>(const DiffArgs<T, D3Q7>&, int, int*, cudaStream_t);
OM_DIFF_SWEEP_API(double)
OM_DIFF_SWEEP_API(float)
OM_DIFF_SWEEP_API(__half)
OM_DIFF_SWEEP_API(__nv_bfloat16)
#undef OM_DIFF_SWEEP_API

}  // namespace om

namespace {

// Capture K sweeps (K even, from an even time) into a CUDA graph once.
template <class T, class L>
om_status diff_capture_t(om_diff* df, int K) {
  if (df->exec && df->graph_k == K) return OM_OK;
  if (df->exec) {
    cudaGraphExecDestroy(df->exec);
    df->exec = nullptr;
  }
  if (!df->cap) OM_CUDA(cudaStreamCreateWithFlags(&df->cap, cudaStreamNonBlocking));
  DiffArgs<T, L> a = diff_args<T, L>(df);
  const unsigned nb = blocks_for(a.nf);
  cudaGraph_t g = nullptr;
  OM_CUDA(cudaStreamBeginCapture(df->cap, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < K; ++k) launch_sweep<T, L>(k & 1, df->var[k & 1], nb, df->cap, a);
  cudaError_t e = cudaStreamEndCapture(df->cap, &g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  e = cudaGraphInstantiate(&df->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
  df->graph_k = K;
  return OM_OK;
}

// Advance nsteps: whole check windows from even times replay the captured
// graph; anything else is launched one sweep at a time.
template <class T, class L>
om_status diff_steps_t(om_diff* df, int64_t nsteps, cudaStream_t s) {
  if (df->ns->nf == 0) {
    df->t += nsteps;
    return OM_OK;
  }
  DiffArgs<T, L> a = diff_args<T, L>(df);
  const unsigned nb = blocks_for(a.nf);
  const int K = df->p.check_every;
  while (nsteps > 0) {
    if (K >= 2 && !(K & 1) && !(df->t & 1) && nsteps >= K) {
      if (df->windows++ > 0) {  // the first whole window as plain launches (see om_flow)
        OM_TRY((diff_capture_t<T, L>(df, K)));
        OM_CUDA(cudaGraphLaunch(df->exec, s));
      } else {
        for (int k = 0; k < K; ++k) launch_sweep<T, L>(k & 1, df->var[k & 1], nb, s, a);
      }
      df->t += K;
      nsteps -= K;
      if (kRebased<T>) diff_rebase<T, L><<<nb, 256, 0, s>>>(a);  // once per window
      continue;
    }
    const bool odd = df->t & 1;
    launch_sweep<T, L>(odd, df->var[odd], nb, s, a);
    ++df->t;
    --nsteps;
  }
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

// Autotuner: time each launch variant of both sweeps (6 even/odd pairs after
// a warm-up pair), keep the fastest per parity (reused for later node sets of
// the same size class in this process); the caller re-initialises.
template <class T, class L>
om_status diff_tune_t(om_diff* df, cudaStream_t s) {
  if (df->ns->nf == 0) return OM_OK;
  return diff_tuned_variants_l<T, L>(diff_args<T, L>(df), df->p.precision, df->var, s);
}

template <class T, class L>
om_status diff_observe_t(om_diff* df, double* out, cudaStream_t s) {
  DiffArgs<T, L> a = diff_args<T, L>(df);
  if (df->t & 1) diff_observe<T, L, true><<<kObsBlocks, kObsThreads, 0, s>>>(a, df->prev, df->partials, df->dprev);
  else diff_observe<T, L, false><<<kObsBlocks, kObsThreads, 0, s>>>(a, df->prev, df->partials, df->dprev);
  launch_finalize(df->partials, kObsBlocks, 5, df->obs_dev, s);
  OM_CUDA(cudaGetLastError());
  OM_CUDA(cudaMemcpyAsync(df->obs_host, df->obs_dev, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
  OM_CUDA(cudaStreamSynchronize(s));
  for (int k = 0; k < 5; ++k) out[k] = df->obs_host[k];
  return OM_OK;
}

template <class T, class L>
om_status diff_extrapolate_t(om_diff* df, double f, cudaStream_t s) {
  if (df->ns->nf == 0 || !df->dprev) return OM_OK;
  DiffArgs<T, L> a = diff_args<T, L>(df);
  diff_extrapolate<T, L><<<blocks_for(a.nf), 256, 0, s>>>(a, df->prev, df->dprev, f);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

template <class T, class L>
om_status diff_export_t(const om_diff* df, double* gd, float* cd, float* jd, cudaStream_t s) {
  const om_nodeset* ns = df->ns;
  if (gd) OM_CUDA(cudaMemsetAsync(gd, 0, sizeof(double) * L::Q * ns->N, s));
  if (cd) OM_CUDA(cudaMemsetAsync(cd, 0, sizeof(float) * ns->N, s));
  if (jd) OM_CUDA(cudaMemsetAsync(jd, 0, sizeof(float) * ns->N, s));
  if (ns->nf == 0) return OM_OK;
  DiffArgs<T, L> a = diff_args<T, L>(df);
  if (df->t & 1) diff_export<T, L, true><<<blocks_for(a.nf), 256, 0, s>>>(a, ns->vox, ns->N, gd, cd, jd);
  else diff_export<T, L, false><<<blocks_for(a.nf), 256, 0, s>>>(a, ns->vox, ns->N, gd, cd, jd);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

template <class T, class L>
om_status diff_import_t(om_diff* df, const double* gd, int linear, cudaStream_t s) {
  if (df->ns->nf == 0) return OM_OK;
  DiffArgs<T, L> a = diff_args<T, L>(df);
  diff_import<T, L><<<blocks_for(a.nf), 256, 0, s>>>(a, df->ns->vox, df->ns->N, gd, linear);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

template <class T, class L>
om_status diff_init_c_t(om_diff* df, const float* c, int64_t stride, int from_linear, cudaStream_t s) {
  df->t = 0;
  if (df->ns->nf == 0) return OM_OK;
  DiffArgs<T, L> a = diff_args<T, L>(df);
  diff_init_c<T, L><<<blocks_for(a.nf), 256, 0, s>>>(a, df->ns->vox, c, stride, from_linear);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

template <class T, class L>
om_status diff_omega_t(om_diff* df, const float* d_nm, cudaStream_t s) {
  if (df->ns->nf == 0) return OM_OK;
  DevBuf<int> bad;
  OM_TRY(bad.alloc(1));
  OM_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
  diff_omega<T><<<blocks_for(df->ns->nf), 256, 0, s>>>(df->ns->vox, d_nm, df->ns->nf, df->p.d_ref_nm,
                                                       df->p.tau_ref, (typename Stg<T>::C*)df->omega,
                                                       bad.p);
  OM_CUDA(cudaGetLastError());
  int hb = 0;
  OM_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  OM_CUDA(cudaStreamSynchronize(s));
  if (hb) return fail(OM_EINVAL, "om_diff_create: a node has a pore size <= 0 (tau_g <= 1/2)");
  return OM_OK;
}

#define OM_DIFF_DISPATCH_L(df, L, fn, ...)                                   \
  switch ((df)->p.precision) {                                               \
    case OM_F64: return fn<double, L>(__VA_ARGS__);                          \
    case OM_F32: return fn<float, L>(__VA_ARGS__);                           \
    case OM_F16DEV: return fn<__half, L>(__VA_ARGS__);                       \
    case OM_BF16DEV: return fn<__nv_bfloat16, L>(__VA_ARGS__);               \
    default: return fail(OM_EINVAL, "unknown precision");                    \
  }
#define OM_DIFF_DISPATCH(df, fn, ...)                                        \
  if ((df)->q == 19) {                                                       \
    OM_DIFF_DISPATCH_L(df, D3Q19, fn, __VA_ARGS__)                           \
  } else {                                                                   \
    OM_DIFF_DISPATCH_L(df, D3Q7, fn, __VA_ARGS__)                            \
  }

size_t storage_bytes(int prec) { return prec == OM_F64 ? 8 : (prec == OM_F32 ? 4 : 2); }

template <class T, class L>
om_status diff_rebase_t(om_diff* df, cudaStream_t s) {
  if (!kRebased<T> || df->ns->nf == 0) return OM_OK;
  DiffArgs<T, L> a = diff_args<T, L>(df);
  diff_rebase<T, L><<<blocks_for(a.nf), 256, 0, s>>>(a);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

om_status diff_observe_any(om_diff* df, double* out, cudaStream_t s) {
  OM_DIFF_DISPATCH(df, diff_observe_t, df, out, s);
}

}  // namespace

om_status om::diff_rebase_any(om_diff* df, cudaStream_t s) { OM_DIFF_DISPATCH(df, diff_rebase_t, df, s); }

extern "C" om_status om_diff_create(const om_nodeset* ns, const float* d_nm_dev,
                                    const om_diff_params* p, void* stream, om_diff** out) {
  if (!ns || !d_nm_dev || !p || !out) return fail(OM_EINVAL, "om_diff_create: null pointer");
  if (p->precision < OM_F64 || p->precision > OM_BF16DEV)
    return fail(OM_EINVAL, "om_diff_create: unknown precision");
  if (p->layout == OM_LAYOUT_DENSE)
    return fail(OM_EINVAL, "om_diff_create: solver objects use the sparse layout (the dense one is om_solve_knudsen's)");
  if (!(p->d_ref_nm > 0.0) || !(p->tau_ref > 0.5) || !(p->c_in != p->c_out))
    return fail(OM_EINVAL, "om_diff_create: need d_ref > 0, tau_ref > 1/2, c_in != c_out");
  if (p->lattice != 7 && p->lattice != 19) return fail(OM_EINVAL, "om_diff_create: lattice must be 7 or 19");
  if (p->accel != OM_ACCEL_NONE && p->accel != OM_ACCEL_EXTRAPOLATE)
    return fail(OM_EINVAL, "om_diff_create: unknown accel");
  cudaStream_t s = as_stream(stream);
  om_diff* df = new om_diff();
  df->ns = ns;
  df->p = *p;
  df->q = p->lattice;
  df->up = p->precision == OM_F16DEV ? 64.0 : 1.0;  // FP16: keep deviations normal numbers
  const size_t cb = p->precision == OM_F64 ? 8 : 4;
  DevBuf<uint8_t> g, om;
  DevBuf<double> prev, part, obs;
  DevBuf<float> cr;
  om_status st = g.alloc((size_t)df->q * ns->pitch * storage_bytes(p->precision));
  if (st == OM_OK && storage_bytes(p->precision) <= 4) st = cr.alloc(ns->pitch);
  if (st == OM_OK) st = om.alloc((size_t)ns->pitch * cb);
  if (st == OM_OK) st = prev.alloc(ns->nf);
  DevBuf<double> dprev;
  if (st == OM_OK && p->accel == OM_ACCEL_EXTRAPOLATE) st = dprev.alloc(ns->nf);
  if (st == OM_OK) st = part.alloc((size_t)kObsBlocks * 8);
  if (st == OM_OK) st = obs.alloc(8);
  double* host = nullptr;
  if (st == OM_OK && cudaMallocHost((void**)&host, 8 * sizeof(double)) != cudaSuccess) {
    (void)cudaGetLastError();
    st = fail(OM_ENOMEM, "om_diff_create: pinned allocation failed");
  }
  if (st != OM_OK) {
    delete df;
    return st;
  }
  df->g = g.take();
  df->omega = om.take();
  df->cr = cr.take();
  df->prev = prev.take();
  df->dprev = p->accel == OM_ACCEL_EXTRAPOLATE ? dprev.take() : nullptr;
  df->partials = part.take();
  df->obs_dev = obs.take();
  df->obs_host = host;
  auto setup = [&]() -> om_status { OM_DIFF_DISPATCH(df, diff_omega_t, df, d_nm_dev, s); };
  auto init = [&]() -> om_status { OM_DIFF_DISPATCH(df, diff_import_t, df, nullptr, 1, s); };
  auto tune = [&]() -> om_status { OM_DIFF_DISPATCH(df, diff_tune_t, df, s); };
  if (p->variant >= 0) df->var[0] = df->var[1] = std::min(p->variant, kDiffVariants - 1);
  st = setup();
  if (st == OM_OK) st = init();
  if (st == OM_OK && p->variant < 0) {
    st = tune();
    if (st == OM_OK) st = init();  // back to the linear profile
  }
  if (st == OM_OK) {
    double o[5];
    st = diff_observe_any(df, o, s);
  }
  if (st != OM_OK) {
    om_diff_destroy(df);
    return st;
  }
  *out = df;
  return OM_OK;
}

extern "C" om_status om_diff_step(om_diff* df, int64_t nsteps, void* stream) {
  if (!df || nsteps < 0) return fail(OM_EINVAL, "om_diff_step: bad argument");
  cudaStream_t s = as_stream(stream);
  OM_DIFF_DISPATCH(df, diff_steps_t, df, nsteps, s);
}

extern "C" om_status om_diff_observe(om_diff* df, double* out, void* stream) {
  if (!df || !out) return fail(OM_EINVAL, "om_diff_observe: null pointer");
  return diff_observe_any(df, out, as_stream(stream));
}

extern "C" om_status om_diff_solve(om_diff* df, double* D_eff_lattice, om_run_info* info,
                                   void* stream) {
  if (!df) return fail(OM_EINVAL, "om_diff_solve: null pointer");
  const om_diff_params& p = df->p;
  if (p.check_every <= 0 || (p.check_every & 1))
    return fail(OM_EINVAL, "om_diff_solve: check_every must be a positive even number");
  cudaStream_t s = as_stream(stream);
  cudaEvent_t e0, e1;
  OM_CUDA(cudaEventCreate(&e0));
  OM_CUDA(cudaEventCreate(&e1));
  double o[5];
  OM_TRY(diff_observe_any(df, o, s));
  double sj_prev = o[0];
  const int64_t t0 = df->t;
  OM_CUDA(cudaEventRecord(e0, s));
  om_status rc = OM_ENOTCONVERGED;
  double rel = 1.0;
  bool diverged = false;
  ExtrapolationTrack track;
  while (df->t - t0 < p.max_steps) {
    int64_t k = std::min<int64_t>(p.check_every, p.max_steps - (df->t - t0));
    OM_TRY(om_diff_step(df, k, stream));
    OM_TRY(diff_observe_any(df, o, s));
    // converged when both the concentration field and the total flux have
    // settled: C can sit at its final profile while the flux still relaxes
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
    if (df->dprev) {
      const double f = track.observe(o[1]);
      if (f > 0.0) {
        auto ex = [&]() -> om_status { OM_DIFF_DISPATCH(df, diff_extrapolate_t, df, std::min(f, 1e3), s); };
        OM_TRY(ex());
      }
    }
  }
  OM_CUDA(cudaEventRecord(e1, s));
  OM_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  OM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const om_nodeset* ns = df->ns;
  if (D_eff_lattice)
    *D_eff_lattice = (o[0] / (double)ns->N) * (double)ns->dom.nx / (p.c_in - p.c_out);
  if (info) {
    info->steps = df->t - t0;
    info->n_nodes = ns->nf;
    info->rel_change = rel;
    info->mass = o[3];
    info->seconds = ms * 1e-3;
    info->mlups = ms > 0 ? (double)ns->nf * (double)info->steps / (ms * 1e-3) / 1e6 : 0.0;
  }
  if (diverged) set_error("om_diff_solve: the populations diverged (non-finite concentration sums)");
  else if (rc != OM_OK) set_error("om_diff_solve: step cap reached before convergence");
  return rc;
}

extern "C" om_status om_diff_get_populations(const om_diff* df, double* g_dev, void* stream) {
  if (!df || !g_dev) return fail(OM_EINVAL, "om_diff_get_populations: null pointer");
  cudaStream_t s = as_stream(stream);
  OM_DIFF_DISPATCH(df, diff_export_t, df, g_dev, (float*)nullptr, (float*)nullptr, s);
}

extern "C" om_status om_diff_get_fields(const om_diff* df, float* c_dev, float* jx_dev, void* stream) {
  if (!df) return fail(OM_EINVAL, "om_diff_get_fields: null pointer");
  cudaStream_t s = as_stream(stream);
  OM_DIFF_DISPATCH(df, diff_export_t, df, (double*)nullptr, c_dev, jx_dev, s);
}

extern "C" om_status om_diff_set_populations(om_diff* df, const double* g_dev, void* stream) {
  if (!df || !g_dev) return fail(OM_EINVAL, "om_diff_set_populations: null pointer");
  cudaStream_t s = as_stream(stream);
  df->t = 0;
  auto imp = [&]() -> om_status { OM_DIFF_DISPATCH(df, diff_import_t, df, g_dev, 0, s); };
  OM_TRY(imp());
  double o[5];
  return diff_observe_any(df, o, s);
}

extern "C" om_status om_diff_init_concentration(om_diff* df, const float* c_dev, int64_t stride, int32_t from_linear,
                                                void* stream) {
  if (!df || !c_dev || stride < 1) return fail(OM_EINVAL, "om_diff_init_concentration: bad argument");
  cudaStream_t s = as_stream(stream);
  auto init = [&]() -> om_status { OM_DIFF_DISPATCH(df, diff_init_c_t, df, c_dev, stride, from_linear, s); };
  OM_TRY(init());
  double o[5];
  return diff_observe_any(df, o, s);
}

extern "C" om_status om_diff_time(const om_diff* df, int64_t* t) {
  if (!df || !t) return fail(OM_EINVAL, "om_diff_time: null pointer");
  *t = df->t;
  return OM_OK;
}

extern "C" om_status om_diff_destroy(om_diff* df) {
  if (!df) return OM_OK;
  if (df->exec) cudaGraphExecDestroy(df->exec);
  if (df->cap) cudaStreamDestroy(df->cap);
  cudaFree(df->g);
  cudaFree(df->omega);
  cudaFree(df->cr);
  cudaFree(df->prev);
  cudaFree(df->dprev);
  cudaFree(df->partials);
  cudaFree(df->obs_dev);
  if (df->obs_host) cudaFreeHost(df->obs_host);
  delete df;
  return OM_OK;
}
