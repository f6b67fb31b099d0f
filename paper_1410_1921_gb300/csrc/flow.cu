// flow.cu -- D3Q19 flow sweep (Sec. 3.1, Eqs. 1-9, App. A) in the AA
// pattern on the fluid-node layout of nodeset.cu.
//
// Collision.  The moment-space MRT of Eqs. 4-7 relaxes every even
// non-conserved moment of the App. A basis with 1/tau and every odd one with
// s_q = 8(2 tau - 1)/(8 tau - 1); its equilibrium moments A1-A9 are the
// moments of the incompressible BGK equilibrium of Eq. 3.  That operator is
// the two-relaxation-time collision
//     f*_i = f_i - w+ (f+_i - e+_i) - w- (f-_i - e-_i) + (1 - w-/2) F_i
// with w+ = 1/tau, w- = s_q, f+-, e+- the symmetric / antisymmetric parts
// of f and f_eq under i -> opposite(i), and the body force g along x entering
// as j* = j + g/2 in f_eq and F_i = 3 w_i e_ix g.  Written per velocity pair
// it costs ~200 flops per node instead of two dense 19x19 products.
// Populations are stored as deviations f_i - w_i (rho0 = 1).
//
// Streaming, AA pattern.  Even steps read and write only the node's own
// slots (post-collision f*_i goes to slot opposite(i)); odd steps read
// slot opposite(i) of the upstream node x - e_i and write slot i of the
// downstream node x + e_i.  Every slot is read and written by one thread
// only, so one population array serves both steps.  A missing neighbour
// (solid or non-transport voxel) is halfway bounce-back: the odd step reads
// the node's own slot i and writes its own slot opposite(i).  x, y and z
// are periodic (body-force driving).
//
// Pressure drive (Sec. 3.3, om_flow_params.drive = OM_DRIVE_PRESSURE).  x
// is not periodic and no force acts; the nodes of the layers x = 0 and
// x = nx - 1 carry densities 1 +- delta_rho/2 by the non-equilibrium
// extrapolation of Guo et al.: before every sweep a boundary kernel forms,
// for each such node b with inward neighbours b1, b2,
//     f_i(b) = f_i^eq(rho_b, u_b) + f_i(b1) - f_i^eq(rho(b1), u(b1)),
// u_b = 2 u(b1) - u(b2) (u(b1) without b2; f^eq(rho_b, 0) without b1), from
// the pre-collision populations of b1 and b2 (their own slots at even times,
// gathered from their neighbours at odd times), into a side buffer that the
// sweep reads in place of b's own populations.  The sweep writes nothing the
// boundary kernel reads, so the two never race.
#include <algorithm>
#include <cmath>

#include "solvers.cuh"

namespace om {

// Launch variants (chosen per parity by the autotuner of om_flow_create),
// all doing identical arithmetic:
//   0  one thread per node, registers left to the compiler;
//   1  one thread per node, registers capped so MINB blocks of 256 threads
//      stay resident per SM (more latency hiding, a few spills);
//   2  a grid of resident blocks only, each thread striding over nodes and
//      loading the next node's coordinates before updating the current one,
//      so that load's latency overlaps the update (odd steps);
//   3  variant 2 with the register cap of variant 1;
//   4  one thread per node with a tighter cap (MINB + 1 blocks);
//   5  variant 2 two nodes deep: the coordinates of the node after next are
//      loaded, and the column-map words of the next node prefetched into
//      L1, while the current node is updated (odd steps);
//   6  even steps: two consecutive nodes per thread, each population of both
//      loaded and stored as one vector of two (twice the bytes per load
//      instruction and per register in flight, which the 16-bit formats
//      need to approach the bandwidth roofline); odd steps as variant 0;
//   7  odd steps from the neighbour records (lattice.cuh): one thread per
//      node reads its two record words and derives its 18 neighbours' node
//      numbers with integer adds, no column-map lookup between the record
//      and the population loads; the slow nodes (faces of the box) follow
//      in the same grid, one thread each, through the column map; even
//      steps as variant 6;
//   8  variant 7 with the register cap of variant 1;
//   9  variant 7 on a resident grid whose threads stride over the nodes
//      (then the slow list) and load the next node's records before
//      updating the current one.
//   Without records (a box beyond their fields) 7-9 run as 6.
// (Odd steps of two nodes per thread, a grid apart, with both lookups and
// all 38 loads issued before either update, were measured slower than
// variant 2: the registers they need halve the resident threads.)
template <class T>
constexpr int kMinBlocks1 = sizeof(T) == 8 ? 3 : 4;

constexpr int kSweepVariants = 13;

template <class T, bool ODD, int MINB>
__global__ void __launch_bounds__(256, MINB) d3q19_sweep(FlowArgs<T> a) {
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.nf) return;
  flow_node<T, ODD>(a, n, n);
}

template <class T, bool ODD, int MINB>
__global__ void __launch_bounds__(256, MINB) d3q19_sweep_strided(FlowArgs<T> a) {
  const uint32_t stride = gridDim.x * blockDim.x;
  uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.nf) return;
  uint32_t c = ODD ? __ldg(a.coord + n) : 0u;
  for (;;) {
    const uint64_t nn = (uint64_t)n + stride;
    const bool more = nn < a.nf;
    uint32_t cn = 0u;
    if (ODD && more) cn = __ldg(a.coord + nn);
    flow_node_at<T, ODD>(a, n, c);
    if (!more) break;
    n = (uint32_t)nn;
    c = cn;
  }
}

template <class T, bool ODD, int MINB>
__global__ void __launch_bounds__(256, MINB) d3q19_sweep_pipelined(FlowArgs<T> a) {
  const uint32_t stride = gridDim.x * blockDim.x;
  uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.nf) return;
  if (!ODD) {
    for (; n < a.nf; n += stride) flow_node_at<T, false>(a, n, 0u);
    return;
  }
  uint32_t c0 = __ldg(a.coord + n);
  uint32_t c1 = (uint64_t)n + stride < a.nf ? __ldg(a.coord + n + stride) : 0u;
  for (;;) {
    const uint64_t nn = (uint64_t)n + stride, nn2 = nn + stride;
    const uint32_t c2 = nn2 < a.nf ? __ldg(a.coord + nn2) : 0u;
    if (nn < a.nf) prefetch_columns<19>(a.col, a.nx, a.ny, a.W, a.px, c1);
    flow_node_at<T, true>(a, n, c0);
    if (nn >= a.nf) break;
    n = (uint32_t)nn;
    c0 = c1;
    c1 = c2;
  }
}

// Odd step of node t from its records, or of slow node slow[t - nf]
template <class T>
__device__ __forceinline__ void flow_odd_rec(const FlowArgs<T>& a, uint32_t t, uint2 r, uint2 q) {
  if (t < a.nf) {
    if (rec_slow(r)) return;  // updated from the slow list
    uint32_t nb[19];
    rec_neighbours19(r, q, t, nb);
    flow_node_nb<T, true>(a, t, nb);
  } else {
    const uint32_t n = __ldg(a.slow + (t - a.nf));
    flow_node_at<T, true>(a, n, __ldg(a.coord + n));
  }
}

// Odd step of a record node with nothing but its populations held across
// the collision: the neighbours (and, for rebased storage, their reference
// densities) are taken from the records before the loads, and again after
// the collision for the stores (variants 10-12; the slow nodes run as their
// own launch, d3q19_sweep_slow, so that the column-map code sets no
// register budget here).
template <class T>
__device__ __forceinline__ void flow_odd_rec_lean(const FlowArgs<T>& a, uint32_t n, uint2 r, uint2 q) {
  using C = typename Stg<T>::C;
  C f[19];
  float rn = 0.f;
  if constexpr (kFlowRebased<T>) rn = a.rr[n];
  {
    uint32_t nb[19];
    rec_neighbours19(r, q, n, nb);
    f[0] = Stg<T>::ld(a.s[0] + n, a.down);
#pragma unroll
    for (int i = 1; i < 19; ++i) {
      const uint32_t o = (uint32_t)q19_opp(i), src = nb[o];
      const uint32_t off = src != kNoNode ? o * a.P + src : (uint32_t)i * a.P + n;
      f[i] = Stg<T>::ld(a.s[0] + off, a.down);
      if constexpr (kFlowRebased<T>)
        if (src != kNoNode) f[i] += (float)q19_w(i) * (a.rr[src] - rn);
    }
  }
  flow_collide(a, n, f);
  order_after(f[16], f[17]);
  asm volatile("" : "+r"(r.x), "+r"(r.y), "+r"(q.x), "+r"(q.y), "+r"(n));
  {
    uint32_t nb[19];
    rec_neighbours19(r, q, n, nb);
    Stg<T>::st(a.s[0] + n, f[0], a.up);
#pragma unroll
    for (int i = 1; i < 19; ++i) {
      const uint32_t dst = nb[i];
      const uint32_t off = dst != kNoNode ? (uint32_t)i * a.P + dst : (uint32_t)q19_opp(i) * a.P + n;
      C v = f[i];
      if constexpr (kFlowRebased<T>)
        if (dst != kNoNode) v -= (float)q19_w(i) * (a.rr[dst] - rn);
      Stg<T>::st(a.s[0] + off, v, a.up);
    }
  }
}

template <class T, int MINB>
__global__ void __launch_bounds__(256, MINB) d3q19_sweep_rec_lean(FlowArgs<T> a) {
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.nf) return;
  const uint2 r = __ldg(a.rec7 + n);
  if (rec_slow(r)) return;
  flow_odd_rec_lean<T>(a, n, r, __ldg(a.rec19 + n));
}

template <class T>
__global__ void __launch_bounds__(256) d3q19_sweep_slow(FlowArgs<T> a) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.nslow) return;
  const uint32_t n = __ldg(a.slow + t);
  flow_node_at<T, true>(a, n, __ldg(a.coord + n));
}

template <class T, int MINB>
__global__ void __launch_bounds__(256, MINB) d3q19_sweep_rec(FlowArgs<T> a) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.nf + a.nslow) return;
  uint2 r = make_uint2(0u, 0u), q = make_uint2(0u, 0u);
  if (t < a.nf) {
    r = __ldg(a.rec7 + t);
    q = __ldg(a.rec19 + t);
  }
  flow_odd_rec<T>(a, t, r, q);
}

template <class T>
__global__ void __launch_bounds__(256) d3q19_sweep_rec_strided(FlowArgs<T> a) {
  const uint32_t stride = gridDim.x * blockDim.x, total = a.nf + a.nslow;
  uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  uint2 r = make_uint2(0u, 0u), q = make_uint2(0u, 0u);
  if (t < a.nf) {
    r = __ldg(a.rec7 + t);
    q = __ldg(a.rec19 + t);
  }
  for (;;) {
    const uint64_t tn = (uint64_t)t + stride;
    uint2 rn = make_uint2(0u, 0u), qn = make_uint2(0u, 0u);
    if (tn < a.nf) {
      rn = __ldg(a.rec7 + tn);
      qn = __ldg(a.rec19 + tn);
    }
    flow_odd_rec<T>(a, t, r, q);
    if (tn >= total) break;
    t = (uint32_t)tn;
    r = rn;
    q = qn;
  }
}

template <class T>
__global__ void __launch_bounds__(256) d3q19_sweep_pair(FlowArgs<T> a) {
  const uint32_t n = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (n >= a.nf) return;
  if (n + 1 == a.nf) flow_node_at<T, false>(a, n, 0u);
  else flow_pair_even<T>(a, n);
}

// Observables (FP64, fixed grid): sum u_x, sum |u_x - prev|, sum |u_x|,
// sum rho-1; prev <- u_x.
template <class T, bool ODD>
__global__ void __launch_bounds__(kObsThreads) d3q19_observe(FlowArgs<T> a, double* prev,
                                                             double* partials) {
  using C = typename Stg<T>::C;
  double acc[4] = {0, 0, 0, 0};
  for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < a.nf; n += gridDim.x * blockDim.x) {
    uint32_t nb[19];
    if (ODD) flow_neighbours(a, a.coord[n], nb);
    C f[19];
    flow_load<T, ODD>(a, n, nb, f);
    double rho = 0, jx = 0;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
      rho += (double)f[i];
      jx += (double)q19_e(i, 0) * (double)f[i];
    }
    const double ux = jx + 0.5 * (double)a.g;
    acc[3] += rho + flow_ref(a, n);
    if (flow_boundary_index(a, n) >= 0) continue;  // pressure drive: velocity sums over interior layers
    acc[0] += ux;
    acc[1] += fabs(ux - prev[n]);
    acc[2] += fabs(ux);
    prev[n] = ux;
  }
  block_reduce_store<4>(acc, partials);
}

template <class T, bool ODD>
__global__ void d3q19_export(FlowArgs<T> a, const int64_t* vox, int64_t N, double* fdense,
                             float* udense) {
  using C = typename Stg<T>::C;
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.nf) return;
  uint32_t nb[19];
  if (ODD) flow_neighbours(a, a.coord[n], nb);
  C f[19];
  flow_load<T, ODD>(a, n, nb, f);
  const int64_t v = vox[n];
  if (fdense) {
    const double r1 = 1.0 + flow_ref(a, n);
#pragma unroll
    for (int i = 0; i < 19; ++i) fdense[i * N + v] = (double)f[i] + q19_w(i) * r1;
  }
  if (udense) {
    double jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
      jx += (double)q19_e(i, 0) * (double)f[i];
      jy += (double)q19_e(i, 1) * (double)f[i];
      jz += (double)q19_e(i, 2) * (double)f[i];
    }
    udense[v] = (float)(jx + 0.5 * (double)a.g);
    udense[N + v] = (float)jy;
    udense[2 * N + v] = (float)jz;
  }
}

template <class T>
__global__ void d3q19_import(FlowArgs<T> a, const int64_t* vox, int64_t N, const double* fdense) {
  using S = Stg<T>;
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.nf) return;
  const int64_t v = vox[n];
  if constexpr (kFlowRebased<T>) a.rr[n] = 0.f;
#pragma unroll
  for (int i = 0; i < 19; ++i) S::st(a.s[i] + n, (typename S::C)(fdense[i * N + v] - q19_w(i)), a.up);
}

// warm start: f_i = f_eq(rho = 1, u = (ux, 0, 0)) in the even layout
template <class T>
__global__ void d3q19_init_u(FlowArgs<T> a, const int64_t* vox, const float* ux, int64_t stride, double scale) {
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.nf) return;
  const double u = warm_velocity(scale * (double)ux[vox[n] * stride]);
  if constexpr (kFlowRebased<T>) a.rr[n] = 0.f;
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const double eu = (double)q19_e(i, 0) * u;
    Stg<T>::st(a.s[i] + n, (typename Stg<T>::C)(q19_w(i) * (3.0 * eu + 4.5 * eu * eu - 1.5 * u * u)), a.up);
  }
}

// Pressure drive: the extrapolated pre-collision deviations of every
// boundary node into bc (Sec. 3.3; see the file comment).  Deviations from
// w_i: f_i^eq - w_i = w_i (rho - 1 + 3 e_i.j + 4.5 (e_i.j)^2 - 1.5 j.j).
template <class C>
__device__ __forceinline__ C feq19_dev(int i, C drho, C jx, C jy, C jz) {
  const C eu = C(q19_e(i, 0)) * jx + C(q19_e(i, 1)) * jy + C(q19_e(i, 2)) * jz;
  return C(q19_w(i)) * (drho + C(3) * eu + C(4.5) * eu * eu - C(1.5) * (jx * jx + jy * jy + jz * jz));
}

template <class T, bool ODD>
__device__ __forceinline__ void flow_moments_at(const FlowArgs<T>& a, uint32_t n, typename Stg<T>::C (&f)[19],
                                                typename Stg<T>::C& r, typename Stg<T>::C (&j)[3]) {
  using C = typename Stg<T>::C;
  uint32_t nb[19];
  if (ODD) flow_neighbours(a, a.coord[n], nb);
  flow_load<T, ODD>(a, n, nb, f);
  r = 0;
  j[0] = j[1] = j[2] = 0;
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    r += f[i];
    j[0] += C(q19_e(i, 0)) * f[i];
    j[1] += C(q19_e(i, 1)) * f[i];
    j[2] += C(q19_e(i, 2)) * f[i];
  }
}

template <class T, bool ODD>
__global__ void d3q19_pressure_bc(FlowArgs<T> a, typename Stg<T>::C* bc, double drho_in, double drho_out) {
  using C = typename Stg<T>::C;
  const uint32_t nbt = a.n_in + a.n_out;
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nbt) return;
  const uint32_t b = k < a.n_in ? k : a.nf - a.n_out + (k - a.n_in);
  int x, y, z;
  unpack_xyz(a.coord[b], x, y, z);
  const int dir = x == 0 ? 1 : -1;
  const C drb = (C)(x == 0 ? drho_in : drho_out);
  const uint32_t b1 = node_at(a.col, a.ny, a.W, x + dir, y, z);
  C out[19];
  if (b1 == kNoNode) {
#pragma unroll
    for (int i = 0; i < 19; ++i) out[i] = feq19_dev<C>(i, drb, C(0), C(0), C(0));
  } else {
    C f1[19], r1, j1[3], ub[3];
    flow_moments_at<T, ODD>(a, b1, f1, r1, j1);
    const uint32_t b2 = node_at(a.col, a.ny, a.W, x + 2 * dir, y, z);
    if (b2 != kNoNode) {
      C f2[19], r2, j2[3];
      flow_moments_at<T, ODD>(a, b2, f2, r2, j2);
      for (int d = 0; d < 3; ++d) ub[d] = C(2) * j1[d] - j2[d];
    } else {
      for (int d = 0; d < 3; ++d) ub[d] = j1[d];
    }
#pragma unroll
    for (int i = 0; i < 19; ++i)
      out[i] = feq19_dev<C>(i, drb, ub[0], ub[1], ub[2]) + (f1[i] - feq19_dev<C>(i, r1, j1[0], j1[1], j1[2]));
  }
#pragma unroll
  for (int i = 0; i < 19; ++i) bc[(size_t)i * nbt + k] = out[i];
}

template <class T>
__global__ void d3q19_rest(FlowArgs<T> a) {
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.nf) return;
  if constexpr (kFlowRebased<T>) a.rr[n] = 0.f;
#pragma unroll
  for (int i = 0; i < 19; ++i) Stg<T>::st(a.s[i] + n, 0, a.up);
}

// rebased storage: every node's reference moved to its current density
// (even time), once per check window
template <class T>
__global__ void d3q19_rebase(FlowArgs<T> a) {
  const uint32_t n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= a.nf) return;
  flow_rebase_node<T>(a, n);
}

}  // namespace om

using namespace om;


namespace {



inline unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

template <class T, bool ODD>
void launch_sweep_p(int variant, unsigned nb, cudaStream_t s, const FlowArgs<T>& a) {
  constexpr int M = kMinBlocks1<T>;
  switch (variant) {
    case 1: d3q19_sweep<T, ODD, M><<<nb, 256, 0, s>>>(a); break;
    case 2: {
      auto k = d3q19_sweep_strided<T, ODD, 0>;
      k<<<resident_grid(k, nb), 256, 0, s>>>(a);
      break;
    }
    case 3: {
      auto k = d3q19_sweep_strided<T, ODD, M>;
      k<<<resident_grid(k, nb), 256, 0, s>>>(a);
      break;
    }
    case 4: d3q19_sweep<T, ODD, M + 1><<<nb, 256, 0, s>>>(a); break;
    case 5: {
      auto k = d3q19_sweep_pipelined<T, ODD, 0>;
      k<<<resident_grid(k, nb), 256, 0, s>>>(a);
      break;
    }
    case 7:
    case 8:
    case 9:
    case 10:
    case 11:
    case 12:
      if (ODD && a.rec7) {
        const unsigned nbr = blocks_for((int64_t)a.nf + a.nslow);
        if (variant >= 10) {
          if (variant == 10) d3q19_sweep_rec_lean<T, 0><<<nb, 256, 0, s>>>(a);
          else if (variant == 11) d3q19_sweep_rec_lean<T, M><<<nb, 256, 0, s>>>(a);
          else d3q19_sweep_rec_lean<T, M - 1><<<nb, 256, 0, s>>>(a);
          if (a.nslow) d3q19_sweep_slow<T><<<blocks_for(a.nslow), 256, 0, s>>>(a);
        } else if (variant == 7) d3q19_sweep_rec<T, 0><<<nbr, 256, 0, s>>>(a);
        else if (variant == 8) d3q19_sweep_rec<T, M><<<nbr, 256, 0, s>>>(a);
        else {
          auto k = d3q19_sweep_rec_strided<T>;
          k<<<resident_grid(k, nbr), 256, 0, s>>>(a);
        }
        break;
      }
      [[fallthrough]];
    case 6:
      if (!ODD) {
        d3q19_sweep_pair<T><<<blocks_for((a.nf + 1) / 2), 256, 0, s>>>(a);
        break;
      }
      [[fallthrough]];
    default: d3q19_sweep<T, ODD, 0><<<nb, 256, 0, s>>>(a); break;
  }
}

template <class T>
void launch_sweep(bool odd, int variant, unsigned nb, cudaStream_t s, const FlowArgs<T>& a) {
  if (odd) launch_sweep_p<T, true>(variant, nb, s, a);
  else launch_sweep_p<T, false>(variant, nb, s, a);
}

}  // namespace

namespace om {

template <class T>
void flow_sweep_variant(bool odd, int variant, const FlowArgs<T>& a, cudaStream_t s) {
  launch_sweep<T>(odd, variant, blocks_for(a.nf), s, a);
}

// Time every launch variant of both sweeps on a (6 even/odd pairs each after
// a warm-up pair; the populations change) and keep the fastest per parity,
// unless a node set of the same size class was tuned before in this process.
template <class T>
om_status flow_tuned_variants(const FlowArgs<T>& a, int precision, int V[2], cudaStream_t s, bool* timed) {
  const int kind = kFlowRebased<T> ? kTuneFlowReb : kTuneFlow;
  if (timed) *timed = false;
  if (a.nf == 0 || tuned_lookup(kind, precision, a.nf, V)) return OM_OK;
  const unsigned nb = blocks_for(a.nf);
  cudaEvent_t ev[3];
  for (auto& e : ev) OM_CUDA(cudaEventCreate(&e));
  float best[2] = {1e30f, 1e30f};
  for (int v = 0; v < kSweepVariants; ++v) {
    float tot[2] = {0.f, 0.f};
    for (int r = 0; r < 7; ++r) {
      OM_CUDA(cudaEventRecord(ev[0], s));
      launch_sweep<T>(false, v, nb, s, a);
      OM_CUDA(cudaEventRecord(ev[1], s));
      launch_sweep<T>(true, v, nb, s, a);
      OM_CUDA(cudaEventRecord(ev[2], s));
      OM_CUDA(cudaEventSynchronize(ev[2]));
      if (r == 0) continue;  // warm-up pair
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
  if (timed) *timed = true;
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

#define OM_FLOW_SWEEP_API(T)                                                                       \
  template void flow_sweep_variant<T>(bool, int, const FlowArgs<T>&, cudaStream_t);               \
  template om_status flow_tuned_variants<T>(const FlowArgs<T>&, int, int*, cudaStream_t, bool*);
OM_FLOW_SWEEP_API(double)
OM_FLOW_SWEEP_API(float)
OM_FLOW_SWEEP_API(__half)
OM_FLOW_SWEEP_API(__nv_bfloat16)
OM_FLOW_SWEEP_API(Reb<float>)
OM_FLOW_SWEEP_API(Reb<__half>)
OM_FLOW_SWEEP_API(Reb<__nv_bfloat16>)
#undef OM_FLOW_SWEEP_API

}  // namespace om

namespace {

// One LB step: the pressure boundary kernel (pressure drive) and the sweep.
template <class T>
void launch_step(const om_flow* fl, bool odd, int variant, unsigned nb, cudaStream_t s, const FlowArgs<T>& a) {
  const uint32_t nbt = a.n_in + a.n_out;
  if (nbt) {
    using C = typename Stg<T>::C;
    const double h = 0.5 * fl->p.delta_rho;
    if (odd) d3q19_pressure_bc<T, true><<<(nbt + 127) / 128, 128, 0, s>>>(a, (C*)fl->bc, h, -h);
    else d3q19_pressure_bc<T, false><<<(nbt + 127) / 128, 128, 0, s>>>(a, (C*)fl->bc, h, -h);
  }
  launch_sweep<T>(odd, variant, nb, s, a);
}

// launch variants of the storage mode T
template <class T>
int* flow_var(om_flow* fl) {
  return kFlowRebased<T> ? fl->varr : fl->var;
}

// Capture K sweeps (K even, from an even time) into a CUDA graph once.
template <class T>
om_status flow_capture_t(om_flow* fl, int K) {
  if (fl->exec && fl->graph_k == K && fl->graph_reb == kFlowRebased<T>) return OM_OK;
  if (fl->exec) {
    cudaGraphExecDestroy(fl->exec);
    fl->exec = nullptr;
  }
  if (!fl->cap) OM_CUDA(cudaStreamCreateWithFlags(&fl->cap, cudaStreamNonBlocking));
  FlowArgs<T> a = flow_args<T>(fl);
  const unsigned nb = blocks_for(a.nf);
  cudaGraph_t g = nullptr;
  OM_CUDA(cudaStreamBeginCapture(fl->cap, cudaStreamCaptureModeThreadLocal));
  const int* V = flow_var<T>(fl);
  for (int k = 0; k < K; ++k) launch_step<T>(fl, k & 1, V[k & 1], nb, fl->cap, a);
  cudaError_t e = cudaStreamEndCapture(fl->cap, &g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  e = cudaGraphInstantiate(&fl->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
  fl->graph_k = K;
  fl->graph_reb = kFlowRebased<T>;
  return OM_OK;
}

// Advance nsteps: whole check windows from even times replay the captured
// graph; anything else is launched one sweep at a time.
template <class T>
om_status flow_steps_t(om_flow* fl, int64_t nsteps, cudaStream_t s) {
  if (fl->ns->nf == 0) {
    fl->t += nsteps;
    return OM_OK;
  }
  FlowArgs<T> a = flow_args<T>(fl);
  const unsigned nb = blocks_for(a.nf);
  const int K = fl->p.check_every;
  const int* V = flow_var<T>(fl);
  while (nsteps > 0) {
    if (K >= 2 && !(K & 1) && !(fl->t & 1) && nsteps >= K) {
      if (fl->windows++ > 0) {
        OM_TRY(flow_capture_t<T>(fl, K));
        OM_CUDA(cudaGraphLaunch(fl->exec, s));
      } else {  // the first whole window as plain launches: one-window calls capture nothing
        for (int k = 0; k < K; ++k) launch_step<T>(fl, k & 1, V[k & 1], nb, s, a);
      }
      fl->t += K;
      nsteps -= K;
      if (kFlowRebased<T>) d3q19_rebase<T><<<nb, 256, 0, s>>>(a);  // once per window
      continue;
    }
    const bool odd = fl->t & 1;
    launch_step<T>(fl, odd, V[odd], nb, s, a);
    ++fl->t;
    --nsteps;
  }
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

// Autotuner: time every launch variant of both sweeps on this node set
// (6 even/odd pairs each after a warm-up pair) and keep the fastest per
// parity; a node set of a size class tuned before in this process reuses
// that choice.  Runs from the rest state and puts the rest state back.
template <class T>
om_status flow_tune_t(om_flow* fl, cudaStream_t s) {
  if (fl->ns->nf == 0) return OM_OK;
  FlowArgs<T> a = flow_args<T>(fl);
  bool timed = false;
  OM_TRY(flow_tuned_variants<T>(a, fl->p.precision, flow_var<T>(fl), s, &timed));
  if (timed) d3q19_rest<T><<<blocks_for(a.nf), 256, 0, s>>>(a);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

template <class T>
om_status flow_observe_t(om_flow* fl, double* out, cudaStream_t s) {
  FlowArgs<T> a = flow_args<T>(fl);
  if (fl->t & 1) d3q19_observe<T, true><<<kObsBlocks, kObsThreads, 0, s>>>(a, fl->prev, fl->partials);
  else d3q19_observe<T, false><<<kObsBlocks, kObsThreads, 0, s>>>(a, fl->prev, fl->partials);
  launch_finalize(fl->partials, kObsBlocks, 4, fl->obs_dev, s);
  OM_CUDA(cudaGetLastError());
  OM_CUDA(cudaMemcpyAsync(fl->obs_host, fl->obs_dev, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  OM_CUDA(cudaStreamSynchronize(s));
  for (int k = 0; k < 4; ++k) out[k] = fl->obs_host[k];
  return OM_OK;
}

template <class T>
om_status flow_export_t(const om_flow* fl, double* fd, float* ud, cudaStream_t s) {
  const om_nodeset* ns = fl->ns;
  if (fd) OM_CUDA(cudaMemsetAsync(fd, 0, sizeof(double) * 19 * ns->N, s));
  if (ud) OM_CUDA(cudaMemsetAsync(ud, 0, sizeof(float) * 3 * ns->N, s));
  if (ns->nf == 0) return OM_OK;
  FlowArgs<T> a = flow_args<T>(fl);
  if (fl->t & 1) d3q19_export<T, true><<<blocks_for(a.nf), 256, 0, s>>>(a, ns->vox, ns->N, fd, ud);
  else d3q19_export<T, false><<<blocks_for(a.nf), 256, 0, s>>>(a, ns->vox, ns->N, fd, ud);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

template <class T>
om_status flow_import_t(om_flow* fl, const double* fd, cudaStream_t s) {
  if (fl->ns->nf == 0) return OM_OK;
  FlowArgs<T> a = flow_args<T>(fl);
  d3q19_import<T><<<blocks_for(a.nf), 256, 0, s>>>(a, fl->ns->vox, fl->ns->N, fd);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

template <class T>
om_status flow_init_u_t(om_flow* fl, const float* ux, int64_t stride, double scale, cudaStream_t s) {
  fl->t = 0;
  if (fl->ns->nf == 0) return OM_OK;
  FlowArgs<T> a = flow_args<T>(fl);
  d3q19_init_u<T><<<blocks_for(a.nf), 256, 0, s>>>(a, fl->ns->vox, ux, stride, scale);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

template <class T>
om_status flow_rest_t(om_flow* fl, cudaStream_t s) {
  if (fl->ns->nf == 0) return OM_OK;
  FlowArgs<T> a = flow_args<T>(fl);
  d3q19_rest<T><<<blocks_for(a.nf), 256, 0, s>>>(a);
  OM_CUDA(cudaGetLastError());
  return OM_OK;
}

// the storage type of the solver's precision and mode (rebased or not)
#define OM_FLOW_DISPATCH(fl, fn, ...)                                                            \
  switch ((fl)->p.precision) {                                                                   \
    case OM_F64: return fn<double>(__VA_ARGS__);                                                 \
    case OM_F32: return (fl)->reb ? fn<Reb<float>>(__VA_ARGS__) : fn<float>(__VA_ARGS__);        \
    case OM_F16DEV: return (fl)->reb ? fn<Reb<__half>>(__VA_ARGS__) : fn<__half>(__VA_ARGS__);   \
    case OM_BF16DEV:                                                                             \
      return (fl)->reb ? fn<Reb<__nv_bfloat16>>(__VA_ARGS__) : fn<__nv_bfloat16>(__VA_ARGS__);   \
    default: return fail(OM_EINVAL, "unknown precision");                                        \
  }

// The mode a (re)initialised solver starts in: FP32 unrebased (its fast
// sweeps; solves enter the rebased mode for their last decades), 16-bit
// rebased throughout (with 8 to 11 mantissa bits, unrebased storage cannot
// resolve a slow flow's velocity at all).
bool starts_rebased(const om_flow* fl) { return fl->rr != nullptr && fl->p.precision != OM_F32; }

// Enter the rebased mode from the current (unrebased) state: the reference
// starts at zero and takes the nodes' densities, the stored deviations lose
// them (an exact change of variables, at an even time).
template <class S>
om_status flow_enter_rebased_s(om_flow* fl, cudaStream_t s) {
  if (fl->ns->nf > 0) {
    OM_CUDA(cudaMemsetAsync(fl->rr, 0, sizeof(float) * fl->ns->nf, s));
    FlowArgs<Reb<S>> a = flow_args<Reb<S>>(fl);
    d3q19_rebase<Reb<S>><<<blocks_for(a.nf), 256, 0, s>>>(a);
    OM_CUDA(cudaGetLastError());
  }
  fl->reb = true;
  return OM_OK;
}
om_status flow_enter_rebased(om_flow* fl, cudaStream_t s) {
  if (fl->reb || !fl->rr || (fl->t & 1)) return OM_OK;
  switch (fl->p.precision) {
    case OM_F32: return flow_enter_rebased_s<float>(fl, s);
    case OM_F16DEV: return flow_enter_rebased_s<__half>(fl, s);
    case OM_BF16DEV: return flow_enter_rebased_s<__nv_bfloat16>(fl, s);
    default: return OM_OK;
  }
}

size_t storage_bytes(int prec) {
  return prec == OM_F64 ? 8 : (prec == OM_F32 ? 4 : 2);
}

om_status flow_observe_any(om_flow* fl, double* out, cudaStream_t s) {
  OM_FLOW_DISPATCH(fl, flow_observe_t, fl, out, s);
}

}  // namespace

extern "C" om_status om_flow_create(const om_nodeset* ns, const om_flow_params* p, void* stream,
                                    om_flow** out) {
  if (!ns || !p || !out) return fail(OM_EINVAL, "om_flow_create: null pointer");
  if (19 * ns->pitch > (int64_t)UINT32_MAX)
    return fail(OM_EINVAL, "om_flow_create: more than 226 M nodes (slot offsets are 32-bit)");
  if (!(p->tau > 0.5)) return fail(OM_EINVAL, "om_flow_create: tau must exceed 1/2");
  if (p->layout == OM_LAYOUT_DENSE)
    return fail(OM_EINVAL, "om_flow_create: solver objects use the sparse layout (the dense one is om_solve_permeability's)");
  if (p->precision < OM_F64 || p->precision > OM_BF16DEV)
    return fail(OM_EINVAL, "om_flow_create: unknown precision");
  if (p->drive != OM_DRIVE_FORCE && p->drive != OM_DRIVE_PRESSURE)
    return fail(OM_EINVAL, "om_flow_create: unknown drive");
  if (p->drive == OM_DRIVE_PRESSURE) {
    if (ns->dom.nx < 4) return fail(OM_EINVAL, "om_flow_create: the pressure drive needs nx >= 4");
    if (!(std::fabs(p->delta_rho) > 0.0 && std::fabs(p->delta_rho) < 0.1))
      return fail(OM_EINVAL, "om_flow_create: the pressure drive needs 0 < |delta_rho| < 0.1");
  }
  cudaStream_t s = as_stream(stream);
  om_flow* fl = new om_flow();
  fl->ns = ns;
  fl->p = *p;
  if (p->drive == OM_DRIVE_PRESSURE && ns->nf > 0) {
    // nodes before column (1, 0) lie at x = 0; from column (nx - 1, 0) on, at x = nx - 1
    uint4 w[2];
    const om_domain& d = ns->dom;
    cudaError_t e = cudaMemcpyAsync(&w[0], ns->col + (size_t)1 * d.ny * ns->W, sizeof(uint4),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&w[1], ns->col + (size_t)(d.nx - 1) * d.ny * ns->W, sizeof(uint4),
                          cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      delete fl;
      return cuda_fail(e, "om_flow_create: boundary ranks", __FILE__, __LINE__);
    }
    fl->n_in = w[0].y;
    fl->n_out = (uint32_t)ns->nf - w[1].y;
  }
  // FP16 storage keeps deviations scaled by 2^10 so they stay normal numbers
  fl->up = p->precision == OM_F16DEV ? 1024.0 : 1.0;
  DevBuf<uint8_t> f;
  DevBuf<double> prev, part, obs;
  DevBuf<float> rr;
  om_status st = f.alloc(19 * (size_t)ns->pitch * storage_bytes(p->precision));
  if (st == OM_OK && storage_bytes(p->precision) <= 4) st = rr.alloc(ns->pitch);
  if (st == OM_OK) st = prev.alloc(ns->nf);
  if (st == OM_OK) st = part.alloc((size_t)kObsBlocks * 8);
  if (st == OM_OK) st = obs.alloc(8);
  DevBuf<uint8_t> bc;
  const size_t nbt = (size_t)fl->n_in + fl->n_out;
  const size_t cbytes = p->precision == OM_F64 ? 8 : 4;  // the storage type's arithmetic type
  if (st == OM_OK && nbt) st = bc.alloc(19 * nbt * cbytes);
  if (st == OM_OK && nbt && cudaMemsetAsync(bc.p, 0, 19 * nbt * cbytes, s) != cudaSuccess)
    st = fail(OM_ECUDA, "om_flow_create: memset failed");
  double* host = nullptr;
  if (st == OM_OK && cudaMallocHost((void**)&host, 8 * sizeof(double)) != cudaSuccess) {
    (void)cudaGetLastError();
    st = fail(OM_ENOMEM, "om_flow_create: pinned allocation failed");
  }
  if (st != OM_OK) {
    delete fl;
    return st;
  }
  fl->f = f.take();
  fl->rr = rr.take();
  fl->prev = prev.take();
  fl->partials = part.take();
  fl->obs_dev = obs.take();
  fl->obs_host = host;
  fl->bc = bc.take();
  auto rest = [&]() -> om_status { OM_FLOW_DISPATCH(fl, flow_rest_t, fl, s); };
  auto tune = [&]() -> om_status { OM_FLOW_DISPATCH(fl, flow_tune_t, fl, s); };
  if (p->variant >= 0)
    fl->var[0] = fl->var[1] = fl->varr[0] = fl->varr[1] = std::min(p->variant, kSweepVariants - 1);
  st = rest();
  if (st == OM_OK && p->variant < 0) st = tune();
  if (st == OM_OK && p->variant < 0 && fl->rr) {  // and the rebased mode's kernels, from rest
    fl->reb = true;
    st = rest();
    if (st == OM_OK) st = tune();
    fl->reb = false;
    if (st == OM_OK) st = rest();
  }
  if (st == OM_OK && starts_rebased(fl)) {
    fl->reb = true;
    st = rest();
  }
  if (st == OM_OK) {
    double o[4];
    st = flow_observe_any(fl, o, s);  // prev <- u_x of the rest state
  }
  if (st != OM_OK) {
    om_flow_destroy(fl);
    return st;
  }
  *out = fl;
  return OM_OK;
}

extern "C" om_status om_flow_step(om_flow* fl, int64_t nsteps, void* stream) {
  if (!fl || nsteps < 0) return fail(OM_EINVAL, "om_flow_step: bad argument");
  cudaStream_t s = as_stream(stream);
  OM_FLOW_DISPATCH(fl, flow_steps_t, fl, nsteps, s);
}

extern "C" om_status om_flow_observe(om_flow* fl, double* out, void* stream) {
  if (!fl || !out) return fail(OM_EINVAL, "om_flow_observe: null pointer");
  return flow_observe_any(fl, out, as_stream(stream));
}

extern "C" om_status om_flow_solve(om_flow* fl, double* k_lattice, om_run_info* info, void* stream) {
  if (!fl) return fail(OM_EINVAL, "om_flow_solve: null pointer");
  const om_flow_params& p = fl->p;
  if (p.check_every <= 0 || (p.check_every & 1))
    return fail(OM_EINVAL, "om_flow_solve: check_every must be a positive even number");
  const bool pressure = p.drive == OM_DRIVE_PRESSURE;
  if (!pressure && !(p.body_force != 0.0)) return fail(OM_EINVAL, "om_flow_solve: body_force must be nonzero");
  if (!pressure && fl->ns->wrap_links == 0) {
    // x is periodic for the flow: with no lattice link across the x boundary
    // it is a wall, and the steady net flux (hence k) is exactly zero
    if (k_lattice) *k_lattice = 0.0;
    if (info) {
      *info = om_run_info{};
      info->n_nodes = fl->ns->nf;
    }
    return fail(OM_ENOPERC, "om_flow_solve: no pore link crosses the periodic x boundary (k = 0)");
  }
  cudaStream_t s = as_stream(stream);
  cudaEvent_t e0, e1;
  OM_CUDA(cudaEventCreate(&e0));
  OM_CUDA(cudaEventCreate(&e1));
  double o[4];
  OM_TRY(flow_observe_any(fl, o, s));  // reference for the first check
  const int64_t t0 = fl->t;
  OM_CUDA(cudaEventRecord(e0, s));
  om_status rc = OM_ENOTCONVERGED;
  double rel = 1.0;
  bool diverged = false;
  while (fl->t - t0 < p.max_steps) {
    int64_t k = std::min<int64_t>(p.check_every, p.max_steps - (fl->t - t0));
    OM_TRY(om_flow_step(fl, k, stream));
    OM_TRY(flow_observe_any(fl, o, s));

    if (!std::isfinite(o[0]) || !std::isfinite(o[2])) {
      diverged = true;
      break;
    }
    rel = o[2] > 0.0 ? o[1] / o[2] : 0.0;
    if (rel < p.conv_tol) {
      rc = OM_OK;
      break;
    }
    // the last decades of the convergence in the rebased mode (single and
    // half precision): its storage resolves the velocity where the
    // unrebased one spends bits on the local density deviation
    if (!fl->reb && fl->rr && rel < kRebaseBelow) OM_TRY(flow_enter_rebased(fl, s));
  }
  OM_CUDA(cudaEventRecord(e1, s));
  OM_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  OM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double nu = (p.tau - 0.5) / 3.0;
  if (k_lattice) {
    const om_domain& d = fl->ns->dom;
    if (pressure)  // Eq. 13: <u_x> over the interior layers, dp = (rho_in - rho_out)/3 over nx - 1
      *k_lattice = nu * (o[0] / ((double)(d.nx - 2) * d.ny * d.nz)) * (double)(d.nx - 1) / (p.delta_rho / 3.0);
    else
      *k_lattice = nu * (o[0] / (double)fl->ns->N) / p.body_force;
  }
  if (info) {
    info->steps = fl->t - t0;
    info->n_nodes = fl->ns->nf;
    info->rel_change = rel;
    info->mass = o[3];
    info->seconds = ms * 1e-3;
    info->mlups = ms > 0 ? (double)fl->ns->nf * (double)info->steps / (ms * 1e-3) / 1e6 : 0.0;
  }
  if (diverged) set_error("om_flow_solve: the populations diverged (non-finite velocity sums)");
  else if (rc != OM_OK) set_error("om_flow_solve: step cap reached before convergence");
  return rc;
}

extern "C" om_status om_flow_get_populations(const om_flow* fl, double* f_dev, void* stream) {
  if (!fl || !f_dev) return fail(OM_EINVAL, "om_flow_get_populations: null pointer");
  cudaStream_t s = as_stream(stream);
  OM_FLOW_DISPATCH(fl, flow_export_t, fl, f_dev, (float*)nullptr, s);
}

extern "C" om_status om_flow_get_velocity(const om_flow* fl, float* u_dev, void* stream) {
  if (!fl || !u_dev) return fail(OM_EINVAL, "om_flow_get_velocity: null pointer");
  cudaStream_t s = as_stream(stream);
  OM_FLOW_DISPATCH(fl, flow_export_t, fl, (double*)nullptr, u_dev, s);
}

extern "C" om_status om_flow_set_populations(om_flow* fl, const double* f_dev, void* stream) {
  if (!fl || !f_dev) return fail(OM_EINVAL, "om_flow_set_populations: null pointer");
  cudaStream_t s = as_stream(stream);
  fl->t = 0;
  fl->reb = starts_rebased(fl);
  auto imp = [&]() -> om_status { OM_FLOW_DISPATCH(fl, flow_import_t, fl, f_dev, s); };
  OM_TRY(imp());
  double o[4];
  return flow_observe_any(fl, o, s);
}

extern "C" om_status om_flow_init_velocity(om_flow* fl, const float* ux_dev, int64_t stride, double scale,
                                           void* stream) {
  if (!fl || !ux_dev || stride < 1) return fail(OM_EINVAL, "om_flow_init_velocity: bad argument");
  cudaStream_t s = as_stream(stream);
  fl->reb = starts_rebased(fl);
  auto init = [&]() -> om_status { OM_FLOW_DISPATCH(fl, flow_init_u_t, fl, ux_dev, stride, scale, s); };
  OM_TRY(init());
  double o[4];
  return flow_observe_any(fl, o, s);
}

extern "C" om_status om_flow_time(const om_flow* fl, int64_t* t) {
  if (!fl || !t) return fail(OM_EINVAL, "om_flow_time: null pointer");
  *t = fl->t;
  return OM_OK;
}

extern "C" om_status om_flow_destroy(om_flow* fl) {
  if (!fl) return OM_OK;
  if (fl->exec) cudaGraphExecDestroy(fl->exec);
  if (fl->cap) cudaStreamDestroy(fl->cap);
  cudaFree(fl->f);
  cudaFree(fl->rr);
  cudaFree(fl->prev);
  cudaFree(fl->partials);
  cudaFree(fl->obs_dev);
  cudaFree(fl->bc);
  if (fl->obs_host) cudaFreeHost(fl->obs_host);
  delete fl;
  return OM_OK;
}
