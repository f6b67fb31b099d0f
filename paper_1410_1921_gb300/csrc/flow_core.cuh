// flow_core.cuh -- device side of the D3Q19 flow sweep (Sec. 3.1, Eqs. 1-9,
// App. A), shared by the single-structure kernels (flow.cu) and the batched
// kernels (batch.cu).  See flow.cu for the scheme.
#pragma once

#include "lattice.cuh"

namespace om {

// Node indices returned by the column map are global slot indices (a batch
// rebases each structure's map by its offset); coordinates are indexed by
// the structure-local node number.
template <class T>
struct FlowArgs {
  T* s[19];  // population i of node n is s[i][n] (kernel parameters: no per-slot registers)
  uint32_t P;  // slot pitch: s[i] == s[0] + i * P, and 19 * P < 2^32
  uint32_t nf;
  const uint4* col;
  const uint32_t* coord;
  int nx, ny, nz, W;
  typename Stg<T>::C wp, wm, g, up, down;
  // Pressure drive (Sec. 3.3): x is not periodic (px = 0); nodes [0, n_in)
  // lie at x = 0 and [nf - n_out, nf) at x = nx - 1, and their pre-collision
  // deviations are bc[i * (n_in + n_out) + k], written before every sweep by
  // the boundary kernel.  Body-force drive: px = 1, n_in = n_out = 0.
  int px = 1;
  uint32_t n_in = 0, n_out = 0;
  const typename Stg<T>::C* bc = nullptr;
  // neighbour records of the node set and its slow nodes (lattice.cuh);
  // rec7 == nullptr when the node set has none
  const uint2* rec7 = nullptr;
  const uint2* rec19 = nullptr;
  const uint32_t* slow = nullptr;
  uint32_t nslow = 0;
  // rebased storage (kFlowRebased<T>): per-node reference density deviation
  float* rr = nullptr;
};

// Reference state of the stored deviations: w_i (rest at rho0 = 1), or in
// the rebased mode (storage type Reb<S>, FP32 and 16-bit) w_i (1 + rr(node)),
// a per-node density the solver moves to the node's current density once
// per check window ("rebasing", as the diffusion does with its
// concentration).  om_flow_solve switches to the rebased mode for the last
// decades of a tight convergence (see flow.cu).  A slow flow's velocity is a small
// difference of populations that also carry the local density deviation
// (body-force driven flow in tortuous pores: delta rho / u ~ 3 L nu / k, 1e2
// to 1e4); without the rebase that deviation takes 7-13 bits of every stored
// value, which biased single-precision k by up to 2e-5 and kept the
// per-node velocity change above 1e-5 in tight pores.  A population that
// changes node is re-referenced by w_i (rr(source) - rr(target)) -- only on
// odd steps, where populations are read from and written to neighbours; the
// collision is unchanged (it is invariant under a shift of the rest part).
template <class T>
constexpr bool kFlowRebased = false;
template <class S>
constexpr bool kFlowRebased<Reb<S>> = true;

// A solve (om_flow_solve, and per structure om_batch_solve) enters the
// rebased mode once the relative change of the velocity field over a check
// window falls below this: two to three decades before a tight test, and
// above the ~1e-5 floor that single-precision rounding puts under that
// change in tight pores without the rebase.
constexpr double kRebaseBelow = 1e-4;

// nb[i] = node number of x + e_i (kNoNode off the node set); periodic y, z,
// and x unless a.px = 0 (no neighbour beyond the x faces)
template <class T>
__device__ __forceinline__ void flow_neighbours(const FlowArgs<T>& a, uint32_t c, uint32_t (&nb)[19]) {
  q19_neighbours(a.col, a.nx, a.ny, a.nz, a.W, a.px, c, nb);
}

// Index of node n among the boundary nodes of the pressure drive, or -1
template <class T>
__device__ __forceinline__ int64_t flow_boundary_index(const FlowArgs<T>& a, uint32_t n) {
  if (n < a.n_in) return n;
  if (a.n_out && n >= a.nf - a.n_out) return (int64_t)a.n_in + (n - (a.nf - a.n_out));
  return -1;
}

// Odd steps: off[i] = element offset from s[0] of the slot that population i
// of node n is read from -- slot opposite(i) of the neighbour x - e_i, or
// the node's own slot i where that neighbour is missing (halfway
// bounce-back).  In the AA pattern the post-collision population
// opposite(i) is written to the same slot, so one offset serves both.
template <class T>
__device__ __forceinline__ void flow_slots_odd(const FlowArgs<T>& a, uint32_t n, const uint32_t (&nb)[19],
                                               uint32_t (&off)[19]) {
  off[0] = n;
#pragma unroll
  for (int i = 1; i < 19; ++i) {
    const uint32_t o = (uint32_t)q19_opp(i), src = nb[o];
    off[i] = src != kNoNode ? o * a.P + src : (uint32_t)i * a.P + n;
  }
}

// pre-collision populations of node n at the current time
template <class T, bool ODD>
__device__ __forceinline__ void flow_load(const FlowArgs<T>& a, uint32_t n, const uint32_t (&nb)[19],
                                          typename Stg<T>::C (&f)[19]) {
  if constexpr (ODD) {
    uint32_t off[19];
    flow_slots_odd(a, n, nb, off);
#pragma unroll
    for (int i = 0; i < 19; ++i) f[i] = Stg<T>::ld(a.s[0] + off[i], a.down);
    if constexpr (kFlowRebased<T>) {
      const float rn = a.rr[n];
#pragma unroll
      for (int i = 1; i < 19; ++i) {
        const uint32_t src = nb[q19_opp(i)];
        if (src != kNoNode) f[i] += (float)q19_w(i) * (a.rr[src] - rn);
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < 19; ++i) f[i] = Stg<T>::ld(a.s[i] + n, a.down);
  }
}

// An empty asm statement taking two values as in-out operands: what reads
// them afterwards cannot be scheduled before the code that produced them
// (keeps the reference gathers of a rebased odd step after the collision).
__device__ __forceinline__ void order_after(float& a, float& b) { asm volatile("" : "+f"(a), "+f"(b)); }
__device__ __forceinline__ void order_after(double& a, double& b) { asm volatile("" : "+d"(a), "+d"(b)); }

template <class C>
__device__ __forceinline__ void trt_collide(C (&f)[19], C wp, C wm, C g) {
  C rho = f[0];
#pragma unroll
  for (int i = 1; i < 19; ++i) rho += f[i];
  C jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int i = 1; i < 19; ++i) {
    if (q19_e(i, 0)) jx += q19_e(i, 0) > 0 ? f[i] : -f[i];
    if (q19_e(i, 1)) jy += q19_e(i, 1) > 0 ? f[i] : -f[i];
    if (q19_e(i, 2)) jz += q19_e(i, 2) > 0 ? f[i] : -f[i];
  }
  const C ux = jx + C(0.5) * g, uy = jy, uz = jz;
  const C usq15 = C(1.5) * (ux * ux + uy * uy + uz * uz);
  const C frc = (C(1) - C(0.5) * wm) * C(3) * g;
  f[0] = f[0] - wp * (f[0] - C(1.0 / 3.0) * (rho - usq15));
#pragma unroll
  for (int i = 1; i < 19; ++i) {
    const int o = q19_opp(i);
    if (o < i) continue;  // each pair once, from its first member
    const C w = C(q19_w(i));
    const C eu = C(q19_e(i, 0)) * ux + C(q19_e(i, 1)) * uy + C(q19_e(i, 2)) * uz;
    const C sym = w * (rho + C(4.5) * eu * eu - usq15);
    const C asym = C(3) * w * eu;
    const C fp = C(0.5) * (f[i] + f[o]);
    const C fm = C(0.5) * (f[i] - f[o]);
    const C A = wp * (fp - sym);
    const C B = wm * (fm - asym) - w * C(q19_e(i, 0)) * frc;
    f[i] = f[i] - A - B;
    f[o] = f[o] - A + B;
  }
}


// Collision of node n's pre-collision deviations f; under the pressure drive
// a boundary node first takes its extrapolated populations.
template <class T>
__device__ __forceinline__ void flow_collide(const FlowArgs<T>& a, uint32_t n, typename Stg<T>::C (&f)[19]) {
  if (a.n_in + a.n_out) {
    const int64_t k = flow_boundary_index(a, n);
    if (k >= 0) {
      const uint32_t nbt = a.n_in + a.n_out;
      // the extrapolated populations are deviations from w_i; rebased storage
      // refers the node's to w_i (1 + rr(n))
      typename Stg<T>::C rn = 0;
      if constexpr (kFlowRebased<T>) rn = a.rr[n];
#pragma unroll
      for (int i = 0; i < 19; ++i) f[i] = a.bc[(size_t)i * nbt + k] - typename Stg<T>::C(q19_w(i)) * rn;
    }
  }
  trt_collide(f, a.wp, a.wm, a.g);
}


// One fused collide-stream update of node n (global slot index) whose
// neighbours are nb (used on odd steps only).  Even steps: read and write the
// node's own slots (post-collision f*_i to slot opposite(i)).  Odd steps:
// read slot opposite(i) of x - e_i, write slot i of x + e_i; a missing
// neighbour is halfway bounce-back (own slot i read, own slot opposite(i)
// written).
template <class T, bool ODD>
__device__ __forceinline__ void flow_node_nb(const FlowArgs<T>& a, uint32_t n, const uint32_t (&nb)[19]) {
  typename Stg<T>::C f[19];
  if constexpr (ODD) {
    uint32_t off[19];
    flow_slots_odd(a, n, nb, off);
#pragma unroll
    for (int i = 0; i < 19; ++i) f[i] = Stg<T>::ld(a.s[0] + off[i], a.down);
    if constexpr (kFlowRebased<T>) {
      // Population i came from x - e_i, and leaves for x + e_i, when its
      // slot offset points into another node's slots: the node index
      // off - (slot array) * P then lies in [0, P) (a bounce-back slot of
      // the node itself gives an index outside it).  The references are
      // gathered again after the collision rather than held across it
      // (fewer live registers; the second reads hit L1).
      const float rn = a.rr[n];
#pragma unroll
      for (int i = 1; i < 19; ++i) {
        const uint32_t src = off[i] - (uint32_t)q19_opp(i) * a.P;
        if (src < a.P) f[i] += (float)q19_w(i) * (a.rr[src] - rn);
      }
      flow_collide(a, n, f);
      order_after(f[16], f[17]);
#pragma unroll
      for (int i = 1; i < 19; ++i) {
        const uint32_t dst = off[q19_opp(i)] - (uint32_t)i * a.P;
        if (dst < a.P) f[i] -= (float)q19_w(i) * (a.rr[dst] - rn);
      }
    } else {
      flow_collide(a, n, f);
    }
#pragma unroll
    for (int i = 0; i < 19; ++i) Stg<T>::st(a.s[0] + off[q19_opp(i)], f[i], a.up);
  } else {
#pragma unroll
    for (int i = 0; i < 19; ++i) f[i] = Stg<T>::ld(a.s[i] + n, a.down);
    flow_collide(a, n, f);
#pragma unroll
    for (int i = 0; i < 19; ++i) Stg<T>::st(a.s[q19_opp(i)] + n, f[i], a.up);
  }
}

// flow_node_nb after the neighbour lookup of the node's coordinates c
template <class T, bool ODD>
__device__ __forceinline__ void flow_node_at(const FlowArgs<T>& a, uint32_t n, uint32_t c) {
  uint32_t nb[19];
  if (ODD) flow_neighbours(a, c, nb);
  flow_node_nb<T, ODD>(a, n, nb);
}

// Even-step update of the two nodes n, n + 1 (n even, n + 1 < nf): each
// population of both moved as one vector (Pair<T>), the collisions those of
// flow_node_nb.
template <class T>
__device__ __forceinline__ void flow_pair_even(const FlowArgs<T>& a, uint32_t n) {
  using C = typename Stg<T>::C;
  C f0[19], f1[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) Pair<T>::ld(a.s[i] + n, a.down, f0[i], f1[i]);
  flow_collide(a, n, f0);
  flow_collide(a, n + 1, f1);
#pragma unroll
  for (int i = 0; i < 19; ++i) Pair<T>::st(a.s[q19_opp(i)] + n, f0[i], f1[i], a.up);
}

// Move node n's reference to its current density (even time only):
// rr += sum_i dev_i, dev_i -= w_i (rr_new - rr_old).
template <class T>
__device__ __forceinline__ void flow_rebase_node(const FlowArgs<T>& a, uint32_t n) {
  if constexpr (kFlowRebased<T>) {
    using S = Stg<T>;
    float f[19], sum = 0.f;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
      f[i] = S::ld(a.s[i] + n, a.down);
      sum += f[i];
    }
    const float old = a.rr[n];
    const float now = old + sum;
    a.rr[n] = now;
#pragma unroll
    for (int i = 0; i < 19; ++i) S::st(a.s[i] + n, f[i] + (float)q19_w(i) * (old - now), a.up);
  }
}

// Reference density deviation of node n (0 for FP64 storage)
template <class T>
__device__ __forceinline__ double flow_ref(const FlowArgs<T>& a, uint32_t n) {
  if constexpr (kFlowRebased<T>) return (double)a.rr[n];
  else return 0.0;
}

// The single-structure solver's sweeps (flow.cu), also run by batches on
// their large structures: one sweep of launch variant `variant` over nodes
// 0 .. a.nf of a's arrays; and the variants timed fastest per parity on a
// node set of a's size class (cached per process; *timed tells whether
// this call timed them, which changes the populations).
template <class T>
void flow_sweep_variant(bool odd, int variant, const FlowArgs<T>& a, cudaStream_t s);
template <class T>
om_status flow_tuned_variants(const FlowArgs<T>& a, int precision, int V[2], cudaStream_t s, bool* timed);

// flow_node_at for node n whose coordinates are coord[ln]
template <class T, bool ODD>
__device__ __forceinline__ void flow_node(const FlowArgs<T>& a, uint32_t n, uint32_t ln) {
  flow_node_at<T, ODD>(a, n, ODD ? a.coord[ln] : 0u);
}

}  // namespace om
