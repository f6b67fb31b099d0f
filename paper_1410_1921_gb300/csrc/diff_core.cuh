// diff_core.cuh -- device side of the Knudsen-diffusion sweep (Sec. 3.2,
// Eqs. 10-12) on D3Q7 or the paper's D3Q19 (the lattice L), shared by the
// single-structure kernels (diff.cu) and the batched kernels (batch.cu, D3Q7).
// See diff.cu for the scheme.
#pragma once

#include <cmath>

#include "lattice.cuh"

namespace om {

template <class T, class L = D3Q7>
struct DiffArgs {
  T* q[L::Q];  // population i of node n is q[i][n]
  uint32_t nf;
  const uint4* col;
  const uint32_t* coord;
  const typename Stg<T>::C* omega;
  int nx, ny, nz, W;
  typename Stg<T>::C s;         // slope of C_lin per lattice cell, (c_out - c_in)/nx
  typename Stg<T>::C up, down;  // storage scale
  double cin, cout;
  float* cr;  // 16-bit storage: per-node reference concentration (see kRebased)
  // neighbour records of the node set and its slow nodes (lattice.cuh);
  // rec7 == nullptr when the node set has none
  const uint2* rec7 = nullptr;
  const uint2* rec19 = nullptr;
  const uint32_t* slow = nullptr;
  uint32_t nslow = 0;
};

// Reference state of the stored deviations.  FP64 storage: a_i C_lin(x),
// the linear inlet-outlet profile, a function of position.  FP32 and 16-bit
// storage: a_i Cr(node), a per-node concentration that the solver moves to
// the node's current C every check window ("rebasing"), so what is stored is
// the small non-equilibrium part plus the drift since the last rebase.
// Deviations from C_lin are ~10 % of C in a tortuous structure; rounding
// them each step biases the flux (Eq. 14) by ~1e-4 relative in FP32 and by
// tens of percent in FP16, while the rebased deviations keep both within the
// convergence tolerance of the FP64 result.
template <class T>
constexpr bool kRebased = sizeof(T) <= 4;

// nb[i] = node of x + e_i, kNoNode for walls and beyond the x faces (those
// links are the Dirichlet half links); periodic y, z
template <class T, class L>
__device__ __forceinline__ void diff_neighbours(const DiffArgs<T, L>& a, uint32_t c, uint32_t (&nb)[L::Q],
                                                int& x) {
  int y, z;
  unpack_xyz(c, x, y, z);
  if constexpr (L::Q == 19) {
    q19_neighbours(a.col, a.nx, a.ny, a.nz, a.W, 0, c, nb);
  } else {
    const int yp = y + 1 == a.ny ? 0 : y + 1, ym = y == 0 ? a.ny - 1 : y - 1;
    const ZPos p = zpos(z, a.nz);
    const uint32_t ny = (uint32_t)a.ny, W = (uint32_t)a.W;
    auto base = [&](int xx, int yy) { return ((uint32_t)xx * ny + (uint32_t)yy) * W; };
    uint32_t self;
    column3(a.col, base(x, y), p, nb[6], self, nb[5]);
    nb[1] = x + 1 < a.nx ? column1(a.col, base(x + 1, y), p) : kNoNode;
    nb[2] = x > 0 ? column1(a.col, base(x - 1, y), p) : kNoNode;
    nb[3] = column1(a.col, base(x, yp), p);
    nb[4] = column1(a.col, base(x, ym), p);
    (void)self;
  }
}

// Reference concentrations an odd step needs (rebased storage): the node's
// own, and each neighbour's (0 where there is none).  Read once into
// registers: the stores of the step could alias them for the compiler.
template <class T, class L>
struct DiffRefs {
  typename Stg<T>::C n, nb[L::Q];
};

template <class T, class L>
__device__ __forceinline__ void diff_refs(const DiffArgs<T, L>& a, uint32_t n, const uint32_t (&nb)[L::Q],
                                          DiffRefs<T, L>& r) {
  using C = typename Stg<T>::C;
  if constexpr (kRebased<T>) {
    r.n = a.cr[n];
#pragma unroll
    for (int i = 1; i < L::Q; ++i) r.nb[i] = nb[i] != kNoNode ? (C)a.cr[nb[i]] : C(0);
  }
}

// Population i of a node at x arrives through the inlet half link x = -1/2
// (e_ix = +1 at x = 0) or the outlet one x = nx - 1/2 (e_ix = -1 at x = nx-1).
template <class L>
__device__ __forceinline__ bool from_inlet(int i, int x) { return L::e(i, 0) == 1 && x == 0; }
template <class L>
__device__ __forceinline__ bool from_outlet(int i, int x, int nx) { return L::e(i, 0) == -1 && x == nx - 1; }

// pre-collision deviations of node n at the current time (odd steps: with
// the reference concentrations r of diff_refs).  FACES = false: the node is
// known to lie off both x faces (x is not used).
template <class T, class L, bool ODD, bool FACES = true>
__device__ __forceinline__ void diff_load_r(const DiffArgs<T, L>& a, uint32_t n, const uint32_t (&nb)[L::Q], int x,
                                            const DiffRefs<T, L>& r, typename Stg<T>::C (&g)[L::Q]) {
  using S = Stg<T>;
  using C = typename S::C;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    if (!ODD || i == 0) {
      g[i] = S::ld(a.q[i] + n, a.down);
    } else {
      const int o = L::opp(i);
      const uint32_t src = nb[o];  // x - e_i
      const bool inlet = FACES && from_inlet<L>(i, x), outlet = FACES && from_outlet<L>(i, x, a.nx);
      const T* p = (src != kNoNode && !inlet && !outlet) ? a.q[o] + src : a.q[i] + n;
      const C v = S::ld(p, a.down);
      const C w = C(L::w(i));
      if constexpr (kRebased<T>) {
        if (inlet) g[i] = -v + C(2) * w * ((C)a.cin - r.n);
        else if (outlet) g[i] = -v + C(2) * w * ((C)a.cout - r.n);
        else if (src != kNoNode) g[i] = v + w * (r.nb[o] - r.n);
        else g[i] = v;
      } else {
        // C_lin(0) = c_in + s/2, C_lin(nx - 1) = c_out - s/2
        if (inlet) g[i] = -v - w * a.s;
        else if (outlet) g[i] = -v + w * a.s;
        else if (src != kNoNode) g[i] = v - w * C(L::e(i, 0)) * a.s;
        else g[i] = v;
      }
    }
  }
}

template <class T, class L, bool ODD>
__device__ __forceinline__ void diff_load(const DiffArgs<T, L>& a, uint32_t n, const uint32_t (&nb)[L::Q], int x,
                                          typename Stg<T>::C (&g)[L::Q]) {
  DiffRefs<T, L> r{};
  if (ODD) diff_refs(a, n, nb, r);
  diff_load_r<T, L, ODD>(a, n, nb, x, r, g);
}

// BGK relaxation of a node's deviations g toward a_i times their sum (the
// reference's own equilibrium part cancels: it is at rest).
template <class L, class C>
__device__ __forceinline__ void diff_relax(C (&g)[L::Q], C om) {
  C cc = g[0];
#pragma unroll
  for (int i = 1; i < L::Q; ++i) cc += g[i];
#pragma unroll
  for (int i = 0; i < L::Q; ++i) g[i] = g[i] - om * (g[i] - C(L::w(i)) * cc);
}

// One fused collide-stream update of node n (global slot index) at x whose
// neighbours are nb (used on odd steps only); the AA read/write pattern of
// flow_node_nb with the anti-bounce-back inlet/outlet and the reference shift.
template <class T, class L, bool ODD, bool FACES = true>
__device__ __forceinline__ void diff_store(const DiffArgs<T, L>& a, uint32_t n, int x, const uint32_t (&nb)[L::Q],
                                           const DiffRefs<T, L>& r, const typename Stg<T>::C (&g)[L::Q]);

template <class T, class L, bool ODD, bool FACES = true>
__device__ __forceinline__ void diff_node_nb(const DiffArgs<T, L>& a, uint32_t n, int x, const uint32_t (&nb)[L::Q]) {
  DiffRefs<T, L> r{};
  if (ODD) diff_refs(a, n, nb, r);
  typename Stg<T>::C g[L::Q];
  diff_load_r<T, L, ODD, FACES>(a, n, nb, x, r, g);
  diff_relax<L>(g, a.omega[n]);
  diff_store<T, L, ODD, FACES>(a, n, x, nb, r, g);
}

// post-collision deviations of node n at x to their slots (see diff_node_nb)
template <class T, class L, bool ODD, bool FACES>
__device__ __forceinline__ void diff_store(const DiffArgs<T, L>& a, uint32_t n, int x, const uint32_t (&nb)[L::Q],
                                           const DiffRefs<T, L>& r, const typename Stg<T>::C (&g)[L::Q]) {
  using S = Stg<T>;
  using C = typename S::C;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const int o = L::opp(i);
    if (!ODD) {
      S::st(a.q[o] + n, g[i], a.up);
    } else if (i == 0) {
      S::st(a.q[0] + n, g[0], a.up);
    } else {
      // leaves through the outlet (e_ix = +1 at nx-1) or the inlet half link
      const bool outlet = FACES && L::e(i, 0) == 1 && x == a.nx - 1, inlet = FACES && L::e(i, 0) == -1 && x == 0;
      T* p = a.q[o] + n;
      C v = g[i];
      const C w = C(L::w(i));
      if constexpr (kRebased<T>) {
        if (outlet) v = -g[i] + C(2) * w * ((C)a.cout - r.n);
        else if (inlet) v = -g[i] + C(2) * w * ((C)a.cin - r.n);
        else if (nb[i] != kNoNode) {
          p = a.q[i] + nb[i];
          v = g[i] + w * (r.n - r.nb[i]);
        }
      } else {
        if (outlet) v = -g[i] + w * a.s;
        else if (inlet) v = -g[i] - w * a.s;
        else if (nb[i] != kNoNode) {
          p = a.q[i] + nb[i];
          v = g[i] - w * C(L::e(i, 0)) * a.s;
        }
      }
      S::st(p, v, a.up);
    }
  }
}

// Even-step update of the two nodes n, n + 1 (n even, n + 1 < nf): each
// population of both moved as one vector (Pair<T>), the relaxations those of
// diff_node_nb.
template <class T, class L>
__device__ __forceinline__ void diff_pair_even(const DiffArgs<T, L>& a, uint32_t n) {
  using C = typename Stg<T>::C;
  C g0[L::Q], g1[L::Q];
#pragma unroll
  for (int i = 0; i < L::Q; ++i) Pair<T>::ld(a.q[i] + n, a.down, g0[i], g1[i]);
  C om0, om1;
  Pair<C>::ld(a.omega + n, C(1), om0, om1);
  diff_relax<L>(g0, om0);
  diff_relax<L>(g1, om1);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) Pair<T>::st(a.q[L::opp(i)] + n, g0[i], g1[i], a.up);
}

// diff_node_nb after the neighbour lookup of the node's coordinates c
template <class T, class L, bool ODD>
__device__ __forceinline__ void diff_node_at(const DiffArgs<T, L>& a, uint32_t n, uint32_t c) {
  uint32_t nb[L::Q];
  int x = 0;
  if (ODD) diff_neighbours(a, c, nb, x);
  diff_node_nb<T, L, ODD>(a, n, x, nb);
}

// Odd step of node t from its records (a node off every face of the box:
// no inlet or outlet link), or of slow node slow[t - nf] through the column
// map; r, q are node t's records (t < nf)
template <class T, class L>
__device__ __forceinline__ void diff_odd_rec(const DiffArgs<T, L>& a, uint32_t t, uint2 r, uint2 q) {
  if (t < a.nf) {
    if (rec_slow(r)) return;  // updated from the slow list
    uint32_t nb[L::Q];
    if constexpr (L::Q == 19) rec_neighbours19(r, q, t, nb);
    else rec_axis<L::Q>(r, t, nb);
    diff_node_nb<T, L, true, false>(a, t, 0, nb);
  } else {
    const uint32_t n = __ldg(a.slow + (t - a.nf));
    diff_node_at<T, L, true>(a, n, __ldg(a.coord + n));
  }
}

// node t's records (the D3Q19 part only for that lattice)
template <class L>
__device__ __forceinline__ void diff_rec_load(const uint2* rec7, const uint2* rec19, uint32_t t, uint32_t nf, uint2& r,
                                              uint2& q) {
  r = make_uint2(0u, 0u);
  q = make_uint2(0u, 0u);
  if (t < nf) {
    r = __ldg(rec7 + t);
    if constexpr (L::Q == 19) q = __ldg(rec19 + t);
  }
}

// diff_node_at for node n whose coordinates are coord[ln]
template <class T, bool ODD, class L = D3Q7>
__device__ __forceinline__ void diff_node(const DiffArgs<T, L>& a, uint32_t n, uint32_t ln) {
  diff_node_at<T, L, ODD>(a, n, ODD ? a.coord[ln] : 0u);
}

// Reference concentration of node n (with coordinates x): C_lin(x) or Cr[n]
template <class T, class L>
__device__ __forceinline__ double diff_ref(const DiffArgs<T, L>& a, uint32_t n, int x) {
  if constexpr (kRebased<T>) return (double)a.cr[n];
  else return a.cin + (double)a.s * ((double)x + 0.5);
}

// Move node n's reference to its current concentration (even time only):
// Cr += sum_i dev_i, dev_i -= a_i (Cr_new - Cr_old).
template <class T, class L>
__device__ __forceinline__ void diff_rebase_node(const DiffArgs<T, L>& a, uint32_t n) {
  if constexpr (kRebased<T>) {
    using S = Stg<T>;
    float d[L::Q], sum = 0.f;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      d[i] = S::ld(a.q[i] + n, a.down);
      sum += d[i];
    }
    const float old = a.cr[n];
    const float now = old + sum;
    a.cr[n] = now;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) S::st(a.q[i] + n, d[i] + (float)L::w(i) * (old - now), a.up);
  }
}

// The single-structure solver's D3Q7 sweeps (diff.cu), also run by batches
// on their large structures: one sweep of launch variant `variant` over
// nodes 0 .. a.nf of a's arrays; and the variants timed fastest per parity
// on a node set of a's size class (cached per process; timing them changes
// the populations).
template <class T>
void diff_sweep_variant(bool odd, int variant, const DiffArgs<T, D3Q7>& a, cudaStream_t s);
template <class T>
om_status diff_tuned_variants(const DiffArgs<T, D3Q7>& a, int precision, int V[2], cudaStream_t s);

// Extrapolated restarts (om_diff_params.accel): the host side of the test
// that the decay of the window-to-window change has settled on one mode.
struct ExtrapolationTrack {
  double last = -1.0;  // sum |dC| of the last window (< 0: none since the start or the last jump)
  double rho[3] = {0.0, 0.0, 0.0};
  int n = 0;           // ratios recorded since then
  // record this window's sum |dC|; returns the factor rho / (1 - rho) to
  // move every node's C by (times its dC) when the last three ratios agree,
  // else 0
  double observe(double sum_abs_dc) {
    if (last > 0.0 && sum_abs_dc > 0.0) {
      rho[0] = rho[1];
      rho[1] = rho[2];
      rho[2] = sum_abs_dc / last;
      ++n;
    }
    last = sum_abs_dc;
    if (n < 3) return 0.0;
    const double r = rho[2];
    if (!(r > 0.0 && r < 0.999)) return 0.0;
    const double tol = 0.02 * (1.0 - r);
    if (std::fabs(rho[2] - rho[1]) > tol || std::fabs(rho[1] - rho[0]) > 0.02 * (1.0 - rho[1])) return 0.0;
    *this = ExtrapolationTrack{};  // start over after the jump
    return r / (1.0 - r);
  }
};

}  // namespace om
