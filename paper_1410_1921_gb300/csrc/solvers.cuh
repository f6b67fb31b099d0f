// solvers.cuh -- the state of the single-structure solver objects of
// include/om.h (om_flow, om_diff) and the kernel arguments built from it,
// shared by the translation units that launch their sweeps.
#pragma once

#include <cmath>

#include "diff_core.cuh"
#include "flow_core.cuh"

struct om_flow {
  const om_nodeset* ns = nullptr;
  om_flow_params p{};
  void* f = nullptr;
  float* rr = nullptr;  // rebased storage: per-node reference density deviation
  double* prev = nullptr;
  double* partials = nullptr;
  double* obs_dev = nullptr;
  double* obs_host = nullptr;  // pinned
  int64_t t = 0;
  double up = 1.0;  // storage scale of reduced-precision formats (stored = deviation * up)
  int var[2] = {0, 0};  // launch variant of the even and odd sweeps
  int varr[2] = {0, 0};  // the same for the rebased mode
  // rebased mode (storage Reb<S>, reference rr): entered by om_flow_solve
  // for the last decades of its convergence, left by any (re)initialisation
  bool reb = false;
  bool graph_reb = false;  // the captured window is of the rebased kernels
  // pressure drive: boundary nodes [0, n_in) and [nf - n_out, nf), their
  // extrapolated populations (storage arithmetic type, [19][n_in + n_out])
  uint32_t n_in = 0, n_out = 0;
  void* bc = nullptr;
  // a captured window of graph_k steps starting at an even time (replayed by
  // *_step); the first whole window runs as plain launches and the graph is
  // captured at the second, so that single-window calls pay no capture
  cudaGraphExec_t exec = nullptr;
  int graph_k = 0;
  int64_t windows = 0;
  cudaStream_t cap = nullptr;
};

struct om_diff {
  const om_nodeset* ns = nullptr;
  om_diff_params p{};
  void* g = nullptr;
  void* omega = nullptr;
  float* cr = nullptr;  // per-node reference concentration (16-bit storage)
  int q = 7;            // lattice: 7 (D3Q7) or 19 (D3Q19)
  double* prev = nullptr;
  double* dprev = nullptr;  // OM_ACCEL_EXTRAPOLATE: each node's change of C over the last window
  double* partials = nullptr;
  double* obs_dev = nullptr;
  double* obs_host = nullptr;
  int64_t t = 0;
  double up = 1.0;      // storage scale (stored = deviation * up)
  int var[2] = {0, 0};  // launch variant of the even and odd sweeps
  // as om_flow's
  cudaGraphExec_t exec = nullptr;
  int graph_k = 0;
  int64_t windows = 0;
  cudaStream_t cap = nullptr;
};

namespace om {

template <class T>
inline FlowArgs<T> flow_args(const om_flow* fl) {
  FlowArgs<T> a;
  const om_nodeset* ns = fl->ns;
  for (int i = 0; i < 19; ++i) a.s[i] = (T*)fl->f + (size_t)i * ns->pitch;
  a.P = (uint32_t)ns->pitch;
  a.nf = (uint32_t)ns->nf;
  a.col = ns->col;
  a.coord = ns->coord;
  a.rec7 = ns->rec7;
  a.rec19 = ns->rec19;
  a.slow = ns->slow;
  a.nslow = (uint32_t)ns->n_slow;
  a.rr = fl->rr;
  a.nx = ns->dom.nx;
  a.ny = ns->dom.ny;
  a.nz = ns->dom.nz;
  a.W = ns->W;
  const double tau = fl->p.tau;
  a.wp = (typename Stg<T>::C)(1.0 / tau);
  a.wm = (typename Stg<T>::C)(8.0 * (2.0 * tau - 1.0) / (8.0 * tau - 1.0));
  a.g = (typename Stg<T>::C)fl->p.body_force;
  a.up = (typename Stg<T>::C)fl->up;
  a.down = (typename Stg<T>::C)(1.0 / fl->up);
  if (fl->p.drive == OM_DRIVE_PRESSURE) {
    a.g = 0;
    a.px = 0;
    a.n_in = fl->n_in;
    a.n_out = fl->n_out;
    a.bc = (const typename Stg<T>::C*)fl->bc;
  }
  return a;
}

template <class T, class L>
inline DiffArgs<T, L> diff_args(const om_diff* df) {
  DiffArgs<T, L> a;
  const om_nodeset* ns = df->ns;
  for (int i = 0; i < L::Q; ++i) a.q[i] = (T*)df->g + (size_t)i * ns->pitch;
  a.nf = (uint32_t)ns->nf;
  a.col = ns->col;
  a.coord = ns->coord;
  a.omega = (const typename Stg<T>::C*)df->omega;
  a.nx = ns->dom.nx;
  a.ny = ns->dom.ny;
  a.nz = ns->dom.nz;
  a.W = ns->W;
  a.s = (typename Stg<T>::C)((df->p.c_out - df->p.c_in) / (double)ns->dom.nx);
  a.up = (typename Stg<T>::C)df->up;
  a.down = (typename Stg<T>::C)(1.0 / df->up);
  a.cin = df->p.c_in;
  a.cout = df->p.c_out;
  a.cr = df->cr;
  a.rec7 = ns->rec7;
  a.rec19 = ns->rec19;
  a.slow = ns->slow;
  a.nslow = (uint32_t)ns->n_slow;
  return a;
}

// move the rebased diffusion's per-node reference to the current
// concentration (diff.cu); OM_OK without work for FP64 storage
om_status diff_rebase_any(om_diff* df, cudaStream_t s);

}  // namespace om
