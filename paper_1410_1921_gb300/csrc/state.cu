// state.cu -- checkpoint and resume of the single-structure solvers.
//
// A solver's evolving state is its stored populations exactly as stored
// (deviations in the storage format), the diffusion's per-node reference
// concentration (FP32 and 16-bit storage), the previous observables of the
// convergence test, and the step counter.  Saved to a host byte image and
// loaded into a solver of the same node set and parameters, it lets that
// solver continue bit for bit as the saved one would have: long diffusion
// runs (10^5 - 10^6 steps) can stop and resume.  Image layout: a header
// (magic, version, solver kind, precision, populations per node, node
// count, step counter, storage scale), then q x nf populations (slot by
// slot), nf doubles of previous observables, nf floats of reference
// concentration where the solver has one.
#include <cstring>

#include "solvers.cuh"

namespace om {
namespace {

constexpr char kMagic[8] = {'O', 'M', 'S', 'T', 'A', 'T', 'E', '1'};

struct StateHeader {
  char magic[8];
  int32_t kind;  // 0 flow, 1 diffusion
  int32_t precision;
  int32_t q;
  int32_t has_cr;
  int64_t nf;
  int64_t t;
  double up;
};

// the arrays of one solver's state
struct StateView {
  int32_t kind, precision, q, has_cr;
  int64_t nf, pitch;
  size_t elem;  // bytes per stored population
  void* pop;
  double* prev;
  float* cr;
  double up;
};

size_t elem_bytes(int prec) { return prec == OM_F64 ? 8 : (prec == OM_F32 ? 4 : 2); }

int64_t image_bytes(const StateView& v) {
  return (int64_t)sizeof(StateHeader) + v.q * v.nf * (int64_t)v.elem + v.nf * 8 + (v.has_cr ? v.nf * 4 : 0);
}

om_status save(const StateView& v, int64_t t, void* host, int64_t bytes, cudaStream_t s, const char* who) {
  if (!host || bytes < image_bytes(v)) return fail(OM_EINVAL, std::string(who) + ": buffer too small");
  StateHeader h{};
  std::memcpy(h.magic, kMagic, sizeof kMagic);
  h.kind = v.kind;
  h.precision = v.precision;
  h.q = v.q;
  h.has_cr = v.has_cr;
  h.nf = v.nf;
  h.t = t;
  h.up = v.up;
  char* p = (char*)host;
  std::memcpy(p, &h, sizeof h);
  p += sizeof h;
  const size_t slot = (size_t)v.nf * v.elem;
  if (v.nf > 0) {
    for (int i = 0; i < v.q; ++i, p += slot)
      OM_CUDA(cudaMemcpyAsync(p, (const char*)v.pop + (size_t)i * v.pitch * v.elem, slot, cudaMemcpyDeviceToHost, s));
    OM_CUDA(cudaMemcpyAsync(p, v.prev, (size_t)v.nf * 8, cudaMemcpyDeviceToHost, s));
    p += (size_t)v.nf * 8;
    if (v.has_cr) OM_CUDA(cudaMemcpyAsync(p, v.cr, (size_t)v.nf * 4, cudaMemcpyDeviceToHost, s));
  }
  OM_CUDA(cudaStreamSynchronize(s));
  return OM_OK;
}

om_status load(const StateView& v, int64_t* t, const void* host, int64_t bytes, cudaStream_t s, const char* who) {
  if (!host || bytes < (int64_t)sizeof(StateHeader)) return fail(OM_EINVAL, std::string(who) + ": no state image");
  StateHeader h;
  std::memcpy(&h, host, sizeof h);
  if (std::memcmp(h.magic, kMagic, sizeof kMagic) != 0) return fail(OM_EINVAL, std::string(who) + ": not a state image");
  if (h.kind != v.kind || h.precision != v.precision || h.q != v.q || h.has_cr != v.has_cr || h.nf != v.nf ||
      h.up != v.up)
    return fail(OM_EINVAL, std::string(who) + ": the image is of another solver kind, precision, lattice or node set");
  if (bytes < image_bytes(v)) return fail(OM_EINVAL, std::string(who) + ": image truncated");
  if (h.t < 0) return fail(OM_EINVAL, std::string(who) + ": bad step counter");
  const char* p = (const char*)host + sizeof h;
  const size_t slot = (size_t)v.nf * v.elem;
  if (v.nf > 0) {
    for (int i = 0; i < v.q; ++i, p += slot)
      OM_CUDA(cudaMemcpyAsync((char*)v.pop + (size_t)i * v.pitch * v.elem, p, slot, cudaMemcpyHostToDevice, s));
    OM_CUDA(cudaMemcpyAsync(v.prev, p, (size_t)v.nf * 8, cudaMemcpyHostToDevice, s));
    p += (size_t)v.nf * 8;
    if (v.has_cr) OM_CUDA(cudaMemcpyAsync(v.cr, p, (size_t)v.nf * 4, cudaMemcpyHostToDevice, s));
  }
  OM_CUDA(cudaStreamSynchronize(s));
  *t = h.t;
  return OM_OK;
}

StateView flow_view(const om_flow* fl) {
  return StateView{0, fl->p.precision, 19, fl->reb ? 1 : 0, fl->ns->nf, fl->ns->pitch, elem_bytes(fl->p.precision),
                   fl->f, fl->prev, fl->rr, fl->up};
}

StateView diff_view(const om_diff* df) {
  return StateView{1, df->p.precision, df->q, df->cr ? 1 : 0, df->ns->nf, df->ns->pitch,
                   elem_bytes(df->p.precision), df->g, df->prev, df->cr, df->up};
}

}  // namespace
}  // namespace om

using namespace om;

extern "C" om_status om_flow_state_size(const om_flow* fl, int64_t* bytes) {
  if (!fl || !bytes) return fail(OM_EINVAL, "om_flow_state_size: null pointer");
  *bytes = image_bytes(flow_view(fl));
  return OM_OK;
}

extern "C" om_status om_flow_save_state(const om_flow* fl, void* host, int64_t bytes, void* stream) {
  if (!fl) return fail(OM_EINVAL, "om_flow_save_state: null pointer");
  return save(flow_view(fl), fl->t, host, bytes, as_stream(stream), "om_flow_save_state");
}

extern "C" om_status om_flow_load_state(om_flow* fl, const void* host, int64_t bytes, void* stream) {
  if (!fl) return fail(OM_EINVAL, "om_flow_load_state: null pointer");
  // the image says whether the saved solver was in its rebased mode (it
  // then carries the reference densities); the solver takes that mode
  bool reb = false;
  if (host && bytes >= (int64_t)sizeof(StateHeader)) {
    StateHeader h;
    std::memcpy(&h, host, sizeof h);
    reb = h.has_cr != 0 && fl->rr != nullptr;
  }
  const bool was = fl->reb;
  fl->reb = reb;
  const om_status st = load(flow_view(fl), &fl->t, host, bytes, as_stream(stream), "om_flow_load_state");
  if (st != OM_OK) fl->reb = was;
  return st;
}

extern "C" om_status om_diff_state_size(const om_diff* df, int64_t* bytes) {
  if (!df || !bytes) return fail(OM_EINVAL, "om_diff_state_size: null pointer");
  *bytes = image_bytes(diff_view(df));
  return OM_OK;
}

extern "C" om_status om_diff_save_state(const om_diff* df, void* host, int64_t bytes, void* stream) {
  if (!df) return fail(OM_EINVAL, "om_diff_save_state: null pointer");
  return save(diff_view(df), df->t, host, bytes, as_stream(stream), "om_diff_save_state");
}

extern "C" om_status om_diff_load_state(om_diff* df, const void* host, int64_t bytes, void* stream) {
  if (!df) return fail(OM_EINVAL, "om_diff_load_state: null pointer");
  return load(diff_view(df), &df->t, host, bytes, as_stream(stream), "om_diff_load_state");
}
