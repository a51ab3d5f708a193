// C ABI of the LJ-MD library (declared in include/ljmd.h): argument checks and
// host <-> device marshalling around the engine. Each md_ctx is one system.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ljmd.h"
#include "ljmd_engine.h"

struct md_ctx {
  ljmd::Engine eng;
  cudaStream_t stream = nullptr;  // library-owned stream for the blocking calls
};

namespace {
using ljmd::set_error;

int cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return MD_ERR_CUDA;
}

int check_ctx(md_ctx* c) {
  if (!c) {
    set_error("null context");
    return MD_ERR_ARG;
  }
  set_error("");
  return MD_OK;
}

int64_t n_of(md_ctx* c) { return c->eng.sys(0).spec.n; }

int h2d(md_ctx* c, double* dst, const double* src, int64_t count) {
  cudaError_t e = cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)count, cudaMemcpyHostToDevice, c->stream);
  return e == cudaSuccess ? MD_OK : cuda_fail(e, "host to device copy");
}

int d2h(md_ctx* c, double* dst, const double* src, int64_t count) {
  cudaError_t e = cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "device to host copy");
  e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? MD_OK : cuda_fail(e, "stream synchronize");
}
}  // namespace

extern "C" {

int md_create(double box_L, int64_t N, double rc, double skin, md_ctx** out) {
  set_error("");
  if (!out) {
    set_error("null output handle");
    return MD_ERR_ARG;
  }
  *out = nullptr;
  md_ctx* c = new (std::nothrow) md_ctx();
  if (!c) {
    set_error("host allocation failed");
    return MD_ERR_OOM;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaStreamCreate");
  }
  std::vector<ljmd::SysSpec> specs{{N, box_L, rc, skin}};
  int r = c->eng.init(specs, MD_FP64);
  if (r != MD_OK) {
    std::string msg = ljmd::last_error_cstr();
    cudaStreamDestroy(c->stream);
    delete c;
    set_error(msg);
    return r;
  }
  *out = c;
  return MD_OK;
}

int md_set_precision(md_ctx* c, int mode) {
  int r = check_ctx(c);
  if (r) return r;
  return c->eng.set_precision(mode);
}

int md_set_validity_rule(md_ctx* c, int rule) {
  int r = check_ctx(c);
  if (r) return r;
  return c->eng.set_rule(rule);
}

int md_set_pair_list(md_ctx* c, int kind) {
  int r = check_ctx(c);
  if (r) return r;
  return c->eng.set_list_kind(kind);
}

int md_set_state(md_ctx* c, const double* x, const double* v) {
  int r = check_ctx(c);
  if (r) return r;
  if (!x || !v) {
    set_error("null state array");
    return MD_ERR_ARG;
  }
  const int64_t n = n_of(c);
  double* st = nullptr;
  if ((r = c->eng.stage(n, &st))) return r;
  if ((r = h2d(c, st, x, 3 * n))) return r;
  if ((r = h2d(c, st + 3 * n, v, 3 * n))) return r;
  if ((r = c->eng.set_state_dev(0, st, st + 3 * n, c->stream))) return r;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? MD_OK : cuda_fail(e, "stream synchronize");
}

int md_set_state_dev(md_ctx* c, const double* x, const double* v, void* stream) {
  int r = check_ctx(c);
  if (r) return r;
  if (!x || !v) {
    set_error("null state array");
    return MD_ERR_ARG;
  }
  return c->eng.set_state_dev(0, x, v, (cudaStream_t)stream);
}

int md_get_checkpoint(md_ctx* c, double* x, double* v, double* xref, double* margin) {
  int r = check_ctx(c);
  if (r) return r;
  if (!x || !v || !xref || !margin) {
    set_error("null checkpoint array");
    return MD_ERR_ARG;
  }
  const int64_t n = n_of(c);
  double* st = nullptr;
  if ((r = c->eng.stage(n, &st))) return r;
  // two arrays at a time through the staging buffer (6 n doubles)
  double m = 0.0;
  if ((r = c->eng.get_checkpoint_dev(0, nullptr, nullptr, st, &m, c->stream))) return r;
  if ((r = d2h(c, xref, st, 3 * n))) return r;
  if ((r = c->eng.get_checkpoint_dev(0, st, st + 3 * n, nullptr, nullptr, c->stream))) return r;
  if ((r = d2h(c, x, st, 3 * n))) return r;
  if ((r = d2h(c, v, st + 3 * n, 3 * n))) return r;
  *margin = m;
  return MD_OK;
}

int md_set_checkpoint(md_ctx* c, const double* x, const double* v, const double* xref, double margin) {
  int r = check_ctx(c);
  if (r) return r;
  if (!x || !v || !xref) {
    set_error("null checkpoint array");
    return MD_ERR_ARG;
  }
  const int64_t n = n_of(c);
  double* st = nullptr;
  if ((r = c->eng.stage(n, &st))) return r;
  if ((r = h2d(c, st, xref, 3 * n))) return r;
  if ((r = h2d(c, st + 3 * n, v, 3 * n))) return r;
  if ((r = c->eng.set_checkpoint_dev(0, st, st + 3 * n, c->stream))) return r;
  if ((r = h2d(c, st, x, 3 * n))) return r;
  return c->eng.finish_checkpoint_dev(0, st, margin, c->stream);
}

int md_get_state(md_ctx* c, double* x, double* v) {
  int r = check_ctx(c);
  if (r) return r;
  const int64_t n = n_of(c);
  double* st = nullptr;
  if ((r = c->eng.stage(n, &st))) return r;
  if ((r = c->eng.get_state_dev(0, x ? st : nullptr, v ? st + 3 * n : nullptr, c->stream))) return r;
  if (x && (r = d2h(c, x, st, 3 * n))) return r;
  if (v && (r = d2h(c, v, st + 3 * n, 3 * n))) return r;
  return MD_OK;
}

int md_get_state_dev(md_ctx* c, double* x, double* v, void* stream) {
  int r = check_ctx(c);
  if (r) return r;
  return c->eng.get_state_dev(0, x, v, (cudaStream_t)stream);
}

int md_step_async(md_ctx* c, int64_t nsteps, double dt, void* stream) {
  int r = check_ctx(c);
  if (r) return r;
  std::vector<double> dts{dt};
  return c->eng.step(nsteps, dts, (cudaStream_t)stream);
}

int md_step(md_ctx* c, int64_t nsteps, double dt) {
  int r = check_ctx(c);
  if (r) return r;
  std::vector<double> dts{dt};
  return c->eng.step(nsteps, dts, c->stream);
}

int md_step_nvt(md_ctx* c, int64_t nsteps, double dt, double T, double Q, double* zeta, double* eta) {
  int r = check_ctx(c);
  if (r) return r;
  if (!zeta || !eta) {
    set_error("null thermostat state");
    return MD_ERR_ARG;
  }
  std::vector<double> d{dt}, t{T}, q{Q}, z{*zeta}, e{*eta};
  r = c->eng.step_nvt(nsteps, d, t, q, z, e, c->stream);
  *zeta = z[0];
  *eta = e[0];
  return r;
}

int md_forces(md_ctx* c, double* f) {
  int r = check_ctx(c);
  if (r) return r;
  if (!f) {
    set_error("null force array");
    return MD_ERR_ARG;
  }
  double* st = nullptr;
  if ((r = c->eng.stage(n_of(c), &st))) return r;
  if ((r = c->eng.forces_dev(0, st, c->stream))) return r;
  return d2h(c, f, st, 3 * n_of(c));
}

int md_forces_dev(md_ctx* c, double* f, void* stream) {
  int r = check_ctx(c);
  if (r) return r;
  if (!f) {
    set_error("null force array");
    return MD_ERR_ARG;
  }
  return c->eng.forces_dev(0, f, (cudaStream_t)stream);
}

int md_observables(md_ctx* c, double* pe, double* virial, double* ke, double* T, double* P) {
  int r = check_ctx(c);
  if (r) return r;
  double o[3];
  if ((r = c->eng.observables(o, c->stream))) return r;
  const int64_t n = n_of(c);
  const double L = c->eng.sys(0).spec.L;
  if (pe) *pe = o[0];
  if (virial) *virial = o[1];
  if (ke) *ke = o[2];
  if (T) *T = n > 1 ? 2.0 * o[2] / (3.0 * (double)(n - 1)) : 0.0;
  if (P) *P = (2.0 * o[2] + o[1]) / (3.0 * L * L * L);
  return MD_OK;
}

int md_kinetic_energy(md_ctx* c, double* ke) {
  int r = check_ctx(c);
  if (r) return r;
  if (!ke) {
    set_error("null output");
    return MD_ERR_ARG;
  }
  double o[3];
  if ((r = c->eng.observables(o, c->stream, false))) return r;
  *ke = o[2];
  return MD_OK;
}

int md_scale_velocities(md_ctx* c, double factor) {
  int r = check_ctx(c);
  if (r) return r;
  std::vector<double> f{factor};
  return c->eng.scale_velocities(f, c->stream);
}

int md_stats(md_ctx* c, int64_t* rebuilds, int64_t* steps) {
  int r = check_ctx(c);
  if (r) return r;
  if (rebuilds) *rebuilds = c->eng.sys(0).rebuilds;
  if (steps) *steps = c->eng.sys(0).steps;
  return MD_OK;
}

int md_build_list(md_ctx* c) {
  int r = check_ctx(c);
  if (r) return r;
  return c->eng.build_lists(c->stream);
}

int md_get_cells(md_ctx* c, int32_t* cell, int32_t* nc_out) {
  int r = check_ctx(c);
  if (r) return r;
  if (nc_out) *nc_out = c->eng.sys(0).nc;
  if (!cell) return MD_OK;
  return c->eng.get_cells(0, cell, c->stream);
}

int md_list_size(md_ctx* c, int64_t* total) {
  int r = check_ctx(c);
  if (r) return r;
  if (!total) {
    set_error("null output");
    return MD_ERR_ARG;
  }
  return c->eng.list_size(0, total, c->stream);
}

int md_debug_set_list_word(md_ctx* c, int64_t slot, int32_t entry, uint32_t word) {
  int r = check_ctx(c);
  if (r) return r;
  return c->eng.debug_set_list_word(0, slot, entry, word, c->stream);
}

int md_get_list(md_ctx* c, int64_t* start, int32_t* partners) {
  int r = check_ctx(c);
  if (r) return r;
  if (!start || !partners) {
    set_error("null output");
    return MD_ERR_ARG;
  }
  return c->eng.get_list(0, start, partners, c->stream);
}

int md_bubbles(md_ctx* c, double side, double gas_density, int32_t* ns_out, uint8_t* counts,
               int64_t* n_bubbles, int64_t* sizes, int64_t cap) {
  int r = check_ctx(c);
  if (r) return r;
  int ns = 0;
  std::vector<uint32_t> cnt;
  std::vector<int64_t> sz;
  if ((r = c->eng.bubbles(0, side, gas_density, &ns, &cnt, &sz, c->stream))) return r;
  if (ns_out) *ns_out = ns;
  if (counts)
    for (size_t q = 0; q < cnt.size(); ++q) counts[q] = (uint8_t)(cnt[q] > 255u ? 255u : cnt[q]);
  if (n_bubbles) *n_bubbles = (int64_t)sz.size();
  if (sizes)
    for (int64_t q = 0; q < (int64_t)sz.size() && q < cap; ++q) sizes[q] = sz[(size_t)q];
  return MD_OK;
}

int md_set_timing(md_ctx* c, int on) {
  int r = check_ctx(c);
  if (r) return r;
  return c->eng.set_timing(on != 0);
}

int md_get_timing(md_ctx* c, double* out8) {
  int r = check_ctx(c);
  if (r) return r;
  if (!out8) {
    set_error("null output");
    return MD_ERR_ARG;
  }
  c->eng.get_timing(out8);
  return MD_OK;
}

int md_pair_stats(md_ctx* c, int64_t* listed, int64_t* within_rc) {
  int r = check_ctx(c);
  if (r) return r;
  if (!listed || !within_rc) {
    set_error("null output");
    return MD_ERR_ARG;
  }
  return c->eng.pair_stats(0, listed, within_rc, c->stream);
}

int md_set_tuning(md_ctx* c, int key, int value) {
  int r = check_ctx(c);
  if (r) return r;
  return c->eng.set_tuning(key, value);
}

int md_get_tuning(md_ctx* c, int key, int* value) {
  int r = check_ctx(c);
  if (r) return r;
  if (!value) {
    set_error("null output");
    return MD_ERR_ARG;
  }
  *value = c->eng.get_tuning(key);
  if (*value < 0) {
    set_error("unknown tuning key");
    return MD_ERR_ARG;
  }
  return MD_OK;
}

void md_destroy(md_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  cudaStream_t s = c->stream;
  delete c;
  if (s) cudaStreamDestroy(s);
}

const char* md_last_error(void) { return ljmd::last_error_cstr(); }

// ----------------------------------------------------------------- batches

struct md_batch {
  ljmd::Engine eng;
  cudaStream_t stream = nullptr;
};

namespace {
int check_batch(md_batch* b) {
  if (!b) {
    set_error("null batch");
    return MD_ERR_ARG;
  }
  set_error("");
  return MD_OK;
}

int check_id(md_batch* b, int id) {
  if (!b->eng.valid_id(id)) {
    set_error("no such system id");
    return MD_ERR_ARG;
  }
  return MD_OK;
}

int new_batch(md_batch** out, md_batch** b) {
  if (!out) {
    set_error("null output handle");
    return MD_ERR_ARG;
  }
  *out = nullptr;
  *b = new (std::nothrow) md_batch();
  if (!*b) {
    set_error("host allocation failed");
    return MD_ERR_OOM;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&(*b)->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete *b;
    *b = nullptr;
    return cuda_fail(e, "cudaStreamCreate");
  }
  return MD_OK;
}

int finish_batch(int r, md_batch* b, md_batch** out) {
  if (r != MD_OK) {
    std::string msg = ljmd::last_error_cstr();
    cudaStreamDestroy(b->stream);
    delete b;
    set_error(msg);
    return r;
  }
  *out = b;
  return MD_OK;
}

ljmd::SysSpec spec_of(const md_sys_desc& d) { return ljmd::SysSpec{d.N, d.box_L, d.rc, d.skin}; }

int bh2d(md_batch* b, double* dst, const double* src, int64_t count) {
  cudaError_t e = cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)count, cudaMemcpyHostToDevice, b->stream);
  return e == cudaSuccess ? MD_OK : cuda_fail(e, "host to device copy");
}

int bd2h(md_batch* b, double* dst, const double* src, int64_t count) {
  cudaError_t e = cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost, b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "device to host copy");
  e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? MD_OK : cuda_fail(e, "stream synchronize");
}
}  // namespace

int md_batch_create(int nsys, const md_sys_desc* desc, int precision, md_batch** out) {
  set_error("");
  if (nsys <= 0 || !desc) {
    set_error("need nsys > 0 and a descriptor array");
    return MD_ERR_ARG;
  }
  md_batch* b = nullptr;
  int r = new_batch(out, &b);
  if (r) return r;
  std::vector<ljmd::SysSpec> specs;
  for (int k = 0; k < nsys; ++k) specs.push_back(spec_of(desc[k]));
  return finish_batch(b->eng.init(specs, precision), b, out);
}

int md_batch_create_arena(int64_t slots, int64_t cells, int64_t list_words, int max_systems, int precision,
                          md_batch** out) {
  set_error("");
  md_batch* b = nullptr;
  int r = new_batch(out, &b);
  if (r) return r;
  ljmd::ArenaCaps caps{slots, cells, list_words, max_systems};
  return finish_batch(b->eng.init_arena(caps, precision), b, out);
}

int md_batch_footprint(const md_sys_desc* desc, int64_t* slots, int64_t* cells, int64_t* list_words) {
  set_error("");
  if (!desc) {
    set_error("null descriptor");
    return MD_ERR_ARG;
  }
  ljmd::SysFootprint f;
  int r = ljmd::footprint(spec_of(*desc), &f, nullptr);
  if (r) return r;
  if (slots) *slots = f.slots;
  if (cells) *cells = f.cells;
  if (list_words) *list_words = f.list_words;
  return MD_OK;
}

int md_batch_add(md_batch* b, const md_sys_desc* desc, int* id) {
  int r = check_batch(b);
  if (r) return r;
  if (!desc || !id) {
    set_error("null argument");
    return MD_ERR_ARG;
  }
  return b->eng.add_system(spec_of(*desc), id);
}

int md_batch_remove(md_batch* b, int id) {
  int r = check_batch(b);
  if (r) return r;
  if ((r = check_id(b, id))) return r;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  return b->eng.remove_system(id);
}

int md_batch_usage(md_batch* b, int64_t* out8) {
  int r = check_batch(b);
  if (r) return r;
  if (!out8) {
    set_error("null output");
    return MD_ERR_ARG;
  }
  b->eng.arena_usage(out8);
  return MD_OK;
}

int md_batch_set_active(md_batch* b, int id, int on) {
  int r = check_batch(b);
  if (r) return r;
  return b->eng.set_active(id, on != 0);
}

int md_batch_set_precision(md_batch* b, int mode) {
  int r = check_batch(b);
  if (r) return r;
  return b->eng.set_precision(mode);
}

int md_batch_set_validity_rule(md_batch* b, int rule) {
  int r = check_batch(b);
  if (r) return r;
  return b->eng.set_rule(rule);
}

int md_batch_set_pair_list(md_batch* b, int kind) {
  int r = check_batch(b);
  if (r) return r;
  return b->eng.set_list_kind(kind);
}

int md_batch_set_state(md_batch* b, int id, const double* x, const double* v) {
  int r = check_batch(b);
  if (r) return r;
  if ((r = check_id(b, id))) return r;
  if (!x || !v) {
    set_error("null state array");
    return MD_ERR_ARG;
  }
  const int64_t n = b->eng.sys(id).spec.n;
  double* st = nullptr;
  if ((r = b->eng.stage(n, &st))) return r;
  if ((r = bh2d(b, st, x, 3 * n))) return r;
  if ((r = bh2d(b, st + 3 * n, v, 3 * n))) return r;
  if ((r = b->eng.set_state_dev(id, st, st + 3 * n, b->stream))) return r;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? MD_OK : cuda_fail(e, "stream synchronize");
}

int md_batch_set_state_dev(md_batch* b, int id, const double* x, const double* v, void* stream) {
  int r = check_batch(b);
  if (r) return r;
  if (!x || !v) {
    set_error("null state array");
    return MD_ERR_ARG;
  }
  return b->eng.set_state_dev(id, x, v, (cudaStream_t)stream);
}

int md_batch_get_state(md_batch* b, int id, double* x, double* v) {
  int r = check_batch(b);
  if (r) return r;
  if ((r = check_id(b, id))) return r;
  const int64_t n = b->eng.sys(id).spec.n;
  double* st = nullptr;
  if ((r = b->eng.stage(n, &st))) return r;
  if ((r = b->eng.get_state_dev(id, x ? st : nullptr, v ? st + 3 * n : nullptr, b->stream))) return r;
  if (x && (r = bd2h(b, x, st, 3 * n))) return r;
  if (v && (r = bd2h(b, v, st + 3 * n, 3 * n))) return r;
  return MD_OK;
}

int md_batch_get_checkpoint(md_batch* b, int id, double* x, double* v, double* xref, double* margin) {
  int r = check_batch(b);
  if (r) return r;
  if ((r = check_id(b, id))) return r;
  if (!x || !v || !xref || !margin) {
    set_error("null checkpoint array");
    return MD_ERR_ARG;
  }
  const int64_t n = b->eng.sys(id).spec.n;
  double* st = nullptr;
  if ((r = b->eng.stage(n, &st))) return r;
  double m = 0.0;
  if ((r = b->eng.get_checkpoint_dev(id, nullptr, nullptr, st, &m, b->stream))) return r;
  if ((r = bd2h(b, xref, st, 3 * n))) return r;
  if ((r = b->eng.get_checkpoint_dev(id, st, st + 3 * n, nullptr, nullptr, b->stream))) return r;
  if ((r = bd2h(b, x, st, 3 * n))) return r;
  if ((r = bd2h(b, v, st + 3 * n, 3 * n))) return r;
  *margin = m;
  return MD_OK;
}

int md_batch_set_checkpoint(md_batch* b, int id, const double* x, const double* v, const double* xref,
                            double margin) {
  int r = check_batch(b);
  if (r) return r;
  if ((r = check_id(b, id))) return r;
  if (!x || !v || !xref) {
    set_error("null checkpoint array");
    return MD_ERR_ARG;
  }
  const int64_t n = b->eng.sys(id).spec.n;
  double* st = nullptr;
  if ((r = b->eng.stage(n, &st))) return r;
  if ((r = bh2d(b, st, xref, 3 * n))) return r;
  if ((r = bh2d(b, st + 3 * n, v, 3 * n))) return r;
  if ((r = b->eng.set_checkpoint_dev(id, st, st + 3 * n, b->stream))) return r;
  if ((r = bh2d(b, st, x, 3 * n))) return r;
  return b->eng.finish_checkpoint_dev(id, st, margin, b->stream);
}

int md_batch_get_state_dev(md_batch* b, int id, double* x, double* v, void* stream) {
  int r = check_batch(b);
  if (r) return r;
  return b->eng.get_state_dev(id, x, v, (cudaStream_t)stream);
}

int md_batch_step_async(md_batch* b, int64_t nsteps, const double* dt, void* stream) {
  int r = check_batch(b);
  if (r) return r;
  if (!dt) {
    set_error("null dt array");
    return MD_ERR_ARG;
  }
  std::vector<double> dts(dt, dt + b->eng.nsys());
  return b->eng.step(nsteps, dts, (cudaStream_t)stream);
}

int md_batch_step(md_batch* b, int64_t nsteps, const double* dt) {
  int r = check_batch(b);
  if (r) return r;
  return md_batch_step_async(b, nsteps, dt, b->stream);
}

int md_batch_step_nvt(md_batch* b, int64_t nsteps, const double* dt, const double* T, const double* Q,
                      double* zeta, double* eta) {
  int r = check_batch(b);
  if (r) return r;
  if (!dt || !T || !Q || !zeta || !eta) {
    set_error("null argument");
    return MD_ERR_ARG;
  }
  const int ns = b->eng.nsys();
  std::vector<double> d(dt, dt + ns), t(T, T + ns), q(Q, Q + ns), z(zeta, zeta + ns), e(eta, eta + ns);
  r = b->eng.step_nvt(nsteps, d, t, q, z, e, b->stream);
  std::copy(z.begin(), z.end(), zeta);
  std::copy(e.begin(), e.end(), eta);
  return r;
}

int md_batch_forces(md_batch* b, int id, double* f) {
  int r = check_batch(b);
  if (r) return r;
  if ((r = check_id(b, id))) return r;
  if (!f) {
    set_error("null force array");
    return MD_ERR_ARG;
  }
  const int64_t n = b->eng.sys(id).spec.n;
  double* st = nullptr;
  if ((r = b->eng.stage(n, &st))) return r;
  if ((r = b->eng.forces_dev(id, st, b->stream))) return r;
  return bd2h(b, f, st, 3 * n);
}

int md_batch_observables_select(md_batch* b, const int32_t* select, double* out) {
  int r = check_batch(b);
  if (r) return r;
  if (!out) {
    set_error("null output");
    return MD_ERR_ARG;
  }
  const int ns = b->eng.nsys();
  std::vector<double> o3((size_t)(3 * ns));
  if ((r = b->eng.observables(o3.data(), b->stream, true, select))) return r;
  for (int k = 0; k < ns; ++k) {
    double* q = out + 5 * k;
    const ljmd::SysHost& h = b->eng.sys(k);
    if (!h.used || !h.active || (select && !select[k])) {
      for (int m = 0; m < 5; ++m) q[m] = 0.0;
      continue;
    }
    const int64_t n = h.spec.n;
    const double L = h.spec.L;
    q[0] = o3[3 * k + 0];
    q[1] = o3[3 * k + 1];
    q[2] = o3[3 * k + 2];
    q[3] = n > 1 ? 2.0 * q[2] / (3.0 * (double)(n - 1)) : 0.0;
    q[4] = (2.0 * q[2] + q[1]) / (3.0 * L * L * L);
  }
  return MD_OK;
}

int md_batch_kinetic_energy(md_batch* b, double* ke) {
  int r = check_batch(b);
  if (r) return r;
  if (!ke) {
    set_error("null output");
    return MD_ERR_ARG;
  }
  const int ns = b->eng.nsys();
  std::vector<double> o3((size_t)(3 * ns));
  if ((r = b->eng.observables(o3.data(), b->stream, false))) return r;
  for (int k = 0; k < ns; ++k) {
    const ljmd::SysHost& h = b->eng.sys(k);
    ke[k] = (h.used && h.active) ? o3[3 * k + 2] : 0.0;
  }
  return MD_OK;
}

int md_batch_scale_velocities(md_batch* b, const double* factor) {
  int r = check_batch(b);
  if (r) return r;
  if (!factor) {
    set_error("null factor array");
    return MD_ERR_ARG;
  }
  std::vector<double> f(factor, factor + b->eng.nsys());
  return b->eng.scale_velocities(f, b->stream);
}

int md_batch_observables(md_batch* b, double* out) { return md_batch_observables_select(b, nullptr, out); }

int md_batch_stats(md_batch* b, int id, int64_t* rebuilds, int64_t* steps) {
  int r = check_batch(b);
  if (r) return r;
  if ((r = check_id(b, id))) return r;
  if (rebuilds) *rebuilds = b->eng.sys(id).rebuilds;
  if (steps) *steps = b->eng.sys(id).steps;
  return MD_OK;
}

int md_batch_set_tuning(md_batch* b, int key, int value) {
  int r = check_batch(b);
  if (r) return r;
  return b->eng.set_tuning(key, value);
}

int md_batch_get_tuning(md_batch* b, int key, int* value) {
  int r = check_batch(b);
  if (r) return r;
  if (!value) {
    set_error("null output");
    return MD_ERR_ARG;
  }
  *value = b->eng.get_tuning(key);
  if (*value < 0) {
    set_error("unknown tuning key");
    return MD_ERR_ARG;
  }
  return MD_OK;
}

int md_batch_set_timing(md_batch* b, int on) {
  int r = check_batch(b);
  if (r) return r;
  return b->eng.set_timing(on != 0);
}

int md_batch_get_timing(md_batch* b, double* out8) {
  int r = check_batch(b);
  if (r) return r;
  if (!out8) {
    set_error("null output");
    return MD_ERR_ARG;
  }
  b->eng.get_timing(out8);
  return MD_OK;
}

void md_batch_destroy(md_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  cudaStream_t s = b->stream;
  delete b;
  if (s) cudaStreamDestroy(s);
}

const char* md_version(void) {
#ifdef LJMD_CHECKS
  return "ljmd 0.1 (sm_103a, checked)";
#else
  return "ljmd 0.1 (sm_103a)";
#endif
}

}  // extern "C"
