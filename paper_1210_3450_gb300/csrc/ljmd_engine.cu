// Host engine of the LJ-MD library: layout of systems in the shared device
// arrays, the velocity-Verlet step loop, the list-validity check of Sec. 2.1 of
// the paper (rebuild when twice the largest displacement since the last build
// reaches the skin) and the rebuild sequence (bin, sort, gather, list build).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "ljmd_engine.h"

namespace ljmd {

namespace {
thread_local std::string g_err;

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));             \
      return e_ == cudaErrorMemoryAllocation ? kErrOOM : kErrCuda;                \
    }                                                                             \
  } while (0)

#define CKL()                                                                     \
  do {                                                                            \
    cudaError_t e_ = cudaGetLastError();                                          \
    if (e_ != cudaSuccess) {                                                      \
      set_error(std::string("kernel launch: ") + cudaGetErrorString(e_));        \
      return kErrCuda;                                                            \
    }                                                                             \
  } while (0)

#define CKR(expr)             \
  do {                        \
    int r_ = (expr);          \
    if (r_ != kOK) return r_; \
  } while (0)

template <class T>
int dmalloc(T** p, int64_t count) {
  *p = nullptr;
  if (count <= 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (size_t)count);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return kErrOOM;
  }
  return kOK;
}

template <class T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

template <class T>
void hfree(T*& p) {
  if (p) cudaFreeHost((void*)p);
  p = nullptr;
}

// Cells per axis: floor(L / rl), lowered by one if the cell side is not
// clearly above rl, and 1 (every pair a candidate) if fewer than 3 remain.
int cells_per_axis(double L, double rl) {
  int nc = (int)std::floor(L / rl);
  if (nc >= 1 && L / nc < rl * (1.0 + 1e-9)) nc -= 1;
  return nc >= 3 ? nc : 1;
}

int initial_kmax(const SysSpec& s, double rl) {
  const double rho = (double)s.n / (s.L * s.L * s.L);
  const double expect = 4.0 / 3.0 * M_PI * rl * rl * rl * rho;
  int64_t k = round_up((int64_t)(1.35 * expect + 32.0), 8);
  const int64_t cap = round_up(std::max<int64_t>(s.n - 1, 1), 8);
  return (int)std::min(k, cap);
}
}  // namespace

void set_error(const std::string& msg) { g_err = msg; }
const char* last_error_cstr() { return g_err.c_str(); }

Engine::~Engine() {
  free_all();
  for (cudaEvent_t e : ev_free_) cudaEventDestroy(e);
  for (TimedPair& p : ev_pending_) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
}

int Engine::set_timing(bool on) {
  timing_ = on;
  for (int k = 0; k < 3; ++k) { t_ms_[k] = 0.0; t_count_[k] = 0; }
  n_launch_ = 0;
  n_rebuild_seq_ = 0;
  return kOK;
}

void Engine::get_timing(double* out8) const {
  out8[0] = t_ms_[kTStep];
  out8[1] = (double)t_count_[kTStep];
  out8[2] = t_ms_[kTList];
  out8[3] = (double)t_count_[kTList];
  out8[4] = t_ms_[kTBin];
  out8[5] = (double)n_rebuild_seq_;
  out8[6] = (double)n_launch_;
  out8[7] = 0.0;
}

void Engine::tmark_begin(int kind, cudaStream_t s) {
  if (!timing_) return;
  auto take = [&]() {
    cudaEvent_t e;
    if (!ev_free_.empty()) { e = ev_free_.back(); ev_free_.pop_back(); }
    else cudaEventCreate(&e);
    return e;
  };
  ev_open_ = TimedPair{take(), take(), kind};
  cudaEventRecord(ev_open_.a, s);
}

void Engine::tmark_end(cudaStream_t s) {
  if (!timing_ || ev_open_.kind < 0) return;
  cudaEventRecord(ev_open_.b, s);
  ev_pending_.push_back(ev_open_);
  ev_open_.kind = -1;
}

// Called after a stream synchronisation: every pending pair has completed.
void Engine::collect_timing() {
  for (TimedPair& p : ev_pending_) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      t_ms_[p.kind] += ms;
      t_count_[p.kind] += 1;
    }
    ev_free_.push_back(p.a);
    ev_free_.push_back(p.b);
  }
  ev_pending_.clear();
}

void Engine::free_all() {
  for (int b = 0; b < 2; ++b) { dfree(d_.x[b]); dfree(d_.xq[b]); }
  dfree(d_.v); dfree(d_.xref); dfree(d_.f); dfree(d_.id); dfree(d_.cell); dfree(d_.ncnt);
  dfree(d_.nbr); dfree(d_.tile_obs); dfree(d_.xtmp); dfree(d_.vtmp); dfree(d_.idtmp);
  dfree(d_.celltmp); dfree(d_.perm); dfree(d_.ccount); dfree(d_.cstart);
  dfree(d_params_); dfree(d_status_); dfree(d_disp2_); dfree(d_rebuild_); dfree(d_tile_sys_);
  dfree(d_obs_); dfree(d_stage_); dfree(d_pairs_);
  hfree(h_status_); hfree(h_disp2_); hfree(h_rebuild_); hfree(h_obs_);
  d_ = DevArrays{};
}

int Engine::init(const std::vector<SysSpec>& specs, int precision) {
  if (specs.empty()) { set_error("no systems"); return kErrArg; }
  if (precision != 0 && precision != 1) { set_error("unknown precision mode"); return kErrArg; }
  precision_ = precision;
  sys_.clear();
  int64_t p = 0, c = 0, l = 0;
  int32_t t = 0;
  stage_n_ = 0;
  max_cells_ = 1;
  for (const SysSpec& s : specs) {
    if (!(s.n > 0) || s.n > ((1 << 26) - 1)) { set_error("N must be in [1, 2^26 - 1]"); return kErrArg; }
    if (!(s.rc > 0.0) || !(s.skin >= 0.0) || !std::isfinite(s.rc) || !std::isfinite(s.skin)) {
      set_error("rc must be > 0 and skin >= 0");
      return kErrArg;
    }
    if (!(s.L > 2.0 * (s.rc + s.skin)) || !(s.L <= 10000.0)) {
      set_error("box side must satisfy 2 (rc + skin) < L <= 10000");
      return kErrArg;
    }
    SysHost h;
    h.spec = s;
    h.rl = s.rc + s.skin;
    // Eq. 1: V(rc) = V'(rc) = 0
    const double irc2 = 1.0 / (s.rc * s.rc);
    const double irc6 = irc2 * irc2 * irc2;
    h.c2 = 6.0 * irc6 * irc6 * irc2 - 3.0 * irc6 * irc2;
    h.c0 = 4.0 * irc6 - 7.0 * irc6 * irc6;
    h.nc = cells_per_axis(s.L, h.rl);
    h.ncell = (int64_t)h.nc * h.nc * h.nc;
    h.kmax = initial_kmax(s, h.rl);
    h.ntiles = (int32_t)((s.n + kTile - 1) / kTile);
    h.p_off = p;
    h.t_off = t;
    h.c_off = c;
    h.l_off = l;
    p += (int64_t)h.ntiles * kTile;
    t += h.ntiles;
    c += h.ncell + 1;
    l += (int64_t)h.ntiles * h.kmax * kTile;
    max_cells_ = std::max(max_cells_, h.ncell);
    stage_n_ = std::max(stage_n_, s.n);
    sys_.push_back(h);
  }
  nslots_ = p;
  ntiles_ = t;
  ncells_ = c;
  nlist_ = l;
  return alloc_all();
}

int Engine::alloc_all() {
  free_all();
  const int ns = nsys();
  for (int b = 0; b < 2; ++b) {
    CKR(dmalloc(&d_.x[b], nslots_));
    CKR(dmalloc(&d_.xq[b], nslots_));
    CK(cudaMemset(d_.x[b], 0, sizeof(double4_32a) * nslots_));
    CK(cudaMemset(d_.xq[b], 0, sizeof(int4) * nslots_));
  }
  CKR(dmalloc(&d_.v, nslots_));
  CKR(dmalloc(&d_.xref, nslots_));
  CKR(dmalloc(&d_.f, nslots_));
  CKR(dmalloc(&d_.id, nslots_));
  CKR(dmalloc(&d_.cell, nslots_));
  CKR(dmalloc(&d_.ncnt, nslots_));
  CKR(dmalloc(&d_.nbr, nlist_));
  CKR(dmalloc(&d_.tile_obs, 3 * (int64_t)ntiles_));
  CKR(dmalloc(&d_.xtmp, nslots_));
  CKR(dmalloc(&d_.vtmp, nslots_));
  CKR(dmalloc(&d_.idtmp, nslots_));
  CKR(dmalloc(&d_.celltmp, nslots_));
  CKR(dmalloc(&d_.perm, nslots_));
  CKR(dmalloc(&d_.ccount, ncells_));
  CKR(dmalloc(&d_.cstart, ncells_));
  CK(cudaMemset(d_.v, 0, sizeof(double4_32a) * nslots_));
  CK(cudaMemset(d_.f, 0, sizeof(double4_32a) * nslots_));
  CK(cudaMemset(d_.xref, 0, sizeof(double4_32a) * nslots_));
  CK(cudaMemset(d_.ncnt, 0, sizeof(int32_t) * nslots_));
  CK(cudaMemset(d_.id, 0xff, sizeof(int32_t) * nslots_));
  CK(cudaMemset(d_.ccount, 0, sizeof(int32_t) * ncells_));
  CK(cudaMemset(d_.cstart, 0, sizeof(int32_t) * ncells_));
  CKR(dmalloc(&d_params_, ns));
  CKR(dmalloc(&d_status_, ns));
  CKR(dmalloc(&d_disp2_, ns));
  CKR(dmalloc(&d_rebuild_, ns));
  CKR(dmalloc(&d_tile_sys_, ntiles_));
  CKR(dmalloc(&d_obs_, 3 * ns));
  CKR(dmalloc(&d_pairs_, 2 * ns));
  CKR(dmalloc(&d_stage_, 6 * stage_n_));
  CK(cudaMemset(d_status_, 0, sizeof(SysStatus) * ns));
  CK(cudaMemset(d_disp2_, 0, sizeof(unsigned long long) * ns));
  CK(cudaMallocHost((void**)&h_status_, sizeof(SysStatus) * ns));
  CK(cudaMallocHost((void**)&h_disp2_, sizeof(unsigned long long) * ns));
  CK(cudaMallocHost((void**)&h_rebuild_, sizeof(int32_t) * ns));
  CK(cudaMallocHost((void**)&h_obs_, sizeof(double) * 3 * ns));
  std::vector<int32_t> ts((size_t)ntiles_);
  for (int k = 0; k < ns; ++k)
    for (int q = 0; q < sys_[k].ntiles; ++q) ts[(size_t)(sys_[k].t_off + q)] = k;
  CK(cudaMemcpy(d_tile_sys_, ts.data(), sizeof(int32_t) * ts.size(), cudaMemcpyHostToDevice));
  return upload_params();
}

int Engine::upload_params() {
  std::vector<SysParams> ps((size_t)nsys());
  for (int k = 0; k < nsys(); ++k) {
    const SysHost& h = sys_[k];
    SysParams& P = ps[(size_t)k];
    std::memset(&P, 0, sizeof(P));
    P.L = h.spec.L;
    P.invL = 1.0 / h.spec.L;
    P.inv_cs = (double)h.nc / h.spec.L;
    P.rc2 = h.spec.rc * h.spec.rc;
    P.rl2 = h.rl * h.rl;
    P.c2 = h.c2;
    P.c0 = h.c0;
    P.dt = h.dt;
    P.qscale = 4294967296.0 / h.spec.L;
    P.qunit = (float)(h.spec.L / 4294967296.0);
    P.rl2q_lo = (float)(P.rl2 * P.qscale * P.qscale * (1.0 - 1e-5));
    P.rl2q_hi = (float)(P.rl2 * P.qscale * P.qscale * (1.0 + 1e-5));
    P.rc2f = (float)P.rc2;
    P.c2f = (float)h.c2;
    P.p_off = h.p_off;
    P.c_off = h.c_off;
    P.l_off = h.l_off;
    P.n = (int32_t)h.spec.n;
    P.nc = h.nc;
    P.kmax = h.kmax;
    P.t_off = h.t_off;
    P.ntiles = h.ntiles;
    P.active = h.active ? 1 : 0;
  }
  CK(cudaMemcpy(d_params_, ps.data(), sizeof(SysParams) * ps.size(), cudaMemcpyHostToDevice));
  return kOK;
}

DevArrays Engine::arrays() const {
  DevArrays a = d_;
  a.params = d_params_;
  a.status = d_status_;
  a.disp2 = d_disp2_;
  a.rebuild = d_rebuild_;
  a.tile_sys = d_tile_sys_;
  a.ntiles = ntiles_;
  return a;
}

int Engine::set_precision(int mode) {
  if (mode != 0 && mode != 1) { set_error("unknown precision mode"); return kErrArg; }
  if (mode != precision_) {
    precision_ = mode;
    for (SysHost& h : sys_) {
      h.f_valid = false;
      if (h.has_state) h.force_rebuild = true;  // refresh the fixed-point shadow
    }
  }
  return kOK;
}

void Engine::set_active(int k, bool on) { sys_[k].active = on; }

int Engine::set_state_dev(int k, const double* x, const double* v, cudaStream_t s) {
  SysHost& h = sys_[k];
  launch_from_caller(arrays(), cur_, x, v, k, h.ntiles, s);
  CKL();
  h.has_state = true;
  h.force_rebuild = true;
  h.f_valid = false;
  return kOK;
}

int Engine::get_state_dev(int k, double* x, double* v, cudaStream_t s) {
  SysHost& h = sys_[k];
  if (!h.has_state) { set_error("no state set"); return kErrState; }
  if (x) launch_to_caller(arrays(), cur_, 0, x, h.spec.n, k, h.ntiles, s);
  if (v) launch_to_caller(arrays(), cur_, 1, v, h.spec.n, k, h.ntiles, s);
  CKL();
  return kOK;
}

int Engine::sync_check(cudaStream_t s) {
  CK(cudaStreamSynchronize(s));
  collect_timing();
  return kOK;
}

// Full rebuild (bin, stable counting sort, gather, list) of the given systems.
int Engine::rebuild(std::vector<int> which, cudaStream_t s) {
  if (which.empty()) return kOK;
  for (int attempt = 0; attempt < 4; ++attempt) {
    for (int k = 0; k < nsys(); ++k) h_rebuild_[k] = 0;
    for (int k : which) h_rebuild_[k] = 1;
    CK(cudaMemcpyAsync(d_rebuild_, h_rebuild_, sizeof(int32_t) * nsys(), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(d_status_, 0, sizeof(SysStatus) * nsys(), s));
    const DevArrays a = arrays();
    tmark_begin(kTBin, s);
    launch_cell_count(a, cur_, s);
    launch_cell_scan(a, nsys(), s);
    launch_scatter(a, s);
    launch_cell_sort(a, nsys(), max_cells_, s);
    launch_gather(a, cur_, s);
    launch_copyback(a, cur_, s);
    tmark_end(s);
    tmark_begin(kTList, s);
    launch_build_list(a, cur_, s);
    tmark_end(s);
    CKL();
    n_launch_ += 7;
    n_rebuild_seq_ += 1;
    CK(cudaMemcpyAsync(h_status_, d_status_, sizeof(SysStatus) * nsys(), cudaMemcpyDeviceToHost, s));
    CKR(sync_check(s));
    bool grow = false;
    for (int k : which) {
      if (h_status_[k].overflow > 0) {
        SysHost& h = sys_[k];
        const int64_t cap = round_up(std::max<int64_t>(h.spec.n - 1, 1), 8);
        const int64_t want = std::min<int64_t>(round_up((int64_t)(h_status_[k].overflow * 1.25) + 16, 8), cap);
        if (want <= h.kmax) { set_error("pair list overflow"); return kErrOverflow; }
        h.kmax = (int)want;
        grow = true;
      }
    }
    if (!grow) {
      for (int k : which) {
        sys_[k].rebuilds += 1;
        sys_[k].force_rebuild = false;
        sys_[k].f_valid = false;
      }
      return kOK;
    }
    // re-lay the list storage with the larger capacities and rebuild every
    // active system that has a state (their old lists moved)
    int64_t l = 0;
    for (SysHost& h : sys_) {
      h.l_off = l;
      l += (int64_t)h.ntiles * h.kmax * kTile;
    }
    nlist_ = l;
    dfree(d_.nbr);
    CKR(dmalloc(&d_.nbr, nlist_));
    CKR(upload_params());
    std::vector<int> all;
    for (int k = 0; k < nsys(); ++k)
      if (sys_[k].active && sys_[k].has_state) all.push_back(k);
    which = all;
  }
  set_error("pair list overflow persists after growing the capacity");
  return kErrOverflow;
}

int Engine::ensure_lists(cudaStream_t s) {
  std::vector<int> which;
  for (int k = 0; k < nsys(); ++k) {
    const SysHost& h = sys_[k];
    if (!h.active) continue;
    if (!h.has_state) { set_error("no state set"); return kErrState; }
    if (h.force_rebuild) which.push_back(k);
  }
  return rebuild(which, s);
}

int Engine::launch_step(double ka, double kb, int flags, cudaStream_t s) {
  const DevArrays a = arrays();
  tmark_begin(kTStep, s);
  if (precision_ == 1) launch_step_fp32(a, cur_, ka, kb, flags, s);
  else launch_step_fp64(a, cur_, ka, kb, flags, s);
  tmark_end(s);
  CKL();
  n_launch_ += 1;
  return kOK;
}

int Engine::pair_stats(int k, int64_t* listed, int64_t* inside, cudaStream_t s) {
  if (!sys_[k].has_state) { set_error("no state set"); return kErrState; }
  CKR(ensure_lists(s));
  CK(cudaMemsetAsync(d_pairs_, 0, sizeof(unsigned long long) * 2 * nsys(), s));
  launch_pair_stats(arrays(), cur_, d_pairs_, s);
  CKL();
  unsigned long long h[2];
  CK(cudaMemcpyAsync(h, d_pairs_ + 2 * k, sizeof(h), cudaMemcpyDeviceToHost, s));
  CKR(sync_check(s));
  *listed = (int64_t)h[0];
  *inside = (int64_t)h[1];
  return kOK;
}

int Engine::ensure_forces(cudaStream_t s) {
  bool need = false;
  for (const SysHost& h : sys_)
    if (h.active && !h.f_valid) need = true;
  if (!need) return kOK;
  CKR(launch_step(0.0, 0.0, kStepStoreF, s));
  for (SysHost& h : sys_)
    if (h.active) h.f_valid = true;
  return kOK;
}

// After a drift: read the displacement maxima, stop on non-finite values, and
// rebuild the systems whose list is no longer valid (2 d_max >= skin).
int Engine::post_drift(cudaStream_t s) {
  CK(cudaMemcpyAsync(h_disp2_, d_disp2_, sizeof(unsigned long long) * nsys(), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h_status_, d_status_, sizeof(SysStatus) * nsys(), cudaMemcpyDeviceToHost, s));
  CK(cudaMemsetAsync(d_disp2_, 0, sizeof(unsigned long long) * nsys(), s));
  CKR(sync_check(s));
  std::vector<int> which;
  for (int k = 0; k < nsys(); ++k) {
    SysHost& h = sys_[k];
    if (!h.active) continue;
    if (h_status_[k].nonfinite) {
      set_error("non-finite position or velocity in system " + std::to_string(k));
      return kErrNonfinite;
    }
    double d2;
    std::memcpy(&d2, &h_disp2_[k], sizeof(double));
    if (!(2.0 * std::sqrt(d2) < h.spec.skin)) which.push_back(k);
  }
  return rebuild(which, s);
}

int Engine::step(int64_t nsteps, const std::vector<double>& dt, cudaStream_t s) {
  if (nsteps < 0) { set_error("nsteps < 0"); return kErrArg; }
  if ((int)dt.size() != nsys()) { set_error("one dt per system required"); return kErrArg; }
  for (int k = 0; k < nsys(); ++k) {
    if (!sys_[k].active) continue;
    if (!std::isfinite(dt[k])) { set_error("dt must be finite"); return kErrArg; }
    sys_[k].dt = dt[k];
  }
  if (nsteps == 0) return kOK;
  CKR(upload_params());
  CKR(ensure_lists(s));
  CKR(ensure_forces(s));
  for (int64_t it = 0; it < nsteps; ++it) {
    if (it == 0) CKR(launch_step(0.0, 0.5, kStepUseStoredF | kStepDrift, s));
    else CKR(launch_step(0.5, 0.5, kStepDrift, s));
    cur_ ^= 1;
    CKR(post_drift(s));
  }
  CKR(launch_step(0.5, 0.0, kStepStoreF, s));
  CKR(sync_check(s));
  for (SysHost& h : sys_) {
    if (!h.active) continue;
    h.f_valid = true;
    h.steps += nsteps;
  }
  return kOK;
}

int Engine::forces_dev(int k, double* f, cudaStream_t s) {
  CKR(ensure_lists(s));
  CKR(ensure_forces(s));
  launch_to_caller(arrays(), cur_, 2, f, sys_[k].spec.n, k, sys_[k].ntiles, s);
  CKL();
  return kOK;
}

int Engine::observables(double* out3, cudaStream_t s) {
  CKR(ensure_lists(s));
  const DevArrays a = arrays();
  launch_pe_virial(a, cur_, s);
  launch_reduce_obs(a, cur_, nsys(), d_obs_, s);
  CKL();
  CK(cudaMemcpyAsync(h_obs_, d_obs_, sizeof(double) * 3 * nsys(), cudaMemcpyDeviceToHost, s));
  CKR(sync_check(s));
  std::memcpy(out3, h_obs_, sizeof(double) * 3 * nsys());
  return kOK;
}

int Engine::build_lists(cudaStream_t s) {
  std::vector<int> which;
  for (int k = 0; k < nsys(); ++k) {
    if (!sys_[k].active) continue;
    if (!sys_[k].has_state) { set_error("no state set"); return kErrState; }
    which.push_back(k);
  }
  return rebuild(which, s);
}

int Engine::get_cells(int k, int32_t* cell, cudaStream_t s) {
  const SysHost& h = sys_[k];
  if (!h.has_state) { set_error("no state set"); return kErrState; }
  CKR(ensure_lists(s));
  std::vector<int32_t> c((size_t)h.spec.n), id((size_t)h.spec.n);
  CK(cudaMemcpyAsync(c.data(), d_.cell + h.p_off, sizeof(int32_t) * h.spec.n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(id.data(), d_.id + h.p_off, sizeof(int32_t) * h.spec.n, cudaMemcpyDeviceToHost, s));
  CKR(sync_check(s));
  for (int64_t q = 0; q < h.spec.n; ++q) cell[id[(size_t)q]] = c[(size_t)q];
  return kOK;
}

int Engine::list_size(int k, int64_t* total, cudaStream_t s) {
  const SysHost& h = sys_[k];
  if (!h.has_state) { set_error("no state set"); return kErrState; }
  CKR(ensure_lists(s));
  std::vector<int32_t> cnt((size_t)h.spec.n);
  CK(cudaMemcpyAsync(cnt.data(), d_.ncnt + h.p_off, sizeof(int32_t) * h.spec.n, cudaMemcpyDeviceToHost, s));
  CKR(sync_check(s));
  int64_t t = 0;
  for (int32_t c : cnt) t += c;
  *total = t;
  return kOK;
}

int Engine::get_list(int k, int64_t* start, int32_t* partners, cudaStream_t s) {
  const SysHost& h = sys_[k];
  if (!h.has_state) { set_error("no state set"); return kErrState; }
  CKR(ensure_lists(s));
  const int64_t n = h.spec.n;
  const int64_t words = (int64_t)h.ntiles * h.kmax * kTile;
  std::vector<int32_t> cnt((size_t)n), id((size_t)n);
  std::vector<uint32_t> lw((size_t)words);
  CK(cudaMemcpyAsync(cnt.data(), d_.ncnt + h.p_off, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(id.data(), d_.id + h.p_off, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(lw.data(), d_.nbr + h.l_off, sizeof(uint32_t) * words, cudaMemcpyDeviceToHost, s));
  CKR(sync_check(s));
  std::vector<int64_t> slot_of((size_t)n);
  for (int64_t q = 0; q < n; ++q) slot_of[(size_t)id[(size_t)q]] = q;
  start[0] = 0;
  for (int64_t i = 0; i < n; ++i) start[i + 1] = start[i] + cnt[(size_t)slot_of[(size_t)i]];
  for (int64_t i = 0; i < n; ++i) {
    const int64_t q = slot_of[(size_t)i];
    const int64_t tl = q / kTile, lane = q % kTile;
    for (int32_t m = 0; m < cnt[(size_t)q]; ++m) {
      const uint32_t e = lw[(size_t)((tl * h.kmax + m) * kTile + lane)];
      partners[start[i] + m] = id[(size_t)(e & kIdxMask)];
    }
  }
  return kOK;
}

}  // namespace ljmd
