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
  for (cudaStream_t& c : cap_)
    if (c) { cudaStreamDestroy(c); c = nullptr; }
  for (cudaEvent_t e : ev_free_) cudaEventDestroy(e);
  for (TimedPair& p : ev_pending_) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
}

int Engine::set_tuning(int key, int value) {
  switch (key) {
    case 0:
      if (value != 64 && value != 128 && value != 256) break;
      tuning_.step_block = value;
      ++struct_ver_;
      return kOK;
    case 1:
      if (value != 1 && value != 2) break;
      tuning_.step_groups = value;
      ++struct_ver_;
      return kOK;
    case 2:
      if (value != 64 && value != 128 && value != 256) break;
      tuning_.list_block = value;
      ++struct_ver_;
      return kOK;
    case 3:
      if (value < 0 || value > 5) break;
      tuning_.list_variant = value;
      ++struct_ver_;
      return kOK;
    case 4:
      if (value != 0 && value != 1) break;
      tuning_.step_hint = value;
      ++struct_ver_;
      return kOK;
    case 5:
      if (value != 0 && value != 1) break;
      graph_ = value != 0;
      return kOK;
    case 6:
      if (value != 0 && value != 1) break;
      tuning_.fp64_queue = value;
      ++struct_ver_;
      return kOK;
    default:
      break;
  }
  set_error("unknown tuning key or value");
  return kErrArg;
}

int Engine::get_tuning(int key) const {
  return key == 0 ? tuning_.step_block : key == 1 ? tuning_.step_groups : key == 2 ? tuning_.list_block
         : key == 3 ? tuning_.list_variant : key == 4 ? tuning_.step_hint : key == 5 ? (graph_ ? 1 : 0)
         : key == 6 ? tuning_.fp64_queue : -1;
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

// ------------------------------------------------------------- ranges

void RangeAlloc::reset(int64_t cap) {
  cap_ = cap;
  free_.clear();
  if (cap > 0) free_[0] = cap;
}

int64_t RangeAlloc::alloc(int64_t len) {
  if (len <= 0) len = 1;
  for (auto it = free_.begin(); it != free_.end(); ++it) {
    if (it->second >= len) {
      const int64_t off = it->first, rest = it->second - len;
      free_.erase(it);
      if (rest > 0) free_[off + len] = rest;
      return off;
    }
  }
  return -1;
}

void RangeAlloc::release(int64_t off, int64_t len) {
  if (len <= 0) len = 1;
  auto it = free_.emplace(off, len).first;
  auto nx = std::next(it);
  if (nx != free_.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    free_.erase(nx);
  }
  if (it != free_.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      free_.erase(it);
    }
  }
}

void RangeAlloc::grow(int64_t new_cap) {
  if (new_cap <= cap_) return;
  const int64_t old = cap_;
  cap_ = new_cap;
  release(old, new_cap - old);
}

int64_t RangeAlloc::free_total() const {
  int64_t t = 0;
  for (const auto& kv : free_) t += kv.second;
  return t;
}

int64_t RangeAlloc::largest_free() const {
  int64_t m = 0;
  for (const auto& kv : free_) m = std::max(m, kv.second);
  return m;
}

int footprint(const SysSpec& s, SysFootprint* f, SysHost* h) {
  if (!(s.n > 0) || s.n > ((1 << 26) - 1)) { set_error("N must be in [1, 2^26 - 1]"); return kErrArg; }
  if (!(s.rc > 0.0) || !(s.skin >= 0.0) || !std::isfinite(s.rc) || !std::isfinite(s.skin)) {
    set_error("rc must be > 0 and skin >= 0");
    return kErrArg;
  }
  if (!(s.L > 2.0 * (s.rc + s.skin)) || !(s.L <= 10000.0)) {
    set_error("box side must satisfy 2 (rc + skin) < L <= 10000");
    return kErrArg;
  }
  SysHost t;
  t.spec = s;
  t.rl = s.rc + s.skin;
  // Eq. 1: V(rc) = V'(rc) = 0
  const double irc2 = 1.0 / (s.rc * s.rc);
  const double irc6 = irc2 * irc2 * irc2;
  t.c2 = 6.0 * irc6 * irc6 * irc2 - 3.0 * irc6 * irc2;
  t.c0 = 4.0 * irc6 - 7.0 * irc6 * irc6;
  t.nc = cells_per_axis(s.L, t.rl);
  t.ncell = (int64_t)t.nc * t.nc * t.nc;
  t.kmax = initial_kmax(s, t.rl);
  t.ntiles = (int32_t)((s.n + kTile - 1) / kTile);
  if (f) {
    f->slots = (int64_t)t.ntiles * kTile;
    f->cells = t.ncell + 1;
    f->list_words = (int64_t)t.ntiles * t.kmax * kTile;
  }
  if (h) *h = t;
  return kOK;
}

// ------------------------------------------------------------- arena

void Engine::free_all() {
  for (int b = 0; b < 2; ++b) { dfree(d_.x[b]); dfree(d_.xq[b]); }
  dfree(d_.v); dfree(d_.xref); dfree(d_.xqref); dfree(d_.f); dfree(d_.facc); dfree(d_.id); dfree(d_.cell); dfree(d_.ncnt);
  dfree(d_.nbr); dfree(d_.tile_obs); dfree(d_.skey); dfree(d_.xf); dfree(d_.vtmp); dfree(d_.idtmp);
  dfree(d_.celltmp); dfree(d_.perm); dfree(d_.sid); dfree(d_.ccount); dfree(d_.cstart); dfree(d_.chunk_sum);
  dfree(d_params_); dfree(d_status_); dfree(d_disp2_); dfree(d_margin_); dfree(d_checks_); dfree(d_rebuild_); dfree(d_order_); dfree(d_tile_sys_);
  dfree(d_obs_); dfree(d_stage_); dfree(d_pairs_); dfree(d_obs_work_); dfree(d_obs_chunk_);
  hfree(h_status_); hfree(h_disp2_); hfree(h_rebuild_); hfree(h_obs_); hfree(h_obs_work_);
  drop_graphs();
  dfree(d_ctl_); dfree(d_reb_count_); hfree(h_ctl_); hfree(h_reb_count_);
  d_ = DevArrays{};
  stage_n_ = 0;
}

int Engine::init(const std::vector<SysSpec>& specs, int precision) {
  if (specs.empty()) { set_error("no systems"); return kErrArg; }
  ArenaCaps caps{0, 0, 0, (int)specs.size()};
  for (const SysSpec& s : specs) {
    SysFootprint f;
    CKR(footprint(s, &f, nullptr));
    caps.slots += f.slots;
    caps.cells += f.cells;
    caps.list_words += f.list_words;
  }
  CKR(init_arena(caps, precision));
  list_growable_ = true;
  for (const SysSpec& s : specs) {
    int id = -1;
    CKR(add_system(s, &id));
  }
  return kOK;
}

int Engine::init_arena(const ArenaCaps& caps, int precision) {
  if (precision < 0 || precision > 5) { set_error("unknown precision mode"); return kErrArg; }
  if (caps.slots <= 0 || caps.cells <= 0 || caps.list_words <= 0 || caps.max_systems <= 0) {
    set_error("arena capacities must be positive");
    return kErrArg;
  }
  precision_ = precision;
  caps_ = caps;
  list_growable_ = false;
  caps_.slots = round_up(caps.slots, kTile);
  caps_.list_words = round_up(caps.list_words, 4 * kTile);
  sys_.assign((size_t)caps.max_systems, SysHost{});
  slot_alloc_.reset(caps_.slots / kTile);  // in tiles
  cell_alloc_.reset(caps_.cells);
  list_alloc_.reset(caps_.list_words / (4 * kTile));  // in 128-word units
  h_tile_sys_.assign((size_t)(caps_.slots / kTile), -1);
  ntiles_ = 0;
  cur_ = 0;
  return alloc_arrays();
}

int Engine::alloc_arrays() {
  free_all();
  const int ns = nsys();
  const int64_t P = caps_.slots, T = caps_.slots / kTile;
  for (int b = 0; b < 2; ++b) {
    CKR(dmalloc(&d_.x[b], P));
    CKR(dmalloc(&d_.xq[b], P + 4));  // 4 spare entries: the list build reads candidates 4 at a time
    CK(cudaMemset(d_.x[b], 0, sizeof(double4_32a) * P));
    CK(cudaMemset(d_.xq[b], 0, sizeof(int4) * (P + 4)));
  }
  CKR(dmalloc(&d_.v, P));
  CKR(dmalloc(&d_.xref, P));
  CKR(dmalloc(&d_.xqref, P));
  CKR(dmalloc(&d_.f, P));
  CKR(dmalloc(&d_.facc, P));
  CK(cudaMemset(d_.facc, 0, sizeof(double4_32a) * P));
  CKR(dmalloc(&d_.id, P));
  CKR(dmalloc(&d_.cell, P));
  CKR(dmalloc(&d_.ncnt, P));
  CKR(dmalloc(&d_.nbr, caps_.list_words));
  CKR(dmalloc(&d_.tile_obs, 3 * T));
  CKR(dmalloc(&d_.skey, P));
  CKR(dmalloc(&d_.xf, P + 4));
  CK(cudaMemset(d_.xf, 0, sizeof(float4) * (P + 4)));
  CKR(dmalloc(&d_.vtmp, P));
  CKR(dmalloc(&d_.idtmp, P));
  CKR(dmalloc(&d_.celltmp, P));
  CKR(dmalloc(&d_.perm, P));
  CKR(dmalloc(&d_.sid, P));
  CKR(dmalloc(&d_.ccount, caps_.cells));
  CKR(dmalloc(&d_.cstart, caps_.cells));
  // a system of ncell cells has at most ncell / kScanChunk + 1 chunks
  d_.chunk_cap = (int32_t)(caps_.cells / kScanChunk + ns + 1);
  CKR(dmalloc(&d_.chunk_sum, (int64_t)d_.chunk_cap * kChunkCopies));
  CK(cudaMemset(d_.v, 0, sizeof(double4_32a) * P));
  CK(cudaMemset(d_.f, 0, sizeof(double4_32a) * P));
  CK(cudaMemset(d_.xref, 0, sizeof(double4_32a) * P));
  CK(cudaMemset(d_.ncnt, 0, sizeof(int32_t) * P));
  CK(cudaMemset(d_.id, 0xff, sizeof(int32_t) * P));
  CK(cudaMemset(d_.ccount, 0, sizeof(int32_t) * caps_.cells));
  CK(cudaMemset(d_.cstart, 0, sizeof(int32_t) * caps_.cells));
  CKR(dmalloc(&d_params_, ns));
  CKR(dmalloc(&d_status_, ns));
  CKR(dmalloc(&d_disp2_, ns));
  CKR(dmalloc(&d_margin_, ns));
  CK(cudaMemset(d_margin_, 0, sizeof(double) * ns));
  CKR(dmalloc(&d_checks_, ns));
  CK(cudaMemset(d_checks_, 0, sizeof(int32_t) * ns));
  CKR(dmalloc(&d_rebuild_, 4 * ns + 2));
  CKR(dmalloc(&d_order_, ns));
  CKR(dmalloc(&d_tile_sys_, T));
  CKR(dmalloc(&d_obs_, 3 * ns));
  CKR(dmalloc(&d_obs_work_, 2 * ns + 1));
  CKR(dmalloc(&d_obs_chunk_, 3 * (T / 256 + ns + 1)));
  CK(cudaMallocHost((void**)&h_obs_work_, sizeof(int32_t) * (2 * ns + 1)));
  CKR(dmalloc(&d_pairs_, 2 * ns));
  CK(cudaMemset(d_status_, 0, sizeof(SysStatus) * ns));
  CK(cudaMemset(d_disp2_, 0, sizeof(unsigned long long) * ns));
  CK(cudaMemset(d_rebuild_, 0, sizeof(int32_t) * ns));
  CK(cudaMemset(d_tile_sys_, 0xff, sizeof(int32_t) * T));
  CK(cudaMallocHost((void**)&h_status_, sizeof(SysStatus) * ns));
  CK(cudaMallocHost((void**)&h_disp2_, sizeof(unsigned long long) * ns));
  CK(cudaMallocHost((void**)&h_rebuild_, sizeof(int32_t) * (4 * ns + 2)));
  CK(cudaMallocHost((void**)&h_obs_, sizeof(double) * 3 * ns));
  CKR(dmalloc(&d_ctl_, 1));
  CKR(dmalloc(&d_reb_count_, ns));
  CK(cudaMemset(d_ctl_, 0, sizeof(GraphCtl)));
  CK(cudaMallocHost((void**)&h_ctl_, sizeof(GraphCtl)));
  CK(cudaMallocHost((void**)&h_reb_count_, sizeof(int32_t) * ns));
  ++struct_ver_;
  return upload_params();
}

int Engine::stage(int64_t n, double** out) {
  if (n > stage_n_) {
    dfree(d_stage_);
    stage_n_ = 0;
    CKR(dmalloc(&d_stage_, 6 * n));
    stage_n_ = n;
  }
  *out = d_stage_;
  return kOK;
}

void Engine::update_extent() {
  int32_t last = 0;
  for (const SysHost& h : sys_) {
    if (!h.used) continue;
    last = std::max(last, h.t_off + h.ntiles);
  }
  ntiles_ = last;
  ++struct_ver_;
}

int Engine::grow_list_arena(int64_t min_extra_units) {
  const int64_t old_units = list_alloc_.cap();
  const int64_t new_units = std::max(old_units + old_units / 2, old_units + min_extra_units);
  uint32_t* nb = nullptr;
  CKR(dmalloc(&nb, new_units * 4 * kTile));
  CK(cudaMemcpy(nb, d_.nbr, sizeof(uint32_t) * old_units * 4 * kTile, cudaMemcpyDeviceToDevice));
  dfree(d_.nbr);
  d_.nbr = nb;
  list_alloc_.grow(new_units);
  caps_.list_words = new_units * 4 * kTile;
  ++struct_ver_;
  return kOK;
}

int Engine::upload_tiles(int k, int32_t value) {
  const SysHost& h = sys_[k];
  for (int q = 0; q < h.ntiles; ++q) h_tile_sys_[(size_t)(h.t_off + q)] = value;
  CK(cudaMemcpy(d_tile_sys_ + h.t_off, h_tile_sys_.data() + h.t_off, sizeof(int32_t) * h.ntiles,
                cudaMemcpyHostToDevice));
  return kOK;
}

int Engine::add_system(const SysSpec& s, int* id) {
  SysHost h;
  SysFootprint f;
  CKR(footprint(s, &f, &h));
  int k = -1;
  for (int q = 0; q < nsys(); ++q)
    if (!sys_[q].used) { k = q; break; }
  if (k < 0) { set_error("arena: no free system record"); return kErrOOM; }
  const int64_t t0 = slot_alloc_.alloc(f.slots / kTile);
  if (t0 < 0) { set_error("arena: not enough free particle slots"); return kErrOOM; }
  const int64_t c0 = cell_alloc_.alloc(f.cells);
  if (c0 < 0) {
    slot_alloc_.release(t0, f.slots / kTile);
    set_error("arena: not enough free cell entries");
    return kErrOOM;
  }
  const int64_t l0 = list_alloc_.alloc(f.list_words / (4 * kTile));
  if (l0 < 0) {
    slot_alloc_.release(t0, f.slots / kTile);
    cell_alloc_.release(c0, f.cells);
    set_error("arena: not enough free list words");
    return kErrOOM;
  }
  h.used = true;
  h.active = true;
  h.t_off = (int32_t)t0;
  h.p_off = t0 * kTile;
  h.c_off = c0;
  h.l_off = l0 * 4 * kTile;
  sys_[k] = h;
  // cell counters of the new range must start at zero
  CK(cudaMemset(d_.ccount + h.c_off, 0, sizeof(int32_t) * (h.ncell + 1)));
  CKR(upload_tiles(k, k));
  update_extent();
  CKR(upload_params(k));
  *id = k;
  return kOK;
}

int Engine::remove_system(int k) {
  if (!valid_id(k)) { set_error("no such system"); return kErrArg; }
  SysHost& h = sys_[k];
  CKR(upload_tiles(k, -1));
  slot_alloc_.release(h.t_off, h.ntiles);
  cell_alloc_.release(h.c_off, h.ncell + 1);
  list_alloc_.release(h.l_off / (4 * kTile), (int64_t)h.ntiles * h.kmax / 4);
  h = SysHost{};
  update_extent();
  return upload_params(k);
}

void Engine::arena_usage(int64_t* o) const {
  o[0] = caps_.slots;
  o[1] = slot_alloc_.free_total() * kTile;
  o[2] = caps_.cells;
  o[3] = cell_alloc_.free_total();
  o[4] = caps_.list_words;
  o[5] = list_alloc_.free_total() * 4 * kTile;
  o[6] = caps_.max_systems;
  int64_t used = 0;
  for (const SysHost& h : sys_) used += h.used ? 1 : 0;
  o[7] = used;
}

int Engine::upload_params(int only) {
  const int k0 = only >= 0 ? only : 0, k1 = only >= 0 ? only + 1 : nsys();
  std::vector<SysParams> ps((size_t)(k1 - k0));
  for (int k = k0; k < k1; ++k) {
    const SysHost& h = sys_[k];
    SysParams& P = ps[(size_t)(k - k0)];
    std::memset(&P, 0, sizeof(P));
    if (!h.used) continue;
    P.L = h.spec.L;
    P.invL = 1.0 / h.spec.L;
    P.inv_cs = (double)h.nc / h.spec.L;
    P.rc2 = h.spec.rc * h.spec.rc;
    P.rl2 = h.rl * h.rl;
    P.c2 = h.c2;
    P.c0 = h.c0;
    P.dt = h.dt;
    P.hdt = 0.5 * h.dt;
    P.qscale = 4294967296.0 / h.spec.L;
    P.qunit = (float)(h.spec.L / 4294967296.0);
    P.rl2q_lo = (float)(P.rl2 * P.qscale * P.qscale * (1.0 - 1e-5));
    P.rl2q_hi = (float)(P.rl2 * P.qscale * P.qscale * (1.0 + 1e-5));
    P.rc2q_hi = (float)(P.rc2 * P.qscale * P.qscale * (1.0 + 1e-5));
    {
      // Float pre-test of the list build: candidate positions rounded to float
      // (error <= u L, u = 2^-24); the particle's position shifted by an image
      // either rounded once from the FP64 sum (error <= 2 u L) or, in the staged
      // build, formed in float from the particle's float position and L as float
      // (error <= 4 u L). So each separation errs by at most e0 = 5 u L (1 + 2^-28)
      // plus u |d|.
      // Near r = rl the float r^2 then errs by less than
      //   rl^2 (2 sqrt(3) e0 / rl + 3 (e0 / rl)^2 + 6 u e0 / rl + 7 u)
      // (separation errors, three float roundings, the FP64 test's own roundings,
      // the thresholds' rounding to float); eps is twice that.
      const double u = 5.9604644775390625e-08;
      const double g = 5.0 * u * h.spec.L * (1.0 + 3.7252902984e-09) / h.rl;
      const double eps = 2.0 * (3.4641016151377544 * g + 3.0 * g * g + 6.0 * u * g + 7.0 * u);
      P.rl2f_lo = std::nextafter((float)(P.rl2 * (1.0 - eps)), 0.0f);
      P.rl2f_hi = std::nextafter((float)(P.rl2 * (1.0 + eps)), 3.0e38f);
    }
    P.skin = h.spec.skin;
    {
      // FP32-force validity threshold: each shadow coordinate is within 1/2 unit
      // of the position, so the integer displacement is compared with
      // (skin / 2 in units - 4)^2
      const double hq = 0.5 * h.spec.skin * (4294967296.0 / h.spec.L) - 4.0;
      P.disp_thr = hq > 0.0 ? hq * hq : 0.0;
    }
    P.rc2f = (float)P.rc2;
    P.c2f = (float)h.c2;
    P.rlf = (float)h.rl;
    P.csf = (float)(h.spec.L / h.nc);
    P.Lf = (float)h.spec.L;
    P.wmargin = (float)(1e-5 * h.spec.L + 1e-6);
    P.p_off = h.p_off;
    P.c_off = h.c_off;
    P.l_off = h.l_off;
    P.n = (int32_t)h.spec.n;
    P.nc = h.nc;
    P.kmax = h.kmax;
    P.t_off = h.t_off;
    P.ntiles = h.ntiles;
    P.active = h.active ? 1 : 0;
    P.rule = rule_;
    P.half = half_ ? 1 : 0;
  }
  CK(cudaMemcpy(d_params_ + k0, ps.data(), sizeof(SysParams) * ps.size(), cudaMemcpyHostToDevice));
  return upload_order();
}

// Order in which rebuild passes take the systems: descending estimated list-build
// cost per tile, so that the warps fetching tiles start the slowest first and a
// pass does not end on a few slow tiles. The estimate counts a particle's
// candidates (9 rows of 3 cells cut to a window of 2 rl, or every particle when
// nc == 1) and half its expected partners. Results do not depend on the order.
int Engine::upload_order() {
  const int ns = nsys();
  if (ns == 0) return kOK;
  std::vector<double> cost((size_t)ns, -1.0);
  for (int k = 0; k < ns; ++k) {
    const SysHost& h = sys_[k];
    if (!h.used) continue;
    const double L = h.spec.L, rho = (double)h.spec.n / (L * L * L);
    const double partners = 4.0 / 3.0 * M_PI * h.rl * h.rl * h.rl * rho;
    const double cs = L / h.nc;
    const double cand = h.nc == 1 ? (double)h.spec.n : 9.0 * cs * cs * 2.0 * h.rl * rho;
    cost[(size_t)k] = cand + 0.5 * partners;
  }
  std::vector<int32_t> order((size_t)ns);
  for (int k = 0; k < ns; ++k) order[(size_t)k] = k;
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t p, int32_t q) { return cost[(size_t)p] > cost[(size_t)q]; });
  order_rank_.assign((size_t)ns, 0);
  for (int i = 0; i < ns; ++i) order_rank_[(size_t)order[(size_t)i]] = i;
  CK(cudaMemcpy(d_order_, order.data(), sizeof(int32_t) * (size_t)ns, cudaMemcpyHostToDevice));
  return kOK;
}

DevArrays Engine::arrays() const {
  DevArrays a = d_;
  a.params = d_params_;
  a.status = d_status_;
  a.disp2 = d_disp2_;
  a.margin = d_margin_;
  a.checks = d_checks_;
  a.rebuild = d_rebuild_;
  a.rebuild_ids = d_rebuild_ + nsys();
  a.sys_order = d_order_;
  a.reb_pref = d_rebuild_ + 2 * nsys();
  a.chunk_pref = d_rebuild_ + 3 * nsys() + 1;
  a.nreb = 0;
  a.tile_next = &d_ctl_->next_tile;
  a.tile_sys = d_tile_sys_;
  a.ntiles = ntiles_;
  return a;
}

int Engine::set_precision(int mode) {
  if (mode < 0 || mode > 5) { set_error("unknown precision mode"); return kErrArg; }
  if (mode != precision_) {
    precision_ = mode;
    ++struct_ver_;
    for (SysHost& h : sys_) {
      h.f_valid = false;
      if (h.has_state) h.force_rebuild = true;  // refresh the fixed-point shadow
    }
  }
  return kOK;
}

int Engine::set_rule(int rule) {
  if (rule != 0 && rule != 1) { set_error("unknown list validity rule"); return kErrArg; }
  if (rule != rule_) {
    rule_ = rule;
    ++struct_ver_;
    // the margin is only tracked under the velocity bound: start from fresh lists
    for (SysHost& h : sys_)
      if (h.has_state) h.force_rebuild = true;
    CKR(upload_params());
  }
  return kOK;
}

int Engine::set_list_kind(int kind) {
  if (kind != 0 && kind != 1) { set_error("unknown pair-list kind"); return kErrArg; }
  if ((kind == 1) != half_) {
    half_ = kind == 1;
    ++struct_ver_;
    for (SysHost& h : sys_) {
      h.f_valid = false;
      if (h.has_state) h.force_rebuild = true;
    }
    CKR(upload_params());
  }
  return kOK;
}

int Engine::set_active(int k, bool on) {
  if (!valid_id(k)) { set_error("no such system"); return kErrArg; }
  SysHost& h = sys_[k];
  if (h.active == on) return kOK;
  if (!on) {
    h.park = cur_;  // its positions stay in this buffer while the others step
  } else if (h.park >= 0) {
    if (h.park != cur_) {
      // the others advanced an odd number of steps: move its positions (and shadows)
      // to the buffer the next launch reads (after all work in flight)
      CK(cudaDeviceSynchronize());
      const size_t nslot = (size_t)h.ntiles * kTile;
      CK(cudaMemcpy(d_.x[cur_] + h.p_off, d_.x[h.park] + h.p_off, sizeof(double4_32a) * nslot,
                    cudaMemcpyDeviceToDevice));
      CK(cudaMemcpy(d_.xq[cur_] + h.p_off, d_.xq[h.park] + h.p_off, sizeof(int4) * nslot,
                    cudaMemcpyDeviceToDevice));
    }
    h.park = -1;
  }
  h.active = on;
  return upload_params(k);
}

int Engine::set_state_dev(int k, const double* x, const double* v, cudaStream_t s) {
  if (!valid_id(k)) { set_error("no such system"); return kErrArg; }
  SysHost& h = sys_[k];
  launch_from_caller(arrays(), cur_of(k), x, v, k, h.ntiles, s);
  CKL();
  h.has_state = true;
  h.force_rebuild = true;
  h.f_valid = false;
  return kOK;
}

int Engine::get_state_dev(int k, double* x, double* v, cudaStream_t s) {
  if (!valid_id(k)) { set_error("no such system"); return kErrArg; }
  SysHost& h = sys_[k];
  if (!h.has_state) { set_error("no state set"); return kErrState; }
  if (x) launch_to_caller(arrays(), cur_of(k), 0, x, h.spec.n, k, h.ntiles, s);
  if (v) launch_to_caller(arrays(), cur_of(k), 1, v, h.spec.n, k, h.ntiles, s);
  CKL();
  return kOK;
}

bool Engine::any_active() const {
  for (const SysHost& h : sys_)
    if (h.used && h.active) return true;
  return false;
}

int Engine::sync_check(cudaStream_t s) {
  CK(cudaStreamSynchronize(s));
  collect_timing();
  if (kChecks) return read_checks(s);
  return kOK;
}

// The device check words stay set once a check has failed (the state is suspect
// from then on), so every later call reports the failure as well.
int Engine::read_checks(cudaStream_t s) {
  std::vector<int32_t> w((size_t)nsys());
  if (w.empty()) return kOK;
  CK(cudaMemcpyAsync(w.data(), d_checks_, sizeof(int32_t) * w.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int k = 0; k < nsys(); ++k)
    if (w[(size_t)k]) {
      set_error("device check failed in system " + std::to_string(k) + " (check bits " + std::to_string(w[(size_t)k]) +
                ")");
      return kErrCheck;
    }
  return kOK;
}

// Full rebuild (bin, stable counting sort, gather, list) of the given systems.
int Engine::rebuild(std::vector<int> which, cudaStream_t s) {
  if (which.empty()) return kOK;
  std::sort(which.begin(), which.end(),
            [&](int p, int q) { return order_rank_[(size_t)p] < order_rank_[(size_t)q]; });
  for (int attempt = 0; attempt < 4; ++attempt) {
    for (int k = 0; k < nsys(); ++k) h_rebuild_[k] = 0;
    int32_t* pref = h_rebuild_ + 2 * nsys();
    int32_t* cpref = h_rebuild_ + 3 * nsys() + 1;
    int32_t tiles = 0, chunks = 0;
    for (size_t q = 0; q < which.size(); ++q) {
      h_rebuild_[which[q]] = 1;
      h_rebuild_[nsys() + q] = which[q];
      pref[q] = tiles;
      cpref[q] = chunks;
      tiles += sys_[which[q]].ntiles;
      chunks += scan_chunks(sys_[which[q]].ncell);
    }
    const int nreb = (int)which.size();
    pref[nreb] = tiles;
    cpref[nreb] = chunks;
    CK(cudaMemcpyAsync(d_rebuild_, h_rebuild_, sizeof(int32_t) * (4 * nsys() + 2), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(d_.chunk_sum, 0, sizeof(int32_t) * (size_t)chunks * kChunkCopies, s));  // totalled by the count
    CK(cudaMemsetAsync(d_status_, 0, sizeof(SysStatus) * nsys(), s));
    CK(cudaMemsetAsync(&d_ctl_->next_tile, 0, sizeof(int32_t), s));
    DevArrays a = arrays();
    a.nreb = nreb;
    tmark_begin(kTBin, s);
    launch_cell_count(a, cur_, s);
    launch_cell_scan(a, nreb, s);
    launch_scatter(a, cur_, s);
    launch_cell_rank(a, cur_, s);
    tmark_end(s);
    tmark_begin(kTList, s);
    launch_build_list(a, cur_, list_tuning(), s);
    tmark_end(s);
    CKL();
    n_launch_ += kRebuildLaunches;
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
        h.old_kmax = h.kmax;
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
    // move the grown systems' lists to larger ranges and rebuild them
    for (int k : which) {
      SysHost& h = sys_[k];
      const int64_t old_units = (int64_t)h.ntiles * h.old_kmax / 4;
      list_alloc_.release(h.l_off / (4 * kTile), old_units);
      int64_t l0 = list_alloc_.alloc((int64_t)h.ntiles * h.kmax / 4);
      if (l0 < 0 && list_growable_) {
        CKR(grow_list_arena((int64_t)h.ntiles * h.kmax / 4));
        l0 = list_alloc_.alloc((int64_t)h.ntiles * h.kmax / 4);
      }
      if (l0 < 0) {
        set_error("arena: not enough free list words to grow a pair list");
        // keep the old capacity (it fits where it was)
        h.kmax = h.old_kmax;
        const int64_t back = list_alloc_.alloc(old_units);
        h.l_off = back * 4 * kTile;
        CKR(upload_params(k));
        return kErrOverflow;
      }
      h.l_off = l0 * 4 * kTile;
      CKR(upload_params(k));
    }
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
  // the kicks are half steps: ka, kb in {0, 1/2} become flags (the kernels take
  // dt/2 from the system parameters, so they need no FP64 compare or product)
  if (ka != 0.0) flags |= kStepKickA;
  if (kb != 0.0) flags |= kStepKickB;
  if ((flags & kStepDrift) && rule_ == 1) flags |= kStepVmax;
  tmark_begin(kTStep, s);
  if (half_) launch_step_half(a, cur_, flags, tuning_, precision_, s);
  else if (precision_ == 1) launch_step_fp32(a, cur_, ka, kb, flags, tuning_, s);
  else launch_step_fp64(a, cur_, ka, kb, flags, tuning_, precision_ >= 2 ? precision_ - 1 : 0, s);
  tmark_end(s);
  CKL();
  n_launch_ += half_ ? 2 : 1;
  return kOK;
}

int Engine::pair_stats(int k, int64_t* listed, int64_t* inside, cudaStream_t s) {
  if (!valid_id(k)) { set_error("no such system"); return kErrArg; }
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

// After a drift: the list-validity decision (k_decide, the kernel the graph loop
// uses), read back with the status words; stop on non-finite values and rebuild
// the systems whose list is no longer valid.
int Engine::post_drift(cudaStream_t s) {
  DevArrays a = arrays();
  a.ctl = d_ctl_;
  launch_decide(a, nsys(), precision_ == 1 ? 1 : 0, rule_ == 1 ? kStepVmax : 0, d_rebuild_, d_rebuild_ + nsys(),
                d_rebuild_ + 2 * nsys(), nullptr, 0, 0, 0, s);
  CKL();
  n_launch_ += 1;
  CK(cudaMemcpyAsync(h_ctl_, d_ctl_, sizeof(GraphCtl), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h_rebuild_, d_rebuild_, sizeof(int32_t) * nsys(), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h_status_, d_status_, sizeof(SysStatus) * nsys(), cudaMemcpyDeviceToHost, s));
  CKR(sync_check(s));
  if (h_ctl_->abort == 2) {
    for (int k = 0; k < nsys(); ++k)
      if (sys_[k].used && sys_[k].active && h_status_[k].nonfinite) {
        set_error("non-finite position or velocity in system " + std::to_string(k));
        return kErrNonfinite;
      }
    set_error("non-finite position or velocity");
    return kErrNonfinite;
  }
  std::vector<int> which;
  for (int k = 0; k < nsys(); ++k)
    if (sys_[k].active && h_rebuild_[k]) which.push_back(k);
  return rebuild(which, s);
}

// ------------------------------------------------ graph-captured step loop

void Engine::drop_graphs() {
  for (int p = 0; p < 2; ++p) {
    if (gexec_[p]) cudaGraphExecDestroy(gexec_[p]);
    gexec_[p] = nullptr;
    gver_[p] = -1;
  }
}

#define CKG(call)                                   \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) {                        \
      set_error(std::string("CUDA graph: ") + cudaGetErrorString(e_)); \
      return kErrCuda;                              \
    }                                               \
  } while (0)

// Loop node (condition set by the second decision of its body) over two steps
// of opposite buffer parity; after each step the decision kernel and a
// conditional node holding the rebuild pass of the other parity.
int Engine::build_graph(cudaGraph_t g, int parity) {
  const DevArrays a0 = arrays();
  DevArrays a = a0;
  a.ctl = d_ctl_;
  int nused = 0;
  for (const SysHost& h : sys_) nused += h.used ? 1 : 0;
  cudaGraphConditionalHandle hw;
  CKG(cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams wp{};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hw;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wn;
  CKG(cudaGraphAddNode(&wn, g, nullptr, nullptr, 0, &wp));
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  cudaGraphConditionalHandle hi[2];
  for (int h = 0; h < 2; ++h) CKG(cudaGraphConditionalHandleCreate(&hi[h], body, 0, cudaGraphCondAssignDefault));
  CKG(cudaStreamBeginCaptureToGraph(cap_[0], body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  int rc = kOK;
  for (int h = 0; h < 2 && rc == kOK; ++h) {
    const int c = parity ^ h;
    // the flags come from the control words (first step of a call, then steady)
    if (half_) launch_step_half(a, c, 0, tuning_, precision_, cap_[0]);
    else if (precision_ == 1) launch_step_fp32(a, c, 0.0, 0.0, 0, tuning_, cap_[0]);
    else launch_step_fp64(a, c, 0.0, 0.0, 0, tuning_, precision_ >= 2 ? precision_ - 1 : 0, cap_[0]);
    launch_decide(a, nsys(), precision_ == 1 ? 1 : 0, rule_ == 1 ? kStepVmax : 0, d_rebuild_, d_rebuild_ + nsys(),
                  d_rebuild_ + 2 * nsys(), d_reb_count_, hi[h], hw, h, cap_[0]);
    cudaStreamCaptureStatus st;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(cap_[0], &st, nullptr, &cg, &deps, &ed, &nd);
    cudaGraphNodeParams ip{};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hi[h];
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t in = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&in, cg, deps, ed, nd, &ip);
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cap_[0], &in, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(cap_[1], ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const int c1 = c ^ 1;
      launch_cell_count(a, c1, cap_[1]);
      launch_cell_scan(a, nused, cap_[1]);
      launch_scatter(a, c1, cap_[1]);
      launch_cell_rank(a, c1, cap_[1]);
      launch_build_list(a, c1, list_tuning(), cap_[1]);
      cudaGraph_t t1 = nullptr;
      e = cudaStreamEndCapture(cap_[1], &t1);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_error(std::string("CUDA graph capture: ") + cudaGetErrorString(e));
      rc = kErrCuda;
    }
  }
  cudaGraph_t t0 = nullptr;
  const cudaError_t e0 = cudaStreamEndCapture(cap_[0], &t0);
  if (rc == kOK && e0 != cudaSuccess) {
    set_error(std::string("CUDA graph capture: ") + cudaGetErrorString(e0));
    rc = kErrCuda;
  }
  if (rc != kOK) {
    cudaGraph_t t1 = nullptr;
    cudaStreamEndCapture(cap_[1], &t1);  // in case the inner capture is still open
    cudaGetLastError();
  }
  return rc;
}

int Engine::capture_graph(int parity) {
  if (gexec_[parity]) cudaGraphExecDestroy(gexec_[parity]);
  gexec_[parity] = nullptr;
  for (cudaStream_t& c : cap_)
    if (!c) CK(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  int rc = build_graph(g, parity);
  if (rc == kOK) {
    const cudaError_t e = cudaGraphInstantiate(&gexec_[parity], g, 0);
    if (e != cudaSuccess) {
      set_error(std::string("CUDA graph instantiate: ") + cudaGetErrorString(e));
      gexec_[parity] = nullptr;
      rc = kErrCuda;
    }
  }
  cudaGraphDestroy(g);
  if (rc == kOK) gver_[parity] = struct_ver_;
  return rc;
}

// Runs up to nsteps (even) steps as one graph launch; *done = steps taken.
int Engine::run_graph(int64_t nsteps, int first_flags, int64_t* done, cudaStream_t s) {
  *done = 0;
  if (!gexec_[cur_] || gver_[cur_] != struct_ver_) CKR(capture_graph(cur_));
  GraphCtl c{};
  c.flags = first_flags;
  c.target = (int32_t)nsteps;
  *h_ctl_ = c;
  CK(cudaMemcpyAsync(d_ctl_, h_ctl_, sizeof(GraphCtl), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(d_reb_count_, 0, sizeof(int32_t) * nsys(), s));
  CK(cudaGraphLaunch(gexec_[cur_], s));
  CK(cudaMemcpyAsync(h_ctl_, d_ctl_, sizeof(GraphCtl), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h_reb_count_, d_reb_count_, sizeof(int32_t) * nsys(), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h_status_, d_status_, sizeof(SysStatus) * nsys(), cudaMemcpyDeviceToHost, s));
  CKR(sync_check(s));
  const GraphCtl r = *h_ctl_;
  *done = r.done;
  if (r.done & 1) cur_ ^= 1;
  n_launch_ += (half_ ? 3 : 2) * (int64_t)r.done + kRebuildLaunches * (int64_t)r.passes;
  n_rebuild_seq_ += r.passes;
  for (int k = 0; k < nsys(); ++k) {
    if (h_reb_count_[k] <= 0) continue;
    sys_[k].rebuilds += h_reb_count_[k];
    sys_[k].force_rebuild = false;
    sys_[k].f_valid = false;
  }
  if (r.abort == 2) {
    for (int k = 0; k < nsys(); ++k)
      if (sys_[k].used && sys_[k].active && h_status_[k].nonfinite) {
        set_error("non-finite position or velocity in system " + std::to_string(k));
        return kErrNonfinite;
      }
    set_error("non-finite position or velocity");
    return kErrNonfinite;
  }
  if (r.abort == 1) {
    // a list overflowed in the last rebuild pass: grow it and rebuild (counted once)
    std::vector<int> which;
    for (int k = 0; k < nsys(); ++k)
      if (sys_[k].used && sys_[k].active && h_status_[k].overflow > 0) {
        which.push_back(k);
        sys_[k].rebuilds -= 1;
      }
    CKR(rebuild(which, s));
  }
  return kOK;
}

int Engine::step(int64_t nsteps, const std::vector<double>& dt, cudaStream_t s) {
  if (nsteps < 0) { set_error("nsteps < 0"); return kErrArg; }
  if ((int)dt.size() != nsys()) { set_error("one dt per system required"); return kErrArg; }
  for (int k = 0; k < nsys(); ++k) {
    if (!sys_[k].active) continue;
    if (!std::isfinite(dt[k])) { set_error("dt must be finite"); return kErrArg; }
    sys_[k].dt = dt[k];
  }
  if (nsteps == 0 || !any_active()) return kOK;  // an empty or fully paused arena: nothing to do
  CKR(upload_params());
  CKR(ensure_lists(s));
  CKR(ensure_forces(s));
  CK(cudaMemsetAsync(d_ctl_, 0, sizeof(GraphCtl), s));
  int64_t it = 0;
  if (graph_ && !timing_) {
    while (nsteps - it >= 2) {
      const int first = (it == 0 ? (kStepUseStoredF | kStepDrift | kStepKickB) : (kStepKickA | kStepKickB | kStepDrift)) |
                        (rule_ == 1 ? kStepVmax : 0);
      int64_t done = 0;
      const int rc = run_graph(std::min<int64_t>(nsteps - it, 1 << 30) & ~int64_t(1), first, &done, s);
      it += done;
      if (rc != kOK) return rc;
    }
  }
  for (; it < nsteps; ++it) {
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

int Engine::get_checkpoint_dev(int k, double* x, double* v, double* xref, double* margin, cudaStream_t s) {
  if (!valid_id(k)) { set_error("no such system"); return kErrArg; }
  SysHost& h = sys_[k];
  if (!h.has_state) { set_error("no state set"); return kErrState; }
  CKR(ensure_lists(s));  // a state set since the last build gets its list (and build positions) now
  const DevArrays a = arrays();
  if (x) launch_to_caller(a, cur_of(k), 4, x, h.spec.n, k, h.ntiles, s);
  if (v) launch_to_caller(a, cur_of(k), 1, v, h.spec.n, k, h.ntiles, s);
  if (xref) launch_to_caller(a, cur_of(k), 5, xref, h.spec.n, k, h.ntiles, s);
  CKL();
  if (margin) CK(cudaMemcpyAsync(margin, d_margin_ + k, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return kOK;
}

// Restore, first part: the build positions and velocities, then the list built
// from them.
int Engine::set_checkpoint_dev(int k, const double* xref, const double* v, cudaStream_t s) {
  CKR(set_state_dev(k, xref, v, s));
  return rebuild(std::vector<int>{k}, s);
}

// Restore, second part: the positions as held (over the freshly built slots) and
// the margin; forces are recomputed before the next step.
int Engine::finish_checkpoint_dev(int k, const double* x, double margin, cudaStream_t s) {
  if (!valid_id(k)) { set_error("no such system"); return kErrArg; }
  SysHost& h = sys_[k];
  launch_positions_by_id(arrays(), cur_of(k), x, h.spec.n, k, s);
  CKL();
  CK(cudaMemcpyAsync(d_margin_ + k, &margin, sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  h.f_valid = false;
  return kOK;
}

int Engine::forces_dev(int k, double* f, cudaStream_t s) {
  if (!valid_id(k)) { set_error("no such system"); return kErrArg; }
  CKR(ensure_lists(s));
  CKR(ensure_forces(s));
  launch_to_caller(arrays(), cur_, 2, f, sys_[k].spec.n, k, sys_[k].ntiles, s);
  CKL();
  return kOK;
}

int Engine::observables(double* out3, cudaStream_t s, bool with_pairs, const int32_t* select) {
  if (with_pairs) CKR(ensure_lists(s));
  const DevArrays a = arrays();
  const int32_t* dsel = nullptr;
  if (select) {
    // the selection rides in the rebuild-flag array (not in use between steps)
    for (int k = 0; k < nsys(); ++k) h_rebuild_[k] = select[k] ? 1 : 0;
    CK(cudaMemcpyAsync(d_rebuild_, h_rebuild_, sizeof(int32_t) * nsys(), cudaMemcpyHostToDevice, s));
    dsel = d_rebuild_;
  }
  launch_pe_virial(a, cur_, with_pairs ? 1 : 0, dsel, s);
  // the systems to reduce and the prefix of their chunk counts
  int nsel = 0, nchunks = 0;
  for (int k = 0; k < nsys(); ++k)
    if (sys_[k].used && sys_[k].active && (!select || select[k])) h_obs_work_[nsel++] = k;
  for (int r = 0; r < nsel; ++r) {
    h_obs_work_[nsel + r] = nchunks;
    nchunks += (sys_[h_obs_work_[r]].ntiles + 255) / 256;
  }
  h_obs_work_[2 * nsel] = nchunks;
  CK(cudaMemcpyAsync(d_obs_work_, h_obs_work_, sizeof(int32_t) * (2 * nsel + 1), cudaMemcpyHostToDevice, s));
  launch_reduce_obs(a, d_obs_work_, nsel, nchunks, d_obs_chunk_, d_obs_, s);
  CKL();
  CK(cudaMemcpyAsync(h_obs_, d_obs_, sizeof(double) * 3 * nsys(), cudaMemcpyDeviceToHost, s));
  CKR(sync_check(s));
  std::memcpy(out3, h_obs_, sizeof(double) * 3 * nsys());
  return kOK;
}

int Engine::step_nvt(int64_t nsteps, const std::vector<double>& dt, const std::vector<double>& T,
                     const std::vector<double>& Q, std::vector<double>& zeta, std::vector<double>& eta,
                     cudaStream_t s) {
  const int ns = nsys();
  if (nsteps < 0 || (int)dt.size() != ns || (int)T.size() != ns || (int)Q.size() != ns ||
      (int)zeta.size() != ns || (int)eta.size() != ns) {
    set_error("step_nvt: one dt, T, Q, zeta, eta per system");
    return kErrArg;
  }
  for (int k = 0; k < ns; ++k) {
    if (!sys_[k].active) continue;
    if (!(Q[k] > 0.0) || !(T[k] >= 0.0) || !std::isfinite(dt[k])) {
      set_error("step_nvt: need Q > 0, T >= 0, finite dt");
      return kErrArg;
    }
  }
  if (nsteps == 0 || !any_active()) return kOK;
  std::vector<double> o3((size_t)(3 * ns)), fac((size_t)ns, 1.0);
  // `halves` consecutive thermostat half steps from one kinetic-energy reduction:
  // each is zeta += dt/4 G, eta += dt/2 zeta, v *= exp(-dt/2 zeta), zeta += dt/4 G'
  // with G = (2 KE - g T) / Q, g = 3 (N - 1); a uniform scale multiplies KE by its
  // square, so the next G needs no new reduction. One velocity scaling at the end.
  auto thermostat = [&](int halves) -> int {
    CKR(observables(o3.data(), s, false));
    for (int k = 0; k < ns; ++k) {
      fac[(size_t)k] = 1.0;
      if (!sys_[k].active) continue;
      const double g = 3.0 * (double)(sys_[k].spec.n - 1);
      double ke = o3[(size_t)(3 * k + 2)];
      for (int h = 0; h < halves; ++h) {
        zeta[k] += 0.25 * dt[k] * (2.0 * ke - g * T[k]) / Q[k];
        eta[k] += 0.5 * dt[k] * zeta[k];
        const double sc = std::exp(-0.5 * dt[k] * zeta[k]);
        fac[(size_t)k] *= sc;
        ke = ke * sc * sc;
        zeta[k] += 0.25 * dt[k] * (2.0 * ke - g * T[k]) / Q[k];
      }
    }
    return scale_velocities(fac, s);
  };
  CKR(ensure_lists(s));
  if (nsteps == 0) return kOK;
  CKR(thermostat(1));
  for (int64_t it = 0; it < nsteps; ++it) {
    CKR(step(1, dt, s));
    // the end of this step and the start of the next are consecutive half steps
    CKR(thermostat(it + 1 < nsteps ? 2 : 1));
  }
  return kOK;
}

int Engine::scale_velocities(const std::vector<double>& factor, cudaStream_t s) {
  if ((int)factor.size() != nsys()) { set_error("one factor per system required"); return kErrArg; }
  for (double f : factor)
    if (!std::isfinite(f)) { set_error("scale factor must be finite"); return kErrArg; }
  CK(cudaMemcpyAsync(d_obs_, factor.data(), sizeof(double) * nsys(), cudaMemcpyHostToDevice, s));
  launch_scale_v(arrays(), d_obs_, s);
  CKL();
  CKR(sync_check(s));
  return kOK;
}

int Engine::bubbles(int k, double side, double gas_density, int* ns_out, std::vector<uint32_t>* counts,
                    std::vector<int64_t>* sizes, cudaStream_t s) {
  if (!valid_id(k)) { set_error("no such system"); return kErrArg; }
  const SysHost& h = sys_[k];
  if (!h.has_state) { set_error("no state set"); return kErrState; }
  if (!(side > 0.0) || !std::isfinite(gas_density)) { set_error("need side > 0"); return kErrArg; }
  const int64_t ns = std::max<int64_t>(1, (int64_t)std::floor(h.spec.L / side));
  const int64_t ncell = ns * ns * ns;
  if (ncell >= ((int64_t)1 << 31) - 1) { set_error("too many subcells (ns^3 >= 2^31)"); return kErrArg; }
  uint32_t* d_counts = nullptr;
  uint32_t* d_size = nullptr;
  int32_t* d_parent = nullptr;
  int* d_err = nullptr;
  int r = dmalloc(&d_counts, ncell);
  if (r == kOK) r = dmalloc(&d_size, ncell);
  if (r == kOK) r = dmalloc(&d_parent, ncell);
  if (r == kOK) r = dmalloc(&d_err, 1);
  if (r != kOK) {
    dfree(d_counts); dfree(d_size); dfree(d_parent); dfree(d_err);
    return r;
  }
  const double vol = std::pow(h.spec.L / (double)ns, 3);
  launch_bubbles(arrays(), cur_of(k), k, h.spec.n, (int)ns, h.spec.L, gas_density * vol, d_counts, d_parent, d_size,
                 d_err, s);
  cudaError_t e = cudaGetLastError();
  std::vector<int32_t> parent((size_t)ncell);
  std::vector<uint32_t> size((size_t)ncell);
  int herr = 0;
  counts->assign((size_t)ncell, 0u);
  if (e == cudaSuccess) e = cudaMemcpyAsync(counts->data(), d_counts, sizeof(uint32_t) * ncell, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(parent.data(), d_parent, sizeof(int32_t) * ncell, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(size.data(), d_size, sizeof(uint32_t) * ncell, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dfree(d_counts); dfree(d_size); dfree(d_parent); dfree(d_err);
  if (e != cudaSuccess) { set_error(std::string("bubbles: ") + cudaGetErrorString(e)); return kErrCuda; }
  if (herr) { set_error("bubbles: union-find retry bound reached"); return kErrTimeout; }
  sizes->clear();
  for (int64_t c = 0; c < ncell; ++c)
    if (parent[(size_t)c] == (int32_t)c) sizes->push_back((int64_t)size[(size_t)c]);
  std::sort(sizes->begin(), sizes->end(), [](int64_t a, int64_t b) { return a > b; });
  *ns_out = (int)ns;
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
  if (!valid_id(k)) { set_error("no such system"); return kErrArg; }
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
  if (!valid_id(k)) { set_error("no such system"); return kErrArg; }
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

int Engine::debug_set_list_word(int k, int64_t slot, int m, uint32_t word, cudaStream_t s) {
  if (!kChecks) { set_error("list words can be written only in the checked build"); return kErrArg; }
  if (!valid_id(k)) { set_error("no such system"); return kErrArg; }
  const SysHost& h = sys_[k];
  if (!h.has_state) { set_error("no state set"); return kErrState; }
  CKR(ensure_lists(s));
  if (slot < 0 || slot >= h.spec.n || m < 0 || m >= h.kmax) { set_error("slot or entry out of range"); return kErrArg; }
  const int64_t w = list_word(h.l_off, (int)(slot / kTile), h.kmax, (int)(slot % kTile), m);
  CK(cudaMemcpyAsync(d_.nbr + w, &word, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
  return sync_check(s);
}

int Engine::get_list(int k, int64_t* start, int32_t* partners, cudaStream_t s) {
  if (!valid_id(k)) { set_error("no such system"); return kErrArg; }
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
      const uint32_t e = lw[(size_t)(list_word(0, (int)tl, h.kmax, (int)lane, m))];
      partners[start[i] + m] = id[(size_t)(e & kIdxMask)];
    }
  }
  return kOK;
}

}  // namespace ljmd
