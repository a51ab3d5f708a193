// Host engine: owns a device-resident arena holding any number of independent
// LJ systems and drives the kernels of one velocity-Verlet step, the
// list-validity check and the rebuild for all of them at once.
//
// The arena has fixed capacities (particle slots, cell entries, list words,
// system records). Systems are added and removed at run time (first-fit range
// allocation), which is what continuous batching needs: a new system takes free
// ranges while the others keep running, and a finished one returns its ranges.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "ljmd_dev.cuh"

namespace ljmd {

struct SysSpec {
  int64_t n;
  double L, rc, skin;
};

struct SysHost {
  SysSpec spec{};
  bool used = false;
  double rl = 0, c2 = 0, c0 = 0;
  int nc = 1;
  int64_t ncell = 1;
  int kmax = 0;
  int old_kmax = 0;
  int64_t p_off = 0, c_off = 0, l_off = 0;
  int32_t t_off = 0, ntiles = 0;
  bool active = false;
  bool has_state = false;
  bool force_rebuild = true;
  bool f_valid = false;
  int64_t rebuilds = 0, steps = 0;
  double dt = 0.0;
  // Position buffer (0/1) of an inactive system: launches advance the other
  // systems' buffers in turn while its positions stay put; -1 = follows the engine.
  int park = -1;
};

struct ArenaCaps {
  int64_t slots;       // particle slots (rounded up to whole 32-slot tiles)
  int64_t cells;       // cell-array entries (a system uses nc^3 + 1)
  int64_t list_words;  // pair-list words
  int max_systems;     // system records
};

// Status codes shared with the C ABI (same values as MD_*).
enum : int { kOK = 0, kErrArg = -1, kErrOOM = -2, kErrOverflow = -3, kErrNonfinite = -4,
             kErrTimeout = -5, kErrCuda = -6, kErrState = -7, kErrCheck = -8 };

void set_error(const std::string& msg);
const char* last_error_cstr();

// First-fit allocator of integer ranges [off, off + len) within [0, cap).
class RangeAlloc {
 public:
  void reset(int64_t cap);
  int64_t alloc(int64_t len);  // offset, or -1 if no free range is long enough
  void release(int64_t off, int64_t len);
  int64_t cap() const { return cap_; }
  void grow(int64_t new_cap);  // append [cap, new_cap) as free
  int64_t free_total() const;
  int64_t largest_free() const;

 private:
  int64_t cap_ = 0;
  std::map<int64_t, int64_t> free_;  // offset -> length
};

// Validates a system and derives its sizes (also used for admission checks).
struct SysFootprint {
  int64_t slots, cells, list_words;
};
int footprint(const SysSpec& s, SysFootprint* f, SysHost* h);

class Engine {
 public:
  Engine() = default;
  ~Engine();
  Engine(const Engine&) = delete;
  Engine& operator=(const Engine&) = delete;

  // Exact-size arena for a fixed set of systems (ids 0..n-1).
  int init(const std::vector<SysSpec>& specs, int precision);
  // Empty arena with the given capacities.
  int init_arena(const ArenaCaps& caps, int precision);
  // Add a system in free ranges; kErrOOM if it does not fit (nothing changes).
  int add_system(const SysSpec& s, int* id);
  int remove_system(int id);
  // out8: slots cap/free, cells cap/free, list cap/free, systems cap/used.
  void arena_usage(int64_t* out8) const;

  int set_precision(int mode);
  // List validity rule: 0 displacement (2 d_max >= skin), 1 velocity bound (DUTC).
  int set_rule(int rule);
  int rule() const { return rule_; }
  // Pair list: 0 full (default), 1 half with Newton's third law (atomic scatter).
  int set_list_kind(int kind);
  int precision() const { return precision_; }
  int nsys() const { return (int)sys_.size(); }
  const SysHost& sys(int k) const { return sys_[k]; }
  bool valid_id(int k) const { return k >= 0 && k < nsys() && sys_[k].used; }

  // State transfer for one system: device arrays of n*3 doubles in caller order.
  int set_state_dev(int k, const double* x, const double* v, cudaStream_t s);
  int get_state_dev(int k, double* x, double* v, cudaStream_t s);
  int forces_dev(int k, double* f, cudaStream_t s);
  // Exact checkpoint of system k (device arrays, caller order): positions as held
  // (not wrapped), velocities, positions at the last list build, and the
  // velocity-bound margin. Restoring rebuilds the list from the build positions
  // (the same slot order and list as at that build), then puts back the positions.
  int get_checkpoint_dev(int k, double* x, double* v, double* xref, double* margin, cudaStream_t s);
  int set_checkpoint_dev(int k, const double* xref, const double* v, cudaStream_t s);
  int finish_checkpoint_dev(int k, const double* x, double margin, cudaStream_t s);

  // Advance every active system by nsteps steps of its own dt (dt per system id;
  // entries of inactive ids are ignored).
  int step(int64_t nsteps, const std::vector<double>& dt, cudaStream_t s);
  // Nose-Hoover NVT (Sec. 4.1): per step a thermostat half step, one
  // velocity-Verlet step, a thermostat half step (reversible splitting); T, Q,
  // zeta, eta per system id (zeta, eta read and updated).
  int step_nvt(int64_t nsteps, const std::vector<double>& dt, const std::vector<double>& T,
               const std::vector<double>& Q, std::vector<double>& zeta, std::vector<double>& eta,
               cudaStream_t s);
  // Observables (pe, virial, ke) of every active system into host out3[3 * nsys].
  // select: nsys flags choosing the systems (NULL = every active system); the
  // entries of unselected systems in out3 are unspecified.
  int observables(double* out3, cudaStream_t s, bool with_pairs = true, const int32_t* select = nullptr);
  // v *= factor[id] for every active system (factor: nsys doubles).
  int scale_velocities(const std::vector<double>& factor, cudaStream_t s);
  // Rebuild the lists of all active systems now.
  int build_lists(cudaStream_t s);
  // Inspection (host arrays, caller order).
  int get_cells(int k, int32_t* cell, cudaStream_t s);
  int list_size(int k, int64_t* total, cudaStream_t s);
  // Checked build only: overwrite list entry m of sorted slot `slot` (a test of the checks).
  int debug_set_list_word(int k, int64_t slot, int m, uint32_t word, cudaStream_t s);
  int get_list(int k, int64_t* start, int32_t* partners, cudaStream_t s);

  int set_active(int k, bool on);
  // Launch shapes: key 0 = step-kernel threads per block (64/128/256), 1 = FP32
  // partner groups per iteration (1/2), 2 = list-build threads per block, 3 =
  // list-build variant, 4 = FP32 load hints, 5 = graph-captured step loop (0/1).
  int set_tuning(int key, int value);
  int get_tuning(int key) const;
  // Per-kernel-class device times (CUDA events on the launching stream).
  int set_timing(bool on);
  void get_timing(double* out8) const;
  int pair_stats(int k, int64_t* listed, int64_t* inside, cudaStream_t s);
  // Bubble identification (Sec. 4.2) of system k at its current positions:
  // ns subcells per axis (side >= `side`), counts per subcell, bubble sizes
  // (subcells) in descending order.
  int bubbles(int k, double side, double gas_density, int* ns, std::vector<uint32_t>* counts,
              std::vector<int64_t>* sizes, cudaStream_t s);
  // Device scratch of at least 6 * n doubles for caller-order staging.
  int stage(int64_t n, double** out);

 private:
  int alloc_arrays();
  void free_all();
  int upload_params(int only = -1);
  int upload_order();
  int upload_tiles(int k, int32_t value);
  int grow_list_arena(int64_t min_extra_units);
  void update_extent();
  int rebuild(std::vector<int> which, cudaStream_t s);
  int ensure_lists(cudaStream_t s);
  int ensure_forces(cudaStream_t s);
  int launch_step(double ka, double kb, int flags, cudaStream_t s);
  int post_drift(cudaStream_t s);
  // Graph-captured step loop (tuning key 5): a CUDA graph whose loop node runs
  // two steps per iteration, each followed by the device-side list-validity
  // decision and a conditional node holding the rebuild pass. The host reads
  // the control words once per graph launch instead of after every step; a
  // list overflow or a non-finite value stops the loop (the host grows the list
  // and resumes, or reports the error), so results equal the host-driven loop's.
  int capture_graph(int parity);
  int build_graph(cudaGraph_t g, int parity);
  void drop_graphs();
  int run_graph(int64_t nsteps, int first_flags, int64_t* done, cudaStream_t s);
  int sync_check(cudaStream_t s);
  bool any_active() const;  // some system takes part in launches
  int read_checks(cudaStream_t s);  // checked build: MD_ERR_CHECK if a device check failed
  DevArrays arrays() const;
  // Buffer holding system k's current positions.
  int cur_of(int k) const { return (!sys_[k].active && sys_[k].park >= 0) ? sys_[k].park : cur_; }
  // Tuning of the list build (the warp-cooperative variant builds full lists only).
  Tuning list_tuning() const {
    Tuning t = tuning_;
    if (half_ && t.list_variant == 4) t.list_variant = 0;
    return t;
  }
  enum TimedKind { kTStep = 0, kTList = 1, kTBin = 2 };
  void tmark_begin(int kind, cudaStream_t s);
  void tmark_end(cudaStream_t s);
  void collect_timing();
  struct TimedPair { cudaEvent_t a, b; int kind; };
  Tuning tuning_{};
  bool timing_ = false;
  std::vector<cudaEvent_t> ev_free_;
  std::vector<TimedPair> ev_pending_;
  TimedPair ev_open_{nullptr, nullptr, -1};
  double t_ms_[3] = {0, 0, 0};
  int64_t t_count_[3] = {0, 0, 0};
  int64_t n_launch_ = 0;
  int64_t n_rebuild_seq_ = 0;
  bool graph_ = true;
  int64_t struct_ver_ = 0;  // bumped whenever captured launches would change
  cudaGraphExec_t gexec_[2] = {nullptr, nullptr};
  int64_t gver_[2] = {-1, -1};
  cudaStream_t cap_[2] = {nullptr, nullptr};
  GraphCtl* d_ctl_ = nullptr;
  GraphCtl* h_ctl_ = nullptr;
  int32_t* d_reb_count_ = nullptr;
  int32_t* h_reb_count_ = nullptr;

  std::vector<SysHost> sys_;
  int precision_ = 0;
  int rule_ = 0;
  bool half_ = false;
  int cur_ = 0;
  ArenaCaps caps_{0, 0, 0, 0};
  bool list_growable_ = false;  // exact-size arenas grow their list storage on demand
  RangeAlloc slot_alloc_, cell_alloc_, list_alloc_;
  int32_t ntiles_ = 0;  // launch extent: tiles up to the last used one
  std::vector<int32_t> h_tile_sys_;

  DevArrays d_{};
  SysParams* d_params_ = nullptr;
  SysStatus* d_status_ = nullptr;
  unsigned long long* d_disp2_ = nullptr;
  double* d_margin_ = nullptr;
  int32_t* d_checks_ = nullptr;  // per system: failed device checks (checked build)
  int32_t* d_rebuild_ = nullptr;  // flags (nsys), compact ids (nsys), tile prefix (nsys + 1), chunk prefix (nsys + 1)
  int32_t* d_tile_sys_ = nullptr;
  int32_t* d_order_ = nullptr;    // system ids by descending list-build cost per tile
  std::vector<int32_t> order_rank_;  // position of each system in that order
  double* d_obs_ = nullptr;
  int32_t* d_obs_work_ = nullptr;  // selected systems and their chunk prefix (observables)
  int32_t* h_obs_work_ = nullptr;
  double* d_obs_chunk_ = nullptr;  // chunk sums (3 doubles per 256 tiles)
  unsigned long long* d_pairs_ = nullptr;
  double* d_stage_ = nullptr;
  int64_t stage_n_ = 0;
  // pinned host mirrors
  SysStatus* h_status_ = nullptr;
  unsigned long long* h_disp2_ = nullptr;
  int32_t* h_rebuild_ = nullptr;  // the same layout as d_rebuild_
  double* h_obs_ = nullptr;
};

}  // namespace ljmd
