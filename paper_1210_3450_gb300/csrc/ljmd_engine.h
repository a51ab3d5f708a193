// Host engine: owns the device arrays of one or more LJ systems and drives the
// kernels of one velocity-Verlet step, the list-validity check and the rebuild.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ljmd_dev.cuh"

namespace ljmd {

struct SysSpec {
  int64_t n;
  double L, rc, skin;
};

struct SysHost {
  SysSpec spec;
  double rl = 0, c2 = 0, c0 = 0;
  int nc = 1;
  int64_t ncell = 1;
  int kmax = 0;
  int64_t p_off = 0, c_off = 0, l_off = 0;
  int32_t t_off = 0, ntiles = 0;
  bool active = true;
  bool has_state = false;
  bool force_rebuild = true;
  bool f_valid = false;
  int64_t rebuilds = 0, steps = 0;
  double dt = 0.0;
};

// Status codes shared with the C ABI (same values as MD_*).
enum : int { kOK = 0, kErrArg = -1, kErrOOM = -2, kErrOverflow = -3, kErrNonfinite = -4,
             kErrTimeout = -5, kErrCuda = -6, kErrState = -7 };

void set_error(const std::string& msg);
const char* last_error_cstr();

class Engine {
 public:
  Engine() = default;
  ~Engine();
  Engine(const Engine&) = delete;
  Engine& operator=(const Engine&) = delete;

  // Lay out and allocate all systems; returns a status code.
  int init(const std::vector<SysSpec>& specs, int precision);
  int set_precision(int mode);
  int precision() const { return precision_; }
  int nsys() const { return (int)sys_.size(); }
  const SysHost& sys(int k) const { return sys_[k]; }

  // State transfer for one system: device arrays of n*3 doubles in caller order.
  int set_state_dev(int k, const double* x, const double* v, cudaStream_t s);
  int get_state_dev(int k, double* x, double* v, cudaStream_t s);
  int forces_dev(int k, double* f, cudaStream_t s);

  // Advance every active system by nsteps steps of its own dt.
  int step(int64_t nsteps, const std::vector<double>& dt, cudaStream_t s);
  // Observables (pe, virial, ke) of every active system into host out3[3 * nsys].
  int observables(double* out3, cudaStream_t s);
  // Rebuild the lists of all active systems now.
  int build_lists(cudaStream_t s);
  // Inspection (host arrays, caller order).
  int get_cells(int k, int32_t* cell, cudaStream_t s);
  int list_size(int k, int64_t* total, cudaStream_t s);
  int get_list(int k, int64_t* start, int32_t* partners, cudaStream_t s);

  void set_active(int k, bool on);
  // Per-kernel-class device times (CUDA events on the launching stream).
  int set_timing(bool on);
  void get_timing(double* out8) const;
  int pair_stats(int k, int64_t* listed, int64_t* inside, cudaStream_t s);
  double* stage() const { return d_stage_; }  // 6 * max n doubles of device scratch

 private:
  int alloc_all();
  void free_all();
  int upload_params();
  int rebuild(std::vector<int> which, cudaStream_t s);
  int ensure_lists(cudaStream_t s);
  int ensure_forces(cudaStream_t s);
  int launch_step(double ka, double kb, int flags, cudaStream_t s);
  int post_drift(cudaStream_t s);
  int sync_check(cudaStream_t s);
  DevArrays arrays() const;
  enum TimedKind { kTStep = 0, kTList = 1, kTBin = 2 };
  void tmark_begin(int kind, cudaStream_t s);
  void tmark_end(cudaStream_t s);
  void collect_timing();
  struct TimedPair { cudaEvent_t a, b; int kind; };
  bool timing_ = false;
  std::vector<cudaEvent_t> ev_free_;
  std::vector<TimedPair> ev_pending_;
  TimedPair ev_open_{nullptr, nullptr, -1};
  double t_ms_[3] = {0, 0, 0};
  int64_t t_count_[3] = {0, 0, 0};
  int64_t n_launch_ = 0;
  int64_t n_rebuild_seq_ = 0;
  unsigned long long* d_pairs_ = nullptr;

  std::vector<SysHost> sys_;
  int precision_ = 0;
  int cur_ = 0;
  int64_t nslots_ = 0, ncells_ = 0, nlist_ = 0, max_cells_ = 1;
  int32_t ntiles_ = 0;

  DevArrays d_{};
  SysParams* d_params_ = nullptr;
  SysStatus* d_status_ = nullptr;
  unsigned long long* d_disp2_ = nullptr;
  int32_t* d_rebuild_ = nullptr;
  int32_t* d_tile_sys_ = nullptr;
  double* d_obs_ = nullptr;
  double* d_stage_ = nullptr;   // caller-order staging (3 * max n doubles x 2)
  int64_t stage_n_ = 0;
  // pinned host mirrors
  SysStatus* h_status_ = nullptr;
  unsigned long long* h_disp2_ = nullptr;
  int32_t* h_rebuild_ = nullptr;
  double* h_obs_ = nullptr;
};

}  // namespace ljmd
