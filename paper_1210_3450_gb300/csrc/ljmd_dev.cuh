// Device-side data layout and kernel declarations of the LJ-MD engine.
//
// Every system lives in a contiguous, 32-aligned range of "slots" of the shared
// particle arrays. Between list builds the particles of a system are stored in
// cell order (Sec. 2.1 grid method; positions sorted by cell give coalesced
// neighbour loads). A warp owns one tile of 32 consecutive slots of one system.
//
// Pair list (Sec. 2.1 "sorted pair list", Fig. 1) in a transposed key-pointer form:
// the partners of the particle in lane l of tile t are grouped four at a time,
//     nbr[list_off + ((t_local * kmax / 4 + k / 4) * 32 + l) * 4 + k % 4],  k < ncnt[slot],
// so each thread reads its next four partners with one 16-byte load and a warp
// reads 512 consecutive bytes per group. An entry packs the partner's slot index
// relative to the system (bits 0..25) and the periodic image of the partner
// (bits 26..31: two bits per axis, 0 = same image, 1 = +L, 2 = -L).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ljmd {

constexpr int kTile = 32;
constexpr int kIdxBits = 26;
constexpr uint32_t kIdxMask = (1u << kIdxBits) - 1u;

// Cells per chunk of the two-pass cell-count scan (256 threads x 4 cells).
constexpr int kScanChunk = 1024;
// Copies of each chunk total that the count kernel adds to (by warp), so that its
// atomics do not all meet on a few words; the scan sums the copies.
constexpr int kChunkCopies = 8;
__host__ __device__ inline int32_t scan_chunks(int64_t ncell) { return (int32_t)((ncell + kScanChunk - 1) / kScanChunk); }

// Word index of list entry k of the particle in lane `lane` of local tile tl
// (kmax is a multiple of 8).
__host__ __device__ inline int64_t list_word(int64_t l_off, int tl, int kmax, int lane, int k) {
  return l_off + (((int64_t)tl * (kmax >> 2) + (k >> 2)) * kTile + lane) * 4 + (k & 3);
}

// Per-system constants (device copy), written by the host.
struct SysParams {
  double L;          // box side
  double invL;       // 1 / L
  double inv_cs;     // nc / L (cells per unit length)
  double rc2;        // rc^2
  double rl2;        // (rc + skin)^2
  double c2, c0;     // Eq. 1 coefficients
  double dt;         // time step of the current md_step call
  double hdt;        // dt / 2 (a half kick)
  double qscale;     // 2^32 / L: fixed-point scale of the shadow positions
  float qunit;       // L / 2^32 as float: fixed-point unit
  float rl2q_lo;     // rl^2 (1 - 1e-5) in fixed-point units^2: certainly inside below
  float rl2q_hi;     // rl^2 (1 + 1e-5) in fixed-point units^2: certainly outside above
  float rl2f_lo;     // rl^2 (1 - eps(L / rl)) as float: the float pre-test's sure inside
  float rl2f_hi;     // rl^2 (1 + eps(L / rl)) as float: the float pre-test's sure outside
  float rc2q_hi;     // rc^2 (1 + 1e-5) in fixed-point units^2: surely outside rc above (FP64 force loop)
  float rc2f;        // rc^2 as float (FP32 force cutoff)
  float c2f;         // c2 as float
  double skin;       // list margin (validity rule 2 d_max >= skin)
  double disp_thr;   // FP32-force form: threshold of the squared fixed-point displacement
  float rlf;         // rc + skin as float
  float csf;         // cell side L / nc as float
  float Lf;          // L as float (the staged list build's image shifts)
  float wmargin;     // margin of the list build's geometric windows (1e-5 L + 1e-6)
  int64_t p_off;     // first slot
  int64_t c_off;     // first cell (cell arrays hold ncell + 1 entries per system)
  int64_t l_off;     // first list word
  int32_t n;         // particles
  int32_t nc;        // cells per axis; 1 = every pair is a candidate
  int32_t kmax;      // list capacity per particle
  int32_t t_off;     // first global tile
  int32_t ntiles;    // tiles of this system
  int32_t active;    // 1 if the system takes part in the current launches
  int32_t rule;      // list validity: 0 displacement (2 d_max >= skin), 1 velocity bound (DUTC)
  int32_t half;      // 1: half list (each pair once, in its lower slot's list; Newton's third law)
};

// Per-system status words written by kernels and read by the host.
struct SysStatus {
  int32_t overflow;   // largest list length that did not fit (0 = none)
  int32_t nonfinite;  // 1 if a position or velocity became non-finite
  int32_t max_count;  // largest list length of the last build
  int32_t pad_;
};

// Kernel flags of the fused force + integration step.
enum StepFlags : int {
  kStepDrift = 1,       // drift x by dt v after the kicks (writes the other x buffer)
  kStepStoreF = 2,      // store F (double) for md_forces / the next call
  kStepUseStoredF = 4,  // take F from the stored buffer instead of the pair loop
  kStepKickA = 8,       // v += dt/2 F completing the previous step
  kStepKickB = 16,      // v += dt/2 F, first half-kick of the next step
  kStepVmax = 32,       // report max |v|^2 of the drift velocities (velocity-bound rule) instead of
                        // the displacement
};

// Control words of the graph-captured step loop (device-resident; NULL in
// DevArrays when the host drives the loop).
struct GraphCtl {
  int32_t abort;   // 1: a pair list overflowed, 2: a non-finite value; the remaining steps do nothing
  int32_t flags;   // StepFlags of the next step
  int32_t nreb;    // systems rebuilding in the current pass
  int32_t done;    // steps taken
  int32_t target;  // steps to take
  int32_t passes;  // rebuild passes taken
  int32_t next_tile;  // list build's work counter
  int32_t pad_;
};

struct DevArrays {
  double4_32a* x[2];      // positions (w unused), ping-pong by step parity
  double4_32a* v;         // velocities
  double4_32a* xref;      // positions at the last list build (FP64 form's check)
  int4* xqref;        // shadow positions at the last list build (FP32-force form's check)
  double4_32a* f;         // stored forces (double); half list: the own-list sums of the step
  double4_32a* facc;      // half list: forces added by the partners' threads (atomics), zeroed on use
  int4* xq[2];        // fixed-point shadow positions (uint32 per axis, wraps at L)
  int32_t* id;        // caller index of each slot, -1 for padding
  int32_t* cell;      // cell of each slot (valid after binning)
  int32_t* ncnt;      // list length of each slot
  uint32_t* nbr;      // list words
  double* tile_obs;   // per-tile (PE, W, KE) partial sums for observables
  // rebuild scratch
  long long* skey;    // sort key (x bits) of each scattered position
  double4_32a* vtmp;
  float4* xf;         // positions as float at the last list build (list pre-test; 4 spare entries)
  int32_t* idtmp;
  int32_t* celltmp;
  int32_t* perm;      // scattered position -> old slot (cell order, arbitrary within a cell)
  int32_t* sid;     // caller index of each scattered position (the ranking's tie-break)
  int32_t* ccount;    // particles per cell (then fill counters)
  int32_t* cstart;    // first slot of each cell (relative to the system), ncell + 1 per system
  // systems
  const SysParams* params;
  SysStatus* status;
  unsigned long long* disp2;  // per system: max squared displacement, or max |v|^2 (double bits)
  double* margin;             // per system: velocity-bound rule's remaining margin
  const int32_t* rebuild;     // per system: 1 if it rebuilds in the current pass
  const int32_t* rebuild_ids; // ids of the systems that rebuild (compact, costliest tiles first)
  const int32_t* sys_order;   // system ids by descending list-build cost per tile
  const int32_t* reb_pref;    // exclusive prefix of the rebuilding systems' tile counts (nreb + 1)
  int32_t* chunk_pref;        // exclusive prefix of the rebuilding systems' cell-chunk counts (nreb + 1)
  int32_t* chunk_sum;         // particles per cell chunk of the rebuilding systems, kChunkCopies partial
                              // sums each (added up by the count)
  int32_t chunk_cap;          // entries of chunk_sum
  int32_t nreb;               // rebuilding systems (host-driven passes; the graph reads ctl->nreb)
  int32_t* tile_next;         // work counter of the list build (reset before each build)
  int32_t* checks;            // per system: failed device checks (bits of CheckBits; checked build)
  const int32_t* tile_sys;  // system of each global tile
  int32_t ntiles;
  GraphCtl* ctl;            // graph-captured loop: step flags, rebuild count, abort word
};

// Device bounds checks of the checked build (compiled with LJMD_CHECKS): a failed
// check sets a bit of the system's check word, the access is skipped or clamped to
// a valid one, and the host reports MD_ERR_CHECK at its next synchronisation. The
// product build compiles them out (check_ok is constant true).
#ifdef LJMD_CHECKS
constexpr bool kChecks = true;
#else
constexpr bool kChecks = false;
#endif
enum CheckBits : int {
  kChkCell = 1,       // binning: cell index outside [0, ncell)
  kChkScatter = 2,    // scatter: position past the end of the particle's cell
  kChkRank = 4,       // in-cell ranking: position past the end of the cell
  kChkGather = 8,     // gather: source slot outside [0, n)
  kChkListEntry = 16, // list build: partner slot outside [0, n), or the particle itself
  kChkPartner = 32,   // pair loops: listed partner slot outside [0, n)
  kChkCount = 64,     // pair loops: list length above the capacity kmax
};
__device__ __forceinline__ bool check_ok(const DevArrays& a, int sys, bool ok, int bit) {
  if (kChecks && !ok) atomicOr(&a.checks[sys], bit);
  return !kChecks || ok;
}

// Launch shapes of the hot kernels (threads per block; partner groups of four
// per FP32 iteration), chosen by the autotuner.
struct Tuning {
  int step_block = 128;
  int step_groups = 2;
  int list_block = 128;
  int list_variant = 5;  // 0..3 per thread (bit 0: fixed-point pre-test; bit 1: row pruning); 4 per warp;
                         // 5 as 0 with each row's candidates staged in shared memory
  int step_hint = 1;     // 1: L1 eviction hints on the FP32 step kernel's loads
  int fp64_queue = 1;    // 1: FP64 force loop classifies pairs first and queues the maybe-inside ones
};

// ---------------------------------------------------------------- launchers
// All launches cover every tile of every active system; warps of inactive
// systems (or of systems not rebuilding, for the rebuild kernels) return early.

// Kernels of one rebuild pass: count (with the scan's chunk totals), scan, scatter,
// rank with gather, list build (which also copies the gathered state back into
// place).
constexpr int kRebuildLaunches = 5;

// Counts the rebuilding systems' particles per cell and per scan chunk; the chunk
// totals must be zero before (the decision or the host-driven pass clears them).
void launch_cell_count(const DevArrays& a, int cur, cudaStream_t s);
// Exclusive scan of the cell counts into the cell starts.
void launch_cell_scan(const DevArrays& a, int nreb, cudaStream_t s);
void launch_scatter(const DevArrays& a, int cur, cudaStream_t s);
// In-cell order and gather into it.
void launch_cell_rank(const DevArrays& a, int cur, cudaStream_t s);
void launch_build_list(const DevArrays& a, int cur, const Tuning& tu, cudaStream_t s);
// Device-side list-validity decision of the graph-captured loop (see GraphCtl).
// reb_count NULL: outside a graph (no step or pass counting, no node conditions).
void launch_decide(const DevArrays& a, int nsys, int fp32, int vflag, int32_t* rebuild, int32_t* rebuild_ids,
                   int32_t* reb_pref, int32_t* reb_count, cudaGraphConditionalHandle h_if,
                   cudaGraphConditionalHandle h_loop, int last, cudaStream_t s);
// mode 0: FP64 reciprocal; 1..4: approximate reciprocal of Sec. 3.3 (8 bits,
// 8 bits corrected, 23 bits, 23 bits corrected)
void launch_step_fp64(const DevArrays& a, int cur, double ka, double kb, int flags, const Tuning& tu,
                      int mode, cudaStream_t s);
// Half list (Newton's third law): pair forces with atomic scatter to the partners,
// then the velocity-Verlet update from own + scattered sums (two launches).
void launch_step_half(const DevArrays& a, int cur, int flags, const Tuning& tu, int precision, cudaStream_t s);
void launch_step_fp32(const DevArrays& a, int cur, double ka, double kb, int flags, const Tuning& tu,
                      cudaStream_t s);
// select: per-system flags (NULL = every active system)
void launch_pe_virial(const DevArrays& a, int cur, int with_pairs, const int32_t* select, cudaStream_t s);
void launch_scale_v(const DevArrays& a, const double* scale, cudaStream_t s);
void launch_pair_stats(const DevArrays& a, int cur, unsigned long long* out2, cudaStream_t s);
// Per-system (PE, W, KE) sums into out3[3 sys] for the nsel systems listed in work
// (ids, then the prefix of their 256-tile chunk counts; nchunks in total); chunk3
// holds 3 doubles per chunk.
void launch_reduce_obs(const DevArrays& a, const int32_t* work, int nsel, int nchunks, double* chunk3, double* out3,
                       cudaStream_t s);
void launch_to_caller(const DevArrays& a, int cur, int which, double* out, int64_t sys_n,
                      int sys, int64_t ntiles_sys, cudaStream_t s);
void launch_positions_by_id(const DevArrays& a, int cur, const double* x, int64_t sys_n, int sys, cudaStream_t s);
void launch_from_caller(const DevArrays& a, int cur, const double* x, const double* v,
                        int sys, int64_t ntiles_sys, cudaStream_t s);

// Bubble identification of system `sys` (Sec. 4.2): subcell counts, gas where
// count < gas_count, union-find labels (root = smallest index), cluster sizes.
void launch_bubbles(const DevArrays& a, int cur, int sys, int64_t n, int ns, double box, double gas_count,
                    uint32_t* counts, int32_t* parent, uint32_t* size, int* err, cudaStream_t s);

}  // namespace ljmd
