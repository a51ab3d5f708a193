/*
 * ljmd.h — C ABI of the GB300 truncated-Lennard-Jones molecular-dynamics library.
 *
 * The library integrates N particles in a cubic periodic box of side L under the
 * truncated LJ potential of Eq. 1 of Watanabe, Suzuki and Ito, "Huge-scale
 * Molecular Dynamics Simulation of Multibubble Nuclei" (arXiv:1210.3450):
 *     V(r) = 4 [ r^-12 - r^-6 + c2 r^2 + c0 ]   for r < rc, 0 otherwise,
 * with c2 = 6 rc^-14 - 3 rc^-8 and c0 = 4 rc^-6 - 7 rc^-12 so that V(rc) = V'(rc) = 0
 * (reduced units: sigma = epsilon = k_B = m = 1). Forces come from a Verlet pair
 * list (radius rl = rc + skin, Sec. 2.1 "bookkeeping method") built from a cell grid
 * (Sec. 2.1 "grid algorithm"): by default a full list without Newton's third law
 * (Sec. 3.3), optionally a half list with it (md_set_pair_list). The time integrator
 * is the second-order symplectic velocity-Verlet scheme (Sec. 3.2, 4.1), optionally
 * with a Nose-Hoover thermostat (md_step_nvt). By default the list is rebuilt when
 * twice the largest displacement since the last build reaches the skin (the
 * list-validity check of Sec. 2.1); md_set_validity_rule selects the velocity bound
 * instead.
 *
 * Conventions for every call:
 *   - Return value 0 (MD_OK) on success, a negative MD_ERR_* code on failure;
 *     md_last_error() then returns a thread-local message.
 *   - Host arrays are caller-owned and only read or written during the call; the
 *     library never keeps a caller pointer. Position, velocity and force arrays are
 *     N x 3 float64 in C order (x0 y0 z0 x1 y1 z1 ...), particle order = the order of
 *     the caller's md_set_state.
 *   - "_dev" variants take device pointers (e.g. a torch tensor's data_ptr) with the
 *     same layout and a cudaStream_t passed as void* (NULL = legacy default stream);
 *     the library orders its work after earlier work on that stream and returns
 *     without synchronising the stream unless stated.
 *   - A context owns all its device memory; calls on one context must not overlap.
 *   - Every call reports CUDA failures as MD_ERR_CUDA. Kernels do not trap: they write
 *     status words (list overflow, non-finite values) that the host checks.
 */
#ifndef LJMD_H
#define LJMD_H

#include <stdint.h>

#if defined(__GNUC__)
#define MD_API __attribute__((visibility("default")))
#else
#define MD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define MD_OK 0
#define MD_ERR_ARG (-1)           /* invalid argument (sizes, box too small, null) */
#define MD_ERR_OOM (-2)           /* device allocation failed                      */
#define MD_ERR_LIST_OVERFLOW (-3) /* list capacity could not be grown enough       */
#define MD_ERR_NONFINITE (-4)     /* a position or velocity became NaN or infinite  */
#define MD_ERR_TIMEOUT (-5)       /* a bounded device wait gave up                 */
#define MD_ERR_CUDA (-6)          /* a CUDA runtime call failed                    */
#define MD_ERR_STATE (-7)         /* call needs a state set by md_set_state first  */
#define MD_ERR_CHECK (-8)         /* a device bounds check failed (checked build)   */

/* Force precision modes (md_set_precision). */
#define MD_FP64 0       /* all pair arithmetic in FP64                                   */
#define MD_FP32_FORCE 1 /* pair forces in FP32 from fixed-point separations; positions,  */
                        /* velocities, list distance tests, energies, virial stay FP64  */
/* FP64 forms whose r^-8 and r^-14 come from an approximate reciprocal y of r^2, as in the
 * paper's FX10 kernel (Sec. 3.3): y is r^2's float reciprocal with its mantissa cut to 8
 * bits (the stand-in for SPARC64 frcpad, relative error < 1/256, Eq. 2) or kept (23 bits);
 * the _CORR forms apply Eqs. 2-7: r^-8 ~ y^4 (5 - 4 y r^2), r^-14 ~ y^7 (8 - 7 y r^2). Energies
 * and the virial stay exact FP64. */
#define MD_FP64_RCP8 2
#define MD_FP64_RCP8_CORR 3
#define MD_FP64_RCP23 4
#define MD_FP64_RCP23_CORR 5

/* Largest particle count of one system (the list packs a slot index in 26 bits). */
#define MD_MAX_N ((int64_t)((1 << 26) - 1))

typedef struct md_ctx md_ctx;

/* ------------------------------------------------------------ single system */

/* Create a system of N particles in a cubic box of side box_L with cutoff rc and list
 * skin (Sec. 2.1: the list radius is rc + skin). Requires 0 < N <= MD_MAX_N, rc > 0,
 * skin >= 0, box_L > 2 (rc + skin) and box_L <= 10000. Precision defaults to MD_FP64.
 * Allocates all device memory on the current CUDA device; *out receives the handle.
 * Errors: MD_ERR_ARG, MD_ERR_OOM, MD_ERR_CUDA. */
MD_API int md_create(double box_L, int64_t N, double rc, double skin, md_ctx** out);

/* Select the force form (MD_FP64, MD_FP32_FORCE, MD_FP64_RCP*). Cached forces are
 * invalidated. */
MD_API int md_set_precision(md_ctx* ctx, int mode);

/* List validity rule (Sec. 2.1: the list is checked every step).
 *   MD_RULE_DISPLACEMENT (default): rebuild when 2 d_max >= skin, d_max the largest
 *     displacement since the last build (exact FP64; in MD_FP32_FORCE the exact integer
 *     displacement of the fixed-point shadow against a threshold 4 units lower).
 *   MD_RULE_DUTC: the velocity bound of the paper's DUTC check: a margin equal to the skin
 *     after each build shrinks every step by 2 v_max dt (v_max the largest drift speed,
 *     FP64) and the list is rebuilt when the margin is no longer positive; it bounds the
 *     displacements from above, so it rebuilds no later than the displacement rule.
 * Changing the rule rebuilds the lists before the next step. Errors: MD_ERR_ARG. */
#define MD_RULE_DISPLACEMENT 0
#define MD_RULE_DUTC 1
MD_API int md_set_validity_rule(md_ctx* ctx, int rule);

/* Pair-list form.
 *   MD_LIST_FULL (default): every particle lists all its partners and sums its own
 *     force (no Newton's third law), as the paper's FX10 kernel (Sec. 3.3).
 *   MD_LIST_HALF: each pair is listed once (Sec. 2.1: pairs i < j; here in the list of the
 *     pair's lower slot in cell order) and its force is added to both particles, the
 *     partner's share by FP64 atomic additions; the step takes two launches (forces,
 *     then the update). The order of the atomic additions varies between runs, so results
 *     vary in the last bits. md_get_list then returns each pair once; md_pair_stats counts
 *     each pair once. The warp-cooperative list build (MD_TUNE_LIST_VARIANT 4) builds full
 *     lists only and gives way to variant 0. Changing the form rebuilds the lists.
 * Errors: MD_ERR_ARG. */
#define MD_LIST_FULL 0
#define MD_LIST_HALF 1
MD_API int md_set_pair_list(md_ctx* ctx, int kind);

/* Copy positions x (N*3, any real values: wrapped into [0, L) on entry) and velocities
 * v (N*3) from host memory; forces a list rebuild before the next force evaluation. */
MD_API int md_set_state(md_ctx* ctx, const double* x, const double* v);

/* Exact checkpoint for resuming a run bit for bit (the paper's product runs last many
 * hours, Sec. 4.1). md_get_checkpoint copies into caller-allocated N*3 arrays the
 * positions as held (between list builds positions are not wrapped, so that the
 * periodic images stored in the list stay valid; they lie within L + skin of the box),
 * the velocities and the positions at the last list build, and the velocity-bound
 * margin (MD_RULE_DUTC). md_set_checkpoint restores them into a context with the same
 * N, L, rc, skin, precision, rule and pair-list form: the list is rebuilt from the build
 * positions (the same particle order and list as at that build) and the positions as
 * held are put back, so that the following steps equal those of the uninterrupted run.
 * Errors: MD_ERR_ARG, MD_ERR_STATE (no state to checkpoint), MD_ERR_CUDA. */
MD_API int md_get_checkpoint(md_ctx* ctx, double* x, double* v, double* x_build, double* margin);
MD_API int md_set_checkpoint(md_ctx* ctx, const double* x, const double* v, const double* x_build,
                             double margin);

/* Same with device pointers (N*3 float64 each), ordered on stream. */
MD_API int md_set_state_dev(md_ctx* ctx, const double* x_dev, const double* v_dev, void* stream);

/* Copy current positions (wrapped, in [0, L)) and velocities into caller arrays (N*3). */
MD_API int md_get_state(md_ctx* ctx, double* x, double* v);

/* Same into device arrays (N*3 float64 each), ordered on stream; x or v may be NULL. */
MD_API int md_get_state_dev(md_ctx* ctx, double* x_dev, double* v_dev, void* stream);

/* Advance nsteps velocity-Verlet steps of size dt (nsteps >= 0). Blocks until done.
 * Errors: MD_ERR_STATE (no state), MD_ERR_NONFINITE, MD_ERR_LIST_OVERFLOW, MD_ERR_CUDA. */
MD_API int md_step(md_ctx* ctx, int64_t nsteps, double dt);

/* Same, ordered on the given stream (the call still waits for the per-step list
 * validity decision, which is read back from the device every step). */
MD_API int md_step_async(md_ctx* ctx, int64_t nsteps, double dt, void* stream);

/* Nose-Hoover NVT steps (the thermostat of Sec. 4.1): each step is a thermostat half
 * step, one velocity-Verlet step (md_step) and a thermostat half step, the reversible
 * splitting: zeta += dt/4 G, eta += dt/2 zeta, v *= exp(-dt/2 zeta), zeta += dt/4 G'
 * with G = (2 KE - 3 (N - 1) T) / Q. zeta and eta (thermostat velocity and position)
 * are read and updated; KE + PE + Q zeta^2 / 2 + 3 (N - 1) T eta is conserved. */
MD_API int md_step_nvt(md_ctx* ctx, int64_t nsteps, double dt, double T, double Q, double* zeta,
                       double* eta);

/* Forces at the current positions (N*3 host array): F_i = sum_j g(r)(x_j - x_i),
 * g = 24 r^-8 - 48 r^-14 + 8 c2 for r < rc (Algorithm 1's bracket, Sec. 3.3). */
MD_API int md_forces(md_ctx* ctx, double* f);

/* Same into a device array (N*3 float64), ordered on stream. */
MD_API int md_forces_dev(md_ctx* ctx, double* f_dev, void* stream);

/* Observables at the current state (any pointer may be NULL):
 *   pe     = sum_{i<j} V(r_ij)                        (Eq. 1)
 *   virial = sum_{i<j} -r_ij V'(r_ij)
 *   ke     = sum_i |v_i|^2 / 2
 *   T      = 2 ke / (3 (N - 1))
 *   P      = (2 ke + virial) / (3 L^3)
 * Sums are accumulated in FP64 in a fixed order (deterministic). */
MD_API int md_observables(md_ctx* ctx, double* pe, double* virial, double* ke, double* T, double* P);

/* Kinetic energy sum_i |v_i|^2 / 2 only (no pair sums; cheaper than md_observables). */
MD_API int md_kinetic_energy(md_ctx* ctx, double* ke);

/* v_i *= factor for every particle (e.g. a velocity-rescaling thermostat between
 * md_step calls). Positions, list and forces stay valid. */
MD_API int md_scale_velocities(md_ctx* ctx, double factor);

/* Counters: list builds since md_create (including forced ones) and steps taken. */
MD_API int md_stats(md_ctx* ctx, int64_t* rebuilds, int64_t* steps);

/* Build the pair list now at the current positions (normally automatic). */
MD_API int md_build_list(md_ctx* ctx);

/* Cell of each particle from the last list build, in caller order (N int32):
 * c = cx + nc (cy + nc cz), c_a = min(floor(x_a nc / L), nc - 1). nc = floor(L / rl),
 * lowered by one when L / nc < rl (1 + 1e-9), and replaced by 1 when below 3 (every
 * pair is then a candidate and every cell is 0); nc_out (may be NULL) receives it. */
MD_API int md_get_cells(md_ctx* ctx, int32_t* cell, int32_t* nc_out);

/* Number of entries of the current full pair list (sum of all list lengths). */
MD_API int md_list_size(md_ctx* ctx, int64_t* total);

/* Checked build only (see md_version): overwrite entry `entry` of the list of the
 * particle in sorted slot `slot` with the raw 32-bit list word `word` (partner slot
 * in bits 0..25, periodic image in bits 26..31), so that a test can show the device
 * checks at work: a pair loop that meets an out-of-range partner records it, skips
 * the partner, and the call returns MD_ERR_CHECK. The list is built first if
 * needed. The product build returns MD_ERR_ARG. */
MD_API int md_debug_set_list_word(md_ctx* ctx, int64_t slot, int32_t entry, uint32_t word);

/* Current full list in caller numbering: start[N+1] (int64) and partners[total] (int32)
 * in the library's internal order per particle (sort to compare as sets). */
MD_API int md_get_list(md_ctx* ctx, int64_t* start, int32_t* partners);

/* Bubble identification (Sec. 4.2): particles are counted in ns^3 subcells, ns =
 * floor(L / side) (the paper: side 3 sigma), a subcell is gas when count / volume <
 * gas_density (the paper: 0.2), and face-neighbouring gas subcells of the periodic
 * simple cubic lattice form one bubble (site percolation). Outputs (may be NULL):
 * ns_out; counts[ns^3] as unsigned char (saturated at 255, the paper's storage);
 * n_bubbles; sizes[min(n_bubbles, cap)] = subcells per bubble, descending.
 * Requires ns^3 < 2^31. Temporary device memory is allocated for the call. */
MD_API int md_bubbles(md_ctx* ctx, double side, double gas_density, int32_t* ns_out, uint8_t* counts,
                      int64_t* n_bubbles, int64_t* sizes, int64_t cap);

/* Pair counts of the current list: entries (listed, r < rl at the build) and those
 * with r < rc at the current positions (FP64 test). */
MD_API int md_pair_stats(md_ctx* ctx, int64_t* listed, int64_t* within_rc);

/* Device timing of the library's own kernels, taken with CUDA events recorded on
 * the stream each kernel is launched on. md_set_timing(ctx, 1) enables it and resets
 * the counters (0 disables). md_get_timing fills out8[8]:
 *   [0] fused force + integration kernel, total ms   [1] its launches
 *   [2] pair-list build kernel, total ms              [3] its launches
 *   [4] binning + sort + gather kernels, total ms     [5] list rebuilds
 *   [6] kernel launches of all kinds                  [7] 0 (reserved)          */
MD_API int md_set_timing(md_ctx* ctx, int on);
MD_API int md_get_timing(md_ctx* ctx, double* out8);

/* Forces without any device allocation, for callers that must not let a library
 * allocate device memory: applications whose device memory belongs to their own
 * allocator or pool (which has to account for every byte), and code that cannot
 * take the device-wide synchronisation that cudaMalloc / cudaFree may cause. The
 * paper has no counterpart of this call; it is a service of this library.
 *   x_dev  N*3 float64 positions on the current device (any real values: wrapped
 *          into [0, box_L) internally), read only;
 *   f_dev  N*3 float64 output on the current device: F_i = sum over j != i with
 *          minimum-image r < rc of (24 r^-8 - 48 r^-14 + 8 c2)(x_j - x_i), the same
 *          pair force as md_forces (no pair list; cells of side >= rc, the particles
 *          of a cell taken in caller order, so the same positions give the same
 *          forces bit for bit from call to call);
 *   stream cudaStream_t as void* (NULL = legacy default stream); the call only
 *          enqueues work on it and returns without synchronising.
 * Limits: 1 <= N <= 65536, rc > 0, 2 rc < box_L <= 10000; larger N returns MD_ERR_ARG.
 * Working memory is one fixed 3.0 MiB device array inside the library (every GPU
 * that loads the library holds it until the process exits); nothing is allocated.
 * The first call on a device looks up that array's device address with that device
 * current; make this first call before any stream capture. All calls share the one
 * array: calls whose work overlaps on the GPU (other streams, other threads) race
 * and must be serialised by the caller. Errors: MD_ERR_ARG, MD_ERR_CUDA. */
MD_API int md_forces_noalloc(const double* x_dev, int64_t N, double box_L, double rc,
                             double* f_dev, void* stream);

/* Measurement utility, not part of the paper's method: the fused multiply-add
 * throughput of one arithmetic pipe of the current device, the denominator of the
 * FP64 force kernel's roofline (that kernel is bound by the FP64 pipe, not HBM).
 *   kind       0: FP64 (DFMA), 1: FP32 (FFMA)
 *   iters      iterations of eight independent chains per thread (64 warps per SM);
 *              about 1e5 (FP64) or 5e6 (FP32) run for a few hundred milliseconds
 *   fma_per_s  output: thread-level FMA instructions per second (flops = 2 x)
 * Launches on the legacy default stream and synchronises it. Errors: MD_ERR_ARG,
 * MD_ERR_CUDA. */
MD_API int md_probe_fma_rate(int kind, int64_t iters, double* fma_per_s);

/* Launch shapes of the hot kernels (results do not depend on them, only speed):
 *   MD_TUNE_STEP_BLOCK   threads per block of the force + integration kernel: 64, 128, 256
 *   MD_TUNE_STEP_GROUPS  FP32-force partners loaded per iteration, in groups of 4: 1, 2
 *   MD_TUNE_LIST_BLOCK   threads per block of the pair-list build: 64, 128, 256
 *   MD_TUNE_LIST_VARIANT pair-list build variant (0..5; the lists are identical):
 *                        0..3 one thread per particle, bit 0 pre-testing candidates
 *                        on the fixed-point shadow positions instead of positions
 *                        rounded to float, bit 1 skipping neighbour rows farther
 *                        than rl in y or z and narrowing the others' x windows;
 *                        4 warp-cooperative (candidates shared by the lanes of a
 *                        row, staged in shared memory); 5 as 0, each row's
 *                        candidates for the whole warp first copied into shared
 *                        memory with coalesced loads
 *   MD_TUNE_STEP_HINT    1: L1 eviction hints on the FP32 step kernel's loads (list
 *                        words not kept in L1, partner positions kept)
 *   MD_TUNE_GRAPH        1: md_step runs its steps in CUDA-graph launches (a loop node of
 *                        two steps, each followed by a device-side list-validity
 *                        decision and a conditional rebuild pass), reading the
 *                        control words once per launch; 0: the host decides after
 *                        every step. Results are identical. Timing (md_set_timing)
 *                        uses the host-driven loop.
 *   MD_TUNE_FP64_QUEUE   1: the FP64 force loops classify each listed pair on the
 *                        fixed-point shadow positions first and run the FP64
 *                        arithmetic only for the pairs that may be inside rc, taken
 *                        from a per-thread queue in list order, so that warps run
 *                        it with full lanes; 0: one plain loop over the list.
 *                        Results are identical bit for bit.
 * Defaults 128 / 2 / 128 / 5 / 1 / 1 / 1. The autotuner (paper_1210_3450_gb300.autotune) times the
 * choices on the caller's own systems and sets the fastest. */
#define MD_TUNE_STEP_BLOCK 0
#define MD_TUNE_STEP_GROUPS 1
#define MD_TUNE_LIST_BLOCK 2
#define MD_TUNE_LIST_VARIANT 3
#define MD_TUNE_STEP_HINT 4
#define MD_TUNE_GRAPH 5
#define MD_TUNE_FP64_QUEUE 6
MD_API int md_set_tuning(md_ctx* ctx, int key, int value);
MD_API int md_get_tuning(md_ctx* ctx, int key, int* value);

/* Release all resources of ctx (NULL is ignored). */
MD_API void md_destroy(md_ctx* ctx);

/* ------------------------------------------------------------ many systems
 * A batch is one device-resident arena holding many independent systems (replicas
 * of uneven size). Every kernel of a step covers all active systems of the batch
 * in one launch (one warp per 32-particle tile, each tile belonging to one system),
 * so a step of the whole batch costs one launch per kernel, not one per system.
 * Systems can be added to and removed from free arena ranges between steps
 * (continuous batching). Each system keeps its own box, cutoff, skin, time step,
 * pair list, list-validity check and rebuild counter; results of a system do not
 * depend on the other systems in the batch (no cross-system arithmetic, fixed
 * per-system reduction order). Ids are small integers in [0, max_systems). */
typedef struct md_batch md_batch;

typedef struct md_sys_desc {
  int64_t N;    /* particles                         */
  double box_L; /* cubic box side                    */
  double rc;    /* cutoff of Eq. 1                   */
  double skin;  /* list margin (list radius rc+skin) */
} md_sys_desc;

/* Batch holding exactly nsys systems with ids 0..nsys-1 (arena sized to fit them).
 * Same limits per system as md_create. */
MD_API int md_batch_create(int nsys, const md_sys_desc* desc, int precision, md_batch** out);

/* Empty arena with capacities: particle slots, cell entries, pair-list words and
 * system records (see md_batch_footprint for what one system needs). */
MD_API int md_batch_create_arena(int64_t slots, int64_t cells, int64_t list_words, int max_systems,
                                 int precision, md_batch** out);

/* Arena space one system needs (particle slots, cell entries, list words);
 * validates desc like md_create. */
MD_API int md_batch_footprint(const md_sys_desc* desc, int64_t* slots, int64_t* cells,
                              int64_t* list_words);

/* Add a system in free arena ranges; *id receives its id. MD_ERR_OOM if it does not
 * fit (the batch is unchanged). The new system is active and needs a state. */
MD_API int md_batch_add(md_batch* b, const md_sys_desc* desc, int* id);

/* Remove a system and return its ranges to the arena. */
MD_API int md_batch_remove(md_batch* b, int id);

/* out8: slots capacity, slots free, cells capacity, cells free, list words capacity,
 * list words free, system records, systems in use. */
MD_API int md_batch_usage(md_batch* b, int64_t* out8);

/* Include (on = 1) or exclude (on = 0) a system from md_batch_step and
 * md_batch_observables (which report zeros for it). An excluded system keeps its state
 * untouched, however many steps the others take, and continues exactly where it stopped
 * when included again: a paused run's result equals its uninterrupted run. Its state
 * can still be read and set while excluded; md_batch_forces returns its forces from its
 * last step. */
MD_API int md_batch_set_active(md_batch* b, int id, int on);

MD_API int md_batch_set_precision(md_batch* b, int mode);
/* List validity rule of every system in the batch (MD_RULE_*), as md_set_validity_rule. */
MD_API int md_batch_set_validity_rule(md_batch* b, int rule);
/* Pair-list form of every system in the batch (MD_LIST_*), as md_set_pair_list. */
MD_API int md_batch_set_pair_list(md_batch* b, int kind);

/* Per-system state transfer, same conventions as md_set_state / md_get_state. */
MD_API int md_batch_set_state(md_batch* b, int id, const double* x, const double* v);
MD_API int md_batch_set_state_dev(md_batch* b, int id, const double* x_dev, const double* v_dev,
                                  void* stream);
MD_API int md_batch_get_state(md_batch* b, int id, double* x, double* v);
MD_API int md_batch_get_state_dev(md_batch* b, int id, double* x_dev, double* v_dev, void* stream);

/* Exact checkpoint of system id, as md_get_checkpoint / md_set_checkpoint: a system can
 * be saved, evicted and resumed later (in this batch, another one, or an md_ctx with the
 * same N, L, rc, skin and settings), continuing bit for bit as if never interrupted. */
MD_API int md_batch_get_checkpoint(md_batch* b, int id, double* x, double* v, double* x_build, double* margin);
MD_API int md_batch_set_checkpoint(md_batch* b, int id, const double* x, const double* v, const double* x_build,
                                   double margin);

/* Advance every active system by nsteps velocity-Verlet steps; dt[id] is the time
 * step of system id (an array of max_systems doubles; entries of inactive ids are
 * ignored). Blocks until done. */
MD_API int md_batch_step(md_batch* b, int64_t nsteps, const double* dt);
MD_API int md_batch_step_async(md_batch* b, int64_t nsteps, const double* dt, void* stream);

/* Nose-Hoover NVT steps for every active system (arrays of max_systems doubles;
 * zeta, eta read and updated), as md_step_nvt. */
MD_API int md_batch_step_nvt(md_batch* b, int64_t nsteps, const double* dt, const double* T,
                             const double* Q, double* zeta, double* eta);

/* Forces of one system at its current positions (N*3 host array). */
MD_API int md_batch_forces(md_batch* b, int id, double* f);

/* Observables of every active system: out[5 * id + {0..4}] = pe, virial, ke, T, P
 * (as md_observables); out holds 5 * max_systems doubles (inactive ids get zeros). */
MD_API int md_batch_observables(md_batch* b, double* out);

/* Same for the systems with select[id] != 0 only (select: max_systems int32); the
 * other entries of out are zero. Costs in proportion to the selected systems. */
MD_API int md_batch_observables_select(md_batch* b, const int32_t* select, double* out);

/* Kinetic energy of every active system: ke[id] (max_systems doubles, 0 if inactive). */
MD_API int md_batch_kinetic_energy(md_batch* b, double* ke);

/* v *= factor[id] for every active system (factor: max_systems doubles). */
MD_API int md_batch_scale_velocities(md_batch* b, const double* factor);

MD_API int md_batch_stats(md_batch* b, int id, int64_t* rebuilds, int64_t* steps);
MD_API int md_batch_set_tuning(md_batch* b, int key, int value);
MD_API int md_batch_get_tuning(md_batch* b, int key, int* value);
MD_API int md_batch_set_timing(md_batch* b, int on);
MD_API int md_batch_get_timing(md_batch* b, double* out8);
MD_API void md_batch_destroy(md_batch* b);

/* Thread-local description of the last error on this thread ("" if none). */
MD_API const char* md_last_error(void);

/* Library version string; it ends in ", checked)" for the checked build.
 *
 * Checked build: the same sources compiled with LJMD_CHECKS. Its kernels verify
 * their indices (cell of a particle, scatter and rank positions within a cell,
 * gather sources, every partner slot the list build appends and every partner slot
 * and list length a pair loop reads). A failed check is recorded in a per-system
 * word and the access is skipped or clamped; the next call that synchronises returns
 * MD_ERR_CHECK, and so does every later one. The product build has no checks. */
MD_API const char* md_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LJMD_H */
