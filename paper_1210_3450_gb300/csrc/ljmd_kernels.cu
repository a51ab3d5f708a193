// CUDA kernels of the LJ-MD hot path for sm_103a.
//
// Paper: Watanabe, Suzuki, Ito, "Huge-scale Molecular Dynamics Simulation of
// Multibubble Nuclei" (arXiv:1210.3450).
//   cell binning (counting sort)          - Sec. 2.1 grid / linked-list method
//   pair-list build with skin             - Sec. 2.1 bookkeeping method, Fig. 1
//   force loop (full list, no 3rd law)    - Sec. 3.3, Algorithm 1, Eq. 1
//   velocity-Verlet update, periodic box  - Sec. 3.2 / 4.1 (second-order symplectic)
//   displacement-triggered list check     - Sec. 2.1 (list validity every step)
//   PE / virial / KE reductions           - Sec. 2.2, 4.3 (energy and pressure)
//
// Work layout: one warp per tile of 32 consecutive slots of one system, one
// thread per particle ("key" particle data stays in registers, Sec. 2.1); the
// partner loop reads the transposed list so each k is one coalesced 128-byte load.
//
// Decisions that must agree bit for bit with a plain FP64 reference (cell of a
// particle, list membership, wrap into the box, displacement) use explicitly
// rounded FP64 intrinsics (__dadd_rn, __dmul_rn, ...), so the compiler cannot fuse
// them into FMAs.
#include <algorithm>

#include "ljmd_dev.cuh"
#include "ljmd_math.cuh"

namespace ljmd {

namespace {

constexpr int kBlock = 128;  // 4 tiles per block
constexpr unsigned kFull = 0xffffffffu;

struct TileCtx {
  int sys;
  int tl;       // tile index within the system
  int local;    // slot index within the system
  int64_t s;    // global slot
  bool act;     // lane holds a particle
  int r;        // rebuild passes: the system's place among the rebuilding systems
};

// Returns false if the whole warp has nothing to do.
__device__ __forceinline__ bool tile_ctx(const DevArrays& a, TileCtx& t, SysParams& P) {
  const int warp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= a.ntiles) return false;
  t.sys = a.tile_sys[warp];
  if (t.sys < 0) return false;  // free tile of the arena
  P = a.params[t.sys];
  if (!P.active) return false;
  t.tl = warp - P.t_off;
  t.local = t.tl * kTile + lane;
  t.s = P.p_off + t.local;
  t.act = t.local < P.n;
  return true;
}

// Slot of a listed partner (list word e); the checked build verifies it.
__device__ __forceinline__ uint32_t partner_slot(const DevArrays& a, int sys, uint32_t e, int n, uint32_t self) {
  const uint32_t j = e & kIdxMask;
  return check_ok(a, sys, j < (uint32_t)n, kChkPartner) ? j : self;
}
// List length of a slot; the checked build verifies it against the capacity.
__device__ __forceinline__ int list_count(const DevArrays& a, int sys, int64_t s, int kmax) {
  const int cnt = a.ncnt[s];
  return check_ok(a, sys, cnt >= 0 && cnt <= kmax, kChkCount) ? cnt : 0;
}

// Tile w of the rebuilding systems (in rebuild order; reb_pref holds the prefix of
// their tile counts): false if its system is inactive.
__device__ __forceinline__ bool reb_tile(const DevArrays& a, int nreb, int w, TileCtx& t, SysParams& P) {
  int lo = 0, hi = nreb - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.reb_pref[mid] <= w) lo = mid;
    else hi = mid - 1;
  }
  t.sys = a.rebuild_ids[lo];
  t.r = lo;
  P = a.params[t.sys];
  if (!P.active) return false;
  t.tl = w - a.reb_pref[lo];
  t.local = t.tl * kTile + (threadIdx.x & 31);
  t.s = P.p_off + t.local;
  t.act = t.local < P.n;
  return true;
}

__device__ __forceinline__ int reb_systems(const DevArrays& a) { return a.ctl ? a.ctl->nreb : a.nreb; }

// Rebuild passes visit only the tiles of the rebuilding systems, each warp
// striding over them (a grid sized to the GPU, not to the arena).
template <class F>
__device__ __forceinline__ void for_rebuild_tiles(const DevArrays& a, F&& body) {
  const int nreb = reb_systems(a);
  const int total = a.reb_pref[nreb];
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); w < total; w += nw) {
    TileCtx t;
    SysParams P;
    if (reb_tile(a, nreb, w, t, P)) body(t, P);
  }
}

}  // namespace

// ------------------------------------------------------------ host <-> slots

__global__ void k_from_caller(DevArrays a, int cur, const double* __restrict__ x,
                              const double* __restrict__ v, int sys) {
  const SysParams P = a.params[sys];
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= (int64_t)P.ntiles * kTile) return;
  const int64_t s = P.p_off + l;
  if (l < P.n) {
    a.x[cur][s] = make_double4_32a(wrap_full(x[3 * l + 0], P.L), wrap_full(x[3 * l + 1], P.L),
                               wrap_full(x[3 * l + 2], P.L), 0.0);
    a.v[s] = make_double4_32a(v[3 * l + 0], v[3 * l + 1], v[3 * l + 2], 0.0);
    a.id[s] = (int32_t)l;
  } else {
    a.x[cur][s] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    a.v[s] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    a.id[s] = -1;
    a.ncnt[s] = 0;
  }
}

// which: 0 = positions (wrapped into [0, L)), 1 = velocities, 2 = stored forces,
// 4 = positions as held (not wrapped), 5 = positions at the last list build
__global__ void k_to_caller(DevArrays a, int cur, int which, double* __restrict__ out, int sys) {
  const SysParams P = a.params[sys];
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= P.n) return;
  const int64_t s = P.p_off + l;
  const int64_t i = a.id[s];
  double4_32a q;
  if (which == 0) {
    q = a.x[cur][s];  // positions drift outside [0, L) between list builds
    q.x = wrap_fast(q.x, P.L);
    q.y = wrap_fast(q.y, P.L);
    q.z = wrap_fast(q.z, P.L);
  } else if (which == 1) {
    q = a.v[s];
  } else if (which == 4) {
    q = a.x[cur][s];
  } else if (which == 5) {
    q = a.xref[s];
  } else {
    q = a.f[s];
  }
  out[3 * i + 0] = q.x;
  out[3 * i + 1] = q.y;
  out[3 * i + 2] = q.z;
}

// --------------------------------------------------------- binning (Sec. 2.1)

// Count with one atomic per distinct cell of the warp: between builds a tile's
// particles (in the previous build's cell order) mostly stay in one or two cells.
// Every lane of the warp calls this (c < 0: no particle).
__device__ __forceinline__ int warp_cell_add(int32_t* counts, int c) {
  const unsigned same = __match_any_sync(kFull, c);
  const int leader = __ffs(same) - 1;
  int base = 0;
  if (c >= 0 && (threadIdx.x & 31) == leader) base = atomicAdd(&counts[c], __popc(same));
  base = __shfl_sync(kFull, base, leader);
  return base + __popc(same & ((1u << (threadIdx.x & 31)) - 1u));  // this lane's place in the group
}

__global__ void k_cell_count(DevArrays a, int cur) {
  for_rebuild_tiles(a, [&](const TileCtx& t, const SysParams& P) {
    // Positions are wrapped into [0, L) only here (at a list build): between
    // builds they move freely so that the periodic images stored in the list
    // stay valid.
    int c = -1;
    if (t.act) {
      const double4_32a x = a.x[cur][t.s];
      const double4_32a w = make_double4_32a(wrap_fast(x.x, P.L), wrap_fast(x.y, P.L), wrap_fast(x.z, P.L), 0.0);
      if (w.x != x.x || w.y != x.y || w.z != x.z) a.x[cur][t.s] = w;
      c = 0;
      if (P.nc > 1) {
        c = cell_of(w, P.inv_cs, P.nc);
        if (!check_ok(a, t.sys, c >= 0 && c < P.nc * P.nc * P.nc, kChkCell)) c = 0;
      }
      a.cell[t.s] = c;
    }
    if (P.nc > 1) {  // uniform over the warp
      warp_cell_add(a.ccount + P.c_off, c);
      // the scan's chunk totals (zeroed by the pass's decision), one atomic per chunk of the warp
      const int copy = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) & (kChunkCopies - 1);
      warp_cell_add(a.chunk_sum, c >= 0 ? (a.chunk_pref[t.r] + c / kScanChunk) * kChunkCopies + copy : -1);
    }
  });
}

// Exclusive scan of the cell counts of the rebuilding systems over chunks of
// kScanChunk cells, so that a large system spreads over many blocks: the count
// kernel also totals each chunk (chunk_sum), and k_cell_starts adds the totals of
// the system's earlier chunks to a block scan of its own chunk and writes the
// starts. Work item w is chunk w - chunk_pref[r] of rebuilding system r. The
// counts are reset to serve as fill counters of the scatter.
constexpr int kScanBlock = kScanChunk / 4;

__device__ __forceinline__ int chunk_system(const DevArrays& a, int nreb, int w) {
  int lo = 0, hi = nreb - 1;
  while (lo < hi) {
    const int m = (lo + hi + 1) >> 1;
    if (a.chunk_pref[m] <= w) lo = m;
    else hi = m - 1;
  }
  return lo;
}

// Sum over the block (every thread receives it); ws holds kScanBlock / 32 ints.
__device__ __forceinline__ int block_sum(int v, int* ws) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = __reduce_add_sync(kFull, v);
  if (lane == 0) ws[w] = v;
  __syncthreads();
  int t = lane < kScanBlock / 32 ? ws[lane] : 0;
  t = __reduce_add_sync(kFull, t);
  __syncthreads();  // ws is reused by the caller's next block-wide step
  return t;
}

__global__ void __launch_bounds__(kScanBlock) k_cell_starts(DevArrays a, int nreb) {
  if (a.ctl) nreb = a.ctl->nreb;
  if (nreb <= 0) return;
  __shared__ int ws[kScanBlock / 32];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int total = a.chunk_pref[nreb];
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const int r = chunk_system(a, nreb, w);
    const int sys = a.rebuild_ids[r];
    const SysParams& P = a.params[sys];
    if (!P.active || !a.rebuild[sys]) continue;  // uniform over the block
    const int64_t ncell = (int64_t)P.nc * P.nc * P.nc;
    const int k = w - a.chunk_pref[r];
    // particles in the system's earlier chunks
    int off = 0;
    for (int q = a.chunk_pref[r] * kChunkCopies + (int)threadIdx.x; q < w * kChunkCopies; q += kScanBlock)
      off += a.chunk_sum[q];
    off = block_sum(off, ws);
    int32_t* cnt = a.ccount + P.c_off;
    int32_t* cst = a.cstart + P.c_off;
    const int64_t c0 = (int64_t)k * kScanChunk + 4 * threadIdx.x;
    int v[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) v[m] = c0 + m < ncell ? cnt[c0 + m] : 0;
    const int tsum = v[0] + v[1] + v[2] + v[3];
    // exclusive scan of tsum over the block
    int incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) ws[wi] = incl;
    __syncthreads();
    int wpre = 0, btot = 0;
#pragma unroll
    for (int q = 0; q < kScanBlock / 32; ++q) {
      const int t = ws[q];
      wpre += q < wi ? t : 0;
      btot += t;
    }
    int run = off + wpre + incl - tsum;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      if (c0 + m < ncell) {
        cst[c0 + m] = run;
        cnt[c0 + m] = 0;
      }
      run += v[m];
    }
    if (threadIdx.x == 0) {
      if ((int64_t)(k + 1) * kScanChunk >= ncell) cst[ncell] = off + btot;  // the system's last chunk
      if (k == 0) a.margin[sys] = P.skin;  // velocity-bound rule: a fresh list has the whole skin
    }
    __syncthreads();  // ws is reused by the next chunk
  }
}

// Scatter into cell order (arbitrary within a cell). Beside the old slot, the
// scattered position receives the particle's sort key (x, then caller index) and
// cell, so that the ranking below reads them contiguously (the caller index goes
// to sid, the cell to the cell scratch).

__global__ void k_scatter(DevArrays a, int cur) {
  for_rebuild_tiles(a, [&](const TileCtx& t, const SysParams& P) {
    if (P.nc == 1) {  // uniform over the warp
      if (t.act) a.perm[t.s] = t.local;
      return;
    }
    const int c = t.act ? a.cell[t.s] : -1;
    const int k = warp_cell_add(a.ccount + P.c_off, c);  // fill counter, one atomic per cell of the warp
    if (!t.act) return;
    const int pos = a.cstart[P.c_off + c] + k;
    if (!check_ok(a, t.sys, pos < a.cstart[P.c_off + c + 1], kChkScatter)) return;
    const int64_t d = P.p_off + pos;
    a.perm[d] = t.local;
    // x >= 0 (wrapped at the count), so its bit pattern orders like the value
    a.skey[d] = __double_as_longlong(a.x[cur][t.s].x);
    a.sid[d] = a.id[t.s];
    a.celltmp[d] = c;
  });
}

// Order the particles of each cell by x, ties by caller index (deterministic), and
// gather each into its slot. A row of neighbouring cells along x is then sorted by
// x as a whole, which lets the list build restrict each row to the window
// |x_j - x_i| < rl. One thread per particle: its place in the cell is the number of
// the cell's particles with a smaller key, counted over the scattered members. It
// then writes the particle there: the positions straight to the arrays that only
// the new order uses (the build-time positions and their shadows), the
// velocities, ids and cells to scratch, which the list build copies back slot by
// slot (copy_back_slot). Every slot of a cell holds that cell in the scratch in
// both orders, so the ranking's reads of it need no barrier. The first member of
// each cell resets the cell's fill counter.
__global__ void k_cell_rank(DevArrays a, int cur) {
  for_rebuild_tiles(a, [&](const TileCtx& t, const SysParams& P) {
    if (!t.act) return;
    const int p = t.local;           // position in the scattered order
    const int i = a.perm[t.s];       // the particle's slot before the rebuild
    int dst = p;                     // nc == 1: one cell, the scattered order is kept
    if (P.nc > 1) {
      const long long* key = a.skey + P.p_off;
      const int32_t* idk = a.sid + P.p_off;  // caller indices in the scattered order
      const int c = a.celltmp[t.s];
      const int lo = a.cstart[P.c_off + c], hi = a.cstart[P.c_off + c + 1];
      if (p == lo) a.ccount[P.c_off + c] = 0;  // ready for the next binning
      const long long ki = key[p];
      const int32_t idi = idk[p];
      int rank = 0;
      for (int q = lo; q < hi; ++q) {
        const long long kj = key[q];
        rank += (kj < ki || (kj == ki && idk[q] < idi)) ? 1 : 0;
      }
      if (!check_ok(a, t.sys, lo + rank < hi, kChkRank)) return;
      dst = lo + rank;
    }
    if (!check_ok(a, t.sys, i >= 0 && i < P.n, kChkGather)) return;
    const int64_t old = P.p_off + i, d = P.p_off + dst;
    const double4_32a x = a.x[cur][old];
    a.xref[d] = x;
    int4 q = fixed4(x, P.qscale);
    a.xqref[d] = q;
    q.w = __float_as_int((float)x.x);  // x as float: the list build's window key
    a.xq[cur][d] = q;
    a.xf[d] = make_float4((float)x.x, (float)x.y, (float)x.z, 0.0f);
    a.vtmp[d] = a.v[old];
    a.idtmp[d] = a.id[old];
    a.celltmp[d] = a.cell[old];
  });
}

// The rebuilt state of one slot back into place. The list build does this for the
// tiles it builds: it reads only the build-time positions, shadows and scratch
// cells, which the copy does not touch, so the copy needs no launch of its own.
__device__ __forceinline__ void copy_back_slot(const DevArrays& a, int cur, int64_t s) {
  a.x[cur][s] = a.xref[s];
  a.v[s] = a.vtmp[s];
  a.id[s] = a.idtmp[s];
  a.cell[s] = a.celltmp[s];
}

// ----------------------------------------------- pair list (Sec. 2.1, Fig. 1)

namespace {

// The FP64 membership test, exactly as the reference writes it: separation,
// periodic image, (dx dx + dy dy) + dz dz < rl^2 without fused operations.
// code = 0xff takes the minimum image d - L nearbyint(d / L) of each axis.
// Returns the image code used, with bit 8 set if the pair is inside.
__device__ __forceinline__ unsigned exact_inside(double xi, double yi, double zi, double xj, double yj, double zj,
                                              unsigned code, double L, double rl2) {
  const double d0 = __dsub_rn(xj, xi), d1 = __dsub_rn(yj, yi), d2 = __dsub_rn(zj, zi);
  if (code == 0xffu) {
    code = 0;
    const double k0 = rint(__ddiv_rn(d0, L)), k1 = rint(__ddiv_rn(d1, L)), k2 = rint(__ddiv_rn(d2, L));
    code |= k0 > 0.5 ? 2u : (k0 < -0.5 ? 1u : 0u);
    code |= (k1 > 0.5 ? 2u : (k1 < -0.5 ? 1u : 0u)) << 2;
    code |= (k2 > 0.5 ? 2u : (k2 < -0.5 ? 1u : 0u)) << 4;
  }
  const double dx = apply_image(d0, code & 3u, L);
  const double dy = apply_image(d1, (code >> 2) & 3u, L);
  const double dz = apply_image(d2, (code >> 4) & 3u, L);
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  return code | (r2 < rl2 ? 0x100u : 0u);  // bit 8: inside
}

// Per-particle state of the list build. The FP64 position and the system's L and
// rl^2 are not kept in registers: the rare exact tests reload them.
struct ListCtx {
  const SysParams* Pp;
  const double4_32a* xs;  // FP64 positions of the system (build-time copy)
  uint32_t* out;          // the particle's list words
  int li;                 // the particle's slot in the system
  int count;
  int kmax;
  bool half;              // half list: only partners in higher slots
  int32_t* chk;           // the system's check word (checked build)
  uint32_t* wp = out;     // where entry `count` goes (entries 4 m .. 4 m + 3 are 16
                          // contiguous bytes; the next four follow 4 kTile words on)
  // The checked build verifies each appended partner: a slot of the system, not
  // the particle itself.
  __device__ __forceinline__ bool entry_ok(uint32_t e) const {
    if (!kChecks) return true;
    const uint32_t j = e & kIdxMask;
    if (j < (uint32_t)Pp->n && j != (uint32_t)li) return true;
    atomicOr(chk, kChkListEntry);
    return false;
  }
  __device__ __forceinline__ void advance() {
    ++count;
    wp += (count & 3) ? 1 : 4 * kTile - 3;
  }
  // Append e when p holds (a predicated store).
  __device__ __forceinline__ void push_if(bool p, uint32_t e) {
    if (!p) return;
    push(e);
  }
  __device__ __forceinline__ void push(uint32_t e) {
    if (!entry_ok(e)) return;
    if (count < kmax) *wp = e;
    advance();
  }
  // Entries up to the next multiple of four hold the particle itself, so that the
  // FP32 step reads whole groups of four without a bound per entry (the pair with
  // itself has r = 0, which its force loop leaves out).
  __device__ __forceinline__ void pad() {
    uint32_t* w = wp;
    for (int c = count; (c & 3) != 0 && c < kmax; ++c) *w++ = (uint32_t)li;
  }
  // Append candidates j0 + k (image bits cbits) for the set bits k of `bits`, in
  // ascending k; the capacity is checked once for all of them.
  __device__ __forceinline__ void push_bits(unsigned bits, int j0, uint32_t cbits) {
    if (count + __popc(bits) <= kmax) {
      while (bits) {
        const int k = __ffs(bits) - 1;
        bits &= bits - 1u;
        const uint32_t e = (uint32_t)(j0 + k) | cbits;
        if (!entry_ok(e)) continue;
        *wp = e;
        advance();
      }
    } else {
      while (bits) {
        const int k = __ffs(bits) - 1;
        bits &= bits - 1u;
        push((uint32_t)(j0 + k) | cbits);
      }
    }
  }
  // Whether candidate j with image code (not 0xff) passes the exact FP64 test.
  __device__ __forceinline__ bool exact_in(int j, unsigned code) const {
    const double4_32a xi = xs[li], xj = xs[j];
    return (exact_inside(xi.x, xi.y, xi.z, xj.x, xj.y, xj.z, code, Pp->L, Pp->rl2) >> 8) & 1u;
  }
  // The exact FP64 test of candidate j with image code (0xff: minimum image).
  __device__ __forceinline__ void exact(int j, unsigned code) {
    const double4_32a xi = xs[li], xj = xs[j];
    const unsigned r = exact_inside(xi.x, xi.y, xi.z, xj.x, xj.y, xj.z, code, Pp->L, Pp->rl2);
    push_if((r >> 8) & 1u, (uint32_t)j | ((r & 0xffu) << kIdxBits));
  }
};

// Candidate pre-tests: squared distance of candidate j (in this range's image)
// from the particle, in float, with sure-inside / sure-outside thresholds.
//   PRE 0: positions rounded to float, key shifted by the range's image;
//          thresholds rl^2 (1 -/+ eps(L / rl)).
//   PRE 1: fixed-point shadow positions (the wrapped 32-bit difference is the
//          minimum image) converted to float; thresholds rl^2 (1 -/+ 1e-5) in
//          fixed-point units (relative error of r^2 below 3.2e-6 for L <= 10^4).
template <int PRE>
struct PreTest;

template <>
struct PreTest<0> {
  const float4* p;
  float cx, cy, cz;  // the particle's position minus the image shift
  float lo2, hi2;
  __device__ __forceinline__ float key(int j) const { return p[j].x; }
  __device__ __forceinline__ float r2(const float4& q) const {
    const float dx = q.x - cx, dy = q.y - cy, dz = q.z - cz;
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  }
  __device__ __forceinline__ float4 load(int j) const { return p[j]; }
};

template <>
struct PreTest<1> {
  const int4* p;
  int qx, qy, qz;
  float lo2, hi2;
  __device__ __forceinline__ float key(int j) const { return __int_as_float(p[j].w); }
  __device__ __forceinline__ float r2(const int4& q) const {
    const float ax = (float)wrapped_diff(q.x, qx);
    const float ay = (float)wrapped_diff(q.y, qy);
    const float az = (float)wrapped_diff(q.z, qz);
    return fmaf(az, az, fmaf(ay, ay, ax * ax));
  }
  __device__ __forceinline__ int4 load(int j) const { return p[j]; }
};

// PRE 0 reading a row's candidates staged in shared memory: slot j sits at
// s[j - base].
struct PreTestS {
  const float4* s;
  int base;
  float cx, cy, cz;
  float lo2, hi2;
  __device__ __forceinline__ float key(int j) const { return s[j - base].x; }
  __device__ __forceinline__ float r2(const float4& q) const {
    const float dx = q.x - cx, dy = q.y - cy, dz = q.z - cz;
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  }
  __device__ __forceinline__ float4 load(int j) const { return s[j - base]; }
};

__device__ __forceinline__ float key_of(const float4& q) { return q.x; }
__device__ __forceinline__ float key_of(const int4& q) { return __int_as_float(q.w); }

// Test the candidates of slot range [lo, hi), all with image `code`, against the
// particle and append the partners in candidate order. The range is ordered by x
// (float key) and only the window xlo <= x_j < xhi can hold partners: the first
// candidate is found by bisection and the sweep stops past xhi. Candidates are
// taken in windows of 32 (eight groups of four independent loads; the slot
// arrays have four spare entries at the end): the pre-test sets a bit per
// candidate that is surely inside and per candidate that may be inside; the
// range end, the particle itself and (half list) the lower slots are masked once
// per window, the rare shell candidates take the exact test, and the accepted
// ones are appended in order.
template <class T_>
__device__ __forceinline__ void sweep_range(const T_& T, ListCtx& o, int lo, int hi, unsigned code,
                                            float xlo, float xhi) {
  int b = hi;
  while (lo < b) {
    const int m = (lo + b) >> 1;
    if (T.key(m) < xlo) lo = m + 1;
    else b = m;
  }
  const uint32_t cbits = code << kIdxBits;
  int j = lo;
  bool more = j < hi;
  while (more) {
    const int j0 = j;
    unsigned in = 0u, may = 0u;
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      if (more) {
        const auto q0 = T.load(j), q1 = T.load(j + 1), q2 = T.load(j + 2), q3 = T.load(j + 3);
        if (!(key_of(q0) < xhi)) {
          more = false;
        } else {
          const float r0 = T.r2(q0), r1 = T.r2(q1), r2 = T.r2(q2), r3 = T.r2(q3);
          if (r0 < T.hi2) may |= 1u << (4 * g);
          if (r1 < T.hi2) may |= 2u << (4 * g);
          if (r2 < T.hi2) may |= 4u << (4 * g);
          if (r3 < T.hi2) may |= 8u << (4 * g);
          if (r0 < T.lo2) in |= 1u << (4 * g);
          if (r1 < T.lo2) in |= 2u << (4 * g);
          if (r2 < T.lo2) in |= 4u << (4 * g);
          if (r3 < T.lo2) in |= 8u << (4 * g);
          j += 4;
          more = j < hi;
        }
      }
    }
    const int nt = min(j, hi) - j0;  // candidates tested in this window
    unsigned valid = nt >= 32 ? ~0u : ((1u << nt) - 1u);
    if ((unsigned)(o.li - j0) < 32u) valid &= ~(1u << (o.li - j0));  // not the particle itself
    if (o.half) {  // half list: keep candidates above the particle's slot
      const int d = o.li - j0;
      if (d >= 31) valid = 0u;
      else if (d >= 0) valid &= ~((2u << d) - 1u);
    }
    may &= valid;
    in &= may;
    unsigned shell = may & ~in;
    while (shell) {  // between the pre-test's thresholds: the exact FP64 test
      const int k = __ffs(shell) - 1;
      shell &= shell - 1u;
      if (o.exact_in(j0 + k, code)) in |= 1u << k;
    }
    o.push_bits(in, j0, cbits);
  }
}

// nc == 1: every particle is a candidate. The fixed-point separation (its wrapped
// difference is the minimum image) rules out the far ones; the rest take the exact
// minimum-image test.
__device__ __forceinline__ void sweep_all(ListCtx& o, const int4* __restrict__ q, float hi2, int n) {
  const int4 qi = q[o.li];
  for (int j = 0; j < n; ++j) {
    const int4 qj = q[j];
    const float ax = (float)wrapped_diff(qj.x, qi.x);
    const float ay = (float)wrapped_diff(qj.y, qi.y);
    const float az = (float)wrapped_diff(qj.z, qi.z);
    if (j != o.li && (!o.half || j > o.li) && fmaf(az, az, fmaf(ay, ay, ax * ax)) < hi2) o.exact(j, 0xffu);
  }
}

}  // namespace

// Full list: every j != i with minimum-image r^2 < rl^2 (strict); one thread per
// particle, candidates from the 27 neighbour cells taken as 9 rows of 3 cells that
// are contiguous in cell order (split in two where a row wraps in x), or from all
// particles when nc == 1. Partners are appended in candidate order
// (deterministic, and the same for every PRE).
//
// The decision is the FP64 test ((dx dx + dy dy) + dz dz < rl^2, no fused
// operations). It is taken first by a float pre-test whose error is bounded: below
// its lower threshold the pair is certainly inside, above the upper one certainly
// outside, and only the thin shell between needs the FP64 test. The result is
// identical to always taking it.
// VAR bit 0: the fixed-point pre-test (else float); bit 1: rows farther than rl
// in y or z are skipped and the x window of each row is narrowed to
// sqrt(rl^2 - dy^2 - dz^2) (dy, dz: distances from the particle to the row).
namespace {

// The 9 neighbour rows of one particle (cells other than nc == 1), swept by
// its own thread.
template <int PRE, bool kPrune>
__device__ __forceinline__ void lane_rows(const DevArrays& a, int cur, const SysParams* __restrict__ Pp, ListCtx& o,
                                          int64_t p_off) {
  const int li = o.li, nc = Pp->nc;
  const double4_32a xi0 = o.xs[li];
  const float rl = Pp->rlf, wm = Pp->wmargin;
  float w = rl + wm;  // half-width of the x window
  PreTest<PRE> T;
  if constexpr (PRE == 0) {
    T.p = a.xf + p_off;
    T.lo2 = Pp->rl2f_lo;
    T.hi2 = Pp->rl2f_hi;
  } else {
    T.p = a.xq[cur] + p_off;
    const int4 qi = T.p[li];
    T.qx = qi.x; T.qy = qi.y; T.qz = qi.z;
    T.lo2 = Pp->rl2q_lo;
    T.hi2 = Pp->rl2q_hi;
  }
  const int32_t* cst = a.cstart + Pp->c_off;
  const int ci = a.celltmp[p_off + li];
  const int cx = ci % nc, cy = (ci / nc) % nc, cz = ci / (nc * nc);
  const int nparts = (cx == 0 || cx == nc - 1) ? 2 : 1;
  const double L = Pp->L;
  // offsets of the particle from its cell's lower y and z faces (row pruning)
  const float cs = Pp->csf;
  const float fy = kPrune ? (float)xi0.y - (float)cy * cs : 0.f;
  const float fz = kPrune ? (float)xi0.z - (float)cz * cs : 0.f;
#pragma unroll 1
  for (int rowi = 0; rowi < 9; ++rowi) {
    const int oz = rowi / 3 - 1, oy = rowi % 3 - 1;
    if (kPrune) {
      // the margin (1e-5 L) is far above the float rounding of x_i and of the
      // cell faces (about 1e-7 L)
      const float dy = fmaxf(0.f, (oy < 0 ? fy : (oy > 0 ? cs - fy : 0.f)) - wm);
      const float dz = fmaxf(0.f, (oz < 0 ? fz : (oz > 0 ? cs - fz : 0.f)) - wm);
      const float rem = rl * rl - dy * dy - dz * dz;
      if (rem <= 0.f) continue;  // the whole row is farther than rl
      w = sqrtf(rem) + wm;
    }
    int nz = cz + oz, ny = cy + oy;
    unsigned shz = 0, shy = 0;
    if (nz < 0) { nz += nc; shz = 2; } else if (nz >= nc) { nz -= nc; shz = 1; }
    if (ny < 0) { ny += nc; shy = 2; } else if (ny >= nc) { ny -= nc; shy = 1; }
    const int row = nc * (ny + nc * nz);
    const double4_32a xi = o.xs[li];  // reloaded (an L1 hit) rather than held in registers
    if constexpr (PRE == 0) {
      // image code 1 adds +L to x_j - x_i, code 2 adds -L: shift the particle instead
      T.cy = (float)(shy == 1 ? xi.y - L : (shy == 2 ? xi.y + L : xi.y));
      T.cz = (float)(shz == 1 ? xi.z - L : (shz == 2 ? xi.z + L : xi.z));
    }
#pragma unroll 1
    for (int part = 0; part < nparts; ++part) {
      int lo, hi;
      unsigned code = (shy << 2) | (shz << 4);
      // cells cx-1..cx+1 of this row: one contiguous range, or two where it wraps
      if (cx == 0) {
        if (part == 0) { lo = cst[row + nc - 1]; hi = cst[row + nc]; code |= 2u; }  // x image -L
        else { lo = cst[row]; hi = cst[row + 2]; }
      } else if (cx == nc - 1) {
        if (part == 0) { lo = cst[row + nc - 2]; hi = cst[row + nc]; }
        else { lo = cst[row]; hi = cst[row + 1]; code |= 1u; }                    // x image +L
      } else {
        lo = cst[row + cx - 1]; hi = cst[row + cx + 2];
      }
      // the particle's x in this range's coordinates (candidates are not shifted)
      const double xs_ = (code & 3u) == 1u ? xi.x - L : ((code & 3u) == 2u ? xi.x + L : xi.x);
      const float xw = (float)xs_;
      if constexpr (PRE == 0) T.cx = xw;
      sweep_range(T, o, lo, hi, code, xw - w, xw + w);
    }
  }
}

// List length, the system's largest length and overflow (one atomic per warp:
// all threads of a system hitting one word serialise).
__device__ __forceinline__ void list_done(const DevArrays& a, int sys, int64_t slot, int count, int kmax,
                                          bool act, unsigned mask, int lane) {
  if (act) a.ncnt[slot] = count < kmax ? count : kmax;
  const int wmax = __reduce_max_sync(mask, act ? count : 0);
  if (lane == __ffs(mask) - 1) {
    atomicMax(&a.status[sys].max_count, wmax);
    if (wmax > kmax) {
      atomicMax(&a.status[sys].overflow, wmax);
      if (a.ctl) atomicMax(&a.ctl->abort, 1);  // graph-captured loop: stop; the host grows the list
    }
  }
}

}  // namespace

namespace {

// Next tile of the rebuilding systems for this warp, from a shared work counter
// (dynamic: tiles differ in cost); false when none is left. Warp-uniform.
__device__ __forceinline__ bool next_rebuild_tile(const DevArrays& a, int& sys, int& tl) {
  const int nreb = reb_systems(a);
  const int total = a.reb_pref[nreb];
  int w = 0;
  if ((threadIdx.x & 31) == 0) w = atomicAdd(a.tile_next, 1);
  w = __shfl_sync(kFull, w, 0);
  if (w >= total) return false;
  int lo = 0, hi = nreb - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.reb_pref[mid] <= w) lo = mid;
    else hi = mid - 1;
  }
  sys = a.rebuild_ids[lo];
  tl = w - a.reb_pref[lo];
  return true;
}

}  // namespace

template <int BLOCK, int VAR>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) k_build_list(DevArrays a, int cur) {
  constexpr int PRE = VAR & 1;
  constexpr bool kPrune = (VAR & 2) != 0;
  const int lane = threadIdx.x & 31;
  int sys, tl;
  while (next_rebuild_tile(a, sys, tl)) {
    const SysParams* __restrict__ Pp = a.params + sys;
    if (!Pp->active) continue;
    const int li = tl * kTile + lane;
    const int n = Pp->n;
    const bool act = li < n;
    const int64_t p_off = Pp->p_off;
    const int kmax = Pp->kmax;
    ListCtx o{Pp, a.xref + p_off, a.nbr + list_word(Pp->l_off, tl, kmax, lane, 0), li, 0, kmax, Pp->half != 0,
              a.checks + sys};
    if (act) copy_back_slot(a, cur, p_off + li);
    if (act) {
      if (Pp->nc == 1) sweep_all(o, a.xq[cur] + p_off, Pp->rl2q_hi, n);
      else lane_rows<PRE, kPrune>(a, cur, Pp, o, p_off);
    }
    if (act) o.pad();
    list_done(a, sys, p_off + li, o.count, kmax, act, kFull, lane);
  }
}

// Warp-cooperative list build: the same lists, in the same order, as
// k_build_list. The lanes of a warp that share a row of cells (y, z) take the
// union of their candidates: for each of the 9 neighbour rows, the cells
// cx_min-1 .. cx_max+1 restricted to the group's x window, read 32 at a time with
// coalesced loads into shared memory and tested by every lane from there
// (broadcast reads). Each lane collects its accepted candidates of a chunk in a
// bit mask (pre-test; the shell resolved by the exact FP64 test) and appends them
// in candidate order. Candidates outside a lane's own three cells are farther
// than the cell side >= rl, so they fail its test; every cell of the union
// appears once, with one image, because a group spans at most nc - 2 cells
// (wider runs of a row are split into several groups). Full lists only.
namespace {

__device__ __forceinline__ void build_tile_warp(const DevArrays& a, int cur, int sys, int tl, float4* buf) {
  const int lane = threadIdx.x & 31;
  const SysParams* __restrict__ Pp = a.params + sys;
  if (!Pp->active) return;  // every return above the loop is uniform over the warp
  const int li = tl * kTile + lane;
  const int n = Pp->n;
  const bool act = li < n;
  const unsigned actm = __ballot_sync(kFull, act);
  const int64_t p_off = Pp->p_off;
  const int kmax = Pp->kmax;
  ListCtx o{Pp, a.xref + p_off, a.nbr + list_word(Pp->l_off, tl, kmax, lane, 0), li, 0, kmax, false, a.checks + sys};
  if (act) copy_back_slot(a, cur, p_off + li);
  const int nc = Pp->nc;
  if (nc == 1) {
    if (act) sweep_all(o, a.xq[cur] + p_off, Pp->rl2q_hi, n);
    if (act) o.pad();
    list_done(a, sys, p_off + li, o.count, kmax, act, kFull, lane);
    return;
  }
  const float4* __restrict__ xf = a.xf + p_off;
  const int32_t* __restrict__ cst = a.cstart + Pp->c_off;
  const double L = Pp->L;
  const float w = Pp->rlf + Pp->wmargin;  // half-width of the x window around each particle
  const float lo2 = Pp->rl2f_lo, hi2 = Pp->rl2f_hi;
  int cx = 0, rkey = -1;
  float xk = 0.f;
  if (act) {
    const int ci = a.celltmp[p_off + li];
    cx = ci % nc;
    rkey = ci / nc;  // row of cells (y, z)
    xk = xf[li].x;
  }
  unsigned todo = actm;
  while (todo) {
    // next group: the remaining lanes of one row whose cells span at most nc - 2
    // (so that the union of their neighbour cells holds each cell once)
    const int gkey = __shfl_sync(kFull, rkey, __ffs(todo) - 1);
    const bool same = ((todo >> lane) & 1u) && rkey == gkey;
    const int cxa = __reduce_min_sync(kFull, same ? cx : 0x7fffffff);
    const unsigned grp = __ballot_sync(kFull, same && cx <= cxa + nc - 3);
    todo &= ~grp;
    const bool mine = (grp >> lane) & 1u;
    const int cxb = __reduce_max_sync(kFull, mine ? cx : -1);
    // x extent of the group: x >= 0, so the float bits order like the values
    const float xmin = __int_as_float(__reduce_min_sync(kFull, mine ? __float_as_int(xk) : 0x7f800000));
    const float xmax = __int_as_float(__reduce_max_sync(kFull, mine ? __float_as_int(xk) : 0));
    const int gcy = gkey % nc, gcz = gkey / nc;
    const int npieces = (cxa == 0 || cxb == nc - 1) ? 2 : 1;
#pragma unroll 1
    for (int rowi = 0; rowi < 9; ++rowi) {
      const int oz = rowi / 3 - 1, oy = rowi % 3 - 1;
      int nz = gcz + oz, ny = gcy + oy;
      unsigned shz = 0, shy = 0;
      if (nz < 0) { nz += nc; shz = 2; } else if (nz >= nc) { nz -= nc; shz = 1; }
      if (ny < 0) { ny += nc; shy = 2; } else if (ny >= nc) { ny -= nc; shy = 1; }
      const int row = nc * (ny + nc * nz);
      const double4_32a xi = o.xs[li];  // padding lanes read their zeroed slot
      // image code 1 adds +L to x_j - x_i, code 2 adds -L: shift the particle instead
      const float cy = (float)(shy == 1 ? xi.y - L : (shy == 2 ? xi.y + L : xi.y));
      const float cz = (float)(shz == 1 ? xi.z - L : (shz == 2 ? xi.z + L : xi.z));
#pragma unroll 1
      for (int piece = 0; piece < npieces; ++piece) {
        int c0, c1;  // first and last cell of this piece (contiguous in cell order)
        unsigned code = (shy << 2) | (shz << 4);
        if (cxa == 0) {
          if (piece == 0) { c0 = c1 = nc - 1; code |= 2u; }  // x image -L
          else { c0 = 0; c1 = cxb + 1; }
        } else if (cxb == nc - 1) {
          if (piece == 0) { c0 = cxa - 1; c1 = nc - 1; }
          else { c0 = c1 = 0; code |= 1u; }                  // x image +L
        } else {
          c0 = cxa - 1; c1 = cxb + 1;
        }
        int lo = cst[row + c0];
        const int hi = cst[row + c1 + 1];
        const float sx = (code & 3u) == 1u ? -(float)L : ((code & 3u) == 2u ? (float)L : 0.f);
        const float xlo = xmin + sx - w, xhi = xmax + sx + w;
        const float cxf = (float)((code & 3u) == 1u ? xi.x - L : ((code & 3u) == 2u ? xi.x + L : xi.x));
        // first candidate of the window (every lane takes the same steps)
        int b = hi;
        while (lo < b) {
          const int m = (lo + b) >> 1;
          if (xf[m].x < xlo) lo = m + 1;
          else b = m;
        }
        const uint32_t cbits = code << kIdxBits;
        for (int j0 = lo; j0 < hi; j0 += 32) {
          const int j = j0 + lane;
          const float4 q = j < hi ? xf[j] : make_float4(0.f, 0.f, 0.f, 0.f);
          const unsigned vm = __ballot_sync(kFull, j < hi && q.x < xhi);  // a prefix: keys ascend
          if (vm == 0) break;
          buf[lane] = q;
          __syncwarp();
          if (mine) {
            unsigned M = 0, C = 0;  // maybe inside (below hi2), certainly inside (below lo2)
#pragma unroll
            for (int t = 0; t < 32; ++t) {
              const float4 c = buf[t];
              const float dx = c.x - cxf, dy = c.y - cy, dz = c.z - cz;
              const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
              M |= r2 < hi2 ? 1u << t : 0u;
              C |= r2 < lo2 ? 1u << t : 0u;
            }
            M &= vm;
            if ((unsigned)(li - j0) < 32u) M &= ~(1u << (li - j0));  // not the particle itself
            C &= M;
            unsigned S = M & ~C;  // in the shell: the exact test decides (rare)
            while (S) {
              const int t = __ffs(S) - 1;
              S &= S - 1;
              const double4_32a xa = o.xs[li], xj = o.xs[j0 + t];
              if (exact_inside(xa.x, xa.y, xa.z, xj.x, xj.y, xj.z, code, L, Pp->rl2) & 0x100u) C |= 1u << t;
            }
            while (C) {
              const int t = __ffs(C) - 1;
              C &= C - 1;
              o.push_if(true, (uint32_t)(j0 + t) | cbits);
            }
          }
          __syncwarp();
          if (vm != kFull) break;
        }
      }
    }
  }
  if (act) o.pad();
    list_done(a, sys, p_off + li, o.count, kmax, act, kFull, lane);
}

}  // namespace

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) k_build_list_warp(DevArrays a, int cur) {
  __shared__ float4 sbuf[BLOCK];
  float4* buf = sbuf + (threadIdx.x & ~31);
  int sys, tl;
  while (next_rebuild_tile(a, sys, tl)) build_tile_warp(a, cur, sys, tl, buf);
}

// List build with rows staged in shared memory: the same lists, in the same
// order, as k_build_list (the same per-thread sweep, pre-test and exact test).
// For each neighbour row (and piece of a row that wraps in x) the warp first
// copies the union of its lanes' candidate ranges into shared memory with
// coalesced loads (up to kStage candidates; a wider union, as where a tile's
// lanes sit on both sides of a box face, is swept from global memory). Each lane
// then bisects for its window and sweeps it from there: the candidate loads of
// the sweep, which in k_build_list wait on L1 and often L2 latency, become
// shared-memory loads. Rows and pieces are visited by the whole warp (a lane
// without a second piece has an empty range).
namespace {

constexpr int kStage = 160;  // staged candidates per warp and row piece

__device__ __forceinline__ void build_tile_staged(const DevArrays& a, int cur, int sys, int tl, float4* buf) {
  const int lane = threadIdx.x & 31;
  const SysParams* __restrict__ Pp = a.params + sys;
  if (!Pp->active) return;  // uniform over the warp
  const int li = tl * kTile + lane;
  const int n = Pp->n;
  const bool act = li < n;
  const int64_t p_off = Pp->p_off;
  const int kmax = Pp->kmax;
  ListCtx o{Pp, a.xref + p_off, a.nbr + list_word(Pp->l_off, tl, kmax, lane, 0), li, 0, kmax, Pp->half != 0,
            a.checks + sys};
  if (act) copy_back_slot(a, cur, p_off + li);
  const int nc = Pp->nc;
  if (nc == 1) {  // uniform over the warp
    if (act) sweep_all(o, a.xq[cur] + p_off, Pp->rl2q_hi, n);
    if (act) o.pad();
    list_done(a, sys, p_off + li, o.count, kmax, act, kFull, lane);
    return;
  }
  const float4* __restrict__ xf = a.xf + p_off;
  const int32_t* __restrict__ cst = a.cstart + Pp->c_off;
  const float w = Pp->rlf + Pp->wmargin;  // half-width of the x window
  PreTest<0> T;
  T.p = xf;
  T.lo2 = Pp->rl2f_lo;
  T.hi2 = Pp->rl2f_hi;
  PreTestS S;
  S.s = buf;
  S.lo2 = T.lo2;
  S.hi2 = T.hi2;
  int cx = 1, cy = 0, cz = 0;
  if (act) {
    const int ci = a.celltmp[p_off + li];
    cx = ci % nc; cy = (ci / nc) % nc; cz = ci / (nc * nc);
  }
  const float Lf = Pp->Lf;
#pragma unroll 1
  for (int rowi = 0; rowi < 9; ++rowi) {
    const int oz = rowi / 3 - 1, oy = rowi % 3 - 1;
    int nz = cz + oz, ny = cy + oy;
    unsigned shz = 0, shy = 0;
    if (nz < 0) { nz += nc; shz = 2; } else if (nz >= nc) { nz -= nc; shz = 1; }
    if (ny < 0) { ny += nc; shy = 2; } else if (ny >= nc) { ny -= nc; shy = 1; }
    const int row = nc * (ny + nc * nz);
    // the particle's float position (reloaded, an L1 hit; padding lanes read their
    // zeroed slot), shifted in float: image code 1 adds +L to x_j - x_i, code 2
    // adds -L, so shift the particle instead (the pre-test's error bound allows
    // for these roundings)
    const float4 fi = xf[li];
    T.cy = shy == 1 ? fi.y - Lf : (shy == 2 ? fi.y + Lf : fi.y);
    T.cz = shz == 1 ? fi.z - Lf : (shz == 2 ? fi.z + Lf : fi.z);
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {
      int lo = 0, hi = 0;
      unsigned code = (shy << 2) | (shz << 4);
      if (act) {
        if (cx == 0) {
          if (part == 0) { lo = cst[row + nc - 1]; hi = cst[row + nc]; code |= 2u; }  // x image -L
          else { lo = cst[row]; hi = cst[row + 2]; }
        } else if (cx == nc - 1) {
          if (part == 0) { lo = cst[row + nc - 2]; hi = cst[row + nc]; }
          else { lo = cst[row]; hi = cst[row + 1]; code |= 1u; }                    // x image +L
        } else if (part == 0) {
          lo = cst[row + cx - 1]; hi = cst[row + cx + 2];
        }
      }
      const bool ne = lo < hi;
      if (!__any_sync(kFull, ne)) continue;  // uniform
      const float xw = (code & 3u) == 1u ? fi.x - Lf : ((code & 3u) == 2u ? fi.x + Lf : fi.x);
      const int u0 = __reduce_min_sync(kFull, ne ? lo : 0x7fffffff);
      const int u1 = __reduce_max_sync(kFull, ne ? hi : -1);
      if (u1 - u0 <= kStage) {
        // stage [u0, u1) and the 3 slots after it (a group of four may read past
        // its range end; the slot arrays have four spare entries)
        for (int k = lane; k < u1 - u0 + 3; k += 32) buf[k] = xf[u0 + k];
        __syncwarp();
        S.base = u0;
        S.cx = xw;
        S.cy = T.cy;
        S.cz = T.cz;
        sweep_range(S, o, lo, hi, code, xw - w, xw + w);
        __syncwarp();  // before the next piece overwrites the buffer
      } else {
        T.cx = xw;
        sweep_range(T, o, lo, hi, code, xw - w, xw + w);
      }
    }
  }
  if (act) o.pad();
    list_done(a, sys, p_off + li, o.count, kmax, act, kFull, lane);
}

}  // namespace

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) k_build_list_staged(DevArrays a, int cur) {
  __shared__ float4 sbuf[BLOCK / 32][kStage + 4];
  int sys, tl;
  while (next_rebuild_tile(a, sys, tl)) build_tile_staged(a, cur, sys, tl, sbuf[threadIdx.x >> 5]);
}

// ------------------------------------- fused force + velocity-Verlet step

namespace {

// Velocity-Verlet update of one particle after its force F is known:
//   v += dt/2 F (flag kStepKickA: completes the previous step), v += dt/2 F (flag
//   kStepKickB: first half-kick of the next step; kept as two roundings so that a
//   run split over several calls equals one uninterrupted call bit for bit), then
//   optionally the drift
//   x' = x + dt v into x[cur ^ 1] (not wrapped: list images stay valid) and the
//   squared displacement since the list build for the validity check.
template <bool kFP32>
__device__ __forceinline__ unsigned long long integrate(const DevArrays& a, const SysParams& P, const TileCtx& t,
                                                        int cur, const double4_32a& xi, double Fx, double Fy,
                                                        double Fz, double ka, double kb, int flags) {
  if (flags & kStepStoreF) a.f[t.s] = make_double4_32a(Fx, Fy, Fz, 0.0);
  double4_32a v = a.v[t.s];
  const double dt = P.dt;
  const double h = P.hdt;
  if (flags & kStepKickA) { v.x = fma(h, Fx, v.x); v.y = fma(h, Fy, v.y); v.z = fma(h, Fz, v.z); }
  if (flags & kStepKickB) { v.x = fma(h, Fx, v.x); v.y = fma(h, Fy, v.y); v.z = fma(h, Fz, v.z); }
  a.v[t.s] = v;
  if (!(flags & kStepDrift)) return 0ull;
  double4_32a xn;
  xn.x = fma(dt, v.x, xi.x);
  xn.y = fma(dt, v.y, xi.y);
  xn.z = fma(dt, v.z, xi.z);
  xn.w = 0.0;
  a.x[cur ^ 1][t.s] = xn;
  if (!(finite_bits(xn.x) && finite_bits(xn.y) && finite_bits(xn.z) && finite_bits(v.x) &&
        finite_bits(v.y) && finite_bits(v.z))) {
    a.status[t.sys].nonfinite = 1;
    return ~0ull;
  }
  // velocity-bound rule: |v|^2 of the drift velocity, (vx vx + vy vy) + vz vz unfused
  // (FP64 work only under that rule)
  auto v2b = [&v]() -> unsigned long long {
    return (unsigned long long)__double_as_longlong(
        __dadd_rn(__dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y)), __dmul_rn(v.z, v.z)));
  };
  if (kFP32) {
    // check in fixed point: exact integer squared displacement of the shadow
    const int4 q = fixed4(xn, P.qscale);
    a.xq[cur ^ 1][t.s] = q;
    if (flags & kStepVmax) return v2b();
    const int4 r = a.xqref[t.s];
    const long long ex = wrapped_diff(q.x, r.x), ey = wrapped_diff(q.y, r.y), ez = wrapped_diff(q.z, r.z);
    return (unsigned long long)(ex * ex) + (unsigned long long)(ey * ey) + (unsigned long long)(ez * ez);
  }
  // the fixed-point shadow, which the FP64 force loop's pre-classification reads
  a.xq[cur ^ 1][t.s] = fixed4(xn, P.qscale);
  if (flags & kStepVmax) return v2b();
  // exact FP64 check, the same operations as the reference
  const double4_32a r = a.xref[t.s];
  const double ex = __dsub_rn(xn.x, r.x), ey = __dsub_rn(xn.y, r.y), ez = __dsub_rn(xn.z, r.z);
  const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
  return (unsigned long long)__double_as_longlong(d2);
}

__device__ __forceinline__ void warp_max_disp(const DevArrays& a, int sys, unsigned long long d2b, int flags) {
  if (!(flags & kStepDrift)) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(kFull, d2b, o);
    d2b = y > d2b ? y : d2b;
  }
  if ((threadIdx.x & 31) == 0 && d2b) atomicMax(&a.disp2[sys], d2b);
}

// FP32 pair force from an exact fixed-point separation; returns 0 for invalid
// slots, for r >= rc and for r = 0 (a list's padding entries name the particle
// itself) without branching (g (24 r^-8 - 48 r^-14 + 8 c2)).
__device__ __forceinline__ void pair_fp32(const int4& qi, const int4& qj, bool valid, float qu, float rc2,
                                          float c2x8, float& fx, float& fy, float& fz) {
  const float dx = (float)wrapped_diff(qj.x, qi.x) * qu;
  const float dy = (float)wrapped_diff(qj.y, qi.y) * qu;
  const float dz = (float)wrapped_diff(qj.z, qi.z) * qu;
  const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  const bool in = valid && r2 < rc2 && r2 > 0.0f;
  const float r2s = in ? r2 : 1.0f;
  float ir2;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ir2) : "f"(r2s));
  ir2 = ir2 * fmaf(-r2s, ir2, 2.0f);  // one Newton step
  const float ir6 = ir2 * ir2 * ir2;
  float g = fmaf(ir2 * ir6, fmaf(-48.0f, ir6, 24.0f), c2x8);
  g = in ? g : 0.0f;
  fx = fmaf(g, dx, fx);
  fy = fmaf(g, dy, fy);
  fz = fmaf(g, dz, fz);
}

}  // namespace

// Loads with L1 eviction hints: list words are read once (no L1 allocation), the
// partners' shadow positions are reused by neighbouring threads (kept in L1).
__device__ __forceinline__ uint4 ld_list(const uint4* p, bool hint) {
  if (!hint) return __ldg(p);
  uint4 r;
  asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
  return r;
}

__device__ __forceinline__ int4 ld_shadow(const int4* p, bool hint) {
  if (!hint) return *p;
  int4 r;
  asm("ld.global.nc.L1::evict_last.v4.s32 {%0, %1, %2, %3}, [%4];"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
  return r;
}

// FP32-force form: pair arithmetic in FP32 from fixed-point separations (the
// wrapped integer difference is already the minimum image). Each iteration
// takes GROUPS x 4 partners (GROUPS 16-byte list loads, then 4 GROUPS gathers in
// flight at once) and the next iteration's list loads are issued before this
// iteration's gathers are used (software pipelining, the role of Algorithm 1's
// unrolling). BLOCK and GROUPS are chosen by the autotuner.
template <int BLOCK, int GROUPS, bool HINT>
__global__ void __launch_bounds__(BLOCK) k_step_fp32(DevArrays a, int cur, double ka, double kb, int flags) {
  if (a.ctl) {  // graph-captured loop (uniform over the grid)
    if (a.ctl->abort) return;
    flags = a.ctl->flags;
  }
  TileCtx t;
  SysParams P;
  if (!tile_ctx(a, t, P)) return;
  const int lane = threadIdx.x & 31;
  double Fx = 0.0, Fy = 0.0, Fz = 0.0;
  double4_32a xi = make_double4_32a(0.0, 0.0, 0.0, 0.0);
  if (t.act) xi = a.x[cur][t.s];
  if (flags & kStepUseStoredF) {
    if (t.act) {
      const double4_32a f = a.f[t.s];
      Fx = f.x; Fy = f.y; Fz = f.z;
    }
  } else if (t.act) {
    const int cnt = list_count(a, t.sys, t.s, P.kmax);
    const uint4* lp4 = (const uint4*)(a.nbr + list_word(P.l_off, t.tl, P.kmax, lane, 0));
    const int4* qs = a.xq[cur] + P.p_off;
    const int4 qi = a.xq[cur][t.s];
    const float qu = P.qunit, rc2 = P.rc2f, c2x8 = 8.0f * P.c2f;
    const uint32_t self = (uint32_t)t.local;
    const uint4 none = make_uint4(self, self, self, self);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    const int ng = (cnt + 3) >> 2;
    uint4 e[GROUPS];
#pragma unroll
    for (int u = 0; u < GROUPS; ++u) e[u] = u < ng ? ld_list(lp4 + (int64_t)u * kTile, HINT) : none;
    for (int g = 0; g < ng; g += GROUPS) {
      uint4 en[GROUPS];
#pragma unroll
      for (int u = 0; u < GROUPS; ++u)
        en[u] = (g + GROUPS + u < ng) ? ld_list(lp4 + (int64_t)(g + GROUPS + u) * kTile, HINT) : none;
        // the list is padded to whole groups of four with the particle itself, and
      // groups past its end read `none` (also the particle itself)
      int4 q[4 * GROUPS];
#pragma unroll
      for (int u = 0; u < GROUPS; ++u) {
        q[4 * u + 0] = ld_shadow(qs + partner_slot(a, t.sys, e[u].x, P.n, self), HINT);
        q[4 * u + 1] = ld_shadow(qs + partner_slot(a, t.sys, e[u].y, P.n, self), HINT);
        q[4 * u + 2] = ld_shadow(qs + partner_slot(a, t.sys, e[u].z, P.n, self), HINT);
        q[4 * u + 3] = ld_shadow(qs + partner_slot(a, t.sys, e[u].w, P.n, self), HINT);
      }
#pragma unroll
      for (int m = 0; m < 4 * GROUPS; ++m) pair_fp32(qi, q[m], true, qu, rc2, c2x8, fx, fy, fz);
#pragma unroll
      for (int u = 0; u < GROUPS; ++u) e[u] = en[u];
    }
    Fx = f2d_bits(fx); Fy = f2d_bits(fy); Fz = f2d_bits(fz);  // exact, no FP64-pipe conversion
  }
  unsigned long long d2b = 0ull;
  if (t.act) d2b = integrate<true>(a, P, t, cur, xi, Fx, Fy, Fz, ka, kb, flags);
  warp_max_disp(a, t.sys, d2b, flags);
}

// Approximate reciprocal of r^2 for the force variants of Sec. 3.3: r^2 rounded
// to float, its correctly rounded float reciprocal, the mantissa cut to 8 bits
// for the stand-in of SPARC64 frcpad (relative error < 1/256, Eq. 2).
template <int BITS>
__device__ __forceinline__ double approx_rcp(double r2) {
  float y = __frcp_rn(__double2float_rn(r2));
  if (BITS < 23) y = __uint_as_float(__float_as_uint(y) & ~((1u << (23 - BITS)) - 1u));
  return (double)y;
}

// Force factor g(r) = 24 r^-8 - 48 r^-14 + 8 c2 for MODE 0 (full FP64 reciprocal)
// or from the approximate reciprocal y: MODE 1 / 3 uncorrected (y^4, y^7) with 8 /
// 23 bits, MODE 2 / 4 corrected by Eqs. 2-7 (y^4 (5 - 4 y r^2), y^7 (8 - 7 y r^2)).
template <int MODE>
__device__ __forceinline__ double force_factor(double r2, double c2x8) {
  if (MODE == 0) {
    const double ir2 = rcp_f64(r2);
    const double ir4 = ir2 * ir2;
    const double ir6 = ir4 * ir2;
    const double ir8 = ir4 * ir4;
    return fma(ir8, fma(-48.0, ir6, 24.0), c2x8);
  }
  const double y = approx_rcp<(MODE <= 2) ? 8 : 23>(r2);
  const double y2 = y * y;
  const double y4 = y2 * y2;
  const double y7 = y4 * y2 * y;
  double ir8 = y4, ir14 = y7;
  if (MODE == 2 || MODE == 4) {
    const double e = y * r2;
    ir8 = y4 * fma(-4.0, e, 5.0);
    ir14 = y7 * fma(-7.0, e, 8.0);
  }
  return fma(24.0, ir8, fma(-48.0, ir14, c2x8));
}

// FP64 form. The FP64 pipe is the bound (on GB300 a warp's FP64 instruction
// holds the pipe about as long as 60 other instructions take to issue), and a
// warp pays for an FP64 instruction whether one lane or all 32 need it. So each
// thread first classifies its listed partners on their fixed-point shadow
// positions (integer separations, float r^2, no FP64 instruction) against
// rc^2 (1 + 1e-5), a bound that no pair inside rc can exceed (each shadow
// coordinate errs by at most half a unit of L / 2^32, and the float r^2 by a few
// parts in 1e7), and queues the list words of the pairs that
// may be inside in shared memory. The FP64 work then runs in rounds in which every
// thread with partners left takes the next pair of its own queue: per pair 3 DADD
// for the separation and 3 for r^2, the exact test r^2 < rc^2 (bit patterns,
// r^2 >= 0), and for pairs inside the reciprocal (3 DFMA after an integer-built
// FP32 seed), the powers and factor (5) and the accumulation (3). A thread's
// queue keeps list order and the pairs left out are outside rc, where the force
// is zero, so every force is summed in the same order as a plain loop over the
// list: the results are the same bit for bit.
constexpr int kQueue64 = 16;  // queued list words per thread (FP64 pair loops)

// The classify-and-queue loop of the FP64 pair loops: every thread of the warp
// calls it (cnt = 0 for a lane without a particle); body(e) runs for the list
// words e of the thread's maybe-inside pairs, in list order, in rounds where
// every thread with a queued pair takes one. qme points at the thread's queue
// column (entry q at qme[q * BLOCK]).
template <int BLOCK, class Body>
__device__ __forceinline__ void queued_pairs(const DevArrays& a, const TileCtx& t, const SysParams& P, int lane,
                                             int cur, int cnt, uint32_t* qme, Body&& body) {
  const uint4* lp4 = (const uint4*)(a.nbr + list_word(P.l_off, t.tl, P.kmax, lane, 0));
  const int4* qs = a.xq[cur] + P.p_off;
  const int4 qi = t.act ? qs[t.local] : make_int4(0, 0, 0, 0);
  const float rc2q = P.rc2q_hi;
  const uint32_t self = (uint32_t)t.local;
  int k = 0;  // next listed partner to classify
  unsigned head = 0u, tail = 0u;
  while (true) {
    const unsigned qn = tail - head;
    const bool left = k < cnt;
    const unsigned has = __ballot_sync(kFull, qn > 0u);
    const unsigned busy = __ballot_sync(kFull, qn > 0u || left);
    if (busy == 0u) break;
    const unsigned room = __ballot_sync(kFull, left && qn <= (unsigned)(kQueue64 - 4));
    if (has == busy || room == 0u) {
      // FP64 round: each thread with a queued pair takes the next one
      if (qn > 0u) {
        const uint32_t e = qme[(head & (kQueue64 - 1)) * BLOCK];
        ++head;
        body(e);
      }
    } else if ((room >> (threadIdx.x & 31)) & 1u) {  // the ballot's bit of this thread
      // classification of the next four listed partners (no FP64 instruction)
      const uint4 w = __ldg(lp4 + (int64_t)(k >> 2) * kTile);
      const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const bool ok = k + m < cnt;
        const int4 qj = qs[ok ? partner_slot(a, t.sys, ws[m], P.n, self) : self];
        const float ax = (float)wrapped_diff(qj.x, qi.x);
        const float ay = (float)wrapped_diff(qj.y, qi.y);
        const float az = (float)wrapped_diff(qj.z, qi.z);
        if (ok && fmaf(az, az, fmaf(ay, ay, ax * ax)) < rc2q) {
          qme[(tail & (kQueue64 - 1)) * BLOCK] = ws[m];
          ++tail;
        }
      }
      k += 4;
    }
  }
}


// QUEUE false: the plain loop over the list (every listed pair takes the FP64
// separation and r^2, the warp pays the force body whenever one lane is inside).
template <int BLOCK, int MODE, bool QUEUE>
__global__ void __launch_bounds__(BLOCK) k_step_fp64(DevArrays a, int cur, double ka, double kb, int flags) {
  __shared__ uint32_t qbuf[QUEUE ? kQueue64 : 1][BLOCK];  // entry q of thread t at [q][t]: no bank conflicts
  if (a.ctl) {  // graph-captured loop (uniform over the grid)
    if (a.ctl->abort) return;
    flags = a.ctl->flags;
  }
  TileCtx t;
  SysParams P;
  if (!tile_ctx(a, t, P)) return;  // uniform over the warp
  const int lane = threadIdx.x & 31;
  double Fx = 0.0, Fy = 0.0, Fz = 0.0;
  double4_32a xi = make_double4_32a(0.0, 0.0, 0.0, 0.0);
  if (t.act) xi = a.x[cur][t.s];
  if (flags & kStepUseStoredF) {
    if (t.act) {
      const double4_32a f = a.f[t.s];
      Fx = f.x; Fy = f.y; Fz = f.z;
    }
  } else if (!QUEUE) {
    if (t.act) {
      const int cnt = list_count(a, t.sys, t.s, P.kmax);
      const uint32_t* lp = a.nbr + list_word(P.l_off, t.tl, P.kmax, lane, 0);
      const double4_32a* xs = a.x[cur] + P.p_off;
      const long long rc2b = __double_as_longlong(P.rc2);
      const double c2x8 = 8.0 * P.c2, L = P.L;
      for (int k = 0; k < cnt; ++k) {
        const uint32_t e = __ldg(lp + (int64_t)(k >> 2) * (4 * kTile) + (k & 3));
        const double4_32a xj = xs[partner_slot(a, t.sys, e, P.n, (uint32_t)t.local)];
        double dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
        const unsigned code = e >> kIdxBits;
        if (code) {
          dx = apply_image(dx, code & 3u, L);
          dy = apply_image(dy, (code >> 2) & 3u, L);
          dz = apply_image(dz, (code >> 4) & 3u, L);
        }
        const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        if (__double_as_longlong(r2) < rc2b) {
          const double g = force_factor<MODE>(r2, c2x8);  // 24 r^-8 - 48 r^-14 + 8 c2
          Fx = fma(g, dx, Fx);
          Fy = fma(g, dy, Fy);
          Fz = fma(g, dz, Fz);
        }
      }
    }
  } else {  // every lane of the warp takes part (inactive ones with an empty list)
    const int cnt = t.act ? list_count(a, t.sys, t.s, P.kmax) : 0;
    const double4_32a* xs = a.x[cur] + P.p_off;
    const long long rc2b = __double_as_longlong(P.rc2);
    const double c2x8 = 8.0 * P.c2, L = P.L;
    const uint32_t self = (uint32_t)t.local;
    queued_pairs<BLOCK>(a, t, P, lane, cur, cnt, &qbuf[0][threadIdx.x], [&](uint32_t e) {
      const double4_32a xj = xs[partner_slot(a, t.sys, e, P.n, self)];
      double dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
      const unsigned code = e >> kIdxBits;
      if (code) {
        dx = apply_image(dx, code & 3u, L);
        dy = apply_image(dy, (code >> 2) & 3u, L);
        dz = apply_image(dz, (code >> 4) & 3u, L);
      }
      const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
      if (__double_as_longlong(r2) < rc2b) {
        const double g = force_factor<MODE>(r2, c2x8);  // 24 r^-8 - 48 r^-14 + 8 c2
        Fx = fma(g, dx, Fx);
        Fy = fma(g, dy, Fy);
        Fz = fma(g, dz, Fz);
      }
    });
  }
  unsigned long long d2b = 0ull;
  if (t.act) d2b = integrate<false>(a, P, t, cur, xi, Fx, Fy, Fz, ka, kb, flags);
  warp_max_disp(a, t.sys, d2b, flags);
}

// ------------------------------------ half list with Newton's third law

// The paper's form before its FX10 kernel (Sec. 2.1 lists each pair once, i < j;
// Sec. 3.3 drops Newton's third law for the SIMD kernel): each pair is listed once,
// in the list of its lower slot; the thread of that slot adds the pair force to
// its own sum and scatters the opposite force to the partner with FP64 atomics.
// The own sum goes to f, the scattered sums to facc; k_integrate_half adds them.
// The order of the atomic additions varies, so results vary in the last bits.
template <int BLOCK, int MODE>
__global__ void __launch_bounds__(BLOCK) k_force_half_fp64(DevArrays a, int cur, int flags) {
  if (a.ctl) {  // graph-captured loop (uniform over the grid)
    if (a.ctl->abort) return;
    flags = a.ctl->flags;
  }
  if (flags & kStepUseStoredF) return;
  TileCtx t;
  SysParams P;
  if (!tile_ctx(a, t, P) || !t.act) return;
  const int lane = threadIdx.x & 31;
  const double4_32a xi = a.x[cur][t.s];
  const int cnt = list_count(a, t.sys, t.s, P.kmax);
  const uint32_t* lp = a.nbr + list_word(P.l_off, t.tl, P.kmax, lane, 0);
  const double4_32a* xs = a.x[cur] + P.p_off;
  double4_32a* fa = a.facc + P.p_off;
  const long long rc2b = __double_as_longlong(P.rc2);
  const double c2x8 = 8.0 * P.c2, L = P.L;
  double Fx = 0.0, Fy = 0.0, Fz = 0.0;
  for (int k = 0; k < cnt; ++k) {
    const uint32_t e = __ldg(lp + (int64_t)(k >> 2) * (4 * kTile) + (k & 3));
    const uint32_t j = partner_slot(a, t.sys, e, P.n, (uint32_t)t.local);
    const double4_32a xj = xs[j];
    double dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
    const unsigned code = e >> kIdxBits;
    if (code) {
      dx = apply_image(dx, code & 3u, L);
      dy = apply_image(dy, (code >> 2) & 3u, L);
      dz = apply_image(dz, (code >> 4) & 3u, L);
    }
    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    if (__double_as_longlong(r2) < rc2b) {
      const double g = force_factor<MODE>(r2, c2x8);
      const double fx = g * dx, fy = g * dy, fz = g * dz;
      Fx += fx;
      Fy += fy;
      Fz += fz;
      atomicAdd(&fa[j].x, -fx);
      atomicAdd(&fa[j].y, -fy);
      atomicAdd(&fa[j].z, -fz);
    }
  }
  a.f[t.s] = make_double4_32a(Fx, Fy, Fz, 0.0);
}

// FP32-force form of the same: pair forces in FP32 from the fixed-point
// separation, own sum in FP32, scattered sums in FP64.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_force_half_fp32(DevArrays a, int cur, int flags) {
  if (a.ctl) {
    if (a.ctl->abort) return;
    flags = a.ctl->flags;
  }
  if (flags & kStepUseStoredF) return;
  TileCtx t;
  SysParams P;
  if (!tile_ctx(a, t, P) || !t.act) return;
  const int lane = threadIdx.x & 31;
  const int cnt = list_count(a, t.sys, t.s, P.kmax);
  const uint32_t* lp = a.nbr + list_word(P.l_off, t.tl, P.kmax, lane, 0);
  const int4* qs = a.xq[cur] + P.p_off;
  const int4 qi = a.xq[cur][t.s];
  double4_32a* fa = a.facc + P.p_off;
  const float qu = P.qunit, rc2 = P.rc2f, c2x8 = 8.0f * P.c2f;
  float fx = 0.f, fy = 0.f, fz = 0.f;
  for (int k = 0; k < cnt; ++k) {
    const uint32_t j = partner_slot(a, t.sys, __ldg(lp + (int64_t)(k >> 2) * (4 * kTile) + (k & 3)), P.n,
                                    (uint32_t)t.local);
    float px = 0.f, py = 0.f, pz = 0.f;
    pair_fp32(qi, qs[j], true, qu, rc2, c2x8, px, py, pz);
    fx += px;
    fy += py;
    fz += pz;
    if (px != 0.f || py != 0.f || pz != 0.f) {
      atomicAdd(&fa[j].x, -f2d_bits(px));
      atomicAdd(&fa[j].y, -f2d_bits(py));
      atomicAdd(&fa[j].z, -f2d_bits(pz));
    }
  }
  a.f[t.s] = make_double4_32a(f2d_bits(fx), f2d_bits(fy), f2d_bits(fz), 0.0);
}

// Velocity-Verlet update of the half-list form: F = own sum + scattered sums
// (the latter reset for the next step), or the stored F.
template <bool kFP32>
__global__ void __launch_bounds__(kBlock) k_integrate_half(DevArrays a, int cur, int flags) {
  if (a.ctl) {
    if (a.ctl->abort) return;
    flags = a.ctl->flags;
  }
  TileCtx t;
  SysParams P;
  if (!tile_ctx(a, t, P)) return;
  double Fx = 0.0, Fy = 0.0, Fz = 0.0;
  double4_32a xi = make_double4_32a(0.0, 0.0, 0.0, 0.0);
  unsigned long long d2b = 0ull;
  if (t.act) {
    xi = a.x[cur][t.s];
    const double4_32a f = a.f[t.s];
    Fx = f.x; Fy = f.y; Fz = f.z;
    if (!(flags & kStepUseStoredF)) {
      const double4_32a g = a.facc[t.s];
      Fx += g.x; Fy += g.y; Fz += g.z;
      a.facc[t.s] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    }
    d2b = integrate<kFP32>(a, P, t, cur, xi, Fx, Fy, Fz, 0.0, 0.0, flags);
  }
  warp_max_disp(a, t.sys, d2b, flags);
}

// ------------------------------------------------- observables (FP64 sums)

// Per particle: 1/2 sum_j V(r) and 1/2 sum_j -r V'(r) over listed partners with
// r < rc (the full list counts each pair twice; a half list once, without the
// 1/2), and 1/2 |v|^2; each tile sums its 32 values in a fixed shuffle order into
// tile_obs[3 t ...]. With V(r) = 4 (r^-12 - r^-6) + 4 c2 r^2 + 4 c0 (Eq. 1) and
// -r V'(r) = 48 r^-12 - 24 r^-6 - 8 c2 r^2, the pair loop only sums r^-12, r^-6
// and r^2 and counts the pairs inside rc. Like the FP64 force loop it classifies
// the listed pairs on the fixed-point shadows first and runs the FP64 arithmetic
// (6 operations for the separation and r^2, 9 for a pair inside rc; the periodic
// image added only where the list word names one, the cutoff tested on bit
// patterns, r^2 >= 0) in full-warp rounds from per-thread queues; the sums keep
// list order, so the results equal a plain loop's bit for bit.
__global__ void __launch_bounds__(kBlock) k_pe_virial(DevArrays a, int cur, int with_pairs,
                                                      const int32_t* __restrict__ select) {
  __shared__ uint32_t qbuf[kQueue64][kBlock];
  TileCtx t;
  SysParams P;
  if (!tile_ctx(a, t, P)) return;           // uniform over the warp
  if (select && !select[t.sys]) return;     // uniform over the warp
  const int lane = threadIdx.x & 31;
  double pe = 0.0, w = 0.0, ke = 0.0;
  if (with_pairs) {  // every lane takes part (inactive ones with an empty list)
    const double4_32a xi = t.act ? a.x[cur][t.s] : make_double4_32a(0.0, 0.0, 0.0, 0.0);
    const double4_32a* xs = a.x[cur] + P.p_off;
    const int cnt = t.act ? list_count(a, t.sys, t.s, P.kmax) : 0;
    const long long rc2b = __double_as_longlong(P.rc2);
    const long long tinyb = __double_as_longlong(1e-30);
    const double L = P.L;
    const uint32_t self = (uint32_t)t.local;
    double s12 = 0.0, s6 = 0.0, sr = 0.0;
    int nin = 0;
    queued_pairs<kBlock>(a, t, P, lane, cur, cnt, &qbuf[0][threadIdx.x], [&](uint32_t e) {
      const double4_32a xj = xs[partner_slot(a, t.sys, e, P.n, self)];
      double dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
      const unsigned code = e >> kIdxBits;
      if (code) {
        dx = apply_image(dx, code & 3u, L);
        dy = apply_image(dy, (code >> 2) & 3u, L);
        dz = apply_image(dz, (code >> 4) & 3u, L);
      }
      const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
      const long long r2b = __double_as_longlong(r2);
      if (r2b < rc2b) {
        // reciprocal within rounding in 3 DFMA (see rcp_f64); IEEE division only for
        // (near-)coincident pairs, outside rcp_f64's range
        const double ir2 = r2b > tinyb ? rcp_f64(r2) : 1.0 / r2;
        const double ir6 = ir2 * ir2 * ir2;
        s12 = fma(ir6, ir6, s12);
        s6 += ir6;
        sr += r2;
        ++nin;
      }
    });
    if (t.act) {
      const double c2 = P.c2;
      pe = 4.0 * (s12 - s6) + 4.0 * fma(c2, sr, P.c0 * (double)nin);
      w = 48.0 * s12 - 24.0 * s6 - 8.0 * c2 * sr;
      if (!P.half) {  // the full list counts each pair twice
        pe *= 0.5;
        w *= 0.5;
      }
    }
  }
  if (t.act) {
    const double4_32a v = a.v[t.s];
    ke = 0.5 * (v.x * v.x + v.y * v.y + v.z * v.z);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    pe += __shfl_xor_sync(kFull, pe, o);
    w += __shfl_xor_sync(kFull, w, o);
    ke += __shfl_xor_sync(kFull, ke, o);
  }
  if (lane == 0) {
    const int64_t g = (int64_t)(P.t_off + t.tl) * 3;
    a.tile_obs[g + 0] = pe;
    a.tile_obs[g + 1] = w;
    a.tile_obs[g + 2] = ke;
  }
}

// Counts of listed pairs and of listed pairs with r < rc (FP64 test), per system.
__global__ void __launch_bounds__(kBlock) k_pair_stats(DevArrays a, int cur, unsigned long long* out2) {
  TileCtx t;
  SysParams P;
  if (!tile_ctx(a, t, P)) return;
  const int lane = threadIdx.x & 31;
  unsigned listed = 0, inside = 0;
  if (t.act) {
    const double4_32a xi = a.x[cur][t.s];
    const double4_32a* xs = a.x[cur] + P.p_off;
    const int cnt = list_count(a, t.sys, t.s, P.kmax);
    const uint32_t* lp = a.nbr + list_word(P.l_off, t.tl, P.kmax, lane, 0);
    listed = (unsigned)cnt;
    for (int k = 0; k < cnt; ++k) {
      const uint32_t e = lp[(int64_t)(k >> 2) * (4 * kTile) + (k & 3)];
      const double4_32a xj = xs[partner_slot(a, t.sys, e, P.n, (uint32_t)t.local)];
      const unsigned code = e >> kIdxBits;
      const double dx = apply_image(xj.x - xi.x, code & 3u, P.L);
      const double dy = apply_image(xj.y - xi.y, (code >> 2) & 3u, P.L);
      const double dz = apply_image(xj.z - xi.z, (code >> 4) & 3u, P.L);
      if (dx * dx + dy * dy + dz * dz < P.rc2) ++inside;
    }
  }
  listed = __reduce_add_sync(kFull, listed);
  inside = __reduce_add_sync(kFull, inside);
  if (lane == 0) {
    atomicAdd(&out2[2 * t.sys + 0], (unsigned long long)listed);
    atomicAdd(&out2[2 * t.sys + 1], (unsigned long long)inside);
  }
}

// Per-system sums of the tile partials (PE, W, KE), in two deterministic stages
// whose partition is relative to each system's first tile (so a system reduces
// the same way alone and in a batch): chunks of 256 tiles, one block each, summed
// by a fixed tree; then one block per system adds its chunk sums in order.
// work: the selected systems' ids (nsel) followed by the prefix of their chunk
// counts (nsel + 1).
constexpr int kObsChunk = 256;

__global__ void __launch_bounds__(kObsChunk) k_obs_chunks(DevArrays a, const int32_t* __restrict__ work, int nsel,
                                                        double* __restrict__ chunk3) {
  const int b = blockIdx.x;
  const int32_t* cpref = work + nsel;
  int lo = 0, hi = nsel - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cpref[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  const int sys = work[lo];
  const SysParams& P = a.params[sys];
  const int q = (b - cpref[lo]) * kObsChunk + (int)threadIdx.x;  // tile within the system
  __shared__ double sh[3][kObsChunk];
  double pe = 0.0, w = 0.0, ke = 0.0;
  if (q < P.ntiles) {
    const double* o = a.tile_obs + (int64_t)(P.t_off + q) * 3;
    pe = o[0];
    w = o[1];
    ke = o[2];
  }
  sh[0][threadIdx.x] = pe;
  sh[1][threadIdx.x] = w;
  sh[2][threadIdx.x] = ke;
  __syncthreads();
  for (int o = kObsChunk / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
      sh[2][threadIdx.x] += sh[2][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    chunk3[3 * b + 0] = sh[0][0];
    chunk3[3 * b + 1] = sh[1][0];
    chunk3[3 * b + 2] = sh[2][0];
  }
}

__global__ void __launch_bounds__(256) k_obs_final(const int32_t* __restrict__ work, int nsel,
                                                 const double* __restrict__ chunk3, double* __restrict__ out3) {
  const int r = blockIdx.x;
  const int sys = work[r];
  const int c0 = work[nsel + r], c1 = work[nsel + r + 1];
  __shared__ double sh[3][256];
  double pe = 0.0, w = 0.0, ke = 0.0;
  for (int c = c0 + (int)threadIdx.x; c < c1; c += 256) {
    pe += chunk3[3 * c + 0];
    w += chunk3[3 * c + 1];
    ke += chunk3[3 * c + 2];
  }
  sh[0][threadIdx.x] = pe;
  sh[1][threadIdx.x] = w;
  sh[2][threadIdx.x] = ke;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
      sh[2][threadIdx.x] += sh[2][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out3[3 * sys + 0] = sh[0][0];
    out3[3 * sys + 1] = sh[1][0];
    out3[3 * sys + 2] = sh[2][0];
  }
}

// ---------------------------------------------------------------- launchers

namespace {
// At least one block: with no tiles its warps return at once (an empty arena).
inline unsigned tile_blocks(const DevArrays& a) {
  return (unsigned)std::max<int64_t>(1, ((int64_t)a.ntiles * kTile + kBlock - 1) / kBlock);
}
}  // namespace

// Positions as held (caller order, not wrapped) into the slots of a system whose
// list was just built, with their fixed-point shadows: a restored checkpoint.
__global__ void k_positions_by_id(DevArrays a, int cur, const double* __restrict__ x, int sys) {
  const SysParams P = a.params[sys];
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= P.n) return;
  const int64_t s = P.p_off + l;
  const int64_t i = a.id[s];
  const double4_32a xv = make_double4_32a(x[3 * i + 0], x[3 * i + 1], x[3 * i + 2], 0.0);
  a.x[cur][s] = xv;
  a.xq[cur][s] = fixed4(xv, P.qscale);
}

void launch_positions_by_id(const DevArrays& a, int cur, const double* x, int64_t sys_n, int sys, cudaStream_t s) {
  if (sys_n <= 0) return;
  k_positions_by_id<<<(unsigned)((sys_n + 255) / 256), 256, 0, s>>>(a, cur, x, sys);
}

void launch_from_caller(const DevArrays& a, int cur, const double* x, const double* v, int sys,
                        int64_t ntiles_sys, cudaStream_t s) {
  const int64_t n = ntiles_sys * kTile;
  k_from_caller<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, cur, x, v, sys);
}

void launch_to_caller(const DevArrays& a, int cur, int which, double* out, int64_t sys_n, int sys,
                      int64_t, cudaStream_t s) {
  if (sys_n <= 0) return;
  k_to_caller<<<(unsigned)((sys_n + 255) / 256), 256, 0, s>>>(a, cur, which, out, sys);
}

// ------------------------------------------ graph-captured loop (decision)

// The list-validity decision after a drift (Sec. 2.1: the list is checked every
// step), for the graph-captured loop and for the host-driven one alike.
// Displacement rule: the FP32-force form compares the squared fixed-point
// displacement (an exact integer) with a threshold lowered by 4 units, the FP64
// forms test 2 sqrt(d2) >= skin. Velocity-bound rule (the DUTC check): the
// margin, the whole skin after a rebuild, shrinks by 2 v_max dt each step, and
// the list is rebuilt when it is no longer positive. Writes the rebuild flags
// and the rebuilding systems (in the order of sys_order: costliest list-build
// tiles first), resets the per-step maxima, and
// in a graph (reb_count set) counts steps, passes and rebuilds and sets the
// conditions of the rebuild node (h_if) and, after the second step of the loop
// body (last), of the loop node (h_loop). A non-finite position or velocity
// stops the loop (abort word 2).
__global__ void __launch_bounds__(1024) k_decide(DevArrays a, int nsys, int fp32, int vflag, int32_t* rebuild,
                                                 int32_t* rebuild_ids, int32_t* reb_pref, int32_t* reb_count,
                                                 cudaGraphConditionalHandle h_if,
                                                 cudaGraphConditionalHandle h_loop, int last) {
  GraphCtl* c = a.ctl;
  const bool graph = reb_count != nullptr;
  if (c->abort) {  // uniform over the block
    if (threadIdx.x == 0 && graph) {
      cudaGraphSetConditional(h_if, 0);
      if (last) cudaGraphSetConditional(h_loop, 0);
    }
    return;
  }
  __shared__ int wsum[32];
  __shared__ long long wsum64[32];
  __shared__ int base_s, bad_s, total_s;
  __shared__ long long total64_s;
  int32_t* chunk_pref = a.chunk_pref;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) { base_s = 0; bad_s = 0; }
  __syncthreads();
  for (int i0 = 0; i0 < nsys; i0 += (int)blockDim.x) {
    const int i = i0 + (int)threadIdx.x;
    const int k = i < nsys ? a.sys_order[i] : -1;
    int need = 0;
    if (k >= 0) {
      const unsigned long long d2 = a.disp2[k];
      a.disp2[k] = 0ull;
      const SysParams& P = a.params[k];
      if (P.active) {
        if (a.status[k].nonfinite) bad_s = 1;
        if (P.rule == 1) {
          // velocity bound (DUTC): the margin shrinks by 2 v_max dt per step; a
          // rebuild restores it (k_cell_starts)
          const double m =
              __dsub_rn(a.margin[k],
                        __dmul_rn(__dmul_rn(2.0, __dsqrt_rn(__longlong_as_double((long long)d2))), P.dt));
          a.margin[k] = m;
          need = (d2 == ~0ull || !(m > 0.0)) ? 1 : 0;
        } else if (fp32) {
          need = (d2 == ~0ull || __ull2double_rn(d2) >= P.disp_thr) ? 1 : 0;
        } else {
          need = !(2.0 * __dsqrt_rn(__longlong_as_double((long long)d2)) < P.skin) ? 1 : 0;
        }
      }
      rebuild[k] = need;
    }
    const unsigned b = __ballot_sync(kFull, need);
    if (lane == 0) wsum[w] = __popc(b);
    __syncthreads();
    if (w == 0) {
      const int v = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
      int incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      wsum[lane] = incl - v;
      if (lane == 31) total_s = incl;
    }
    __syncthreads();
    if (need) {
      rebuild_ids[base_s + wsum[w] + __popc(b & ((1u << lane) - 1u))] = k;
      if (graph) reb_count[k] += 1;
      a.status[k].overflow = 0;
      a.status[k].max_count = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) base_s += total_s;
    __syncthreads();
  }
  // prefixes of the rebuilding systems' tile counts (the rebuild kernels' work
  // list) and of their cell-chunk counts (the cell scan's work list), as one
  // scan of the pair packed in 64 bits
  const int nreb_all = base_s;
  long long carry = 0;
  for (int r0 = 0; r0 < nreb_all; r0 += (int)blockDim.x) {
    const int r = r0 + (int)threadIdx.x;
    long long v = 0;
    if (r < nreb_all) {
      const SysParams& P = a.params[rebuild_ids[r]];
      v = ((long long)scan_chunks((int64_t)P.nc * P.nc * P.nc) << 32) | (unsigned)P.ntiles;
    }
    long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum64[w] = incl;
    __syncthreads();
    if (w == 0) {
      const long long ws = lane < (int)(blockDim.x >> 5) ? wsum64[lane] : 0;
      long long wi = ws;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(kFull, wi, o);
        if (lane >= o) wi += y;
      }
      wsum64[lane] = wi - ws;
      if (lane == 31) total64_s = wi;
    }
    __syncthreads();
    if (r < nreb_all) {
      const long long e = carry + wsum64[w] + incl - v;
      reb_pref[r] = (int32_t)(e & 0xffffffffll);
      chunk_pref[r] = (int32_t)(e >> 32);
    }
    carry += total64_s;
    __syncthreads();
  }
  // the pass's chunk totals start at zero (the count kernel adds to them)
  for (int q = (int)threadIdx.x; q < (int)(carry >> 32) * kChunkCopies; q += (int)blockDim.x) a.chunk_sum[q] = 0;
  if (threadIdx.x == 0) {
    const int nreb = base_s;
    reb_pref[nreb] = (int32_t)(carry & 0xffffffffll);
    chunk_pref[nreb] = (int32_t)(carry >> 32);
    *a.tile_next = 0;
    c->done += 1;
    if (bad_s) {
      c->abort = 2;
      if (graph) {
        cudaGraphSetConditional(h_if, 0);
        if (last) cudaGraphSetConditional(h_loop, 0);
      }
      return;
    }
    c->nreb = nreb;
    c->passes += nreb > 0 ? 1 : 0;
    c->flags = kStepKickA | kStepKickB | kStepDrift | vflag;
    if (graph) {
      cudaGraphSetConditional(h_if, nreb > 0 ? 1u : 0u);
      if (last) cudaGraphSetConditional(h_loop, c->done < c->target ? 1u : 0u);
    }
  }
}

void launch_decide(const DevArrays& a, int nsys, int fp32, int vflag, int32_t* rebuild, int32_t* rebuild_ids,
                   int32_t* reb_pref, int32_t* reb_count, cudaGraphConditionalHandle h_if,
                   cudaGraphConditionalHandle h_loop, int last, cudaStream_t s) {
  // one block; as many warps as the systems need (a single warp for one system)
  const int threads = std::max(32, std::min(1024, (nsys + 31) / 32 * 32));
  k_decide<<<1, threads, 0, s>>>(a, nsys, fp32, vflag, rebuild, rebuild_ids, reb_pref, reb_count, h_if, h_loop,
                                 last);
}

// Binning kernels of a rebuild pass: at most 64 blocks of 128 per SM; warps stride
// over the rebuilding systems' tiles.
inline unsigned bin_blocks(const DevArrays& a) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(((int64_t)a.ntiles + 3) / 4, 152 * 64));
}

void launch_cell_count(const DevArrays& a, int cur, cudaStream_t s) {
  k_cell_count<<<bin_blocks(a), kBlock, 0, s>>>(a, cur);
}
void launch_cell_scan(const DevArrays& a, int nreb, cudaStream_t s) {
  // blocks stride over the chunks: one wave of 8 blocks per SM at most
  const unsigned g = (unsigned)std::max(1, std::min(a.chunk_cap, 152 * 8));
  k_cell_starts<<<g, kScanBlock, 0, s>>>(a, nreb);
}
void launch_scatter(const DevArrays& a, int cur, cudaStream_t s) {
  k_scatter<<<bin_blocks(a), kBlock, 0, s>>>(a, cur);
}
void launch_cell_rank(const DevArrays& a, int cur, cudaStream_t s) {
  k_cell_rank<<<bin_blocks(a), kBlock, 0, s>>>(a, cur);
}
namespace {
inline unsigned blocks_of(const DevArrays& a, int block) {
  return (unsigned)std::max<int64_t>(1, ((int64_t)a.ntiles * kTile + block - 1) / block);
}
}  // namespace

// Rebuild passes: warps stride over (or fetch) the rebuilding systems' tiles, so
// the grids are sized to the GPU (two waves of resident warps) or to the arena's
// tiles if fewer.
constexpr int kSMs = 152;
inline unsigned reb_blocks(const DevArrays& a, int block, int blocks_per_sm) {
  const int64_t all = ((int64_t)a.ntiles * kTile + block - 1) / block;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(all, (int64_t)kSMs * blocks_per_sm * 2));
}

template <int VAR>
static void launch_build_list_v(const DevArrays& a, int cur, int block, cudaStream_t s) {
  switch (block) {
    case 64: k_build_list<64, VAR><<<reb_blocks(a, 64, 16), 64, 0, s>>>(a, cur); break;
    case 256: k_build_list<256, VAR><<<reb_blocks(a, 256, 4), 256, 0, s>>>(a, cur); break;
    default: k_build_list<128, VAR><<<reb_blocks(a, 128, 8), 128, 0, s>>>(a, cur); break;
  }
}

void launch_build_list(const DevArrays& a, int cur, const Tuning& tu, cudaStream_t s) {
  switch (tu.list_variant) {
    case 5:
      switch (tu.list_block) {
        case 64: k_build_list_staged<64><<<reb_blocks(a, 64, 16), 64, 0, s>>>(a, cur); break;
        case 256: k_build_list_staged<256><<<reb_blocks(a, 256, 4), 256, 0, s>>>(a, cur); break;
        default: k_build_list_staged<128><<<reb_blocks(a, 128, 8), 128, 0, s>>>(a, cur); break;
      }
      break;
    case 4:
      switch (tu.list_block) {
        case 64: k_build_list_warp<64><<<reb_blocks(a, 64, 16), 64, 0, s>>>(a, cur); break;
        case 256: k_build_list_warp<256><<<reb_blocks(a, 256, 4), 256, 0, s>>>(a, cur); break;
        default: k_build_list_warp<128><<<reb_blocks(a, 128, 8), 128, 0, s>>>(a, cur); break;
      }
      break;
    case 1: launch_build_list_v<1>(a, cur, tu.list_block, s); break;
    case 2: launch_build_list_v<2>(a, cur, tu.list_block, s); break;
    case 3: launch_build_list_v<3>(a, cur, tu.list_block, s); break;
    default: launch_build_list_v<0>(a, cur, tu.list_block, s); break;
  }
}
template <int MODE, bool QUEUE>
static void launch_step_fp64_m(const DevArrays& a, int cur, double ka, double kb, int flags, int block,
                               cudaStream_t s) {
  switch (block) {
    case 64: k_step_fp64<64, MODE, QUEUE><<<blocks_of(a, 64), 64, 0, s>>>(a, cur, ka, kb, flags); break;
    case 256: k_step_fp64<256, MODE, QUEUE><<<blocks_of(a, 256), 256, 0, s>>>(a, cur, ka, kb, flags); break;
    default: k_step_fp64<128, MODE, QUEUE><<<blocks_of(a, 128), 128, 0, s>>>(a, cur, ka, kb, flags); break;
  }
}

template <bool QUEUE>
static void launch_step_fp64_q(const DevArrays& a, int cur, double ka, double kb, int flags, const Tuning& tu,
                               int mode, cudaStream_t s) {
  switch (mode) {
    case 1: launch_step_fp64_m<1, QUEUE>(a, cur, ka, kb, flags, tu.step_block, s); break;
    case 2: launch_step_fp64_m<2, QUEUE>(a, cur, ka, kb, flags, tu.step_block, s); break;
    case 3: launch_step_fp64_m<3, QUEUE>(a, cur, ka, kb, flags, tu.step_block, s); break;
    case 4: launch_step_fp64_m<4, QUEUE>(a, cur, ka, kb, flags, tu.step_block, s); break;
    default: launch_step_fp64_m<0, QUEUE>(a, cur, ka, kb, flags, tu.step_block, s); break;
  }
}

void launch_step_fp64(const DevArrays& a, int cur, double ka, double kb, int flags, const Tuning& tu,
                      int mode, cudaStream_t s) {
  if (tu.fp64_queue) launch_step_fp64_q<true>(a, cur, ka, kb, flags, tu, mode, s);
  else launch_step_fp64_q<false>(a, cur, ka, kb, flags, tu, mode, s);
}
template <int MODE>
static void launch_force_half_fp64_m(const DevArrays& a, int cur, int flags, int block, cudaStream_t s) {
  switch (block) {
    case 64: k_force_half_fp64<64, MODE><<<blocks_of(a, 64), 64, 0, s>>>(a, cur, flags); break;
    case 256: k_force_half_fp64<256, MODE><<<blocks_of(a, 256), 256, 0, s>>>(a, cur, flags); break;
    default: k_force_half_fp64<128, MODE><<<blocks_of(a, 128), 128, 0, s>>>(a, cur, flags); break;
  }
}

void launch_step_half(const DevArrays& a, int cur, int flags, const Tuning& tu, int precision, cudaStream_t s) {
  if (precision == 1) {
    switch (tu.step_block) {
      case 64: k_force_half_fp32<64><<<blocks_of(a, 64), 64, 0, s>>>(a, cur, flags); break;
      case 256: k_force_half_fp32<256><<<blocks_of(a, 256), 256, 0, s>>>(a, cur, flags); break;
      default: k_force_half_fp32<128><<<blocks_of(a, 128), 128, 0, s>>>(a, cur, flags); break;
    }
    k_integrate_half<true><<<tile_blocks(a), kBlock, 0, s>>>(a, cur, flags);
    return;
  }
  switch (precision) {
    case 2: launch_force_half_fp64_m<1>(a, cur, flags, tu.step_block, s); break;
    case 3: launch_force_half_fp64_m<2>(a, cur, flags, tu.step_block, s); break;
    case 4: launch_force_half_fp64_m<3>(a, cur, flags, tu.step_block, s); break;
    case 5: launch_force_half_fp64_m<4>(a, cur, flags, tu.step_block, s); break;
    default: launch_force_half_fp64_m<0>(a, cur, flags, tu.step_block, s); break;
  }
  k_integrate_half<false><<<tile_blocks(a), kBlock, 0, s>>>(a, cur, flags);
}

void launch_step_fp32(const DevArrays& a, int cur, double ka, double kb, int flags, const Tuning& tu,
                      cudaStream_t s) {
  const int b = tu.step_block, g = tu.step_groups;
#define LJMD_STEP32(B, G, H) k_step_fp32<B, G, H><<<blocks_of(a, B), B, 0, s>>>(a, cur, ka, kb, flags)
#define LJMD_STEP32B(G, H)             \
  if (b == 64) LJMD_STEP32(64, G, H);  \
  else if (b == 256) LJMD_STEP32(256, G, H); \
  else LJMD_STEP32(128, G, H)
  if (tu.step_hint) {
    if (g == 2) { LJMD_STEP32B(2, true); } else { LJMD_STEP32B(1, true); }
  } else {
    if (g == 2) { LJMD_STEP32B(2, false); } else { LJMD_STEP32B(1, false); }
  }
#undef LJMD_STEP32B
#undef LJMD_STEP32
}
void launch_pe_virial(const DevArrays& a, int cur, int with_pairs, const int32_t* select, cudaStream_t s) {
  k_pe_virial<<<tile_blocks(a), kBlock, 0, s>>>(a, cur, with_pairs, select);
}

// v *= factor for every particle of the systems with scale[sys] != 1.
__global__ void k_scale_v(DevArrays a, const double* __restrict__ scale) {
  TileCtx t;
  SysParams P;
  if (!tile_ctx(a, t, P) || !t.act) return;
  const double f = scale[t.sys];
  if (f == 1.0) return;
  double4_32a v = a.v[t.s];
  v.x *= f;
  v.y *= f;
  v.z *= f;
  a.v[t.s] = v;
}

void launch_scale_v(const DevArrays& a, const double* scale, cudaStream_t s) {
  k_scale_v<<<tile_blocks(a), kBlock, 0, s>>>(a, scale);
}
void launch_pair_stats(const DevArrays& a, int cur, unsigned long long* out2, cudaStream_t s) {
  k_pair_stats<<<tile_blocks(a), kBlock, 0, s>>>(a, cur, out2);
}
void launch_reduce_obs(const DevArrays& a, const int32_t* work, int nsel, int nchunks, double* chunk3, double* out3,
                       cudaStream_t s) {
  if (nsel <= 0 || nchunks <= 0) return;
  k_obs_chunks<<<nchunks, kObsChunk, 0, s>>>(a, work, nsel, chunk3);
  k_obs_final<<<nsel, 256, 0, s>>>(work, nsel, chunk3, out3);
}

}  // namespace ljmd
