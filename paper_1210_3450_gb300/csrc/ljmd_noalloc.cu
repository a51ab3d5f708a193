// Allocation-free force entry point (md_forces_noalloc).
//
// Some callers cannot let a library call cudaMalloc: applications whose device
// memory is owned by their own allocator or memory pool (which must account for
// every byte and may already hold nearly all of it), and code that cannot afford
// the implicit device-wide synchronisation of cudaMalloc / cudaFree. For them this
// file offers one call that computes truncated-LJ forces for positions the caller
// passes in, into a force array the caller passes in, and keeps every piece of
// working memory in one fixed file-scope device array instead of allocating it.
//
// The working memory (cell counters, cell starts, per-particle cells, the
// scattered caller indices, the cell-sorted copy of the positions) lives in
// g_noalloc_scratch below; every GPU
// that loads this library holds that array until the process exits. Host code
// cannot use the symbol g_noalloc_scratch as a device address (it names a host
// stand-in), so the device address is looked up with cudaGetSymbolAddress, once
// per device, with that device current, on the first call made on that device.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "ljmd.h"
#include "ljmd_dev.cuh"
#include "ljmd_engine.h"
#include "ljmd_math.cuh"

namespace ljmd {
namespace {

constexpr int64_t kNaMaxN = 65536;      // particles per call
constexpr int64_t kNaMaxCells = 32768;  // cell grid of at most 32^3 cells
constexpr int kNaMaxDevices = 64;

// Layout of the scratch array (bytes, each part 256-aligned).
constexpr size_t kOffCount = 0;                                          // int[kNaMaxCells]
constexpr size_t kOffStart = kOffCount + 4 * kNaMaxCells;                // int[kNaMaxCells + 1]
constexpr size_t kOffCell = kOffStart + 4 * (kNaMaxCells + 256);         // int[kNaMaxN]
constexpr size_t kOffIdx = kOffCell + 4 * kNaMaxN;                       // int[kNaMaxN]
constexpr size_t kOffPos = kOffIdx + 4 * kNaMaxN;                        // double4_32a[kNaMaxN]
constexpr size_t kScratchBytes = kOffPos + 32 * kNaMaxN;                 // 3.0 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct NaParams {
  double L, inv_cs, rc2, c2x8;
  int n, nc;
};

struct NaScratch {
  int* count;
  int* start;
  int* cell;
  int* idx;          // caller indices scattered into cell order (arbitrary within a cell)
  double4_32a* pos;  // wrapped positions in cell order, by caller index within a cell; w = caller index
};

__device__ __forceinline__ NaScratch na_view(unsigned char* base) {
  NaScratch s;
  s.count = (int*)(base + kOffCount);
  s.start = (int*)(base + kOffStart);
  s.cell = (int*)(base + kOffCell);
  s.idx = (int*)(base + kOffIdx);
  s.pos = (double4_32a*)(base + kOffPos);
  return s;
}

__global__ void k_na_clear(unsigned char* base, int ncell) {
  NaScratch s = na_view(base);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) s.count[c] = 0;
}

__global__ void k_na_bin(unsigned char* base, NaParams p, const double* __restrict__ x) {
  NaScratch s = na_view(base);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.n) return;
  const double4_32a w = make_double4_32a(wrap_full(x[3 * i + 0], p.L), wrap_full(x[3 * i + 1], p.L),
                                         wrap_full(x[3 * i + 2], p.L), 0.0);
  const int c = p.nc > 1 ? cell_of(w, p.inv_cs, p.nc) : 0;
  s.cell[i] = c;
  atomicAdd(&s.count[c], 1);
}

// Single block: exclusive scan of the counts; counts become fill counters.
__global__ void __launch_bounds__(1024) k_na_scan(unsigned char* base, int ncell) {
  NaScratch s = na_view(base);
  __shared__ int wsum[32];
  __shared__ int total;
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  int carry = 0;
  for (int b0 = 0; b0 < ncell; b0 += 1024) {
    const int c = b0 + tid;
    const int v = c < ncell ? s.count[c] : 0;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[wp] = incl;
    __syncthreads();
    if (wp == 0) {
      const int ws = wsum[lane];
      int wi = ws;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += y;
      }
      wsum[lane] = wi - ws;
      if (lane == 31) total = wi;
    }
    __syncthreads();
    if (c < ncell) {
      s.start[c] = carry + wsum[wp] + incl - v;
      s.count[c] = 0;
    }
    carry += total;
    __syncthreads();
  }
  if (tid == 0) s.start[ncell] = carry;
}

// Caller indices into their cells' ranges, in arrival order.
__global__ void k_na_scatter(unsigned char* base, NaParams p) {
  NaScratch s = na_view(base);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.n) return;
  const int c = s.cell[i];
  s.idx[s.start[c] + atomicAdd(&s.count[c], 1)] = i;
}

// Each particle's place in its cell is the number of the cell's particles with a
// smaller caller index, so the cell-sorted positions, and with them the order of
// every force sum, do not depend on the order of the atomics above: the same
// positions give the same forces bit for bit.
__global__ void k_na_rank(unsigned char* base, NaParams p, const double* __restrict__ x) {
  NaScratch s = na_view(base);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.n) return;
  const int c = s.cell[i];
  const int lo = s.start[c], hi = s.start[c + 1];
  int rank = 0;
  for (int q = lo; q < hi; ++q) rank += s.idx[q] < i ? 1 : 0;
  s.pos[lo + rank] = make_double4_32a(wrap_full(x[3 * i + 0], p.L), wrap_full(x[3 * i + 1], p.L),
                                      wrap_full(x[3 * i + 2], p.L), (double)i);
}

// Force on caller particle i from every j in the 27 neighbour cells (or from all
// particles when nc == 1), minimum image, r < rc: the same pair force as the
// list-based kernels, F_i = sum_j (24 r^-8 - 48 r^-14 + 8 c2)(x_j - x_i).
__global__ void k_na_force(unsigned char* base, NaParams p, const double* __restrict__ x,
                           double* __restrict__ f) {
  NaScratch s = na_view(base);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.n) return;
  const double xi = wrap_full(x[3 * i + 0], p.L), yi = wrap_full(x[3 * i + 1], p.L),
               zi = wrap_full(x[3 * i + 2], p.L);
  const long long rc2b = __double_as_longlong(p.rc2);
  double fx = 0.0, fy = 0.0, fz = 0.0;
  auto pair = [&](const double4_32a& q, double sx, double sy, double sz) {
    if ((int)q.w == i) return;
    const double dx = (q.x - xi) + sx, dy = (q.y - yi) + sy, dz = (q.z - zi) + sz;
    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    if (__double_as_longlong(r2) < rc2b) {
      const double ir2 = rcp_f64(r2);
      const double ir4 = ir2 * ir2;
      const double g = fma(ir4 * ir4, fma(-48.0, ir4 * ir2, 24.0), p.c2x8);
      fx = fma(g, dx, fx);
      fy = fma(g, dy, fy);
      fz = fma(g, dz, fz);
    }
  };
  if (p.nc > 1) {
    const int nc = p.nc;
    const int ci = s.cell[i];
    const int cx = ci % nc, cy = (ci / nc) % nc, cz = ci / (nc * nc);
    for (int oz = -1; oz <= 1; ++oz) {
      int nz = cz + oz;
      double sz = 0.0;
      if (nz < 0) { nz += nc; sz = -p.L; } else if (nz >= nc) { nz -= nc; sz = p.L; }
      for (int oy = -1; oy <= 1; ++oy) {
        int ny = cy + oy;
        double sy = 0.0;
        if (ny < 0) { ny += nc; sy = -p.L; } else if (ny >= nc) { ny -= nc; sy = p.L; }
        for (int ox = -1; ox <= 1; ++ox) {
          int nx = cx + ox;
          double sx = 0.0;
          if (nx < 0) { nx += nc; sx = -p.L; } else if (nx >= nc) { nx -= nc; sx = p.L; }
          const int c = nx + nc * (ny + nc * nz);
          for (int q = s.start[c]; q < s.start[c + 1]; ++q) pair(s.pos[q], sx, sy, sz);
        }
      }
    }
  } else {
    for (int q = 0; q < p.n; ++q) {
      const double4_32a pj = s.pos[q];
      pair(pj, -p.L * rint((pj.x - xi) / p.L), -p.L * rint((pj.y - yi) / p.L),
           -p.L * rint((pj.z - zi) / p.L));
    }
  }
  f[3 * i + 0] = fx;
  f[3 * i + 1] = fy;
  f[3 * i + 2] = fz;
}

std::mutex g_na_mu;
unsigned char* g_na_addr[kNaMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
int na_scratch(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return MD_ERR_CUDA;
  }
  if (dev < 0 || dev >= kNaMaxDevices) {
    set_error("device ordinal out of range for md_forces_noalloc");
    return MD_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return MD_ERR_CUDA;
    }
    g_na_addr[dev] = (unsigned char*)p;
  }
  *out = g_na_addr[dev];
  return MD_OK;
}

}  // namespace
}  // namespace ljmd

extern "C" int md_forces_noalloc(const double* x_dev, int64_t N, double box_L, double rc,
                                 double* f_dev, void* stream) {
  using namespace ljmd;
  set_error("");
  if (!x_dev || !f_dev) {
    set_error("null device array");
    return MD_ERR_ARG;
  }
  if (N < 1 || N > kNaMaxN) {
    set_error("md_forces_noalloc: N must be in [1, 65536] (fixed scratch size)");
    return MD_ERR_ARG;
  }
  if (!(rc > 0.0) || !std::isfinite(rc) || !(box_L > 2.0 * rc) || !(box_L <= 10000.0)) {
    set_error("md_forces_noalloc: need rc > 0 and 2 rc < L <= 10000");
    return MD_ERR_ARG;
  }
  unsigned char* base = nullptr;
  int r = na_scratch(&base);
  if (r != MD_OK) return r;
  NaParams p;
  p.L = box_L;
  p.n = (int)N;
  // cells per axis, floor(L / rc), clamped in double before the conversion (L / rc
  // can exceed the int range); lowered by one where rounding could make a cell
  // narrower than rc, and at most 32 (coarser cells stay valid: side > rc)
  const double q = std::floor(box_L / rc);
  int nc = q > 33.0 ? 33 : (int)q;
  if (nc >= 1 && box_L / nc < rc * (1.0 + 1e-9)) nc -= 1;
  if (nc > 32) nc = 32;
  p.nc = nc >= 3 ? nc : 1;
  p.inv_cs = (double)p.nc / box_L;
  p.rc2 = rc * rc;
  const double irc2 = 1.0 / p.rc2, irc6 = irc2 * irc2 * irc2;
  p.c2x8 = 8.0 * (6.0 * irc6 * irc6 * irc2 - 3.0 * irc6 * irc2);
  const int ncell = p.nc * p.nc * p.nc;
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned blocks = (unsigned)((N + 255) / 256);
  k_na_clear<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(base, ncell);
  k_na_bin<<<blocks, 256, 0, s>>>(base, p, x_dev);
  k_na_scan<<<1, 1024, 0, s>>>(base, ncell);
  k_na_scatter<<<blocks, 256, 0, s>>>(base, p);
  k_na_rank<<<blocks, 256, 0, s>>>(base, p, x_dev);
  k_na_force<<<blocks, 256, 0, s>>>(base, p, x_dev, f_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("md_forces_noalloc launch: ") + cudaGetErrorString(e));
    return MD_ERR_CUDA;
  }
  return MD_OK;
}
