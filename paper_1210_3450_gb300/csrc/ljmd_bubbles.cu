// Bubble identification (Sec. 4.2 of the paper): particles are counted in
// subcells of side >= 3 sigma, a subcell is gas when its density is below a
// threshold (0.2 in the paper), and face-neighbouring gas subcells of the
// periodic simple cubic lattice form one bubble (site percolation). The paper
// gathers the counts on one node and clusters serially; here both steps run on
// the GPU: a histogram with atomics, then a lock-free union-find whose root is
// always the smallest subcell index of a cluster (so labels are deterministic).
#include "ljmd_dev.cuh"
#include "ljmd_math.cuh"

namespace ljmd {
namespace {

// Subcell of every particle of system `sys`, counted with atomics.
__global__ void k_sub_count(DevArrays a, int cur, int sys, int ns, double inv_side, uint32_t* counts) {
  const SysParams P = a.params[sys];
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= P.n) return;
  const double4_32a x = a.x[cur][P.p_off + l];
  const int cx = cell_axis(wrap_fast(x.x, P.L), inv_side, ns);
  const int cy = cell_axis(wrap_fast(x.y, P.L), inv_side, ns);
  const int cz = cell_axis(wrap_fast(x.z, P.L), inv_side, ns);
  atomicAdd(&counts[cx + (int64_t)ns * (cy + (int64_t)ns * cz)], 1u);
}

// parent[c] = c for gas subcells (count < gas_count), -1 otherwise.
__global__ void k_gas_init(const uint32_t* counts, int64_t ncell, double gas_count, int32_t* parent) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  parent[c] = (double)counts[c] < gas_count ? (int32_t)c : -1;
}

// parent[] is read and written by threads on every SM while the union runs, so
// its accesses are relaxed atomics at GPU scope: a plain load may be served from
// this SM's L1 and keep returning a root that another SM has linked meanwhile
// (each compare-and-swap would then fail until the retry bound).
__device__ __forceinline__ int32_t ld_parent(const int32_t* p) {
  int32_t v;
  asm volatile("ld.relaxed.gpu.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_parent(int32_t* p, int32_t v) {
  asm volatile("st.relaxed.gpu.s32 [%0], %1;" : : "l"(p), "r"(v) : "memory");
}

// Root of c (parent chains only ever point to smaller indices).
__device__ __forceinline__ int32_t uf_find(int32_t* parent, int32_t c) {
  int32_t p = ld_parent(parent + c);
  while (p != c) {
    const int32_t g = ld_parent(parent + p);
    if (g != p) st_parent(parent + c, g);  // path halving (benign race: g is an ancestor)
    c = p;
    p = g;
  }
  return c;
}

// Join the clusters of a and b: the larger root is linked under the smaller.
// Each failed compare-and-swap means another thread linked that root first;
// the retry count is bounded and overruns are reported in *err.
__device__ __forceinline__ void uf_union(int32_t* parent, int32_t a, int32_t b, int* err) {
  for (int it = 0; it < 1 << 20; ++it) {
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a == b) return;
    if (a < b) {
      const int32_t t = a;
      a = b;
      b = t;
    }
    // a > b: link root a under b if a is still a root
    if (atomicCAS(&parent[a], a, b) == a) return;
  }
  atomicExch(err, 1);
}

__global__ void k_gas_union(int32_t* parent, int ns, int* err) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ncell = (int64_t)ns * ns * ns;
  if (c >= ncell || parent[c] < 0) return;
  const int cx = (int)(c % ns), cy = (int)((c / ns) % ns), cz = (int)(c / ((int64_t)ns * ns));
  const int64_t nb[3] = {((cx + 1) % ns) + (int64_t)ns * (cy + (int64_t)ns * cz),
                         cx + (int64_t)ns * (((cy + 1) % ns) + (int64_t)ns * cz),
                         cx + (int64_t)ns * (cy + (int64_t)ns * ((cz + 1) % ns))};
#pragma unroll
  for (int q = 0; q < 3; ++q)
    if (ld_parent(parent + nb[q]) >= 0) uf_union(parent, (int32_t)c, (int32_t)nb[q], err);
}

// Final labels (roots) and cluster sizes.
__global__ void k_gas_label(int32_t* parent, int64_t ncell, uint32_t* size) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncell || parent[c] < 0) return;
  const int32_t r = uf_find(parent, (int32_t)c);
  parent[c] = r;
  atomicAdd(&size[r], 1u);
}

}  // namespace

void launch_bubbles(const DevArrays& a, int cur, int sys, int64_t n, int ns, double box, double gas_count,
                    uint32_t* counts, int32_t* parent, uint32_t* size, int* err, cudaStream_t s) {
  const int64_t ncell = (int64_t)ns * ns * ns;
  const unsigned gc = (unsigned)((ncell + 255) / 256);
  cudaMemsetAsync(counts, 0, sizeof(uint32_t) * ncell, s);
  cudaMemsetAsync(size, 0, sizeof(uint32_t) * ncell, s);
  cudaMemsetAsync(err, 0, sizeof(int), s);
  if (n > 0) k_sub_count<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, cur, sys, ns, (double)ns / box, counts);
  k_gas_init<<<gc, 256, 0, s>>>(counts, ncell, gas_count, parent);
  k_gas_union<<<gc, 256, 0, s>>>(parent, ns, err);
  k_gas_label<<<gc, 256, 0, s>>>(parent, ncell, size);
}

}  // namespace ljmd
