// Device helpers shared by the kernels: periodic wrap, cell index, fixed-point
// shadow coordinates, list image codes and the FP64 reciprocal used by the
// pair-force loops.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ljmd {

// x - L floor(x / L), then the same fix-ups as the reference wrap.
static __device__ __forceinline__ double wrap_full(double x, double L) {
  double w = __dsub_rn(x, __dmul_rn(L, floor(__ddiv_rn(x, L))));
  if (w < 0.0) w = __dadd_rn(w, L);
  if (w >= L) w = __dsub_rn(w, L);
  if (w < 0.0 || w >= L) w = 0.0;
  return w;
}

// Wrap only when outside [0, L): for x >= 0 the bit pattern orders like the value,
// and negative values (sign bit set) or NaN compare above L's bit pattern.
static __device__ __forceinline__ double wrap_fast(double x, double L) {
  if ((unsigned long long)__double_as_longlong(x) >= (unsigned long long)__double_as_longlong(L))
    x = wrap_full(x, L);
  return x;
}

// floor(y) for 0 <= y < 2^31 by integer operations on the bits (negative y
// gives -1, NaN gives 0x7fffffff; callers clamp).
static __device__ __forceinline__ int floor_bits(double y) {
  const long long b = __double_as_longlong(y);
  if (b < 0) return -1;
  const int ef = (int)(b >> 52);
  if (ef < 1023) return 0;                      // 0 <= y < 1
  if (ef > 1023 + 30) return 0x7fffffff;        // too large (or inf / NaN)
  const unsigned long long m = (unsigned long long)(b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  return (int)(m >> (1075 - ef));
}

// Cell index along one axis: min(floor(x * nc / L), nc - 1), the product rounded
// once in FP64 exactly as the reference computes it, the floor on the bits.
static __device__ __forceinline__ int cell_axis(double x, double inv_cs, int nc) {
  int k = floor_bits(__dmul_rn(x, inv_cs));
  if (k > nc - 1) k = nc - 1;
  if (k < 0) k = 0;
  return k;
}

static __device__ __forceinline__ int cell_of(const double4_32a& x, double inv_cs, int nc) {
  return cell_axis(x.x, inv_cs, nc) + nc * (cell_axis(x.y, inv_cs, nc) + nc * cell_axis(x.z, inv_cs, nc));
}

// Round a double to the nearest integer (ties to even) and keep the low 32 bits,
// with integer operations only (no FP64-pipe conversion). Same result as
// (int)(unsigned)__double2ll_rn(y) for |y| < 2^62.
static __device__ __forceinline__ int round_low32(double y) {
  const long long b = __double_as_longlong(y);
  const int ef = (int)((b >> 52) & 0x7FF);
  if (ef < 1022) return 0;  // |y| < 0.5 (or zero / subnormal)
  const unsigned long long m = (unsigned long long)(b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int shift = 1075 - ef;  // y = m 2^-shift
  unsigned long long r;
  if (shift <= 0) {
    r = m << (-shift);
  } else {
    r = m >> shift;
    const unsigned long long rem = m & ((1ull << shift) - 1ull), half = 1ull << (shift - 1);
    if (rem > half || (rem == half && (r & 1ull))) ++r;
  }
  if (b < 0) r = 0ull - r;
  return (int)(unsigned)r;
}

// Fixed-point shadow coordinate: round(x 2^32 / L) mod 2^32. Differences of two
// such values, taken as wrapped 32-bit integers, are minimum-image separations.
static __device__ __forceinline__ int to_fixed(double x, double qscale) {
  return round_low32(x * qscale);
}

// Exact float -> double with integer operations (subnormal floats become zero).
static __device__ __forceinline__ double f2d_bits(float f) {
  const unsigned fb = __float_as_uint(f);
  const unsigned ex = (fb >> 23) & 0xFFu;
  const unsigned sign = fb & 0x80000000u;
  if (ex == 0u) return __longlong_as_double((long long)sign << 32);
  const unsigned hi = sign | ((ex == 0xFFu ? 0x7FFu : ex + 896u) << 20) | ((fb & 0x7FFFFFu) >> 3);
  return __longlong_as_double(((long long)hi << 32) | ((long long)(fb & 7u) << 29));
}

static __device__ __forceinline__ int4 fixed4(const double4_32a& x, double qscale) {
  return make_int4(to_fixed(x.x, qscale), to_fixed(x.y, qscale), to_fixed(x.z, qscale), 0);
}

static __device__ __forceinline__ int wrapped_diff(int a, int b) { return (int)((unsigned)a - (unsigned)b); }

static __device__ __forceinline__ bool finite_bits(double v) {
  return ((unsigned long long)__double_as_longlong(v) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

// Apply the periodic image encoded in a list word (two bits per axis).
static __device__ __forceinline__ double apply_image(double d, unsigned code2, double L) {
  if (code2 == 1u) return __dadd_rn(d, L);
  if (code2 == 2u) return __dsub_rn(d, L);
  return d;
}

// 1 / r2 in FP64 without the FP64 divide sequence: a float seed built from the
// top mantissa bits by integer operations, a hardware reciprocal estimate, and one
// cubically convergent correction y = y0 (1 + e + e^2), e = 1 - r2 y0. The seed's
// relative error is below 2^-21, so the result is within rounding of 1 / r2.
// Valid for 1e-37 < r2 < 1e37.
static __device__ __forceinline__ double rcp_f64(double r2) {
  const long long b = __double_as_longlong(r2);
  const int hi = (int)(b >> 32);
  const unsigned lo = (unsigned)b;
  const int fb = (((hi >> 20) - 896) << 23) | ((hi & 0xFFFFF) << 3) | (int)(lo >> 29);
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(__int_as_float(fb)));
  const int yb = __float_as_int(yf);
  const long long db = ((long long)((((yb >> 23) + 896) << 20) | ((yb & 0x7FFFFF) >> 3)) << 32) |
                       ((long long)(yb & 7) << 29);
  const double y0 = __longlong_as_double(db);
  const double e = fma(-r2, y0, 1.0);
  return fma(y0, fma(e, e, e), y0);
}


}  // namespace ljmd
