// Shared device-side definitions of libdp (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/dp.h"

namespace dp {

// ---------------------------------------------------------------------------
// Device-side status word bits (written by kernels, read by the host after a
// launch).  Kernels never trap: they record the problem and return.
// ---------------------------------------------------------------------------
enum : int {
  kFlagRebuild = 1 << 0,   // neighbour skin lists must be rebuilt
  kFlagOverflow = 1 << 1,  // a skin list exceeded its capacity
  kFlagMirror = 1 << 2,    // a skin entry had no mirror entry (internal error)
  kFlagTimeout = 1 << 3,   // a bounded device-side wait gave up
  kFlagNonFinite = 1 << 4  // non-finite energy or force, or beyond the exact sums' range
};

// One periodic system of a batch.  Atoms [atom0, atom0 + natom) belong to it.
struct SysInfo {
  double L[3];     // box lengths
  double cs[3];    // cell edge per direction (cells >= rc + skin)
  int atom0, natom;
  int cell0;       // first cell of this system in the batch's cell arrays
  int nc[3];       // cells per direction (>= 3 when use_cells)
  int use_cells;   // 0: brute force over atoms and images (boxes < 3 cells)
  int nimg[3];     // image range for brute force
  int pad;
};

// One entry of a skin (Verlet) list: neighbour atom j and its image m relative
// to UNWRAPPED positions: r_ij = x_j - x_i + m * L (constant while atoms move).
struct SkinEntry {
  int j, mx, my, mz;
};

// ---------------------------------------------------------------------------
// Exact FP64 helpers: no contraction into FMA, so distances that decide
// neighbour membership and order are the plain IEEE products and sums.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double wrap_coord(double x, double L, double* f_out) {
  double f = floor(__ddiv_rn(x, L));
  *f_out = f;
  return __dsub_rn(x, __dmul_rn(L, f));
}

// r = (w_j - w_i) + n * L per component, d2 = (x*x + y*y) + z*z
__device__ __forceinline__ double sep_exact(const double* wi, const double* wj, const int* n,
                                            const double* L, double* r) {
  for (int a = 0; a < 3; ++a) {
    double t = __dsub_rn(wj[a], wi[a]);
    double u = __dmul_rn((double)n[a], L[a]);
    r[a] = __dadd_rn(t, u);
  }
  return __dadd_rn(__dadd_rn(__dmul_rn(r[0], r[0]), __dmul_rn(r[1], r[1])), __dmul_rn(r[2], r[2]));
}

// Neighbour order: (d2, j, n) lexicographic.  d2 >= 0 is never NaN, and the
// bit patterns of non-negative doubles order like their values, so d2 is
// compared as a 64-bit integer (integer pipe, not the FP64 one).
__device__ __forceinline__ bool key_less(double da, int ja, const int* na, double db, int jb,
                                         const int* nb) {
  const long long ia = __double_as_longlong(da), ib = __double_as_longlong(db);
  if (ia != ib) return ia < ib;
  if (ja != jb) return ja < jb;
  for (int a = 0; a < 3; ++a)
    if (na[a] != nb[a]) return na[a] < nb[a];
  return false;
}

// Smooth switch sw(r) and d sw/dr (quintic smoothstep between rs and rc).
template <typename T>
__device__ __forceinline__ void smooth_switch(T r, T rs, T rc, T* sw, T* dsw) {
  if (r < rs) {
    *sw = T(1);
    *dsw = T(0);
  } else if (r < rc) {
    T inv = T(1) / (rc - rs);
    T u = (r - rs) * inv;
    T u2 = u * u;
    *sw = u2 * u * (T(-6) * u2 + T(15) * u - T(10)) + T(1);
    T um1 = u - T(1);
    *dsw = T(-30) * u2 * um1 * um1 * inv;
  } else {
    *sw = T(0);
    *dsw = T(0);
  }
}

template <typename T>
__device__ __forceinline__ T dtanh(T x);
template <>
__device__ __forceinline__ float dtanh<float>(float x) { return tanhf(x); }
template <>
__device__ __forceinline__ double dtanh<double>(double x) { return tanh(x); }

template <typename T>
__device__ __forceinline__ T dsqrt(T x);
template <>
__device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }
template <>
__device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }

template <typename T>
__device__ __forceinline__ T dexp(T x);
template <>
__device__ __forceinline__ float dexp<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double dexp<double>(double x) { return exp(x); }

// ------------------------------------------------------------------ exact sums
// Sums whose order depends on the skin list (and so on when it was last
// rebuilt) are accumulated in 128-bit fixed point at 2^-80 resolution: integer
// addition is associative, so the result is the same for any order.
constexpr double kFix = 0x1p80, kUnfix = 0x1p-80;

// v * 2^80 as a 128-bit integer, truncated toward zero; `bad` is set for a
// value that is not finite or too large (|v| >= 2^46) to be represented.
__device__ __forceinline__ __int128 to_fixed(double v, bool* bad) {
  const double a = fabs(v);
  if (!(a < 0x1p46)) {
    *bad = true;
    return 0;
  }
  const double s = a * kFix;                // exact: power-of-two scaling
  const double hi = floor(s * 0x1p-64);     // exact, < 2^62
  const double lo = s - hi * 0x1p64;        // exact, 0 <= lo < 2^64
  const unsigned __int128 u =
      ((unsigned __int128)(unsigned long long)hi << 64) | (unsigned long long)lo;
  return v < 0 ? -(__int128)u : (__int128)u;
}

// The same conversions from the bit patterns, in integer arithmetic only
// (this part's FP64 pipe retires about two lanes per clock per SM): for a
// binary floating-point value m 2^(e - bias - mbits), v 2^80 truncated toward
// zero is m shifted by e - bias - mbits + 80.  Same results as to_fixed.
__device__ __forceinline__ __int128 shift_fixed(unsigned long long m, int sh, bool neg) {
  unsigned __int128 u;
  if (sh >= 0) u = (unsigned __int128)m << sh;
  else u = sh > -64 ? (unsigned __int128)(m >> -sh) : 0;
  return neg ? -(__int128)u : (__int128)u;
}
__device__ __forceinline__ __int128 to_fixed_f32(float v, bool* bad) {
  const unsigned b = __float_as_uint(v);
  const int e = (int)((b >> 23) & 0xffu);
  if (e >= 127 + 46) {   // |v| >= 2^46, infinite or NaN
    *bad = true;
    return 0;
  }
  const unsigned long long m = (b & 0x7fffffu) | (e ? 0x800000u : 0u);
  return shift_fixed(m, (e ? e : 1) - 127 - 23 + 80, (b >> 31) != 0);
}
__device__ __forceinline__ __int128 to_fixed_f64(double v, bool* bad) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ffu);
  if (e >= 1023 + 46) {
    *bad = true;
    return 0;
  }
  const unsigned long long m = (b & 0xfffffffffffffull) | (e ? (1ull << 52) : 0ull);
  return shift_fixed(m, (e ? e : 1) - 1023 - 52 + 80, (b >> 63) != 0);
}

// a + b in 128-bit fixed point; *bad is set when the sum leaves the signed
// 128-bit range (|sum| >= 2^47 at 2^-80 resolution), where it would wrap
__device__ __forceinline__ __int128 fixed_add(__int128 a, __int128 b, bool* bad) {
  const __int128 r = (__int128)((unsigned __int128)a + (unsigned __int128)b);
  *bad |= ((a ^ r) & (b ^ r)) < 0;
  return r;
}

__device__ __forceinline__ __int128 warp_sum_fixed(__int128 v, bool* bad) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)v, o);
    const long long hi = __shfl_xor_sync(0xffffffffu, (long long)(v >> 64), o);
    v = fixed_add(v, (__int128)(((unsigned __int128)(unsigned long long)hi << 64) | lo), bad);
  }
  return v;
}

// the 128-bit sum as a double (deterministic; two roundings at most)
__device__ __forceinline__ double from_fixed(__int128 v) {
  const long long hi = (long long)(v >> 64);
  const unsigned long long lo = (unsigned long long)v;
  return ((double)hi * 0x1p64 + (double)lo) * kUnfix;
}

__device__ __forceinline__ double quiet_nan() { return __longlong_as_double(0x7ff8000000000000LL); }

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace dp
