// Plain (unfused) graph-family potential, FP32 / FP64, one simple kernel per
// operation.  The paper (Sec. II) describes DPA3 as a GNN whose line-graph
// series carries bond and angle representations; the library's reading:
//
//   init   n_i = W_type[t_i];  e_ip = tanh(s_ip w_e + b_e),  s = sw(r)/r
//   layer  (a) u = n Wm;  m_i = (1/nmax) sum_p sw_ip (e_ip * u_j);
//              n_i <- n_i + tanh([n_i, m_i] Wn + bn)
//          (b) e_ip <- e_ip + tanh(n_i Wa + n_j Wb + e_ip Wc + be)
//          (c) q = e Wp; for the angle slots p (r < rca, at most na, nearest):
//              a_ip = sum_l Wphi[l] * (1/na) sum_{k != p} swa_ip swa_ik P_l(c_pk) q_ik
//              e_ip <- e_ip + swa_ip tanh(a_ip Wq + bq)
//   energy e_i = fitting_{t_i}(n_i)
//
// and the hand-written adjoint.  Gradients that flow to a neighbour's node
// (through u_j and n_j Wb) are gathered over the neighbour's incoming slots
// in a fixed order (skin list + mirror index), so results are reproducible.
#include <math.h>

#include <string>
#include <algorithm>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "gemm.cuh"
#include "mp.cuh"
#include "gemm_tc.cuh"
#include "kernels.cuh"
#include "model.h"

namespace dp {
namespace gf {

// slot of element idx of a (slots x ed) array: a shift when ed is a power of
// two (ed_shift >= 0), else a division
__device__ __forceinline__ long long slot_of(long long idx, int ed, int ed_shift) {
  return ed_shift >= 0 ? (idx >> ed_shift) : idx / ed;
}

// four consecutive values (16- or 32-byte aligned) as vector loads
__device__ __forceinline__ void ld4(const float* p, float* v) {
  const float4 u = *reinterpret_cast<const float4*>(p);
  v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w;
}
__device__ __forceinline__ void ld4(const double* p, double* v) {
  const double2 u = reinterpret_cast<const double2*>(p)[0], w = reinterpret_cast<const double2*>(p)[1];
  v[0] = u.x; v[1] = u.y; v[2] = w.x; v[3] = w.y;
}
// two consecutive values (8- or 16-byte aligned) as one vector load
__device__ __forceinline__ void ld2(const float* p, float* v) {
  const float2 u = *reinterpret_cast<const float2*>(p);
  v[0] = u.x; v[1] = u.y;
}
__device__ __forceinline__ void ld2(const double* p, double* v) {
  const double2 u = *reinterpret_cast<const double2*>(p);
  v[0] = u.x; v[1] = u.y;
}
__device__ __forceinline__ void st4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double* v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
// the mixed form keeps some per-slot arrays in 16 bits, in the type of its
// tensor-core operands (FP16; BF16 when built with DP_GF_BF16)
#ifdef DP_GF_BF16
using gf16_t = __nv_bfloat16;
#else
using gf16_t = __half;
#endif
// four consecutive 16-bit values (8-byte aligned) as FP32, and back (rounded)
__device__ __forceinline__ void ld4(const __half* p, float* v) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void ld4(const __nv_bfloat16* p, float* v) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
// two 16-bit values as raw bits, and their FP32 values (a batch of loads is
// issued before any conversion: in-order issue would otherwise make the warp
// wait for each load at its conversion)
__device__ __forceinline__ uint32_t ld2raw(const __half* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ uint32_t ld2raw(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}
__device__ __forceinline__ float2 raw2f(uint32_t u, const __half*) {
  return __half22float2(*reinterpret_cast<const __half2*>(&u));
}
__device__ __forceinline__ float2 raw2f(uint32_t u, const __nv_bfloat16*) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
}
__device__ __forceinline__ void st4(__half* p, const float* v) {
  const __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
  *reinterpret_cast<uint2*>(p) = make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
}
__device__ __forceinline__ void st4(__nv_bfloat16* p, const float* v) {
  const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
  *reinterpret_cast<uint2*>(p) = make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
}


// ------------------------------------------------------------------ kernels
// geometry of every slot: distance, switches, s = sw/r, unit vector
template <typename T>
__global__ void k_env(long long P, int nmax, int na, const int* __restrict__ sel_j,
                      const double* __restrict__ sel_r, double rs, double rc, double rsa,
                      double rca, T* __restrict__ d, T* __restrict__ sw, T* __restrict__ dsw,
                      T* __restrict__ sa, T* __restrict__ dsa, T* __restrict__ s,
                      T* __restrict__ rh) {
  long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= P) return;
  int p = (int)(e % nmax);
  if (sel_j[e] < 0) {
    d[e] = T(1); sw[e] = dsw[e] = sa[e] = dsa[e] = s[e] = T(0);
    rh[3 * e] = rh[3 * e + 1] = rh[3 * e + 2] = T(0);
    return;
  }
  double r[3] = {sel_r[3 * e], sel_r[3 * e + 1], sel_r[3 * e + 2]};
  double dd = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  T a, b;
  smooth_switch((T)dd, (T)rs, (T)rc, &a, &b);
  d[e] = (T)dd; sw[e] = a; dsw[e] = b; s[e] = a / (T)dd;
  for (int q = 0; q < 3; ++q) rh[3 * e + q] = (T)(r[q] / dd);
  if (dd < rca && p < na) {
    smooth_switch((T)dd, (T)rsa, (T)rca, &a, &b);
    sa[e] = a; dsa[e] = b;
  } else {
    sa[e] = dsa[e] = T(0);
  }
}

template <typename T, typename E = T>   // E: storage of the edge state (T, or 16 bits)
__global__ void k_init(int n, int nmax, int nd, int ed, const int* __restrict__ types,
                       const int* __restrict__ sel_j, const T* __restrict__ s,
                       const T* __restrict__ Wt, const T* __restrict__ we,
                       const T* __restrict__ be0, T* __restrict__ node, E* __restrict__ edge) {
  int i = blockIdx.x;
  for (int c = threadIdx.x; c < nd; c += blockDim.x) node[(size_t)i * nd + c] = Wt[types[i] * nd + c];
  if ((ed & 3) == 0) {   // four columns per thread, one 16-byte store
    const int eq = ed >> 2;
    for (int idx = threadIdx.x; idx < nmax * eq; idx += blockDim.x) {
      const int p = idx / eq, c = (idx - p * eq) << 2;
      const size_t e = (size_t)i * nmax + p;
      T v[4] = {T(0), T(0), T(0), T(0)};
      if (sel_j[e] >= 0) {
        const T se = s[e];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = dtanh(se * we[c + q] + be0[c + q]);
      }
      st4(edge + e * ed + c, v);
    }
    return;
  }
  for (int idx = threadIdx.x; idx < nmax * ed; idx += blockDim.x) {
    int p = idx / ed, c = idx % ed;
    size_t e = (size_t)i * nmax + p;
    edge[e * ed + c] = E(sel_j[e] >= 0 ? dtanh(s[e] * we[c] + be0[c]) : T(0));
  }
}

// m_i = (1/nmax) sum_p sw_ip e_ip * u_j(p); one block per atom
template <typename T>
__global__ void k_msg(int nmax, int ed, T inv_nmax, const int* __restrict__ sel_j,
                      const T* __restrict__ sw, const T* __restrict__ edge,
                      const T* __restrict__ u, T* __restrict__ m) {
  int i = blockIdx.x;
  for (int c = threadIdx.x; c < ed; c += blockDim.x) {
    T acc = T(0);
    for (int p = 0; p < nmax; ++p) {
      size_t e = (size_t)i * nmax + p;
      int j = sel_j[e];
      if (j < 0) break;
      acc += sw[e] * edge[e * ed + c] * u[(size_t)j * ed + c];
    }
    m[(size_t)i * ed + c] = acc * inv_nmax;
  }
}

// The same, one warp per atom: lane l owns columns 2l, 2l + 1 (+ 64 k), and
// four slots' rows are read before any is summed (a 16-bit edge row as raw
// bits, converted at the sum); the sum runs over the slots in order and stops
// at the first empty one, as above (the kept slots are a prefix of the
// list).  ed even.  Eight slots per batch for 16-bit rows measured slower.
template <typename T, typename E = T>   // E: storage of the edge state
__global__ void k_msg_warp(int n, int nmax, int ed, T inv_nmax, const int* __restrict__ sel_j,
                           const T* __restrict__ sw, const E* __restrict__ edge,
                           const T* __restrict__ u, T* __restrict__ m) {
  constexpr bool k16 = sizeof(E) == 2;
  constexpr int B = 4;
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  const size_t base = (size_t)i * nmax;
  for (int c = 2 * lane; c < ed; c += 64) {
    T a0 = T(0), a1 = T(0);
    bool done = false;
    for (int p = 0; p < nmax && !done; p += B) {
      int jj[B];
      T sv[B], e0[B], e1[B], u0[B], u1[B];
      uint32_t er[B];   // 16-bit edge rows, converted below
#pragma unroll
      for (int q = 0; q < B; ++q) {
        jj[q] = p + q < nmax ? sel_j[base + p + q] : -1;
        if (jj[q] >= 0) {
          const size_t e = base + p + q;
          T uv[2];
          sv[q] = sw[e];
          if constexpr (k16) {
            er[q] = ld2raw(edge + e * ed + c);
          } else {
            T ev[2];
            ld2(edge + e * ed + c, ev);
            e0[q] = ev[0]; e1[q] = ev[1];
          }
          ld2(u + (size_t)jj[q] * ed + c, uv);
          u0[q] = uv[0]; u1[q] = uv[1];
        }
      }
#pragma unroll
      for (int q = 0; q < B; ++q) {
        if (jj[q] < 0) {
          done = true;
          break;
        }
        if constexpr (k16) {
          const float2 ev = raw2f(er[q], edge);
          e0[q] = ev.x; e1[q] = ev.y;
        }
        a0 += sv[q] * e0[q] * u0[q];
        a1 += sv[q] * e1[q] * u1[q];
      }
    }
    m[(size_t)i * ed + c] = a0 * inv_nmax;
    m[(size_t)i * ed + c + 1] = a1 * inv_nmax;
  }
}

template <typename T>
__global__ void k_add(long long n, const T* __restrict__ a, const T* __restrict__ b,
                      T* __restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] + b[i];
}

template <typename T>
__global__ void k_copy(long long n, const T* __restrict__ a, T* __restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i];
}

// (b): v = tanh(A_i + B_j + C_e + be), e1 = e + v on real slots
template <typename T>
__global__ void k_edge(long long P, int nmax, int ed, int ed_shift, const int* __restrict__ sel_j,
                       const T* __restrict__ Ai, const T* __restrict__ Bj,
                       const T* __restrict__ Ce, const T* __restrict__ be,
                       const T* __restrict__ e_in, T* __restrict__ v, T* __restrict__ e1) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P * ed) return;
  long long e = slot_of(idx, ed, ed_shift);
  int c = (int)(idx - e * ed);
  int j = sel_j[e];
  if (j < 0) {
    v[idx] = T(0);
    e1[idx] = T(0);
    return;
  }
  long long i = e / nmax;
  T y = dtanh(Ai[i * ed + c] + Bj[(long long)j * ed + c] + Ce[idx] + be[c]);
  v[idx] = y;
  e1[idx] = e_in[idx] + y;
}

constexpr int kMaxNa = 64;

// acc[i] += c[i] * x for i < N (N even); FP32 as packed pair instructions
template <int N>
__device__ __forceinline__ void fma_n(double* acc, const double* c, double x) {
#pragma unroll
  for (int i = 0; i < N; ++i) acc[i] += c[i] * x;
}
template <int N>
__device__ __forceinline__ void fma_n(float* acc, const float* c, float x) {
#pragma unroll
  for (int h = 0; h < N; h += 2)
    asm("{\n\t.reg .b64 ra, rb, rc;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %4};\n\tmov.b64 rc, {%0, %1};\n\t"
        "fma.rn.f32x2 rc, ra, rb, rc;\n\tmov.b64 {%0, %1}, rc;\n\t}"
        : "+f"(acc[h]), "+f"(acc[h + 1])
        : "f"(c[h]), "f"(c[h + 1]), "f"(x));
}
// sum_i a[i] b[i] for i < N (N even), as two interleaved partial sums
template <int N, typename T>
__device__ __forceinline__ T dot_n(const T* a, const T* b) {
  T s0 = T(0), s1 = T(0);
#pragma unroll
  for (int i = 0; i < N; i += 2) {
    s0 += a[i] * b[i];
    s1 += a[i + 1] * b[i + 1];
  }
  return s0 + s1;
}

// Angle channel by monomial sums.  The angle sums weight q_k by
// sum_l Wphi[l][c] P_l(u_p . u_k) for l <= 3 (unit vectors u).  In the power
// basis P_l(x) = sum_n A_ln x^n (P2 = 1.5 x^2 - 0.5, P3 = 2.5 x^3 - 1.5 x),
// so the weight is sum_n beta_n[c] x^n with beta_n[c] = sum_l Wphi[l][c] A_ln,
// and (u . v)^n = sum_{|m| = n} mult(m) u^m v^m over the monomials
// u^m = ux^mx uy^my uz^mz of degree n (multinomial weights mult(m) = n! /
// (mx! my! mz!)).  Hence, for an atom with angle slots k < nang,
//   sum_{k != p} sa_k q_k[c] sum_n beta_n[c] (u_p . u_k)^n
//     = sum_m u_p^m YB_m[c] - sa_p q_p[c] sum_n beta_n[c] (u_p . u_p)^n,
//   YB_m[c] = mult(m) beta_|m|[c] Y_m[c],   Y_m[c] = sum_k sa_k u_k^m q_k[c]
// (the k = p term is taken out of the full sum).  This is an identity between
// polynomials in the unit-vector components, so its derivatives are those of
// the pairwise form as well; it costs two passes of 20 multiply-adds per
// (slot, column) instead of four per (slot, partner, column).
constexpr int kMono = 20;
// sa-weighted monomials are stored in two halves of 10 at offsets 0 and 12 of
// a 24-wide row, so that each half starts on a 16-byte boundary
constexpr int kMonoSa = 24;
__host__ __device__ constexpr int monosa_at(int m) { return m < 10 ? m : m + 2; }
// the 20 monomials of degree <= 3 in this order: 1 | x y z | xx yy zz xy xz yz |
// xxx yyy zzz xxy xxz xyy yyz xzz yzz xyz
__host__ __device__ constexpr int mono_deg(int m) { return m == 0 ? 0 : m < 4 ? 1 : m < 10 ? 2 : 3; }
__host__ __device__ constexpr int mono_mult(int m) {
  return m == 19 ? 6 : (m >= 13 ? 3 : (m >= 7 && m < 10 ? 2 : 1));
}
template <typename T>
__device__ __forceinline__ void monomials(T x, T y, T z, T* m) {
  m[0] = T(1); m[1] = x; m[2] = y; m[3] = z;
  m[4] = x * x; m[5] = y * y; m[6] = z * z; m[7] = x * y; m[8] = x * z; m[9] = y * z;
  m[10] = m[4] * x; m[11] = m[5] * y; m[12] = m[6] * z; m[13] = m[4] * y; m[14] = m[4] * z;
  m[15] = x * m[5]; m[16] = m[5] * z; m[17] = x * m[6]; m[18] = y * m[6]; m[19] = m[7] * z;
}
// d/du of sum_m g[m] u^m
template <typename T>
__device__ __forceinline__ void monomial_grad(T x, T y, T z, const T* g, T* d) {
  d[0] = g[1] + T(2) * x * g[4] + y * g[7] + z * g[8] + T(3) * x * x * g[10] + T(2) * x * y * g[13] +
         T(2) * x * z * g[14] + y * y * g[15] + z * z * g[17] + y * z * g[19];
  d[1] = g[2] + T(2) * y * g[5] + x * g[7] + z * g[9] + T(3) * y * y * g[11] + x * x * g[13] +
         T(2) * x * y * g[15] + T(2) * y * z * g[16] + z * z * g[18] + x * z * g[19];
  d[2] = g[3] + T(2) * z * g[6] + x * g[8] + y * g[9] + T(3) * z * z * g[12] + x * x * g[14] +
         y * y * g[16] + T(2) * x * z * g[17] + T(2) * y * z * g[18] + x * y * g[19];
}
template <typename T>
__device__ __forceinline__ void ld20(const T* p, T* v) {
#pragma unroll
  for (int i = 0; i < kMono; i += 4) ld4(p + i, v + i);
}

// Angle-channel blocks: kAngThreads threads per atom.  Column phases give
// each column of a 64-column block two threads (kAngCols = kAngThreads / 2).
constexpr int kAngThreads = 128, kAngCols = kAngThreads / 2;

// beta[4 c + n] = sum_l Wphi[l][c] A_ln (Wphi stored [4][ed])
template <typename T>
__device__ void angle_beta(T* beta, const T* Wphi, int ed) {
  for (int c = threadIdx.x; c < ed; c += blockDim.x) {
    const T w0 = Wphi[c], w1 = Wphi[ed + c], w2 = Wphi[2 * ed + c], w3 = Wphi[3 * ed + c];
    beta[4 * c] = w0 - T(0.5) * w2;
    beta[4 * c + 1] = w1 - T(1.5) * w3;
    beta[4 * c + 2] = T(1.5) * w2;
    beta[4 * c + 3] = T(2.5) * w3;
  }
}
// per angle slot s < nang: mono[s] = u_s^m, monosa[s] = sa_s u_s^m (24-wide
// rows), and xpow[s] = (u_s . u_s)^n, n < 4
template <typename T>
__device__ void angle_mono(T* mono, T* monosa, T* xpow, int nang, const T* gsa, const T* grh) {
  for (int s = threadIdx.x; s < nang; s += blockDim.x) {
    T m[kMono];
    const T x = grh[3 * s], y = grh[3 * s + 1], z = grh[3 * s + 2], sp = gsa[s];
    monomials(x, y, z, m);
    const T xx = m[4] + m[5] + m[6];
#pragma unroll
    for (int i = 0; i < kMono; ++i) {
      mono[s * kMono + i] = m[i];
      monosa[s * kMonoSa + monosa_at(i)] = sp * m[i];
    }
    xpow[4 * s] = T(1);
    xpow[4 * s + 1] = xx;
    xpow[4 * s + 2] = xx * xx;
    xpow[4 * s + 3] = xx * xx * xx;
  }
}
// One half (monomials 10 H .. 10 H + 9) of the weighted sums of column c over
// the angle slots: out[c][m] = scale mult(m) beta_|m|[c] sum_k monosa[k][m] x_k[c]
// for NX arrays x at once (the monomials are read once for all of them)
template <int H, int NX, typename T>
__device__ __forceinline__ void angle_ysum(T* const* out, const T* beta, const T* monosa, int nang,
                                           const T* const* xs, int ld, int c, const T* scale) {
  T acc[NX][10];
#pragma unroll
  for (int x = 0; x < NX; ++x)
#pragma unroll
    for (int j = 0; j < 10; ++j) acc[x][j] = T(0);
  for (int k = 0; k < nang; ++k) {
    T w[10];
    const T* row = monosa + k * kMonoSa + 12 * H;
    ld4(row, w);
    ld4(row + 4, w + 4);
    ld2(row + 8, w + 8);
#pragma unroll
    for (int x = 0; x < NX; ++x) fma_n<10>(acc[x], w, xs[x][k * ld + c]);
  }
  T b[4];
  ld4(beta + 4 * c, b);
#pragma unroll
  for (int x = 0; x < NX; ++x)
#pragma unroll
    for (int j = 0; j < 10; ++j)
      out[x][c * kMono + 10 * H + j] = scale[x] * T(mono_mult(10 * H + j)) * b[mono_deg(10 * H + j)] * acc[x][j];
}

// Asynchronous element copies global -> shared (cp.async, completion per
// thread by commit group; a block barrier then publishes them)
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The angle kernels are persistent: a block loops over atoms i = blockIdx.x,
// + gridDim.x, ... and, while it works on one atom, copies the next atom's
// slot switches (na) and unit vectors (3 na) into the other of two buffers.
// The slots' q and da rows are read from global memory where they are used
// (through L1): staging them in shared memory as well cost resident blocks
// and made both kernels slower.
template <typename T>
struct AngleBuf {
  T *sa, *rh;
};
template <typename T>
__device__ __forceinline__ AngleBuf<T> angle_buf(T* start, int na, int b) {
  T* p = start + (size_t)b * 4 * na;
  AngleBuf<T> u;
  u.sa = p;
  u.rh = p + na;
  return u;
}
// start the copies of atom i's slot data into u (one commit group per thread)
template <typename T>
__device__ __forceinline__ void angle_fetch(const AngleBuf<T>& u, int ca, long long base, const T* sa,
                                            const T* rh) {
  if (threadIdx.x < ca) cp_async_elem(u.sa + threadIdx.x, sa + base + threadIdx.x);
  for (int idx = threadIdx.x; idx < 3 * ca; idx += blockDim.x) cp_async_elem(u.rh + idx, rh + 3 * base + idx);
  cp_async_commit();
}
// Next atom's copies started, this atom's awaited; returns the angle count
// (the slots with swa > 0, a prefix of the nearest-first list), counted by
// the block barrier that also publishes the copies.  Thread t < ca copied
// switch t itself, so it may read it before the barrier.
template <typename T>
__device__ __forceinline__ int angle_next(const AngleBuf<T>& cur, const AngleBuf<T>& nxt, int i, int n,
                                          int nmax, int ca, const T* sa, const T* rh) {
  const int nx = i + gridDim.x;
  if (nx < n) {
    angle_fetch(nxt, ca, (long long)nx * nmax, sa, rh);
    cp_async_wait<1>();
  } else {
    cp_async_wait<0>();
  }
  return __syncthreads_count(threadIdx.x < ca && cur.sa[threadIdx.x] > T(0));
}

// (c) forward: a_p[c] = (1/na) sa_p sum_{k != p} sa_k q_k[c] sum_l Wphi[l][c] P_l(u_p . u_k)
// for the angle slots p of each atom, by the monomial sums above.  q and a
// hold the angle rows only: slot p < ca of atom i at row i ca + p (ca =
// min(na, nmax)); rows from the atom's angle count up to ca get a = 0.
// Shared memory: beta (ed x 4), the slots' monomials, sa-weighted monomials
// and (u . u)^n (na x 20, na x 24, na x 4), YB (ed x 20), then two slot-data
// buffers.
template <typename T>
__global__ void __launch_bounds__(kAngThreads) k_angle(int n, int nmax, int na, int ca, int ed, T inv_na,
                                                       const T* __restrict__ sa,
                                                       const T* __restrict__ rh,
                                                       const T* __restrict__ q,
                                                       const T* __restrict__ Wphi,
                                                       T* __restrict__ a) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* beta = reinterpret_cast<T*>(sm_raw);
  T* mono = beta + (size_t)ed * 4;
  T* monosa = mono + (size_t)na * kMono;
  T* xpow = monosa + (size_t)na * kMonoSa;
  T* YB = xpow + (size_t)na * 4;
  T* bufs = YB + (size_t)ed * kMono;
  angle_beta(beta, Wphi, ed);
  int i = blockIdx.x;
  if (i < n) angle_fetch(angle_buf(bufs, na, 0), ca, (long long)i * nmax, sa, rh);
  const int cl = threadIdx.x % kAngCols, half = threadIdx.x / kAngCols;
  for (int it = 0; i < n; ++it, i += gridDim.x) {
    const AngleBuf<T> cur = angle_buf(bufs, na, it & 1);
    const int nang = angle_next(cur, angle_buf(bufs, na, (it + 1) & 1), i, n, nmax, ca, sa, rh);
    const long long abase = (long long)i * ca;
    const T* qs = q + abase * ed;
    const int ld = ed;
    angle_mono(mono, monosa, xpow, nang, cur.sa, cur.rh);
    __syncthreads();
    for (int c = cl; c < ed; c += kAngCols) {   // YB: half of the monomials per thread
      T* const out[1] = {YB};
      const T* const xs[1] = {qs};
      const T one[1] = {T(1)};
      if (half == 0) angle_ysum<0, 1>(out, beta, monosa, nang, xs, ld, c, one);
      else angle_ysum<1, 1>(out, beta, monosa, nang, xs, ld, c, one);
    }
    __syncthreads();
    for (int c = cl; c < ed; c += kAngCols) {   // a: every second slot per thread
      T yb[kMono], b[4];
      ld20(YB + c * kMono, yb);
      ld4(beta + 4 * c, b);
      for (int p = half; p < nang; p += 2) {
        T m[kMono], xp[4];
        ld20(mono + p * kMono, m);
        ld4(xpow + 4 * p, xp);
        const T z = b[0] + b[1] * xp[1] + b[2] * xp[2] + b[3] * xp[3];
        const T sp = cur.sa[p];
        a[(abase + p) * ed + c] = inv_na * sp * (dot_n<kMono>(m, yb) - sp * qs[p * ld + c] * z);
      }
    }
    for (int idx = threadIdx.x; idx < (ca - nang) * ed; idx += blockDim.x)
      a[(abase + nang) * ed + idx] = T(0);
    __syncthreads();   // the monomials, YB and this buffer are rewritten next
  }
}

// e += swa * t on the angle rows (t by angle row i ca + p, e and swa by slot
// i nmax + p; the other slots keep e_{l+1} = e1, swa being 0 there)
template <typename T>
__global__ void k_angle_out(long long PA, int ed, int ed_shift, int nmax, int ca,
                            const T* __restrict__ sa, const T* __restrict__ t, T* __restrict__ e) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= PA * ed) return;
  const long long m = slot_of(idx, ed, ed_shift), i = m / ca;
  const long long row = i * nmax + (m - i * ca);
  const int c = (int)(idx - m * ed);
  e[row * ed + c] += sa[row] * t[idx];
}

// e_i = y3 . F4 + c4 (FP64) and delta3
template <typename T>
__global__ void k_fit_out(int n, int f3, const int* __restrict__ types, const T* __restrict__ y3,
                          const T* __restrict__ F4, const T* __restrict__ c4,
                          double* __restrict__ atom_e, T* __restrict__ d3,
                          const unsigned char* __restrict__ seed) {
  long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (wid >= n) return;
  int a = (int)wid, t = types[a];
  const T sd = seed && !seed[a] ? T(0) : T(1);   // energy seed of the adjoint
  double acc = 0.0;
  for (int b = lane; b < f3; b += 32) {
    T y = y3[(long long)a * f3 + b], w = F4[t * f3 + b];
    acc += (double)y * (double)w;
    d3[(long long)a * f3 + b] = sd * w * (T(1) - y * y);
  }
  acc = warp_sum(acc);
  if (lane == 0) atom_e[a] = acc + (double)c4[t];
}

// ------------------------------------------------------------------ adjoint kernels
// (c): dsa += de . t, dz = de * swa * (1 - t^2) on the angle rows (t, dz by
// angle row m = i ca + p; de, swa, dsa by slot i nmax + p)
template <typename T>
__global__ void k_angle_out_bwd(long long PA, int ed, int nmax, int ca, const T* __restrict__ sa,
                                const T* __restrict__ t, const T* __restrict__ de,
                                T* __restrict__ dz, T* __restrict__ dsa_e) {
  long long m = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (m >= PA) return;
  const long long i = m / ca, e = i * nmax + (m - i * ca);
  T s = sa[e];
  T acc = T(0);
  for (int c = lane; c < ed; c += 32) {
    T tv = t[m * ed + c], g = de[e * ed + c];
    acc += g * tv;
    dz[m * ed + c] = g * s * (T(1) - tv * tv);
  }
  acc = warp_sum(acc);
  if (lane == 0 && s > T(0)) dsa_e[e] += acc;
}
// The same with 16 threads per angle row, four columns each (ed a multiple
// of 4); the dsa sum closes with a fixed-order reduction over the 16 lanes.
template <typename T, typename Z = T>   // Z: storage of dz (T, or 16 bits)
__global__ void k_angle_out_bwd4(long long PA, int ed, int nmax, int ca, const T* __restrict__ sa,
                                 const T* __restrict__ t, const T* __restrict__ de,
                                 Z* __restrict__ dz, T* __restrict__ dsa_e) {
  const long long m = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 4;
  const int l16 = threadIdx.x & 15;
  if (m >= PA) return;   // the whole 16-lane group leaves together
  const unsigned mask = 0xFFFFu << (threadIdx.x & 16);
  const int i32 = (int)m / ca;   // angle rows < 2^31
  const long long i = i32, e = i * nmax + (m - i * ca);
  const T s = sa[e];
  T acc = T(0);
  for (int c = 4 * l16; c < ed; c += 64) {
    T tv[4], g[4], z[4];
    ld4(t + m * ed + c, tv);
    ld4(de + e * ed + c, g);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      acc += g[q] * tv[q];
      z[q] = g[q] * s * (T(1) - tv[q] * tv[q]);
    }
    st4(dz + m * ed + c, z);
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) acc += __shfl_xor_sync(mask, acc, o);
  if (l16 == 0 && s > T(0)) dsa_e[e] += acc;
}

// (c) adjoint of a_p for each atom, with g_p[c] = dE/da_p[c] (da) and the
// forward's YB recomputed:
//   dY_m[c] = (1/na) mult(m) beta_|m|[c] sum_p sa_p u_p^m g_p[c]            (dYB)
//   dq_k[c] = sa_k (sum_m u_k^m dY_m[c] - (1/na) sa_k g_k[c] Z_k[c]),
//             Z_k[c] = sum_n beta_n[c] (u_k . u_k)^n
// and per slot s, from H_m(s) = sum_c g_s[c] YB_m[c], K_m(s) = sum_c q_s[c] dY_m[c]
// and D_n(s) = sum_c g_s[c] q_s[c] beta_n[c]:
//   dE/dsa_s  = (1/na) (sum_m u_s^m H_m - 2 sa_s sum_n D_n x^n) + sum_m u_s^m K_m
//   dE/du_s^m = sa_s ((1/na) H_m + K_m)
//   dE/dx     = -(1/na) sa_s^2 (D_1 + 2 D_2 x + 3 D_3 x^2),   x = u_s . u_s
// dE/du_s then follows by differentiating the monomials (plus 2 u_s dE/dx).
// q, da and dq hold the angle rows only (row i ca + p).  Shared memory: beta,
// the monomials (as in the forward), YB and dYB (ed x 20 each), the per-slot
// sums H, K, D (na x 44), then two slot-data buffers.
template <typename T, typename DQ = T>   // DQ: storage of dq (T, or 16 bits)
__global__ void __launch_bounds__(kAngThreads) k_angle_bwd(int n, int nmax, int na, int ca, int ed, T inv_na,
                                                           const T* __restrict__ sa,
                                                           const T* __restrict__ rh,
                                                           const T* __restrict__ q,
                                                           const T* __restrict__ Wphi,
                                                           const T* __restrict__ da,
                                                           DQ* __restrict__ dq, T* __restrict__ dsa_e,
                                                           T* __restrict__ drh) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  constexpr int kHKD = 2 * kMono + 4;
  T* beta = reinterpret_cast<T*>(sm_raw);
  T* mono = beta + (size_t)ed * 4;
  T* monosa = mono + (size_t)na * kMono;
  T* xpow = monosa + (size_t)na * kMonoSa;
  T* YB = xpow + (size_t)na * 4;
  T* dYB = YB + (size_t)ed * kMono;
  T* hkd = dYB + (size_t)ed * kMono;
  T* bufs = hkd + (size_t)na * kHKD;
  angle_beta(beta, Wphi, ed);
  int i = blockIdx.x;
  if (i < n) angle_fetch(angle_buf(bufs, na, 0), ca, (long long)i * nmax, sa, rh);
  const int cl = threadIdx.x % kAngCols, half = threadIdx.x / kAngCols;
  for (int it = 0; i < n; ++it, i += gridDim.x) {
    const AngleBuf<T> cur = angle_buf(bufs, na, it & 1);
    const int nang = angle_next(cur, angle_buf(bufs, na, (it + 1) & 1), i, n, nmax, ca, sa, rh);
    const long long base = (long long)i * nmax, abase = (long long)i * ca;
    const T* das = da + abase * ed;
    const T* qs = q + abase * ed;
    const int ld = ed;
    angle_mono(mono, monosa, xpow, nang, cur.sa, cur.rh);
    __syncthreads();
    for (int c = cl; c < ed; c += kAngCols) {   // YB and dYB, half of the monomials per thread
      T* const out[2] = {YB, dYB};
      const T* const xs[2] = {qs, das};
      const T sc[2] = {T(1), inv_na};
      if (half == 0) angle_ysum<0, 2>(out, beta, monosa, nang, xs, ld, c, sc);
      else angle_ysum<1, 2>(out, beta, monosa, nang, xs, ld, c, sc);
    }
    __syncthreads();
    for (int c = cl; c < ed; c += kAngCols) {   // dq: every second slot per thread
      T dyb[kMono], b[4];
      ld20(dYB + c * kMono, dyb);
      ld4(beta + 4 * c, b);
      for (int p = half; p < nang; p += 2) {
        T m[kMono], xp[4];
        ld20(mono + p * kMono, m);
        ld4(xpow + 4 * p, xp);
        const T z = b[0] + b[1] * xp[1] + b[2] * xp[2] + b[3] * xp[3];
        const T sp = cur.sa[p];
        dq[(abase + p) * ed + c] = DQ(sp * (dot_n<kMono>(m, dyb) - inv_na * sp * das[p * ld + c] * z));
      }
    }
    for (int idx = threadIdx.x; idx < (ca - nang) * ed; idx += blockDim.x)
      dq[(abase + nang) * ed + idx] = DQ(T(0));
    // H, K (and D) of two slots and four monomials per thread, summed over the
    // columns in order
    const int npair = (nang + 1) >> 1;
    for (int tile = threadIdx.x; tile < npair * 5; tile += blockDim.x) {
      const int p0 = 2 * (tile / 5), mb = 4 * (tile % 5);
      const int p1 = min(p0 + 1, nang - 1);
      T h[2][4], k[2][4], d[2][4];
#pragma unroll
      for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int j = 0; j < 4; ++j) h[x][j] = k[x][j] = d[x][j] = T(0);
      auto column = [&](int c, const T* g, const T* qv) {
        T yb[4], dy[4];
        ld4(YB + c * kMono + mb, yb);
        ld4(dYB + c * kMono + mb, dy);
#pragma unroll
        for (int x = 0; x < 2; ++x) {
          fma_n<4>(h[x], yb, g[x]);
          fma_n<4>(k[x], dy, qv[x]);
        }
        if (mb == 0) {
          T b[4];
          ld4(beta + 4 * c, b);
#pragma unroll
          for (int x = 0; x < 2; ++x) fma_n<4>(d[x], b, g[x] * qv[x]);
        }
      };
      if ((ed & 3) == 0) {   // the two slots' rows four columns per load
        for (int c = 0; c < ed; c += 4) {
          T g4[2][4], q4[2][4];
          ld4(das + p0 * ld + c, g4[0]);
          ld4(das + p1 * ld + c, g4[1]);
          ld4(qs + p0 * ld + c, q4[0]);
          ld4(qs + p1 * ld + c, q4[1]);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const T g[2] = {g4[0][u], g4[1][u]}, qv[2] = {q4[0][u], q4[1][u]};
            column(c + u, g, qv);
          }
        }
      } else {
        for (int c = 0; c < ed; ++c) {
          const T g[2] = {das[p0 * ld + c], das[p1 * ld + c]};
          const T qv[2] = {qs[p0 * ld + c], qs[p1 * ld + c]};
          column(c, g, qv);
        }
      }
#pragma unroll
      for (int x = 0; x < 2; ++x) {
        const int p = p0 + x;
        if (p >= nang) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          hkd[p * kHKD + mb + j] = h[x][j];
          hkd[p * kHKD + kMono + mb + j] = k[x][j];
          if (mb == 0) hkd[p * kHKD + 2 * kMono + j] = d[x][j];
        }
      }
    }
    __syncthreads();
    // switch and unit-vector terms: one thread per angle slot
    for (int s = threadIdx.x; s < nang; s += blockDim.x) {
      T m[kMono], hh[kMono], kk[kMono], dd[4], xp[4];
      ld20(mono + s * kMono, m);
      ld20(hkd + s * kHKD, hh);
      ld20(hkd + s * kHKD + kMono, kk);
      ld4(hkd + s * kHKD + 2 * kMono, dd);
      ld4(xpow + 4 * s, xp);
      const T sp = cur.sa[s];
      const T dsp = inv_na * (dot_n<kMono>(m, hh) -
                              T(2) * sp * (dd[0] + dd[1] * xp[1] + dd[2] * xp[2] + dd[3] * xp[3])) +
                    dot_n<kMono>(m, kk);
      T dm[kMono];
#pragma unroll
      for (int j = 0; j < kMono; ++j) dm[j] = sp * (inv_na * hh[j] + kk[j]);
      const T dx = -inv_na * sp * sp * (dd[1] + T(2) * dd[2] * xp[1] + T(3) * dd[3] * xp[2]);
      const T ux = cur.rh[3 * s], uy = cur.rh[3 * s + 1], uz = cur.rh[3 * s + 2];
      T dr[3];
      monomial_grad(ux, uy, uz, dm, dr);
      dsa_e[base + s] += dsp;
      drh[3 * (base + s)] += dr[0] + T(2) * dx * ux;
      drh[3 * (base + s) + 1] += dr[1] + T(2) * dx * uy;
      drh[3 * (base + s) + 2] += dr[2] + T(2) * dx * uz;
    }
    __syncthreads();   // the monomials, the sums and this buffer are rewritten next
  }
}

// (b): dy = de1 (1 - v^2) on real slots
template <typename T>
__global__ void k_dtanh(long long n, const T* __restrict__ g, const T* __restrict__ y,
                        T* __restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = g[i] * (T(1) - y[i] * y[i]);
}
// the same, four elements per thread (n4 = n / 4; 16-byte aligned arrays)
template <typename T>
__global__ void k_dtanh4(long long n4, const T* __restrict__ g, const T* __restrict__ y,
                         T* __restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n4) return;
  T gv[4], yv[4];
  ld4(g + 4 * i, gv);
  ld4(y + 4 * i, yv);
#pragma unroll
  for (int q = 0; q < 4; ++q) gv[q] *= T(1) - yv[q] * yv[q];
  st4(out + 4 * i, gv);
}

// (b) fused per atom: dy = de1 (1 - v^2) on every slot row and the atom's sum
// of those rows (block per atom; ed a multiple of 4, at most 4 x blockDim).
// Thread t owns the column quad t mod (ed / 4) and the rows congruent to
// t / (ed / 4); the row groups' partial sums are added in group order.  v and
// dy are stored as V and Y (16 bits in the mixed form); the sums add the
// products before dy is rounded to Y.
template <typename T, typename V = T, typename Y = T>
__global__ void k_dtanh_rowsum(int nmax, int ed, const T* __restrict__ g, const V* __restrict__ y,
                               Y* __restrict__ dy, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* part = reinterpret_cast<T*>(sm_raw);   // [row group][ed]
  const int cqn = ed >> 2, nrg = blockDim.x / cqn;
  const int cq = threadIdx.x % cqn, rg = threadIdx.x / cqn;
  const size_t base = (size_t)blockIdx.x * nmax * ed;
  T acc[4] = {T(0), T(0), T(0), T(0)};
  if (rg < nrg)
    for (int p = rg; p < nmax; p += nrg) {
      const size_t o = base + (size_t)p * ed + 4 * cq;
      T gv[4], yv[4];
      ld4(g + o, gv);
      ld4(y + o, yv);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        gv[q] *= T(1) - yv[q] * yv[q];
        acc[q] += gv[q];
      }
      st4(dy + o, gv);
    }
  if (rg < nrg) st4(part + (size_t)rg * ed + 4 * cq, acc);
  __syncthreads();
  if (rg == 0) {
    T tot[4] = {T(0), T(0), T(0), T(0)};
    for (int r = 0; r < nrg; ++r) {
      T v[4];
      ld4(part + (size_t)r * ed + 4 * cq, v);
#pragma unroll
      for (int q = 0; q < 4; ++q) tot[q] += v[q];
    }
    st4(out + (size_t)blockIdx.x * ed + 4 * cq, tot);
  }
}

// per atom: sum over its own slots (rows of dy)
template <typename T>
__global__ void k_rowsum(int nmax, int ed, const T* __restrict__ x, T* __restrict__ out) {
  int i = blockIdx.x;
  for (int c = threadIdx.x; c < ed; c += blockDim.x) {
    T acc = T(0);
    for (int p = 0; p < nmax; ++p) acc += x[((size_t)i * nmax + p) * ed + c];
    out[(size_t)i * ed + c] = acc;
  }
}

// (a) per kept slot: de += (1/nmax) sw dm_i * u_j;  X = (1/nmax) sw dm_i * e (for du_j);
// dsw += (1/nmax) sum_c dm_i e u_j
template <typename T>
__global__ void k_msg_bwd(long long P, int nmax, int ed, int ldm, T inv_nmax,
                          const int* __restrict__ sel_j, const T* __restrict__ sw,
                          const T* __restrict__ e, const T* __restrict__ u,
                          const T* __restrict__ dm, T* __restrict__ de, T* __restrict__ X,
                          T* __restrict__ dsw_e) {
  long long s = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (s >= P) return;
  int j = sel_j[s];
  if (j < 0) return;   // an empty slot: no message, and its X row is never gathered
  long long i = s / nmax;
  T acc = T(0);
  for (int c = lane; c < ed; c += 32) {
    T g = dm[i * ldm + c], ev = e[s * ed + c], uv = u[(long long)j * ed + c];
    de[s * ed + c] += inv_nmax * sw[s] * g * uv;
    X[s * ed + c] = inv_nmax * sw[s] * g * ev;
    acc += g * ev * uv;
  }
  acc = warp_sum(acc);
  if (lane == 0) dsw_e[s] += inv_nmax * acc;
}

// The same with 16 threads per slot, four columns each (ed, ldm multiples of
// 4, 16-byte aligned rows); the dsw sum closes with a fixed-order reduction
// over the 16 lanes.
template <typename T>
__global__ void k_msg_bwd4(long long P, int nmax, int ed, int ldm, T inv_nmax,
                           const int* __restrict__ sel_j, const T* __restrict__ sw,
                           const T* __restrict__ e, const T* __restrict__ u,
                           const T* __restrict__ dm, T* __restrict__ de, T* __restrict__ X,
                           T* __restrict__ dsw_e) {
  const long long s = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 4;
  const int l16 = threadIdx.x & 15;
  if (s >= P) return;   // the whole 16-lane group leaves together
  const int j = sel_j[s];
  if (j < 0) return;    // likewise: an empty slot
  const unsigned mask = 0xFFFFu << (threadIdx.x & 16);
  const long long i = (int)s / nmax;   // slots < 2^31
  const T f = inv_nmax * sw[s];
  T acc = T(0);
  for (int c = 4 * l16; c < ed; c += 64) {
    T g[4], ev[4], uv[4], d[4], x[4];
    ld4(dm + i * ldm + c, g);
    ld4(e + s * ed + c, ev);
    ld4(u + (long long)j * ed + c, uv);
    ld4(de + s * ed + c, d);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      d[q] += f * g[q] * uv[q];
      x[q] = f * g[q] * ev[q];
      acc += g[q] * ev[q] * uv[q];
    }
    st4(de + s * ed + c, d);
    st4(X + s * ed + c, x);
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) acc += __shfl_xor_sync(mask, acc, o);
  if (l16 == 0) dsw_e[s] += inv_nmax * acc;
}

// dn = dn1 + dnm[:, :nd]
template <typename T>
__global__ void k_add_strided(int n, int nd, int ld, const T* __restrict__ a, const T* __restrict__ b,
                              T* __restrict__ out) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * nd) return;
  long long i = idx / nd;
  int c = (int)(idx % nd);
  out[idx] = a[idx] + b[i * ld + c];
}

// edge init adjoint and the final pair gradient g = dE/dr
template <typename T>
__global__ void k_pair_grad(long long P, int nmax, int ed, int atom0, const int* __restrict__ sel_j,
                            const T* __restrict__ d, const T* __restrict__ sw,
                            const T* __restrict__ dsw, const T* __restrict__ dsa,
                            const T* __restrict__ rh, const T* __restrict__ e0,
                            const T* __restrict__ we, const T* __restrict__ de,
                            const T* __restrict__ dsw_e, const T* __restrict__ dsa_e,
                            const T* __restrict__ drh, T* __restrict__ g) {
  long long s = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (s >= P) return;
  if (sel_j[s] < 0) {
    if (lane < 3) g[3 * s + lane] = T(0);
    return;
  }
  T ds = T(0);
  for (int c = lane; c < ed; c += 32) {
    T ev = e0[s * ed + c];
    ds += de[s * ed + c] * (T(1) - ev * ev) * we[c];
  }
  ds = warp_sum(ds);
  if (lane != 0) return;
  T dd = d[s];
  T radial = ds * (dsw[s] / dd - sw[s] / (dd * dd)) + dsw_e[s] * dsw[s] + dsa_e[s] * dsa[s];
  const T* r = rh + 3 * s;
  const T* dr = drh + 3 * s;
  T proj = dr[0] * r[0] + dr[1] * r[1] + dr[2] * r[2];
  for (int a = 0; a < 3; ++a) g[3 * s + a] = radial * r[a] + (dr[a] - proj * r[a]) / dd;
  (void)atom0;
  (void)nmax;
}
// The same with 16 threads per slot, four columns each (ed a multiple of 4);
// the ds sum closes with a fixed-order reduction over the 16 lanes.
template <typename T, typename E = T>   // E: storage of the edge state
__global__ void k_pair_grad4(long long P, int ed, const int* __restrict__ sel_j, const T* __restrict__ d,
                             const T* __restrict__ sw, const T* __restrict__ dsw,
                             const T* __restrict__ dsa, const T* __restrict__ rh,
                             const E* __restrict__ e0, const T* __restrict__ we,
                             const T* __restrict__ de, const T* __restrict__ dsw_e,
                             const T* __restrict__ dsa_e, const T* __restrict__ drh, T* __restrict__ g) {
  const long long s = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 4;
  const int l16 = threadIdx.x & 15;
  if (s >= P) return;   // the whole 16-lane group leaves together
  if (sel_j[s] < 0) {   // likewise
    if (l16 < 3) g[3 * s + l16] = T(0);
    return;
  }
  const unsigned mask = 0xFFFFu << (threadIdx.x & 16);
  T ds = T(0);
  for (int c = 4 * l16; c < ed; c += 64) {
    T ev[4], dv[4], wv[4];
    ld4(de + s * ed + c, dv);   // e0 last: a 16-bit e0 is converted right after its load
    ld4(we + c, wv);
    ld4(e0 + s * ed + c, ev);
#pragma unroll
    for (int q = 0; q < 4; ++q) ds += dv[q] * (T(1) - ev[q] * ev[q]) * wv[q];
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) ds += __shfl_xor_sync(mask, ds, o);
  if (l16 != 0) return;
  const T dd = d[s];
  const T radial = ds * (dsw[s] / dd - sw[s] / (dd * dd)) + dsw_e[s] * dsw[s] + dsa_e[s] * dsa[s];
  const T* r = rh + 3 * s;
  const T* dr = drh + 3 * s;
  const T proj = dr[0] * r[0] + dr[1] * r[1] + dr[2] * r[2];
  for (int a = 0; a < 3; ++a) g[3 * s + a] = radial * r[a] + (dr[a] - proj * r[a]) / dd;
}

// ------------------------------------------------------------------ host side
template <typename T>
class PlainGf : public Model {
 public:
  ~PlainGf() override {
    for (cudaStream_t x : fit_st_) cudaStreamDestroy(x);
    for (cudaEvent_t x : fit_ev_) cudaEventDestroy(x);
    if (fork_ev_) cudaEventDestroy(fork_ev_);
    for (void* p : allocs_) cudaFree(p);
  }
  bool init(const GfDims& m, const double* w, int n_atoms, const int* types, std::string* err);
  int run(const NbrView& nv, const int* types, double* atom_e, cudaStream_t st) override;
  void bind_flags(int* flags) override { flags_ = flags; }
  bool set_energy_seed(const unsigned char* seed) override {
    seed_ = seed;
    return true;
  }
  // FP32 storage with every matrix product on the tensor cores (BF16 operands)
  void use_tensor_cores() { tc_ = true; }
  const float* grad32() const override { return grad_as<float>(); }
  const double* grad64() const override { return grad_as<double>(); }
  size_t bytes() const override { return bytes_; }

 private:
  // one matrix product: the tensor-core GEMM in the mixed form, else SIMT
  void mm(const Gemm<T>& g, cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
      if (tc_ && g.alpha == 1.f && g.a_rk == 1 && g.c_rn == 1 && (g.b_rn == 1 || g.b_rk == 1) &&
          gemm_tc_shape_ok(g.N, g.K) && g.a_rm % 4 == 0 &&
          (reinterpret_cast<uintptr_t>(g.A) & 15) == 0 && g.c_rm % 4 == 0 &&
          (reinterpret_cast<uintptr_t>(g.C) & 15) == 0 &&
          (reinterpret_cast<uintptr_t>(g.aux) & 15) == 0 &&
          (reinterpret_cast<uintptr_t>(g.bias) & 15) == 0) {   // 16-byte rows of A, C, aux; bias
        GemmTc t{};
        t.M = g.M; t.N = g.N; t.K = g.K;
        t.A = g.A; t.lda = g.a_rm; t.a_rows = g.a_rows;
        t.B = g.B; t.b_nk = g.b_rn == 1 ? 0 : 1; t.ldb = g.b_rn == 1 ? g.b_rk : g.b_rn;
        t.C = g.C; t.ldc = g.c_rm; t.c_rows = g.c_rows;
        t.bias = g.bias; t.beta = g.beta; t.epi = g.epi; t.aux = g.aux;
        t.status = flags_;
#ifdef DP_GF_BF16
        t.fp16 = 0;
#else
        t.fp16 = 1;
#endif
        // products over atom rows (node features, fitting) take the
        // activations as a 16-bit high part plus remainder: they carry most of
        // the 16-bit error and cost little; products over slot rows keep one
        t.split = g.M <= n_ ? 1 : 0;
        gemm_tc(t, st);
        return;
      }
    }
    gemm(g, 1, st);
  }
  // per atom j: the sum of x over every kept slot (i, p) whose neighbour is j,
  // in increasing (i, p) order whatever the skin list's order
  template <typename S>
  void gather_in(const NbrView& nv, const S* x, T* out, cudaStream_t st) {
    int warps = 4;
    while (warps > 1 && sizeof(int) * 2 * nv.cap * warps > 48 * 1024) --warps;
    k_mp_gather<T, S><<<ceil_div(n_, warps), warps * 32, sizeof(int) * 2 * nv.cap * warps, st>>>(
        n_, m_.nmax, m_.nmax, m_.ed, nv.cap, nv.skin, nv.skin_cnt, nv.mirror, nv.selpos, x,
        nullptr, out);
  }
  // mixed form: the edge update of layer l as the epilogue of e Wc on the
  // tensor cores (Ce never reaches memory); false when not applicable
  bool edge_fused(int l, const NbrView& nv, cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
      const int Ed = m_.ed;
      if (!tc_ || !gemm_tc_shape_ok(Ed, Ed) || Ed % 4 != 0) return false;
      GemmTc t{};
      t.M = (int)((long long)n_ * m_.nmax); t.N = Ed; t.K = Ed;
      t.A = ee_[l]; t.lda = Ed;
      t.B = Wc_[l]; t.ldb = Ed; t.b_nk = 0;
      t.C = ee_[l + 1]; t.ldc = Ed;   // e1; the angle channel then updates its rows in place
      t.bias = be_[l]; t.epi = 3;
      t.sel_j = nv.sel_j; t.nmax = m_.nmax; t.Ai = Ai_; t.Bj = Bj_; t.e_in = ee_[l]; t.v_out = vv_[l];
      if (s16_) {
        t.v16 = reinterpret_cast<uint16_t*>(vv16_[l]);
        t.a16 = t.e16 = reinterpret_cast<const uint16_t*>(ee16_[l]);
        t.o16 = reinterpret_cast<uint16_t*>(ee16_[l + 1]);
      }
      t.status = flags_;
#ifdef DP_GF_BF16
      t.fp16 = 0;
#else
      t.fp16 = 1;
#endif
      t.split = 0;   // slot rows: one 16-bit activation operand
      gemm_tc(t, st);
      return true;
    } else {
      (void)l; (void)nv; (void)st;
      return false;
    }
  }
  // mixed form: t = tanh(a Wq + bq) and e_{l+1} = e1 + swa t in one product's
  // epilogue, over the angle rows (e_{l+1} holds e1 and is updated in place);
  // false when not applicable
  bool angle_out_fused(int l, cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
      const int Ed = m_.ed;
      if (!tc_ || !gemm_tc_shape_ok(Ed, Ed) || Ed % 4 != 0) return false;
      GemmTc t{};
      t.M = (int)((long long)n_ * nac_); t.N = Ed; t.K = Ed;
      t.A = aa_; t.lda = Ed;
      t.B = Wq_[l]; t.ldb = Ed; t.b_nk = 0;
      t.C = tt_[l]; t.ldc = Ed;
      t.bias = bq_[l]; t.epi = 4;
      t.sa = sa_; t.e_in = ee_[l + 1]; t.v_out = ee_[l + 1]; t.x_rows = ang_rows_;
      if (s16_) {
        t.e16 = reinterpret_cast<const uint16_t*>(ee16_[l + 1]);
        t.o16 = reinterpret_cast<uint16_t*>(ee16_[l + 1]);
      }
      t.status = flags_;
#ifdef DP_GF_BF16
      t.fp16 = 0;
#else
      t.fp16 = 1;
#endif
      t.split = 0;   // slot rows: one 16-bit activation operand
      gemm_tc(t, st);
      return true;
    } else {
      (void)l; (void)st;
      return false;
    }
  }
  // mixed form: de += dy Wc^T with the message adjoint of layer l in the same
  // product's epilogue (de += f dm_i u_j, X = f dm_i e, dsw on kept slots);
  // false when not applicable (then the two run separately)
  bool msg_fusable() const {
    if constexpr (std::is_same<T, float>::value)
      return tc_ && gemm_tc_shape_ok(m_.ed, m_.ed) && m_.ed % 4 == 0 && m_.nd % 4 == 0;
    else
      return false;
  }
  void msg_fused(int l, const NbrView& nv, cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
      const int Ed = m_.ed, Nd = m_.nd;
      GemmTc t{};
      t.M = (int)((long long)n_ * m_.nmax); t.N = Ed; t.K = Ed;
      t.A = dy_; t.lda = Ed;
      if (s16_) t.a16 = reinterpret_cast<const uint16_t*>(dy16_);
      t.B = Wc_[l]; t.ldb = Ed; t.b_nk = 1;
      t.C = de_; t.ldc = Ed; t.beta = 1.f; t.epi = 5;
      t.sel_j = nv.sel_j; t.nmax = m_.nmax; t.sw = sw_; t.dm = dnm_ + Nd; t.lddm = Nd + Ed;
      t.u = uu_[l]; t.e_in = ee_[l]; t.x_out = X_; t.dsw = dsw_e_; t.inv_nmax = 1.f / (float)m_.nmax;
      if (s16_) {
        t.x16 = reinterpret_cast<uint16_t*>(X16_);
        t.e16 = reinterpret_cast<const uint16_t*>(ee16_[l]);
      }
      t.status = flags_;
#ifdef DP_GF_BF16
      t.fp16 = 0;
#else
      t.fp16 = 1;
#endif
      t.split = 0;   // slot rows: one 16-bit activation operand
      gemm_tc(t, st);
    } else {
      (void)l; (void)nv; (void)st;
    }
  }
  // one product whose A operand is stored in 16 bits (mixed form only); the
  // rest of g as for mm()
  template <typename A16>
  void mm_a16(Gemm<T> g, const A16* a16, cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
      GemmTc t{};
      t.M = g.M; t.N = g.N; t.K = g.K;
      t.a16 = reinterpret_cast<const uint16_t*>(a16); t.lda = g.a_rm; t.a_rows = g.a_rows;
      t.B = g.B; t.b_nk = g.b_rn == 1 ? 0 : 1; t.ldb = g.b_rn == 1 ? g.b_rk : g.b_rn;
      t.C = g.C; t.ldc = g.c_rm; t.c_rows = g.c_rows;
      t.bias = g.bias; t.beta = g.beta; t.epi = g.epi; t.aux = g.aux;
      t.status = flags_;
#ifdef DP_GF_BF16
      t.fp16 = 0;
#else
      t.fp16 = 1;
#endif
      gemm_tc(t, st);
    } else {
      (void)g; (void)a16; (void)st;
    }
  }
  // the angle channel's q = e_{l+1} Wp over the angle rows (their slots'
  // rows of e gathered); in the mixed form from the 16-bit edge state
  void q_product(int l, cudaStream_t st) {
    const int Ed = m_.ed;
    if constexpr (std::is_same<T, float>::value) {
      if (s16_) {
        GemmTc t{};
        t.M = (int)((long long)n_ * nac_); t.N = Ed; t.K = Ed;
        t.a16 = reinterpret_cast<const uint16_t*>(ee16_[l + 1]); t.lda = Ed; t.a_rows = ang_rows_;
        t.B = Wp_[l]; t.ldb = Ed; t.b_nk = 0;
        t.C = qq_[l]; t.ldc = Ed;
        t.status = flags_;
#ifdef DP_GF_BF16
        t.fp16 = 0;
#else
        t.fp16 = 1;
#endif
        gemm_tc(t, st);
        return;
      }
    }
    Gemm<T> g = gemm_rowmajor<T>((int)((long long)n_ * nac_), Ed, Ed, ee_[l + 1], Ed, Wp_[l], Ed, qq_[l], Ed);
    g.a_rows = ang_rows_;
    mm(g, st);
  }
  bool tc_ = false;
  // mixed form: v (the edge update's tanh, kept for the adjoint), dy (the
  // A operand of de += dy Wc^T) and X (the message adjoint's per-slot rows)
  // stored in 16 bits, the operand type (S16; T itself outside the mixed form)
  using S16 = typename std::conditional<std::is_same<T, float>::value, gf16_t, T>::type;
  bool s16_ = false;
  std::vector<S16*> vv16_;
  // the edge state e_0 .. e_L in 16 bits as well (mixed form): the tensor-core
  // products round it to 16 bits anyway, and its residual updates e1 = e + v,
  // e_{l+1} = e1 + swa t are rounded once per layer
  std::vector<S16*> ee16_;
  // and the angle channel's adjoints dz and dq, which only ever feed a
  // product as its A operand (rounded to 16 bits there anyway)
  S16 *dz16_ = nullptr, *dq16_ = nullptr;
  S16 *dy16_ = nullptr, *X16_ = nullptr;
  int* flags_ = nullptr;
  const unsigned char* seed_ = nullptr;   // energy seed (device, optional)
  // shared-memory variants of the angle kernels (see k_angle, k_angle_bwd):
  int angle_grid_ = 1, angle_bwd_grid_ = 1;
  size_t angle_smem_ = 0, angle_bwd_smem_ = 0;

  template <typename U>
  const U* grad_as() const {
    if constexpr (std::is_same<T, U>::value) return g_;
    else return nullptr;
  }
  template <typename U>
  bool dalloc(U** p, size_t count, std::string* err) {
    size_t b = sizeof(U) * (count ? count : 1);
    cudaError_t e = cudaMalloc((void**)p, b);
    if (e != cudaSuccess) {
      *err = std::string("graph model: ") + cudaGetErrorString(e);
      cudaGetLastError();
      return false;
    }
    allocs_.push_back(*p);
    bytes_ += b;
    return true;
  }
  bool upload(T** p, const double* src, size_t count, std::string* err) {
    if (!dalloc(p, count, err)) return false;
    std::vector<T> h(src, src + count);
    return cudaMemcpy(*p, h.data(), sizeof(T) * count, cudaMemcpyHostToDevice) == cudaSuccess;
  }
  GfDims m_{};
  int n_ = 0;
  long long P_ = 0;
  // the angle channel works on angle rows only: slot p < nac_ = min(na, nmax)
  // of atom i is angle row i nac_ + p, at slot ang_rows_[i nac_ + p] = i nmax + p
  int nac_ = 0;
  int* ang_rows_ = nullptr;
  // weights
  T *Wt_, *we_, *be0_;
  std::vector<T*> Wm_, Wn_, bn_, Wa_, Wb_, Wc_, be_, Wp_, Wphi_, Wq_, bq_;
  std::vector<T*> F1_, c1_, F2_, c2_, F3_, c3_;
  T *F4_, *c4_;
  int* fit_rows_;
  std::vector<std::pair<int, int>> fit_ranges_;
  // the species' fitting products run concurrently: one stream each, forked
  // from and joined back to the evaluation's stream by events
  std::vector<cudaStream_t> fit_st_;
  std::vector<cudaEvent_t> fit_ev_;
  cudaEvent_t fork_ev_ = nullptr;
  void fit_fork(cudaStream_t st) {
    cudaEventRecord(fork_ev_, st);
    for (cudaStream_t x : fit_st_) cudaStreamWaitEvent(x, fork_ev_, 0);
  }
  void fit_join(cudaStream_t st) {
    for (size_t t = 0; t < fit_st_.size(); ++t) {
      cudaEventRecord(fit_ev_[t], fit_st_[t]);
      cudaStreamWaitEvent(st, fit_ev_[t], 0);
    }
  }
  // geometry
  T *d_, *sw_, *dsw_, *sa_, *dsa_, *s_, *rh_;
  // states
  std::vector<T*> nn_, ee_, hh_, uu_, mm_, vv_, qq_, tt_;   // qq_, tt_ by angle row
  T *Ai_, *Bj_, *Ce_, *aa_;
  T *y1_, *y2_, *y3_, *d1_, *d2_, *d3_;
  // adjoint
  T *dn_, *dn1_, *de_, *dy_, *dz_, *da_, *dq_, *du_, *dx_, *dnm_, *X_, *sdy_, *gat_;   // aa_, dz_, da_, dq_ by angle row
  T *dsw_e_, *dsa_e_, *drh_, *g_;
  std::vector<void*> allocs_;
  size_t bytes_ = 0;
};

template <typename T>
bool PlainGf<T>::init(const GfDims& m, const double* w, int n_atoms, const int* types,
                      std::string* err) {
  m_ = m;
  n_ = n_atoms;
  const int Nd = m.nd, Ed = m.ed, L = m.n_layers, S = m.n_species, NM = m.nmax;
  P_ = (long long)n_atoms * NM;
  if (P_ > 2147483647LL) {   // slot indices are 32-bit in the products and kernels
    *err = "graph model: atoms x nmax must stay below 2^31";
    return false;
  }
  size_t off = 0;
  auto take = [&](T** p, size_t cnt) {
    bool ok = upload(p, w + off, cnt, err);
    off += cnt;
    return ok;
  };
  bool ok = take(&Wt_, (size_t)S * Nd) && take(&we_, Ed) && take(&be0_, Ed);
  Wm_.resize(L); Wn_.resize(L); bn_.resize(L); Wa_.resize(L); Wb_.resize(L); Wc_.resize(L);
  be_.resize(L); Wp_.resize(L); Wphi_.resize(L); Wq_.resize(L); bq_.resize(L);
  for (int l = 0; l < L && ok; ++l)
    ok = take(&Wm_[l], (size_t)Nd * Ed) && take(&Wn_[l], (size_t)(Nd + Ed) * Nd) &&
         take(&bn_[l], Nd) && take(&Wa_[l], (size_t)Nd * Ed) && take(&Wb_[l], (size_t)Nd * Ed) &&
         take(&Wc_[l], (size_t)Ed * Ed) && take(&be_[l], Ed) && take(&Wp_[l], (size_t)Ed * Ed) &&
         take(&Wphi_[l], 4 * (size_t)Ed) && take(&Wq_[l], (size_t)Ed * Ed) && take(&bq_[l], Ed);
  F1_.resize(S); c1_.resize(S); F2_.resize(S); c2_.resize(S); F3_.resize(S); c3_.resize(S);
  std::vector<double> F4, c4;
  for (int t = 0; t < S && ok; ++t) {
    ok = take(&F1_[t], (size_t)Nd * m.f1) && take(&c1_[t], m.f1) &&
         take(&F2_[t], (size_t)m.f1 * m.f2) && take(&c2_[t], m.f2) &&
         take(&F3_[t], (size_t)m.f2 * m.f3) && take(&c3_[t], m.f3);
    F4.insert(F4.end(), w + off, w + off + m.f3);
    off += m.f3;
    c4.push_back(w[off]);
    off += 1;
  }
  if (!ok || !upload(&F4_, F4.data(), F4.size(), err) || !upload(&c4_, c4.data(), c4.size(), err))
    return false;
  // fitting row groups
  std::vector<int> rows;
  fit_ranges_.assign(S, {0, 0});
  for (int t = 0; t < S; ++t) {
    int start = (int)rows.size();
    for (int i = 0; i < n_atoms; ++i)
      if (types[i] == t) rows.push_back(i);
    fit_ranges_[t] = {start, (int)rows.size() - start};
  }
  if (!dalloc(&fit_rows_, rows.size(), err)) return false;
  fit_st_.assign(S, nullptr);
  fit_ev_.assign(S, nullptr);
  for (int t = 0; t < S; ++t)
    if (cudaStreamCreateWithFlags(&fit_st_[t], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&fit_ev_[t], cudaEventDisableTiming) != cudaSuccess) {
      *err = "graph model: cannot create the fitting streams";
      return false;
    }
  if (cudaEventCreateWithFlags(&fork_ev_, cudaEventDisableTiming) != cudaSuccess) {
    *err = "graph model: cannot create the fitting streams";
    return false;
  }
  if (!rows.empty()) cudaMemcpy(fit_rows_, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice);
  const size_t N = n_atoms, P = P_;
  nac_ = std::min(m.na, NM);
  const size_t PA = (size_t)n_atoms * nac_;
  {
    std::vector<int> ar(PA);
    for (size_t q = 0; q < PA; ++q) ar[q] = (int)((q / nac_) * NM + q % nac_);
    if (!dalloc(&ang_rows_, PA, err)) return false;
    if (PA) cudaMemcpy(ang_rows_, ar.data(), sizeof(int) * PA, cudaMemcpyHostToDevice);
  }
  ok = dalloc(&d_, P, err) && dalloc(&sw_, P, err) && dalloc(&dsw_, P, err) &&
       dalloc(&sa_, P, err) && dalloc(&dsa_, P, err) && dalloc(&s_, P, err) &&
       dalloc(&rh_, 3 * P, err);
  nn_.resize(L + 1); ee_.resize(L + 1);
  hh_.resize(L); uu_.resize(L); mm_.resize(L); vv_.resize(L); qq_.resize(L); tt_.resize(L);
  // the mixed form's products and epilogues take the 16-bit rows (every
  // width it accepts has ed a multiple of 16 and nd of 16)
  s16_ = tc_ && std::is_same<T, float>::value && Ed % 16 == 0 && Ed <= 256 && Nd % 4 == 0;
  vv16_.assign(L, nullptr);
  dy_ = X_ = nullptr;
  ee16_.assign(L + 1, nullptr);
  for (int l = 0; l <= L && ok; ++l)
    ok = dalloc(&nn_[l], N * Nd, err) &&
         (s16_ ? dalloc(&ee16_[l], P * Ed, err) : dalloc(&ee_[l], P * Ed, err));
  for (int l = 0; l < L && ok; ++l)
    ok = dalloc(&hh_[l], N * Nd, err) && dalloc(&uu_[l], N * Ed, err) &&
         dalloc(&mm_[l], N * Ed, err) && (s16_ ? dalloc(&vv16_[l], P * Ed, err) : dalloc(&vv_[l], P * Ed, err)) && dalloc(&qq_[l], PA * Ed, err) &&
         dalloc(&tt_[l], PA * Ed, err);
  // the angle kernels hold their monomial sums in shared memory, with two
  // slot-data buffers (switches and unit vectors): beta (ed x 4), the slots'
  // monomials (na x 48) and YB (ed x 20), and in the adjoint also dYB (ed x
  // 20) and the per-slot sums (na x 44)
  const size_t kMaxSmem = 232448, na_ = (size_t)m.na, ed_ = (size_t)m.ed,
               fixed = (4 * ed_ + (kMono + kMonoSa + 4) * na_ + kMono * ed_) * sizeof(T),
               fixed_bwd = fixed + (kMono * ed_ + (2 * kMono + 4) * na_) * sizeof(T),
               geo = 2 * na_ * 4 * sizeof(T);
  if (fixed_bwd + geo > kMaxSmem) {
    *err = "graph model: the angle channel's sums do not fit in shared memory";
    return false;
  }
  angle_smem_ = fixed + geo;
  angle_bwd_smem_ = fixed_bwd + geo;
  const int angle_smem = (int)angle_smem_, angle_bwd_smem = (int)angle_bwd_smem_;
  if (cudaFuncSetAttribute(k_angle<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, angle_smem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_angle_bwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, angle_bwd_smem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_angle_bwd<T, S16>, cudaFuncAttributeMaxDynamicSharedMemorySize, angle_bwd_smem) !=
          cudaSuccess) {
    *err = "graph model: angle kernels cannot get their shared memory";
    return false;
  }
  {  // persistent grids: the blocks that fit on the device at once
    int dev = 0, sms = 0, bf = 0, bb = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bf, k_angle<T>, kAngThreads, angle_smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bb, k_angle_bwd<T>, kAngThreads, angle_bwd_smem) !=
            cudaSuccess) {
      *err = "graph model: cannot size the angle kernels' grids";
      return false;
    }
    angle_grid_ = std::max(1, std::min(n_atoms, sms * std::max(1, bf)));
    angle_bwd_grid_ = std::max(1, std::min(n_atoms, sms * std::max(1, bb)));
  }
  ok = ok && dalloc(&Ai_, N * Ed, err) && dalloc(&Bj_, N * Ed, err) && dalloc(&Ce_, P * Ed, err) &&
       dalloc(&aa_, PA * Ed, err) && dalloc(&y1_, N * m.f1, err) && dalloc(&y2_, N * m.f2, err) &&
       dalloc(&y3_, N * m.f3, err) && dalloc(&d1_, N * m.f1, err) && dalloc(&d2_, N * m.f2, err) &&
       dalloc(&d3_, N * m.f3, err) && dalloc(&dn_, N * Nd, err) && dalloc(&dn1_, N * Nd, err) &&
       dalloc(&de_, P * Ed, err) && (s16_ ? dalloc(&dy16_, P * Ed, err) : dalloc(&dy_, P * Ed, err)) &&
       (s16_ ? dalloc(&dz16_, PA * Ed, err) : dalloc(&dz_, PA * Ed, err)) && dalloc(&da_, PA * Ed, err) &&
       (s16_ ? dalloc(&dq16_, PA * Ed, err) : dalloc(&dq_, PA * Ed, err)) &&
       dalloc(&du_, N * Ed, err) && dalloc(&dx_, N * Nd, err) && dalloc(&dnm_, N * (Nd + Ed), err) &&
       (s16_ ? dalloc(&X16_, P * Ed, err) : dalloc(&X_, P * Ed, err)) && dalloc(&sdy_, N * Ed, err) && dalloc(&gat_, N * Ed, err) &&
       dalloc(&dsw_e_, P, err) && dalloc(&dsa_e_, P, err) && dalloc(&drh_, 3 * P, err) &&
       dalloc(&g_, 3 * P, err);
  return ok;
}

template <typename T>
int PlainGf<T>::run(const NbrView& nv, const int* types, double* atom_e, cudaStream_t st) {
  const GfDims& m = m_;
  const int Nd = m.nd, Ed = m.ed, L = m.n_layers, NM = m.nmax, NA = m.na, S = m.n_species, n = n_;
  const long long P = P_, PE = P * Ed;
  const T inv_nmax = T(1) / T(NM), inv_na = T(1) / T(NA);
  const int CA = nac_;
  const long long PA = (long long)n * CA;
  int k = 0;
  auto grid = [](long long n_) { return ceil_div(n_, 256); };
  k_env<T><<<grid(P), 256, 0, st>>>(P, NM, NA, nv.sel_j, nv.sel_r, m.rs, m.rc, m.rsa, m.rca, d_, sw_,
                                     dsw_, sa_, dsa_, s_, rh_);
  if (s16_)
    k_init<T, S16><<<n, 128, 0, st>>>(n, NM, Nd, Ed, types, nv.sel_j, s_, Wt_, we_, be0_, nn_[0], ee16_[0]);
  else
    k_init<T><<<n, 128, 0, st>>>(n, NM, Nd, Ed, types, nv.sel_j, s_, Wt_, we_, be0_, nn_[0], ee_[0]);
  k += 2;
  const size_t angle_smem = angle_smem_, angle_bwd_smem = angle_bwd_smem_;
  const int ed_shift = (Ed & (Ed - 1)) == 0 ? __builtin_ctz((unsigned)Ed) : -1;
  for (int l = 0; l < L; ++l) {
    // (a)
    mm(gemm_rowmajor<T>(n, Ed, Nd, nn_[l], Nd, Wm_[l], Ed, uu_[l], Ed), st);
    if (s16_)
      k_msg_warp<T, S16><<<ceil_div((long long)n * 32, 256), 256, 0, st>>>(n, NM, Ed, inv_nmax, nv.sel_j,
                                                                            sw_, ee16_[l], uu_[l], mm_[l]);
    else if (Ed % 2 == 0)
      k_msg_warp<T><<<ceil_div((long long)n * 32, 256), 256, 0, st>>>(n, NM, Ed, inv_nmax, nv.sel_j, sw_,
                                                                       ee_[l], uu_[l], mm_[l]);
    else
      k_msg<T><<<n, 64, 0, st>>>(NM, Ed, inv_nmax, nv.sel_j, sw_, ee_[l], uu_[l], mm_[l]);
    {
      Gemm<T> g = gemm_rowmajor<T>(n, Nd, Nd, nn_[l], Nd, Wn_[l], Nd, hh_[l], Nd);
      g.bias = bn_[l];
      mm(g, st);
      g = gemm_rowmajor<T>(n, Nd, Ed, mm_[l], Ed, Wn_[l] + (size_t)Nd * Nd, Nd, hh_[l], Nd);
      g.beta = T(1);
      g.epi = 1;
      mm(g, st);
    }
    k_add<T><<<grid((long long)n * Nd), 256, 0, st>>>((long long)n * Nd, nn_[l], hh_[l], nn_[l + 1]);
    // (b)
    mm(gemm_rowmajor<T>(n, Ed, Nd, nn_[l + 1], Nd, Wa_[l], Ed, Ai_, Ed), st);
    mm(gemm_rowmajor<T>(n, Ed, Nd, nn_[l + 1], Nd, Wb_[l], Ed, Bj_, Ed), st);
    if (edge_fused(l, nv, st)) {
      --k;   // one launch instead of two
    } else {
      mm(gemm_rowmajor<T>((int)P, Ed, Ed, ee_[l], Ed, Wc_[l], Ed, Ce_, Ed), st);
      k_edge<T><<<grid(PE), 256, 0, st>>>(P, NM, Ed, ed_shift, nv.sel_j, Ai_, Bj_, Ce_, be_[l],
                                          ee_[l], vv_[l], ee_[l + 1]);
    }
    // (c) on the angle rows; e_{l+1} holds e1 until the angle update below
    q_product(l, st);
    k_angle<T><<<angle_grid_, kAngThreads, angle_smem, st>>>(n, NM, NA, CA, Ed, inv_na, sa_, rh_, qq_[l],
                                                             Wphi_[l], aa_);
    if (angle_out_fused(l, st)) {
      --k;   // one launch instead of two
    } else {
      Gemm<T> g = gemm_rowmajor<T>((int)PA, Ed, Ed, aa_, Ed, Wq_[l], Ed, tt_[l], Ed);
      g.bias = bq_[l];
      g.epi = 1;
      mm(g, st);
      k_angle_out<T><<<grid(PA * Ed), 256, 0, st>>>(PA, Ed, ed_shift, NM, CA, sa_, tt_[l], ee_[l + 1]);
    }
    k += 14;
  }
  // fitting: each species' rows on its own stream (disjoint rows of y1..y3)
  fit_fork(st);
  for (int t = 0; t < S; ++t) {
    auto rg = fit_ranges_[t];
    if (rg.second == 0) continue;
    const int* rws = fit_rows_ + rg.first;
    cudaStream_t fs = fit_st_[t];
    Gemm<T> g = gemm_rowmajor<T>(rg.second, m.f1, Nd, nn_[L], Nd, F1_[t], m.f1, y1_, m.f1);
    g.a_rows = rws; g.c_rows = rws; g.bias = c1_[t]; g.epi = 1;
    mm(g, fs);
    g = gemm_rowmajor<T>(rg.second, m.f2, m.f1, y1_, m.f1, F2_[t], m.f2, y2_, m.f2);
    g.a_rows = rws; g.c_rows = rws; g.bias = c2_[t]; g.epi = 1;
    mm(g, fs);
    g = gemm_rowmajor<T>(rg.second, m.f3, m.f2, y2_, m.f2, F3_[t], m.f3, y3_, m.f3);
    g.a_rows = rws; g.c_rows = rws; g.bias = c3_[t]; g.epi = 1;
    mm(g, fs);
    k += 3;
  }
  fit_join(st);
  k_fit_out<T><<<ceil_div((long long)n * 32, 256), 256, 0, st>>>(n, m.f3, types, y3_, F4_, c4_, atom_e, d3_,
                                                                 seed_);
  fit_fork(st);
  for (int t = 0; t < S; ++t) {
    auto rg = fit_ranges_[t];
    if (rg.second == 0) continue;
    const int* rws = fit_rows_ + rg.first;
    Gemm<T> g{};
    g.M = rg.second; g.N = m.f2; g.K = m.f3;
    g.A = d3_; g.a_rm = m.f3; g.a_rk = 1;
    g.B = F3_[t]; g.b_rk = 1; g.b_rn = m.f3;
    g.C = d2_; g.c_rm = m.f2; g.c_rn = 1; g.nb2 = 1;
    g.a_rows = rws; g.c_rows = rws; g.alpha = T(1); g.epi = 2; g.aux = y2_;
    mm(g, fit_st_[t]);
    g.N = m.f1; g.K = m.f2; g.A = d2_; g.a_rm = m.f2; g.B = F2_[t]; g.b_rn = m.f2;
    g.C = d1_; g.c_rm = m.f1; g.aux = y1_;
    mm(g, fit_st_[t]);
    g.N = Nd; g.K = m.f1; g.A = d1_; g.a_rm = m.f1; g.B = F1_[t]; g.b_rn = m.f1;
    g.C = dn_; g.c_rm = Nd; g.epi = 0; g.aux = nullptr;
    mm(g, fit_st_[t]);
    k += 3;
  }
  fit_join(st);
  // ---- adjoint through the layers
  // adjoint accumulators start at zero (all-zero bytes are 0.0 in FP32 and FP64)
  cudaMemsetAsync(de_, 0, sizeof(T) * PE, st);
  cudaMemsetAsync(dsw_e_, 0, sizeof(T) * P, st);
  cudaMemsetAsync(dsa_e_, 0, sizeof(T) * P, st);
  cudaMemsetAsync(drh_, 0, sizeof(T) * 3 * P, st);
  k += 1;   // k_fit_out
  for (int l = L - 1; l >= 0; --l) {
    // (c): de holds dE/de_{l+1}; it becomes dE/de1 in place (e_{l+1} = e1 + swa t)
    if (s16_)
      k_angle_out_bwd4<T, S16><<<grid(PA * 16), 256, 0, st>>>(PA, Ed, NM, CA, sa_, tt_[l], de_, dz16_, dsa_e_);
    else if (Ed % 4 == 0)
      k_angle_out_bwd4<T><<<grid(PA * 16), 256, 0, st>>>(PA, Ed, NM, CA, sa_, tt_[l], de_, dz_, dsa_e_);
    else
      k_angle_out_bwd<T><<<grid(PA * 32), 256, 0, st>>>(PA, Ed, NM, CA, sa_, tt_[l], de_, dz_, dsa_e_);
    {  // da = dz Wq^T (angle rows)
      Gemm<T> g{};
      g.M = (int)PA; g.N = Ed; g.K = Ed;
      g.A = dz_; g.a_rm = Ed; g.a_rk = 1;
      g.B = Wq_[l]; g.b_rk = 1; g.b_rn = Ed;
      g.C = da_; g.c_rm = Ed; g.c_rn = 1; g.nb2 = 1; g.alpha = T(1);
      if (s16_) mm_a16(g, dz16_, st);
      else mm(g, st);
    }
    if (s16_)
      k_angle_bwd<T, S16><<<angle_bwd_grid_, kAngThreads, angle_bwd_smem, st>>>(
          n, NM, NA, CA, Ed, inv_na, sa_, rh_, qq_[l], Wphi_[l], da_, dq16_, dsa_e_, drh_);
    else
      k_angle_bwd<T><<<angle_bwd_grid_, kAngThreads, angle_bwd_smem, st>>>(
          n, NM, NA, CA, Ed, inv_na, sa_, rh_, qq_[l], Wphi_[l], da_, dq_, dsa_e_, drh_);
    {  // de1 = de + dq Wp^T, in place on the angle rows' slots (dq is 0 elsewhere)
      Gemm<T> g{};
      g.M = (int)PA; g.N = Ed; g.K = Ed;
      g.A = dq_; g.a_rm = Ed; g.a_rk = 1;
      g.B = Wp_[l]; g.b_rk = 1; g.b_rn = Ed;
      g.C = de_; g.c_rm = Ed; g.c_rn = 1; g.nb2 = 1; g.alpha = T(1); g.beta = T(1);
      g.c_rows = ang_rows_;
      if (s16_) mm_a16(g, dq16_, st);
      else mm(g, st);
    }
    // (b): de now holds dE/de1; it becomes dE/de_l (e1 = e_l + tanh(...))
    const bool fused_rowsum = Ed % 4 == 0 && Ed <= 1024;
    if (fused_rowsum)   // dy and its per-atom row sum sdy in one pass
      if (s16_)
        k_dtanh_rowsum<T, S16, S16><<<n, 256, 256 / (Ed / 4) * Ed * sizeof(T), st>>>(NM, Ed, de_, vv16_[l],
                                                                                     dy16_, sdy_);
      else
        k_dtanh_rowsum<T><<<n, 256, 256 / (Ed / 4) * Ed * sizeof(T), st>>>(NM, Ed, de_, vv_[l], dy_, sdy_);
    else if (PE % 4 == 0)
      k_dtanh4<T><<<grid(PE / 4), 256, 0, st>>>(PE / 4, de_, vv_[l], dy_);
    else
      k_dtanh<T><<<grid(PE), 256, 0, st>>>(PE, de_, vv_[l], dy_);
    const bool fused_msg = msg_fusable();
    if (!fused_msg) {  // de += dy Wc^T (else below, with the message adjoint)
      Gemm<T> g{};
      g.M = (int)P; g.N = Ed; g.K = Ed;
      g.A = dy_; g.a_rm = Ed; g.a_rk = 1;
      g.B = Wc_[l]; g.b_rk = 1; g.b_rn = Ed;
      g.C = de_; g.c_rm = Ed; g.c_rn = 1; g.nb2 = 1; g.alpha = T(1); g.beta = T(1);
      mm(g, st);
    }
    if (!fused_rowsum) k_rowsum<T><<<n, 64, 0, st>>>(NM, Ed, dy_, sdy_);
    if (s16_) gather_in(nv, dy16_, gat_, st);
    else gather_in(nv, dy_, gat_, st);
    k_copy<T><<<grid((long long)n * Nd), 256, 0, st>>>((long long)n * Nd, dn_, dn1_);
    {  // dn1 += sdy Wa^T + gat Wb^T
      Gemm<T> g{};
      g.M = n; g.N = Nd; g.K = Ed;
      g.A = sdy_; g.a_rm = Ed; g.a_rk = 1;
      g.B = Wa_[l]; g.b_rk = 1; g.b_rn = Ed;
      g.C = dn1_; g.c_rm = Nd; g.c_rn = 1; g.nb2 = 1; g.alpha = T(1); g.beta = T(1);
      mm(g, st);
      g.A = gat_; g.B = Wb_[l];
      mm(g, st);
    }
    // (a)
    k_dtanh<T><<<grid((long long)n * Nd), 256, 0, st>>>((long long)n * Nd, dn1_, hh_[l], dx_);
    {  // dnm = dx Wn^T  (n x (Nd + Ed))
      Gemm<T> g{};
      g.M = n; g.N = Nd + Ed; g.K = Nd;
      g.A = dx_; g.a_rm = Nd; g.a_rk = 1;
      g.B = Wn_[l]; g.b_rk = 1; g.b_rn = Nd;
      g.C = dnm_; g.c_rm = Nd + Ed; g.c_rn = 1; g.nb2 = 1; g.alpha = T(1);
      mm(g, st);
    }
    k_add_strided<T><<<grid((long long)n * Nd), 256, 0, st>>>(n, Nd, Nd + Ed, dn1_, dnm_, dn_);
    if (fused_msg)
      msg_fused(l, nv, st);
    else if (Ed % 4 == 0 && Nd % 4 == 0)
      k_msg_bwd4<T><<<grid(P * 16), 256, 0, st>>>(P, NM, Ed, Nd + Ed, inv_nmax, nv.sel_j, sw_, ee_[l],
                                                  uu_[l], dnm_ + Nd, de_, X_, dsw_e_);
    else
      k_msg_bwd<T><<<grid(P * 32), 256, 0, st>>>(P, NM, Ed, Nd + Ed, inv_nmax, nv.sel_j, sw_, ee_[l],
                                                 uu_[l], dnm_ + Nd, de_, X_, dsw_e_);
    if (s16_) gather_in(nv, X16_, du_, st);
    else gather_in(nv, X_, du_, st);
    {  // dn += du Wm^T
      Gemm<T> g{};
      g.M = n; g.N = Nd; g.K = Ed;
      g.A = du_; g.a_rm = Ed; g.a_rk = 1;
      g.B = Wm_[l]; g.b_rk = 1; g.b_rn = Ed;
      g.C = dn_; g.c_rm = Nd; g.c_rn = 1; g.nb2 = 1; g.alpha = T(1); g.beta = T(1);
      mm(g, st);
    }
    k += 18 - (fused_rowsum ? 1 : 0) - (fused_msg ? 1 : 0);
  }
  if (s16_)
    k_pair_grad4<T, S16><<<grid(P * 16), 256, 0, st>>>(P, Ed, nv.sel_j, d_, sw_, dsw_, dsa_, rh_, ee16_[0],
                                                       we_, de_, dsw_e_, dsa_e_, drh_, g_);
  else if (Ed % 4 == 0)
    k_pair_grad4<T><<<grid(P * 16), 256, 0, st>>>(P, Ed, nv.sel_j, d_, sw_, dsw_, dsa_, rh_, ee_[0], we_, de_,
                                                  dsw_e_, dsa_e_, drh_, g_);
  else
    k_pair_grad<T><<<grid(P * 32), 256, 0, st>>>(P, NM, Ed, 0, nv.sel_j, d_, sw_, dsw_, dsa_, rh_, ee_[0],
                                                 we_, de_, dsw_e_, dsa_e_, drh_, g_);
  return k + 1;
}

}  // namespace gf

size_t gf_weight_count(const GfDims& m) {
  size_t Nd = m.nd, Ed = m.ed, S = m.n_species;
  size_t t = S * Nd + 2 * Ed;
  t += (size_t)m.n_layers * (Nd * Ed + (Nd + Ed) * Nd + Nd + 2 * Nd * Ed + Ed * Ed + Ed + Ed * Ed +
                             4 * Ed + Ed * Ed + Ed);
  t += S * (Nd * m.f1 + m.f1 + (size_t)m.f1 * m.f2 + m.f2 + (size_t)m.f2 * m.f3 + m.f3 + m.f3 + 1);
  return t;
}

bool gf_mixed_supported(const GfDims& m, std::string* why) {
  const int dims[6] = {m.nd, m.ed, m.nd + m.ed, m.f1, m.f2, m.f3};
  for (int d : dims)
    if (!gemm_tc_shape_ok(d, 16)) {
      *why = "the mixed graph form needs node, edge and fitting widths (and node + edge) that "
             "are multiples of 16, at most 256";
      return false;
    }
  return true;
}

Model* make_plain_gf(const GfDims& m, bool f64, bool tensor_cores, const double* weights,
                     int n_atoms, const int* types_host, std::string* err) {
  if (m.na > gf::kMaxNa) {
    *err = "graph model supports at most 64 angle neighbours";
    return nullptr;
  }
  if (tensor_cores) {
    if (!gf_mixed_supported(m, err) || !gemm_tc_prepare(err)) return nullptr;
    auto* p = new gf::PlainGf<float>();
    p->use_tensor_cores();
    if (!p->init(m, weights, n_atoms, types_host, err)) { delete p; return nullptr; }
    return p;
  }
  if (f64) {
    auto* p = new gf::PlainGf<double>();
    if (!p->init(m, weights, n_atoms, types_host, err)) { delete p; return nullptr; }
    return p;
  }
  auto* p = new gf::PlainGf<float>();
  if (!p->init(m, weights, n_atoms, types_host, err)) { delete p; return nullptr; }
  return p;
}

}  // namespace dp
