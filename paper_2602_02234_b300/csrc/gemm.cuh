// Generic batched SIMT GEMM used by the plain (unfused) FP32 / FP64 paths.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace dp {

// =========================================================================
// Generic batched SIMT GEMM: C(m,n) = alpha * sum_k A(m,k) B(k,n) [+ bias]
//                                     [+ beta C] then epilogue
// with arbitrary element strides, a two-level batch index and optional row
// gather (A) / scatter (C).  64 x 64 tile, 16-deep K slices, 4 x 4 per thread.
// =========================================================================
template <typename T>
struct Gemm {
  int M, N, K;
  const T* A;
  long long a_rm, a_rk, a_b1, a_b2;
  const T* B;
  long long b_rk, b_rn, b_b1, b_b2;
  T* C;
  long long c_rm, c_rn, c_b1, c_b2;
  int nb2;               // batch = b1 * nb2 + b2
  const int* a_rows;     // optional: row of A for m
  const int* c_rows;     // optional: row of C for m
  const T* bias;         // optional [N]
  const T* aux;          // epilogue 2: C *= 1 - aux(m,n)^2 (aux laid out like C)
  T alpha, beta;
  int epi;               // 0 none, 1 tanh, 2 times (1 - aux^2)
};

template <typename T>
__global__ void __launch_bounds__(256) k_gemm(Gemm<T> g, long long batch) {
  constexpr int BM = 64, BN = 64, BK = 16;
  long long b = (long long)blockIdx.y + (long long)gridDim.y * blockIdx.z;
  if (b >= batch) return;
  long long b1 = b / g.nb2, b2 = b % g.nb2;
  int tiles_n = (g.N + BN - 1) / BN;
  int tm = blockIdx.x / tiles_n, tn = blockIdx.x % tiles_n;
  const T* A = g.A + b1 * g.a_b1 + b2 * g.a_b2;
  const T* B = g.B + b1 * g.b_b1 + b2 * g.b_b2;
  T* C = g.C + b1 * g.c_b1 + b2 * g.c_b2;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  long long arow[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int e = tid + 256 * q;
    int m = tm * BM + e / BK;
    arow[q] = m < g.M ? (g.a_rows ? (long long)g.a_rows[m] : (long long)m) : -1;
  }
  for (int k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int e = tid + 256 * q;
      int mm = e / BK, kk = e % BK, k = k0 + kk;
      T v = T(0);
      if (arow[q] >= 0 && k < g.K) v = A[arow[q] * g.a_rm + (long long)k * g.a_rk];
      As[kk][mm] = v;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int e = tid + 256 * q;
      int kk = e / BN, nn = e % BN, k = k0 + kk, n = tn * BN + nn;
      T v = T(0);
      if (k < g.K && n < g.N) v = B[(long long)k * g.b_rk + (long long)n * g.b_rn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bb[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int m = tm * BM + ty + 16 * i;
    if (m >= g.M) continue;
    long long row = g.c_rows ? (long long)g.c_rows[m] : (long long)m;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int n = tn * BN + tx + 16 * j;
      if (n >= g.N) continue;
      long long o = row * g.c_rm + (long long)n * g.c_rn;
      T v = g.alpha * acc[i][j];
      if (g.bias) v += g.bias[n];
      if (g.beta != T(0)) v += g.beta * C[o];
      if (g.epi == 1) v = dtanh(v);
      else if (g.epi == 2) {
        T y = g.aux[b1 * g.c_b1 + b2 * g.c_b2 + o];
        v *= T(1) - y * y;
      }
      C[o] = v;
    }
  }
}

// =========================================================================
// FP32 fast path for one (unbatched) product with row-major A (unit column
// stride), B row-major (K x N, unit column stride) or stored transposed (unit
// row stride) and row-major C: 128 x 128
// tiles, 8-deep K slices, 8 x 8 outputs per thread from two 4-wide fragments
// in each direction, the next slice's float4 loads in registers while the
// current one is multiplied out of the other shared buffer.  Same result
// definition as k_gemm (sums in increasing k per output), same epilogues.
// =========================================================================
constexpr int kSgBM = 128, kSgBN = 128, kSgBK = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_sgemm128(Gemm<T> g) {
  static_assert(std::is_same<T, float>::value, "FP32 only");
  __shared__ __align__(16) float As[2][kSgBK][kSgBM];
  __shared__ __align__(16) float Bs[2][kSgBK][kSgBN];
  const int tiles_n = (g.N + kSgBN - 1) / kSgBN;
  const int tm = blockIdx.x / tiles_n, tn = blockIdx.x - tm * tiles_n;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // loads: A slice 128 x 8 (thread: row tid >> 1, columns 4 (tid & 1) .. +3),
  // B slice 8 x 128 (thread: row tid >> 5, columns 4 (tid & 31) .. +3)
  const int am = tid >> 1, ak = (tid & 1) << 2;
  const int bk = tid >> 5, bn = (tid & 31) << 2;
  const long long m_ld = (long long)tm * kSgBM + am;
  const long long arow = m_ld < g.M ? (g.a_rows ? (long long)g.a_rows[m_ld] : m_ld) : -1;
  const float* Ap = arow >= 0 ? g.A + arow * g.a_rm : nullptr;
  const int n_ld = tn * kSgBN + bn;
  auto load_a = [&](int k0) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    const int k = k0 + ak;
    if (Ap) {
      if (k + 3 < g.K) {
        v = *reinterpret_cast<const float4*>(Ap + k);
      } else {
        if (k < g.K) v.x = Ap[k];
        if (k + 1 < g.K) v.y = Ap[k + 1];
        if (k + 2 < g.K) v.z = Ap[k + 2];
      }
    }
    return v;
  };
  // B (K x N) with unit column stride: four columns of one row; B stored
  // transposed (unit row stride, b_rk == 1): four rows of one column, like A
  const bool bt = g.b_rn != 1;
  const int tn_ld = tn * kSgBN + am;   // transposed B: column of this thread
  auto load_b = [&](int k0) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!bt) {
      const int k = k0 + bk;
      if (k < g.K && n_ld < g.N) v = *reinterpret_cast<const float4*>(g.B + (long long)k * g.b_rk + n_ld);
    } else if (tn_ld < g.N) {
      const int k = k0 + ak;
      const float* Bp = g.B + (long long)tn_ld * g.b_rn;
      if (k + 3 < g.K) {
        v = *reinterpret_cast<const float4*>(Bp + k);
      } else {
        if (k < g.K) v.x = Bp[k];
        if (k + 1 < g.K) v.y = Bp[k + 1];
        if (k + 2 < g.K) v.z = Bp[k + 2];
      }
    }
    return v;
  };
  auto store_b = [&](int bf, float4 v) {
    if (!bt) {
      *reinterpret_cast<float4*>(&Bs[bf][bk][bn]) = v;
    } else {
      Bs[bf][ak][am] = v.x; Bs[bf][ak + 1][am] = v.y; Bs[bf][ak + 2][am] = v.z; Bs[bf][ak + 3][am] = v.w;
    }
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  float4 ra = load_a(0), rb = load_b(0);
  int buf = 0;
  As[0][ak][am] = ra.x; As[0][ak + 1][am] = ra.y; As[0][ak + 2][am] = ra.z; As[0][ak + 3][am] = ra.w;
  store_b(0, rb);
  __syncthreads();
  for (int k0 = 0; k0 < g.K; k0 += kSgBK) {
    const bool more = k0 + kSgBK < g.K;
    if (more) {
      ra = load_a(k0 + kSgBK);
      rb = load_b(k0 + kSgBK);
    }
#pragma unroll
    for (int kk = 0; kk < kSgBK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][4 * ty]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][4 * ty + 64]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][4 * tx]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][4 * tx + 64]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      buf ^= 1;
      As[buf][ak][am] = ra.x; As[buf][ak + 1][am] = ra.y; As[buf][ak + 2][am] = ra.z;
      As[buf][ak + 3][am] = ra.w;
      store_b(buf, rb);
      __syncthreads();
    }
  }
  // outputs: rows 4 ty + i (i < 4) and 64 + 4 ty + i - 4, columns likewise
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long long m = (long long)tm * kSgBM + (i < 4 ? 4 * ty + i : 64 + 4 * ty + i - 4);
    if (m >= g.M) continue;
    const long long row = g.c_rows ? (long long)g.c_rows[m] : m;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int n = tn * kSgBN + (j < 4 ? 4 * tx + j : 64 + 4 * tx + j - 4);
      if (n >= g.N) continue;
      const long long o = row * g.c_rm + n;
      float v = g.alpha * acc[i][j];
      if (g.bias) v += g.bias[n];
      if (g.beta != 0.f) v += g.beta * g.C[o];
      if (g.epi == 1) v = tanhf(v);
      else if (g.epi == 2) {
        const float y = g.aux[o];
        v *= 1.f - y * y;
      }
      g.C[o] = v;
    }
  }
}

// =========================================================================
// FP32 batched small products (M, N <= 128, any K, any element strides, no
// row gather): one CTA of 256 threads per batch item (persistent over items),
// 32-deep K slices staged in shared memory in k-major order (each operand
// read along whichever of its strides is 1), and a register tile of 8 rows x
// TN columns per thread (rows 4 ty .. + 3 and 64 + 4 ty .. + 3; columns
// likewise for TN = 8, 2 tx .. + 1 for TN = 2).  Sums in increasing k.
// =========================================================================
constexpr int kBgK = 32, kBgLd = 132;

// X(r, k) = X[r s_r + k s_k] for r < R, k0 <= k < k0 + 32, into S[k - k0][r]
// (zero outside R x K), read along whichever stride is 1, four elements at a
// time where the rows are 16-byte aligned
__device__ __forceinline__ void stage_slice(const float* X, long long s_r, long long s_k, int R, int K,
                                            int k0, float (*S)[kBgLd]) {
  const int tid = threadIdx.x;
  const bool al = (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  if (s_k == 1 && al && s_r % 4 == 0) {          // rows contiguous in k
    for (int i = tid; i < 128 * (kBgK / 4); i += 256) {
      const int r = i >> 3, kk = (i & 7) << 2, k = k0 + kk;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < R) {
        const float* x = X + (long long)r * s_r + k;
        if (k + 3 < K) {
          v = *reinterpret_cast<const float4*>(x);
        } else {
          if (k < K) v.x = x[0];
          if (k + 1 < K) v.y = x[1];
          if (k + 2 < K) v.z = x[2];
        }
      }
      S[kk][r] = v.x;
      S[kk + 1][r] = v.y;
      S[kk + 2][r] = v.z;
      S[kk + 3][r] = v.w;
    }
  } else if (s_r == 1 && al && s_k % 4 == 0) {   // columns contiguous in r
    for (int i = tid; i < kBgK * 32; i += 256) {
      const int kk = i >> 5, r = (i & 31) << 2, k = k0 + kk;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k < K) {
        const float* x = X + (long long)k * s_k + r;
        if (r + 3 < R) {
          v = *reinterpret_cast<const float4*>(x);
        } else {
          if (r < R) v.x = x[0];
          if (r + 1 < R) v.y = x[1];
          if (r + 2 < R) v.z = x[2];
        }
      }
      *reinterpret_cast<float4*>(&S[kk][r]) = v;
    }
  } else {
    for (int i = tid; i < 128 * kBgK; i += 256) {
      const int kk = i >> 7, r = i & 127, k = k0 + kk;
      S[kk][r] = (r < R && k < K) ? X[(long long)r * s_r + (long long)k * s_k] : 0.f;
    }
  }
}

template <int TN>
__global__ void __launch_bounds__(256, TN == 2 ? 4 : 2) k_bgemm_small(Gemm<float> g, long long batch) {
  __shared__ __align__(16) float As[kBgK][kBgLd];
  __shared__ __align__(16) float Bs[kBgK][kBgLd];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (long long b = blockIdx.x; b < batch; b += gridDim.x) {
    const long long b1 = b / g.nb2, b2 = b - b1 * g.nb2;
    const float* A = g.A + b1 * g.a_b1 + b2 * g.a_b2;
    const float* B = g.B + b1 * g.b_b1 + b2 * g.b_b2;
    float* C = g.C + b1 * g.c_b1 + b2 * g.c_b2;
    float acc[8][TN];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < g.K; k0 += kBgK) {
      __syncthreads();   // the previous slice (or item) has been read
      // A(m, k) -> As[k - k0][m] and B(k, n) -> Bs[k - k0][n]; rows beyond
      // M (N) and k beyond K are zero
      stage_slice(A, g.a_rm, g.a_rk, g.M, g.K, k0, As);
      stage_slice(B, g.b_rn, g.b_rk, g.N, g.K, k0, Bs);
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < kBgK; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][4 * ty]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][64 + 4 * ty]);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        float bv[TN];
        if constexpr (TN == 8) {
          const float4 c0 = *reinterpret_cast<const float4*>(&Bs[kk][4 * tx]);
          const float4 c1 = *reinterpret_cast<const float4*>(&Bs[kk][64 + 4 * tx]);
          bv[0] = c0.x; bv[1] = c0.y; bv[2] = c0.z; bv[3] = c0.w;
          bv[4] = c1.x; bv[5] = c1.y; bv[6] = c1.z; bv[7] = c1.w;
        } else {
          const float2 c0 = *reinterpret_cast<const float2*>(&Bs[kk][2 * tx]);
          bv[0] = c0.x; bv[1] = c0.y;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], bv[j], acc[i][j]);
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int m = i < 4 ? 4 * ty + i : 64 + 4 * ty + i - 4;
      if (m >= g.M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int n = TN == 8 ? (j < 4 ? 4 * tx + j : 64 + 4 * tx + j - 4) : 2 * tx + j;
        if (n >= g.N) continue;
        const long long o = (long long)m * g.c_rm + (long long)n * g.c_rn;
        float v = g.alpha * acc[i][j];
        if (g.bias) v += g.bias[n];
        if (g.beta != 0.f) v += g.beta * C[o];
        if (g.epi == 1) v = tanhf(v);
        else if (g.epi == 2) {
          const float y = g.aux[b1 * g.c_b1 + b2 * g.c_b2 + o];
          v *= 1.f - y * y;
        }
        C[o] = v;
      }
    }
  }
}

template <typename T>
inline bool sgemm128_ok(const Gemm<T>& g, long long batch) {
  if constexpr (!std::is_same<T, float>::value) {
    return false;
  } else {
    auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    const bool b_rows = g.b_rn == 1 && g.b_rk % 4 == 0 && g.N % 4 == 0;   // B row-major
    const bool b_cols = g.b_rk == 1 && g.b_rn % 4 == 0;                   // B stored transposed
    return batch == 1 && g.a_rk == 1 && (b_rows || b_cols) && g.c_rn == 1 && g.a_rm % 4 == 0 &&
           al16(g.A) && al16(g.B) && g.M >= kSgBM &&
           g.K >= kSgBK && g.N >= 96;   // narrower products keep the 64 x 64 tiles
  }
}

template <typename T>
inline void gemm(const Gemm<T>& g, long long batch, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || batch <= 0) return;
  if constexpr (std::is_same<T, float>::value) {
    static int sms = 0;
    if (sms == 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (sms <= 0) sms = 148;
    }
    if (batch > 1 && g.M <= 128 && g.N <= 128 && !g.a_rows && !g.c_rows) {
      const long long grid = std::min<long long>(batch, (long long)sms * 8);
      if (g.N <= 32) k_bgemm_small<2><<<(unsigned)grid, 256, 0, st>>>(g, batch);
      else k_bgemm_small<8><<<(unsigned)grid, 256, 0, st>>>(g, batch);
      return;
    }
    if (sgemm128_ok(g, batch)) {
      const long long tiles = ((long long)(g.M + kSgBM - 1) / kSgBM) * ((g.N + kSgBN - 1) / kSgBN);
      // small products keep the 64 x 64 tiles, which give the GPU more CTAs
      if (tiles >= 2LL * sms && tiles <= 0x7fffffffLL) {
        k_sgemm128<float><<<(unsigned)tiles, 256, 0, st>>>(g);
        return;
      }
    }
  }
  int tiles = ((g.M + 63) / 64) * ((g.N + 63) / 64);
  long long by = batch < 65535 ? batch : 65535;
  long long bz = (batch + by - 1) / by;
  k_gemm<T><<<dim3(tiles, (unsigned)by, (unsigned)bz), 256, 0, st>>>(g, batch);
}

template <typename T>
inline Gemm<T> gemm_rowmajor(int M, int N, int K, const T* A, long long lda, const T* B,
                             long long ldb, T* C, long long ldc) {
  Gemm<T> g{};
  g.M = M; g.N = N; g.K = K;
  g.A = A; g.a_rm = lda; g.a_rk = 1;
  g.B = B; g.b_rk = ldb; g.b_rn = 1;
  g.C = C; g.c_rm = ldc; g.c_rn = 1;
  g.nb2 = 1;
  g.alpha = T(1);
  g.beta = T(0);
  return g;
}

}  // namespace dp
