// Generic batched SIMT GEMM used by the plain (unfused) FP32 / FP64 paths.
#pragma once

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

template <typename T>
inline void gemm(const Gemm<T>& g, long long batch, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || batch <= 0) return;
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
