// Kernels shared by the paths whose adjoint gathers per-slot values onto the
// neighbour atom (cross-atom message passing of the attention family, the
// graph family's messages): the atom channel's initial value and the reverse
// gather.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace dp {

// a stored per-slot value as the accumulation type
__device__ __forceinline__ float mp_val(float x) { return x; }
__device__ __forceinline__ double mp_val(double x) { return x; }
__device__ __forceinline__ float mp_val(__half x) { return __half2float(x); }
__device__ __forceinline__ float mp_val(__nv_bfloat16 x) { return __bfloat162float(x); }

// h_i = Wt[t_i]
template <typename T>
__global__ void k_mp_init(int n, int m1, const int* __restrict__ types, const T* __restrict__ Wt,
                          T* __restrict__ h) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)n * m1) return;
  const int i = (int)(q / m1), f = (int)(q % m1);
  h[q] = Wt[(long long)types[i] * m1 + f];
}

// dq_j = (sum over the slots (i, p) naming j of dG'_ip) * (1 - U_j^2), slot
// (i, p) being row i * row_stride + p of dG (U null: the plain sum).  The
// slots are found through j's skin list and summed in increasing i * nmax + p,
// so the result does not depend on the order the skin list holds them in.
// dG may be stored in 16 bits (S = __half or __nv_bfloat16 with T = float).
// One warp per atom; shared memory: 2 x cap ints per warp.
template <typename T, typename S = T>
__global__ void k_mp_gather(int n, int nmax, int row_stride, int m1, int cap,
                            const SkinEntry* __restrict__ skin, const int* __restrict__ skin_cnt, const int* __restrict__ mirror,
                            const short* __restrict__ selpos, const S* __restrict__ dG,
                            const T* __restrict__ U, T* __restrict__ dq) {
  extern __shared__ int mp_smem[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + wib;
  if (j >= n) return;
  int* keys = mp_smem + (size_t)wib * 2 * cap;
  int* ord = keys + cap;
  const int cnt = skin_cnt[j];
  int k = 0;
  for (int base = 0; base < cnt; base += 32) {
    const int c = base + lane;
    bool take = false;
    int key = 0;
    if (c < cnt) {
      const long long e = (long long)j * cap + c;
      const int i = skin[e].j, cp = mirror[e];
      if (cp >= 0) {
        const int p = selpos[(long long)i * cap + cp];
        if (p >= 0) {
          take = true;
          key = i * nmax + p;
        }
      }
    }
    const unsigned b = __ballot_sync(0xffffffffu, take);
    if (take) keys[k + __popc(b & ((1u << lane) - 1u))] = key;
    k += __popc(b);
  }
  __syncwarp();
  for (int q = lane; q < k; q += 32) {
    const int kq = keys[q];
    int r = 0;
    for (int t = 0; t < k; ++t) r += keys[t] < kq ? 1 : 0;
    const int i = kq / nmax;
    ord[r] = i * row_stride + (kq - i * nmax);     // the slot's row of dG
  }
  __syncwarp();
  if ((m1 & 1) == 0) {
    // lane owns column pairs 2 lane + 64 q; four rows in flight, summed in order
    for (int f = 2 * lane; f < m1; f += 64) {
      T a0 = T(0), a1 = T(0);
      int t = 0;
      for (; t + 4 <= k; t += 4) {
        T x0[4], x1[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const S* r = dG + (long long)ord[t + q] * m1 + f;
          x0[q] = mp_val(r[0]);
          x1[q] = mp_val(r[1]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          a0 += x0[q];
          a1 += x1[q];
        }
      }
      for (; t < k; ++t) {
        const S* r = dG + (long long)ord[t] * m1 + f;
        a0 += mp_val(r[0]);
        a1 += mp_val(r[1]);
      }
      if (U) {
        const T u0 = U[(long long)j * m1 + f], u1 = U[(long long)j * m1 + f + 1];
        a0 *= T(1) - u0 * u0;
        a1 *= T(1) - u1 * u1;
      }
      dq[(long long)j * m1 + f] = a0;
      dq[(long long)j * m1 + f + 1] = a1;
    }
    return;
  }
  for (int f = lane; f < m1; f += 32) {
    T acc = T(0);
    for (int t = 0; t < k; ++t) acc += mp_val(dG[(long long)ord[t] * m1 + f]);
    if (U) {
      const T u = U[(long long)j * m1 + f];
      acc *= T(1) - u * u;
    }
    dq[(long long)j * m1 + f] = acc;
  }
}

// The same sum for 128-wide features stored in the fused kernels' row-fastest
// layout: float4 group g of slot row p of atom i at (i * 32 + g) * 128 + p.
// Lane g owns columns 4g..4g+3.  Slots are visited in increasing i * nmax + p.
static __global__ void k_mp_gather4(int n, int nmax, int cap, const SkinEntry* __restrict__ skin,
                             const int* __restrict__ skin_cnt, const int* __restrict__ mirror,
                             const short* __restrict__ selpos, const float4* __restrict__ dG,
                             const float* __restrict__ U, float* __restrict__ dq) {
  extern __shared__ int mp_smem4[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + wib;
  if (j >= n) return;
  int* keys = mp_smem4 + (size_t)wib * 2 * cap;
  int* ord = keys + cap;
  const int cnt = skin_cnt[j];
  int k = 0;
  for (int base = 0; base < cnt; base += 32) {
    const int c = base + lane;
    bool take = false;
    int key = 0;
    if (c < cnt) {
      const long long e = (long long)j * cap + c;
      const int i = skin[e].j, cp = mirror[e];
      if (cp >= 0) {
        const int p = selpos[(long long)i * cap + cp];
        if (p >= 0) {
          take = true;
          key = i * nmax + p;
        }
      }
    }
    const unsigned b = __ballot_sync(0xffffffffu, take);
    if (take) keys[k + __popc(b & ((1u << lane) - 1u))] = key;
    k += __popc(b);
  }
  __syncwarp();
  for (int q = lane; q < k; q += 32) {
    const int kq = keys[q];
    int r = 0;
    for (int t = 0; t < k; ++t) r += keys[t] < kq ? 1 : 0;
    const int i = kq / nmax;
    ord[r] = i * 32 * 128 + (kq - i * nmax);     // float4 index of the slot's group 0
  }
  __syncwarp();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int t = 0; t < k; ++t) {
    const float4 v = dG[(long long)ord[t] + lane * 128];
    acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
  }
  const float4 u = reinterpret_cast<const float4*>(U + (long long)j * 128)[lane];
  reinterpret_cast<float4*>(dq + (long long)j * 128)[lane] =
      make_float4(acc.x * (1.f - u.x * u.x), acc.y * (1.f - u.y * u.y), acc.z * (1.f - u.z * u.z),
                  acc.w * (1.f - u.w * u.w));
}

}  // namespace dp
