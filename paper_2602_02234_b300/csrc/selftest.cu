// Diagnostics: one 128 x N x K BF16 tensor-core product on the device, with
// the operands staged in shared memory in K-major or MN-major core-matrix
// layout, so tests can check the tcgen05 operand conventions the fused
// kernels rely on against a host reference.
#include <math.h>

#include <string>

#include "common.cuh"
#include "tc.cuh"

namespace dp {

static constexpr int kStRegionA = 64 * 1024;
static constexpr int kStRegionB = 128 * 1024;
static constexpr int kStSmem = kStRegionA + kStRegionB + 64;

__global__ void __launch_bounds__(128) k_selftest_mma(int N, int K, const float* __restrict__ A,
                                                      const float* __restrict__ B, int a_mn,
                                                      int b_mn, uint32_t a_lbo, uint32_t a_sbo,
                                                      uint32_t b_lbo, uint32_t b_sbo,
                                                      float* __restrict__ D,
                                                      int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* As = sm;
  unsigned char* Bs = sm + kStRegionA;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kStRegionA + kStRegionB);
  uint32_t* tptr = reinterpret_cast<uint32_t*>(sm + kStRegionA + kStRegionB + 16);
  const int t = threadIdx.x;
  for (int i = t; i < (kStRegionA + kStRegionB) / 16; i += blockDim.x)
    reinterpret_cast<int4*>(sm)[i] = make_int4(0, 0, 0, 0);
  __syncthreads();
  for (int idx = t; idx < 128 * K; idx += blockDim.x) {
    int r = idx / K, k = idx % K;
    uint32_t off = a_mn ? tc::mnmajor_off(r, k, 128) : tc::kmajor_off(r, k, K);
    *reinterpret_cast<__nv_bfloat16*>(As + off) = __float2bfloat16(A[idx]);
  }
  for (int idx = t; idx < N * K; idx += blockDim.x) {
    int r = idx / K, k = idx % K;
    uint32_t off = b_mn ? tc::mnmajor_off(r, k, N) : tc::kmajor_off(r, k, K);
    *reinterpret_cast<__nv_bfloat16*>(Bs + off) = __float2bfloat16(B[idx]);
  }
  if (t == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
  }
  if (t < 32) {
    tc::tmem_alloc(tptr, 256);
    tc::tmem_relinquish();
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tptr;
  if (t == 0) {
    const uint32_t idesc = tc::idesc_bf16(128, N, a_mn, b_mn);
    for (int k0 = 0; k0 < K; k0 += 16) {
      uint32_t a_addr = tc::smem_u32(As) + (a_mn ? (k0 / 8) * (128 / 8) * 128 : (k0 / 8) * 128);
      uint32_t b_addr = tc::smem_u32(Bs) + (b_mn ? (k0 / 8) * (N / 8) * 128 : (k0 / 8) * 128);
      tc::mma_bf16(tbase, tc::make_desc(a_addr, a_lbo, a_sbo), tc::make_desc(b_addr, b_lbo, b_sbo),
                   idesc, k0 > 0 ? 1u : 0u);
    }
    tc::mma_commit(bar);
  }
  bool ok = tc::mbar_wait(bar, 0, 1LL << 24);
  if (!ok) atomicOr(status, 1);
  tc::fence_after_sync();
  const int w = t >> 5, lane = t & 31;
  if (ok) {
    for (int c = 0; c < N; c += 32) {
      float v[32];
      tc::tmem_ld32(tbase + ((uint32_t)(32 * w) << 16) + (uint32_t)c, v);
      for (int q = 0; q < 32; ++q)
        if (c + q < N) D[(32 * w + lane) * N + c + q] = v[q];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (t < 32) tc::tmem_dealloc(tbase, 256);
}

}  // namespace dp

using namespace dp;

// Largest byte offset an operand descriptor can reach for a tile of `rows`
// rows (any assignment of the two strides to the two directions).
static long long reach(long long start, int rows, uint32_t lbo, uint32_t sbo) {
  long long big = lbo > sbo ? lbo : sbo;
  return start + (long long)(rows / 8 + 2) * big + 128;
}

extern "C" int dp_selftest_mma(int n, int k, int a_mn, int b_mn, int swap, const float* A,
                               const float* B, float* D) {
  if (n < 16 || n > 256 || n % 16 || k < 16 || k > 128 || k % 16 || !A || !B || !D)
    return DP_ERR_ARG;
  // strides between neighbouring core matrices along K and along rows
  uint32_t a_k = a_mn ? 128u * (128 / 8) : 128u, a_r = a_mn ? 128u : 128u * (k / 8);
  uint32_t b_k = b_mn ? 128u * (n / 8) : 128u, b_r = b_mn ? 128u : 128u * (k / 8);
  uint32_t a_lbo = swap ? a_r : a_k, a_sbo = swap ? a_k : a_r;
  uint32_t b_lbo = swap ? b_r : b_k, b_sbo = swap ? b_k : b_r;
  long long a_start = a_mn ? (long long)(k / 8 - 2) * 16 * 128 : (long long)(k / 8 - 2) * 128;
  long long b_start = b_mn ? (long long)(k / 8 - 2) * (n / 8) * 128 : (long long)(k / 8 - 2) * 128;
  if (reach(a_start, 128, a_lbo, a_sbo) > kStRegionA || reach(b_start, n, b_lbo, b_sbo) > kStRegionB)
    return DP_ERR_ARG;  // a descriptor could reach outside the staged region
  float *dA = nullptr, *dB = nullptr, *dD = nullptr;
  int* dS = nullptr;
  int rc = DP_OK;
  if (cudaMalloc(&dA, sizeof(float) * 128 * k) || cudaMalloc(&dB, sizeof(float) * n * k) ||
      cudaMalloc(&dD, sizeof(float) * 128 * n) || cudaMalloc(&dS, sizeof(int))) {
    rc = DP_ERR_OOM;
  } else {
    cudaMemcpy(dA, A, sizeof(float) * 128 * k, cudaMemcpyHostToDevice);
    cudaMemcpy(dB, B, sizeof(float) * n * k, cudaMemcpyHostToDevice);
    cudaMemset(dD, 0, sizeof(float) * 128 * n);
    cudaMemset(dS, 0, sizeof(int));
    cudaFuncSetAttribute(k_selftest_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, kStSmem);
    k_selftest_mma<<<1, 128, kStSmem>>>(n, k, dA, dB, a_mn, b_mn, a_lbo, a_sbo, b_lbo, b_sbo, dD, dS);
    cudaError_t e = cudaDeviceSynchronize();
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&st, dS, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(D, dD, sizeof(float) * 128 * n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = DP_ERR_CUDA;
    else if (st) rc = DP_ERR_TIMEOUT;
  }
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dD);
  cudaFree(dS);
  return rc;
}

// A bounded wait that is made to run out: an mbarrier that nothing arrives on,
// polled max_polls times by every thread, exactly as the fused kernels wait
// for their tensor-core products and bulk copies.  The kernel records the
// timeout in a status word and returns normally.
__global__ void k_selftest_timeout(long long max_polls, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    dp::tc::mbar_init(&bar, 1);
    dp::tc::fence_mbar_init();
  }
  __syncthreads();
  bool ok = dp::tc::mbar_wait(&bar, 0, max_polls);
  ok = __syncthreads_and(ok) != 0;
  if (!ok && threadIdx.x == 0) atomicOr(status, dp::kFlagTimeout);
}

extern "C" int dp_selftest_timeout(long long max_polls) {
  if (max_polls < 1 || max_polls > (1LL << 20)) return DP_ERR_ARG;
  int* d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return DP_ERR_OOM;
  cudaMemset(d, 0, sizeof(int));
  k_selftest_timeout<<<1, 128>>>(max_polls, d);
  int st = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&st, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return DP_ERR_CUDA;
  return (st & dp::kFlagTimeout) ? DP_ERR_TIMEOUT : DP_OK;
}

// Issue-to-completion cost of 128 x N x 16 tensor-core products from shared
// memory: `reps` groups of 64 products (8 chains of K = 128 into four
// 128-column accumulators), issued by `issuers` threads (lane 0 of warps
// 0 .. issuers-1, each committing its own share), each group waited for.
// Thread 0's clock64 over all groups, divided by the products.
constexpr int kRateTile = 128 * 128 * 2;

__global__ void __launch_bounds__(512) k_selftest_mma_rate(int N, int issuers, int reps,
                                                           unsigned long long* cycles,
                                                           int* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tptr;
  __shared__ __align__(8) uint64_t bar;
  const int t = threadIdx.x, warp = t >> 5;
  for (int i = t; i < 2 * kRateTile / 16; i += blockDim.x)
    reinterpret_cast<int4*>(sm)[i] = make_int4(0, 0, 0, 0);
  if (t == 0) {
    dp::tc::mbar_init(&bar, (uint32_t)issuers);
    dp::tc::fence_mbar_init();
  }
  if (warp == 0) {
    dp::tc::tmem_alloc(&tptr, 512);
    dp::tc::tmem_relinquish();
  }
  dp::tc::fence_async_smem();
  dp::tc::fence_before_sync();
  __syncthreads();
  dp::tc::fence_after_sync();
  const uint32_t tb = tptr;
  const uint32_t a = dp::tc::smem_u32(sm), b = dp::tc::smem_u32(sm + kRateTile);
  const uint32_t idesc = dp::tc::idesc_bf16(128, N, 0, 0);
  // K-major 128 x 128 tiles: a K step of 16 is two core matrices (256 bytes)
  const uint64_t da0 = dp::tc::make_desc(a, 128u, 16u * 128u);
  const uint64_t db0 = dp::tc::make_desc(b, 128u, 16u * 128u);
  bool ok = true;
  uint32_t phase = 0;
  const unsigned long long t0 = clock64();
  for (int r = 0; r < reps; ++r) {
    if ((t & 31) == 0 && warp < issuers) {
      for (int g = warp; g < 8; g += issuers)
        for (int ks = 0; ks < 8; ++ks)
          dp::tc::mma_bf16(tb + (uint32_t)((g & 3) * 128), da0 + 16u * ks, db0 + 16u * ks, idesc,
                           ks > 0 ? 1u : 0u);
      dp::tc::mma_commit(&bar);
    }
    if (t == 0) ok = ok && dp::tc::mbar_wait(&bar, phase & 1u, 1LL << 22);
    phase ^= 1u;
    ok = __syncthreads_and(ok) != 0;
    dp::tc::fence_after_sync();
    if (!ok) break;
  }
  if (t == 0) {
    *cycles = clock64() - t0;
    if (!ok) atomicOr(status, dp::kFlagTimeout);
  }
  dp::tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) dp::tc::tmem_dealloc(tb, 512);
}

extern "C" int dp_selftest_mma_rate(int n, int issuers, int reps, double* cycles_per_mma) {
  if (n < 16 || n > 128 || n % 16 || issuers < 1 || issuers > 8 || reps < 1 || reps > 100000 ||
      !cycles_per_mma)
    return DP_ERR_ARG;
  unsigned long long* dc = nullptr;
  int* ds = nullptr;
  if (cudaMalloc(&dc, sizeof(unsigned long long)) != cudaSuccess) return DP_ERR_OOM;
  if (cudaMalloc(&ds, sizeof(int)) != cudaSuccess) {
    cudaFree(dc);
    return DP_ERR_OOM;
  }
  cudaMemset(ds, 0, sizeof(int));
  cudaFuncSetAttribute(k_selftest_mma_rate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       2 * kRateTile);
  unsigned long long c = 0;
  int st = 0;
  cudaError_t e = cudaSuccess;
  for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {   // the first pass warms up
    k_selftest_mma_rate<<<1, 512, 2 * kRateTile>>>(n, issuers, reps, dc, ds);
    e = cudaDeviceSynchronize();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&c, dc, sizeof(c), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&st, ds, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(dc);
  cudaFree(ds);
  if (e != cudaSuccess) return DP_ERR_CUDA;
  if (st & dp::kFlagTimeout) return DP_ERR_TIMEOUT;
  *cycles_per_mma = (double)c / ((double)reps * 64.0);
  return DP_OK;
}
