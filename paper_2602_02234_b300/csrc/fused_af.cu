// Fused attention-family model on the fifth-generation tensor cores.
//
// Same model as the plain path (paper Sec. II: "repinit" embedding, "repformer"
// residual self-attention, "fitting-net"; the library's reading of them), in
// three kernels per evaluation:
//
//   k_af_fwd   one CTA per SM, persistent over atoms; per atom the 128
//              neighbour slots are the 128 rows of every tile.  Environment
//              and softmax in FP32 registers (several threads per row, each
//              owning 32-column chunks of it), every matrix
//              product a tcgen05.mma from shared-memory 16-bit tiles (FP16
//              by default, BF16 when built with DP_FUSED_BF16) into FP32
//              tensor memory.  Writes the descriptor D (16-bit), T (FP32),
//              the layer inputs G_l (16-bit tiles) and LayerNorm 1/sigma.
//   k_fit      tiles of 128 atoms of one species: fitting MLP forward, atomic
//              energies (FP64 sum of FP32 products) and the input-gradient
//              chain down to dE/dD, all products on the tensor cores.
//   k_af_bwd   per atom again: recomputes Q, K, V and the softmax of each
//              layer from the stored G_l and runs the hand-written adjoint
//              to g_ij = dE/dr_ij.
//
// Tensor memory columns of the per-atom kernels: [0,128) R0, [128,256) R1,
// [256,384) R2 (the FP32 residual stream G, or its gradient), [384,512) R3.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "gemm.cuh"
#include "kernels.cuh"
#include "model.h"
#include "mp.cuh"
#include "tc.cuh"

namespace dp {
namespace fz {

// Tensor-core operand type: FP16 by default (10-bit mantissa; the backward
// seed is scaled by kGradScale to keep gradients in FP16's normal range), BF16
// when built with -DDP_FUSED_BF16.
#ifdef DP_FUSED_BF16
typedef __nv_bfloat16 op_t;
constexpr uint32_t kFmt = 1;
__device__ __forceinline__ uint32_t pack2(float a, float b) { return tc::pack_bf16(a, b); }
__device__ __forceinline__ float2 unpack2(uint32_t u) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
}
__device__ __forceinline__ float op2f(op_t v) { return __bfloat162float(v); }
__device__ __forceinline__ op_t f2op(float v) { return __float2bfloat16(v); }
#else
typedef __half op_t;
constexpr uint32_t kFmt = 0;
__device__ __forceinline__ uint32_t pack2(float a, float b) { return tc::pack_f16(a, b); }
__device__ __forceinline__ float2 unpack2(uint32_t u) {
  return __half22float2(*reinterpret_cast<const __half2*>(&u));
}
__device__ __forceinline__ float op2f(op_t v) { return __half2float(v); }
__device__ __forceinline__ op_t f2op(float v) { return __float2half_rn(v); }
#endif
constexpr float kGradScale = 4096.f;

constexpr int kW = 128;          // embedding / attention width and rows per atom tile
constexpr int kSplit = 4;                 // per-atom kernels: threads per neighbour row
constexpr int kThreads = kW * kSplit;     // 512 threads, 16 warps
constexpr int kStride = 32 * kSplit;      // column step between a thread's 32-column chunks
constexpr int kFitThreads = 128; // fitting kernel: one thread per atom row
constexpr long long kPolls = 1LL << 22;
constexpr uint32_t R0 = 0, R1 = 128, R2 = 256, R3 = 384;
constexpr int kTile = kW * kW * 2;  // one 128 x 128 16-bit tile: 32 KB
constexpr int kDH = 32;             // head width (4 heads over the 128 attention columns)

// Thread roles of the per-atom kernels.  Thread t serves neighbour row
// r = t mod 128, which is tensor-memory lane r (warp t/32 reads lane quarter
// (t/32) mod 4), and part p = t / 128 of that row's columns: the 32-column
// chunks starting at 32p, 32p + 32 kSplit, ...  Row sums over all columns
// combine the kSplit partial sums through `row_all` / `row_sum`.
__device__ __forceinline__ int row_id() { return threadIdx.x & (kW - 1); }
__device__ __forceinline__ int part_id() { return threadIdx.x >> 7; }
__device__ __forceinline__ uint32_t lane_base() {
  return (uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16;
}

// shared-memory map of the per-atom kernels (bytes)
constexpr int SM_G = 0, SM_Q = kTile, SM_K = 2 * kTile, SM_V = 3 * kTile, SM_P = 4 * kTile,
              SM_W = 5 * kTile, SM_MISC = 6 * kTile;
struct Misc {
  uint8_t ones[16 * kW * 2];  // 16 x 128 K-major operand: row 0 ones (column sums)
  uint8_t rhb[16 * kW * 2];   // rows 0..2: unit-vector components of each slot
  // per neighbour slot k: cl[0][k] = log2 sw (-inf if empty), cl[1..3][k] = unit vector
  __align__(16) float cl[4][kW];
  float4 xch[kSplit][kW];     // exchange of per-row partial results
  float sw[kW], dsw[kW], s[kW], d[kW];
  float rh[kW][3];
  float Rt[kW][4];
  __align__(16) float T[4][kW];   // also a bulk-copy destination
  float dT[4][kW];
  float dRt[kW][4];
  float drc[kW][3];
  float dswa[kW];
  int tj[kW];
  int mask;
  int nvalid;
  uint32_t tptr;
  int pad;
  unsigned long long bar, wbar, pbar, xbar;
};
constexpr int kSmemAtom = SM_MISC + (int)sizeof(Misc) + 64;
static_assert(kSmemAtom <= 227 * 1024, "per-atom shared memory");

struct Params {
  int n, nmax, e1, e2, m2, n_layers, heads, dh;
  int m1;                                 // real embedding width; columns [m1, 128) are padding
  float inv_m1;
  int atom0;                              // atoms [atom0, n) are evaluated
  float rs, rc, inv_nmax, inv_sqrt_d;
  const int* sel_j;
  const double* sel_r;
  const int* types;
  // 16-bit weight tiles (core-matrix layout), see the host packing below
  const uint8_t *W2T, *W3T, *W2R, *W3R;  // per species
  const uint8_t *WqT, *WkT, *WvT, *WoT;  // per layer, 32 KB each
  const uint8_t *WqR, *WkR, *WvR, *WoR;
  const float *W1, *b1, *b2, *b3, *bo;   // FP32 vectors
  uint8_t* Gst;                           // [n][L+1][32 KB]
  float* rstd;                            // [n][L][128]
  float* smx;                             // [n][L][heads][128] softmax log2-normaliser beta
  op_t* D;                                // [n][128 * m2]
  float* Tm;                              // [n][4][128]
  const float* dD;                        // [n][128 * m2]
  float* g;                               // [n][nmax][3]
  int* status;
  // cross-atom message passing: one launch per layer, this one does layers
  // [lb, le) (without message passing lb = 0, le = n_layers)
  int mp, lb, le, cap;
  uint8_t* Gpst;                          // [n][L][32 KB] layer inputs after the message
  // FP32 per-slot state between launches in a row-fastest layout: float4 group
  // g (columns 4g..4g+3) of slot row r of atom a at float4 index (a * 32 + g) * 128 + r,
  // so the 32 rows a warp holds move as one contiguous 512-byte access
  float* Gf32;                            // [n][32][128] float4: residual stream
  const float* U;                         // [L][cap][128] tanh(h Wm + bm) of each layer
  float* hbuf;                            // [n][128] atom channel h
  float* dG32;                            // [n][32][128] float4: scaled dE/dG' of the layer just done
  const float* hgrad;                     // [n][128] scaled dE/dh
  float* accs;                            // [n][8][128] dR~ (4), gate (3), dE/dsw between launches
};

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ uint64_t dK(uint32_t base, int Kx, int row0, int k0) {
  return tc::make_desc(base + (uint32_t)(((row0 >> 3) * (Kx >> 3) + (k0 >> 3)) * 128), 128u,
                       (uint32_t)((Kx >> 3) * 128));
}
// MN-major view of a K-major-stored tile: operand MN index = stored column,
// operand K index = stored row.
__device__ __forceinline__ uint64_t dMN(uint32_t base, int Kx, int mn0, int k0) {
  return tc::make_desc(base + (uint32_t)(((k0 >> 3) * (Kx >> 3) + (mn0 >> 3)) * 128),
                       (uint32_t)((Kx >> 3) * 128), 128u);
}

// An MMA operand: a K-major tile (Kx stored columns) read either directly
// (rows = operand M/N, stored columns koff.. = operand K) or through its
// MN-major view (stored columns mn0.. = operand M/N, stored rows koff.. = K).
struct Opnd {
  uint32_t base;
  int Kx, mn, mn0, koff;
};
__device__ __forceinline__ uint64_t odesc(const Opnd& o, int ks) {
  return o.mn ? dMN(o.base, o.Kx, o.mn0, o.koff + ks) : dK(o.base, o.Kx, 0, o.koff + ks);
}
__device__ __forceinline__ Opnd kop(const uint8_t* p, int Kx, int koff = 0) {
  return Opnd{tc::smem_u32(p), Kx, 0, 0, koff};
}
__device__ __forceinline__ Opnd mnop(const uint8_t* p, int Kx, int mn0, int koff = 0) {
  return Opnd{tc::smem_u32(p), Kx, 1, mn0, koff};
}
// Issue D (+)= A B over K (thread 0 only): K/16 instructions of 128 x N x 16.
// The descriptors are formed once: a K step of 16 moves a K-major operand by
// two core matrices (256 bytes) and an MN-major one by two row groups
// (32 Kx bytes); the start-address field counts 16-byte units and stays below
// 2^14 for any shared-memory address.
__device__ __forceinline__ void mma_issue(uint32_t d, const Opnd& A, const Opnd& B, int N, int K,
                                          bool acc) {
  const uint32_t id = tc::idesc_f16(128, N, A.mn, B.mn, kFmt);
  uint64_t da = odesc(A, 0), db = odesc(B, 0);
  const uint64_t ia = A.mn ? (uint64_t)(2 * A.Kx) : 16u, ib = B.mn ? (uint64_t)(2 * B.Kx) : 16u;
  for (int ks = 0; ks < K; ks += 16, da += ia, db += ib)
    tc::mma_bf16(d, da, db, id, (acc || ks > 0) ? 1u : 0u);
}

__device__ __forceinline__ void zero_smem(uint8_t* dst, int bytes) {
  int4* d = reinterpret_cast<int4*>(dst);
  for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = make_int4(0, 0, 0, 0);
}

// 8 consecutive values of row r, columns c..c+7 (c multiple of 8), as one
// 16-byte store into a K-major tile with Kx columns
__device__ __forceinline__ void store8(uint8_t* tile, int r, int c, int Kx, const float* v) {
  uint4 u;
  u.x = pack2(v[0], v[1]);
  u.y = pack2(v[2], v[3]);
  u.z = pack2(v[4], v[5]);
  u.w = pack2(v[6], v[7]);
  *reinterpret_cast<uint4*>(tile + tc::kmajor_off(r, c, Kx)) = u;
}
__device__ __forceinline__ void load8(const uint8_t* tile, int r, int c, int Kx, float* v) {
  uint4 u = *reinterpret_cast<const uint4*>(tile + tc::kmajor_off(r, c, Kx));
  const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float2 f = unpack2(w4[q]);
    v[2 * q] = f.x;
    v[2 * q + 1] = f.y;
  }
}
// store columns c..c+31 of row r, those below `ncol` only (ncol multiple of 8)
__device__ __forceinline__ void store32(uint8_t* tile, int r, int c, int Kx, int ncol,
                                        const float* v) {
#pragma unroll
  for (int q = 0; q < 32; q += 8)
    if (c + q < ncol) store8(tile, r, c + q, Kx, v + q);
}

// tanh by the hardware approximation (one instruction, relative error about
// 2^-11), for the embedding layers whose outputs only ever serve as 16-bit
// operands (rounded to the same size anyway).  G0, which also enters the FP32
// residual stream, and the fitting layers, which give the energy, use tanhf:
// their forward values must stay consistent with the 1 - y^2 the backward
// uses, or the forces stop being the gradient of the energy (NVE drift).
__device__ __forceinline__ float tanh_hw(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// The kSplit partial results of this thread's row, in part order.  Every
// thread of the block calls it (two barriers).  All threads of a row then
// combine the same values in the same order, so they never disagree on a row
// statistic.
__device__ __forceinline__ void row_all(Misc* m, float4 v, float4* all) {
  const int r = row_id();
  m->xch[part_id()][r] = v;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kSplit; ++i) all[i] = m->xch[i][r];
  __syncthreads();
}
__device__ __forceinline__ float4 row_sum(Misc* m, float4 v) {
  float4 all[kSplit];
  row_all(m, v, all);
  float4 s = all[0];
#pragma unroll
  for (int i = 1; i < kSplit; ++i) {
    s.x += all[i].x;
    s.y += all[i].y;
    s.z += all[i].z;
    s.w += all[i].w;
  }
  return s;
}

// Completion tracking on one mbarrier: every thread polls (bounded) and the
// outcome is made uniform across the CTA, so a timeout never strands part of
// the block at a barrier.
struct Bar {
  unsigned long long* bar;
  uint32_t phase;
  uint32_t commits = 1;   // arrivals the barrier takes per phase (product groups)
  __device__ bool wait(int* status) {
    bool ok = tc::mbar_wait(reinterpret_cast<uint64_t*>(bar), phase & 1u, kPolls);
    phase ^= 1u;
    ok = __syncthreads_and(ok) != 0;
    if (!ok && threadIdx.x == 0) atomicOr(status, kFlagTimeout);
    tc::fence_after_sync();
    return ok;
  }
  // Completion of tensor-core products: thread 0 polls, the block barrier
  // passes its outcome on (and orders the later tensor-memory loads).
  __device__ bool wait_mma(int* status) {
    bool ok = true;
    if (threadIdx.x == 0) ok = tc::mbar_wait(reinterpret_cast<uint64_t*>(bar), phase & 1u, kPolls);
    phase ^= 1u;
    ok = __syncthreads_and(ok) != 0;
    if (!ok && threadIdx.x == 0) atomicOr(status, kFlagTimeout);
    tc::fence_after_sync();
    return ok;
  }
};

__device__ __forceinline__ void before_mma() {
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
}

// Bulk (TMA) copy of `bytes` from global memory into a shared buffer,
// completing on `b`.  All threads call it; thread 0 issues after a barrier
// that orders every earlier access to the buffer before the copy.
__device__ __forceinline__ void bulk_load(Bar& b, uint8_t* dst, const void* src, uint32_t bytes) {
  tc::fence_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    tc::mbar_expect_tx(reinterpret_cast<uint64_t*>(b.bar), bytes);
    tc::bulk_g2s(dst, src, bytes, reinterpret_cast<uint64_t*>(b.bar));
  }
}

// Thread 0 only, after a barrier that ordered every earlier access to `dst`:
// arm `b` for `arm` bytes when arm > 0 (one arrival: the first copy of a group
// carries the group's total), then start the copy.
__device__ __forceinline__ void issue_copy(Bar& b, uint8_t* dst, const void* src, uint32_t bytes,
                                           uint32_t arm) {
  if (arm) tc::mbar_expect_tx(reinterpret_cast<uint64_t*>(b.bar), arm);
  tc::bulk_g2s(dst, src, bytes, reinterpret_cast<uint64_t*>(b.bar));
}

// Thread 0: the selected neighbours of the atom this CTA takes next, into L2
// while the current one runs (the environment set-up reads them first).
__device__ __forceinline__ void prefetch_env(const Params& p, int next) {
  tc::prefetch_l2(p.sel_j, (size_t)next * p.nmax * sizeof(int), (size_t)p.nmax * sizeof(int));
  tc::prefetch_l2(p.sel_r, (size_t)next * p.nmax * 3 * sizeof(double), (size_t)p.nmax * 3 * sizeof(double));
}

// One product group: barrier, issue by thread 0, commit to `mb` (as many
// times as the barrier takes arrivals), wait.
#define MMA_GROUP(mb, status, ...)                                   \
  do {                                                               \
    before_mma();                                                    \
    if (threadIdx.x == 0) {                                          \
      __VA_ARGS__;                                                   \
      for (uint32_t c_ = 0; c_ < (mb).commits; ++c_)                 \
        tc::mma_commit(reinterpret_cast<uint64_t*>((mb).bar));       \
    }                                                                \
    if (!(mb).wait_mma(status)) return false;                        \
  } while (0)
// The same with four issuing threads (lane 0 of warps 0-3), each issuing its
// own products (those that accumulate into one region stay with one thread)
// and committing once; `mb` takes four arrivals per phase.  A single thread
// issues one 128 x n x 16 product about every 72 cycles; four of them reach
// the rate the shared-memory operand reads allow (about 46 cycles for n <= 32).
#define MMA_GROUP4(mb, status, P0, P1, P2, P3)                       \
  do {                                                               \
    before_mma();                                                    \
    if ((threadIdx.x & 31) == 0 && threadIdx.x < 128) {              \
      const int w_ = threadIdx.x >> 5;                               \
      if (w_ == 0) { P0; }                                           \
      else if (w_ == 1) { P1; }                                      \
      else if (w_ == 2) { P2; }                                      \
      else { P3; }                                                   \
      tc::mma_commit(reinterpret_cast<uint64_t*>((mb).bar));         \
    }                                                                \
    if (!(mb).wait_mma(status)) return false;                        \
  } while (0)

// ------------------------------------------------------------------ environment
// Row t: switch, s = sw/r, R~, unit vector; empty slots zero.
__device__ void env_row(const Params& p, int atom, Misc* m, int t) {
  int j = t < p.nmax ? p.sel_j[(size_t)atom * p.nmax + t] : -1;
  if (j < 0) {
    m->sw[t] = 0.f; m->dsw[t] = 0.f; m->s[t] = 0.f; m->d[t] = 1.f;
    for (int a = 0; a < 3; ++a) m->rh[t][a] = 0.f;
    for (int a = 0; a < 4; ++a) m->Rt[t][a] = 0.f;
    m->cl[0][t] = -INFINITY;
    m->cl[1][t] = m->cl[2][t] = m->cl[3][t] = 0.f;
    m->tj[t] = -1;
    return;
  }
  size_t o = ((size_t)atom * p.nmax + t) * 3;
  float r[3] = {(float)p.sel_r[o], (float)p.sel_r[o + 1], (float)p.sel_r[o + 2]};
  float d = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  float sw, dsw;
  smooth_switch(d, p.rs, p.rc, &sw, &dsw);
  float s = sw / d;
  m->sw[t] = sw; m->dsw[t] = dsw; m->s[t] = s; m->d[t] = d;
  m->Rt[t][0] = s;
  for (int a = 0; a < 3; ++a) {
    m->rh[t][a] = r[a] / d;
    m->Rt[t][1 + a] = s * r[a] / d;
  }
  m->cl[0][t] = sw > 0.f ? log2f(sw) : -INFINITY;
  for (int a = 0; a < 3; ++a) m->cl[1 + a][t] = r[a] / d;
  m->tj[t] = p.types[j];
}

__device__ void atom_setup(const Params& p, int atom, Misc* m) {
  const int t = threadIdx.x;
  if (t == 0) {
    m->mask = 0;
    m->nvalid = 0;
  }
  __syncthreads();
  if (t < kW) {
    env_row(p, atom, m, t);
    if (m->tj[t] >= 0) {
      atomicOr(&m->mask, 1 << m->tj[t]);
      atomicMax(&m->nvalid, t + 1);
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------ embedding
// Species loop over the set bits of `mask` in increasing order: the weight
// block of species sp (bytes at base + sp * stride) arrives in one of two free
// tiles, the next species' block is already on its way into the other one
// while body(sp, tile) runs.  Barriers k0, k1 belong to the two tiles.
template <typename F>
__device__ bool species_loop(unsigned mask, const uint8_t* base, size_t stride, uint32_t bytes,
                             uint8_t* t0, uint8_t* t1, Bar& k0, Bar& k1, int* status, F&& body) {
  if (!mask) return true;
  int sp = __ffs(mask) - 1;
  int slot = 0;
  bulk_load(k0, t0, base + (size_t)sp * stride, bytes);
  while (sp >= 0) {
    const unsigned rest = sp < 31 ? mask & ~((2u << sp) - 1u) : 0u;
    const int nx = rest ? __ffs(rest) - 1 : -1;
    if (nx >= 0) bulk_load(slot ? k0 : k1, slot ? t0 : t1, base + (size_t)nx * stride, bytes);
    if (!(slot ? k1 : k0).wait(status)) return false;
    if (!body(sp, slot ? t1 : t0)) return false;
    sp = nx;
    slot ^= 1;
  }
  return true;
}

// Species loop in pairs: the set bits of `mask` in increasing order, two at a
// time; both species' weight blocks arrive together (tiles t0, t1 on k0, k1)
// and body(sa, t0, sb, t1) issues both products in one group (sb = -1 when
// the count is odd).  Most atoms see two species, so one product group does
// the work of two.
template <typename F>
__device__ bool species_pairs(unsigned mask, const uint8_t* base, size_t stride, uint32_t bytes,
                              uint8_t* t0, uint8_t* t1, Bar& k0, Bar& k1, int* status, F&& body) {
  while (mask) {
    const int sa = __ffs(mask) - 1;
    mask &= mask - 1u;
    const int sb = mask ? __ffs(mask) - 1 : -1;
    if (sb >= 0) mask &= mask - 1u;
    tc::fence_async_smem();
    __syncthreads();   // every earlier access to t0 and t1 is done
    if (threadIdx.x == 0) {
      issue_copy(k0, t0, base + (size_t)sa * stride, bytes, bytes);
      if (sb >= 0) issue_copy(k1, t1, base + (size_t)sb * stride, bytes, bytes);
    }
    if (!k0.wait(status)) return false;
    if (sb >= 0 && !k1.wait(status)) return false;
    if (!body(sa, t0, sb, t1)) return false;
  }
  return true;
}

// Layer 1 on the SIMT cores into the K-major tile H1, layer 2 on the tensor
// cores two species at a time into H2 (16-bit); weights through tiles w0, w1.
__device__ bool embed_h2(const Params& p, uint8_t* sm, Misc* m, uint32_t tb, Bar& mb, Bar& k0,
                         Bar& k1, uint8_t* H1, uint8_t* H2, uint8_t* w0, uint8_t* w1) {
  const int r = row_id(), pt = part_id();
  const uint32_t lo = lane_base();
  const int tj = m->tj[r];
  const float s = m->s[r];
  for (int c = 8 * pt; c < p.e1; c += 8 * kSplit) {
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      v[q] = tj >= 0 ? tanh_hw(s * p.W1[tj * p.e1 + c + q] + p.b1[tj * p.e1 + c + q]) : 0.f;
    store8(H1, r, c, p.e1, v);
  }
  for (int c = 8 * pt; c < p.e2; c += 8 * kSplit) {
    float z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    store8(H2, r, c, p.e2, z);
  }
  const uint32_t bytes = p.e2 * p.e1 * 2;
  const uint32_t rb = p.e2 <= 64 ? R0 + 64 : R1;   // the second species' accumulator
  return species_pairs((unsigned)m->mask, p.W2T, bytes, bytes, w0, w1, k0, k1, p.status,
                       [&](int sa, uint8_t* Wa, int sb, uint8_t* Wb) -> bool {
    MMA_GROUP4(mb, p.status, mma_issue(tb + R0, kop(H1, p.e1), kop(Wa, p.e1), p.e2, p.e1, false),
               if (sb >= 0) mma_issue(tb + rb, kop(H1, p.e1), kop(Wb, p.e1), p.e2, p.e1, false), (void)0,
               (void)0);
    const bool mine = tj >= 0 && (tj == sa || tj == sb);
    if (__any_sync(0xffffffffu, mine)) {
      for (int c = 16 * pt; c < p.e2; c += 16 * kSplit) {
        float v[16];
        if (sb >= 0) {
          float u[16];
          tc::tmem_ld16x2(tb + lo + R0 + c, v, tb + lo + rb + c, u);
          if (tj == sb) {
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = u[q];
          }
        } else {
          tc::tmem_ld16(tb + lo + R0 + c, v);
        }
        if (mine) {
#pragma unroll
          for (int q = 0; q < 16; ++q) v[q] = tanh_hw(v[q] + p.b2[tj * p.e2 + c + q]);
          store8(H2, r, c, p.e2, v);
          store8(H2, r, c + 8, p.e2, v + 8);
        }
      }
    }
    tc::fence_before_sync();
    return true;
  });
}

// G0 into the G tile (16-bit) and R2 (FP32).  Tiles: H1 in Q, H2 in K,
// weights through W and P.
__device__ bool embed_forward(const Params& p, uint8_t* sm, Misc* m, uint32_t tb, Bar& mb, Bar& wb,
                              Bar& xb) {
  const int r = row_id(), pt = part_id();
  const uint32_t lo = lane_base();
  uint8_t* H2 = sm + SM_K;
  uint8_t* Gt = sm + SM_G;
  if (!embed_h2(p, sm, m, tb, mb, wb, xb, sm + SM_Q, H2, sm + SM_W, sm + SM_P)) return false;
  const int tj = m->tj[r];
  zero_smem(Gt, kTile);
  {
    float z[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) z[q] = 0.f;
    for (int c = 32 * pt; c < kW; c += kStride) tc::tmem_st32(tb + lo + R2 + c, z);
  }
  const uint32_t bytes = kW * p.e2 * 2;
  // two species per product group: the first into R1, the second into R3
  return species_pairs((unsigned)m->mask, p.W3T, bytes, bytes, sm + SM_W, sm + SM_P, wb, xb,
                       p.status, [&](int sa, uint8_t* Wa, int sb, uint8_t* Wb) -> bool {
    MMA_GROUP4(mb, p.status, mma_issue(tb + R1, kop(H2, p.e2), kop(Wa, p.e2), kW, p.e2, false),
               if (sb >= 0) mma_issue(tb + R3, kop(H2, p.e2), kop(Wb, p.e2), kW, p.e2, false), (void)0,
               (void)0);
    const bool mine = tj >= 0 && (tj == sa || tj == sb);
    const uint32_t racc = sb >= 0 && tj == sb ? R3 : R1;
    if (__any_sync(0xffffffffu, mine)) {
      for (int c = 32 * pt; c < kW; c += kStride) {
#pragma unroll
        for (int c16 = 0; c16 < 32; c16 += 16) {
          float v[16], g[16];
          tc::tmem_ld16x2(tb + lo + R1 + c + c16, v, tb + lo + R2 + c + c16, g);
          if (sb >= 0) {
            float u[16];
            tc::tmem_ld16(tb + lo + R3 + c + c16, u);
            if (racc == R3) {
#pragma unroll
              for (int q = 0; q < 16; ++q) v[q] = u[q];
            }
          }
          if (mine) {
#pragma unroll
            for (int q = 0; q < 16; ++q) g[q] = tanhf(v[q] + p.b3[tj * kW + c + c16 + q]);   // G0 enters the FP32 residual stream
            store8(Gt, r, c + c16, kW, g);
            store8(Gt, r, c + c16 + 8, kW, g + 8);
          }
          tc::tmem_st16(tb + lo + R2 + c + c16, g);
        }
      }
    }
    tc::fence_before_sync();
    return true;
  });
}

// The three input projections of layer l arrive (on xb) in the Q, K and V
// tiles themselves.
__device__ void load_qkv_weights(const Params& p, int l, uint8_t* sm, Bar& xb) {
  tc::fence_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) {
    issue_copy(xb, sm + SM_Q, p.WqT + (size_t)l * kTile, kTile, 3 * kTile);
    issue_copy(xb, sm + SM_K, p.WkT + (size_t)l * kTile, kTile, 0);
    issue_copy(xb, sm + SM_V, p.WvT + (size_t)l * kTile, kTile, 0);
  }
}

// Q, K, V of one layer from the G tile in one product group (R0, R1, R3),
// then drained as 16-bit tiles over their weights.
__device__ bool qkv(const Params& p, uint8_t* sm, uint32_t tb, Bar& mb, Bar& xb) {
  const int r = row_id(), pt = part_id();
  const uint32_t lo = lane_base();
  if (!xb.wait(p.status)) return false;
  MMA_GROUP4(mb, p.status, mma_issue(tb + R0, kop(sm + SM_G, kW), kop(sm + SM_Q, kW), kW, kW, false),
             mma_issue(tb + R1, kop(sm + SM_G, kW), kop(sm + SM_K, kW), kW, kW, false),
             mma_issue(tb + R3, kop(sm + SM_G, kW), kop(sm + SM_V, kW), kW, kW, false), (void)0);
  const uint32_t src[3] = {R0, R1, R3};
  uint8_t* dst[3] = {sm + SM_Q, sm + SM_K, sm + SM_V};
#pragma unroll
  for (int q3 = 0; q3 < 3; ++q3)
    for (int c = 32 * pt; c < kW; c += kStride) {
      float v[32];
      tc::tmem_ld32(tb + lo + src[q3] + c, v);
      store32(dst[q3], r, c, kW, kW, v);
    }
  tc::fence_before_sync();
  return true;
}

// Packed FP32 pairs: two neighbour columns per instruction.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }

__device__ __forceinline__ float2 bc2(float x) { return make_float2(x, x); }

// gate r^_j . r^_k for the column pair (k, k+1); rj holds row j's components twice
__device__ __forceinline__ float2 gate2(const float2* rj, const Misc* m, int k) {
  return ffma2(rj[0], ld2(&m->cl[1][k]), ffma2(rj[1], ld2(&m->cl[2][k]), fmul2(rj[2], ld2(&m->cl[3][k]))));
}

// Softmax normaliser of row r of the head scores in tensor memory.  With
// u_jk = S_jk log2(e)/sqrt(d) + log2 sw_k (-inf for an empty column) the
// weights are w_jk = 2^(u_jk - beta_j), beta_j = log2 sum_k 2^u_jk; the parts of
// a row merge their partial (maximum, sum) pairs.  beta = +inf for an empty
// row, so that all its weights vanish.
// Each thread's part is one 32-column chunk, whose
// e_k = 2^(u_k - m) (m = the chunk's maximum) it leaves in tensor memory in
// place of the scores, so that the weights need no second exponential:
// w_k = e_k 2^(m - beta).  Returns {beta, 2^(m - beta)}.
static_assert(kStride == kW, "one 32-column chunk per thread");
__device__ float2 softmax_beta_keep(const Params& p, Misc* m, uint32_t taddr) {
  const float a = p.inv_sqrt_d * 1.4426950408889634f;
  const int nv = m->nvalid;
  const int c = 32 * part_id();
  float mx = -INFINITY, z = 0.f;
  if (c < nv) {
    float v[32];
    tc::tmem_ld32(taddr + c, v);
#pragma unroll
    for (int q = 0; q < 32; q += 2) {
      const float2 u = ffma2(make_float2(v[q], v[q + 1]), bc2(a), ld2(&m->cl[0][c + q]));
      v[q] = u.x;
      v[q + 1] = u.y;
      mx = fmaxf(mx, fmaxf(u.x, u.y));
    }
    const float2 nref = bc2(mx == -INFINITY ? 0.f : -mx);
    float2 zc[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
    for (int q = 0; q < 32; q += 2) {
      const float2 u = fadd2(make_float2(v[q], v[q + 1]), nref);
      v[q] = exp2f(u.x);
      v[q + 1] = exp2f(u.y);
      zc[(q >> 1) & 1] = fadd2(zc[(q >> 1) & 1], make_float2(v[q], v[q + 1]));
    }
    z = (zc[0].x + zc[1].x) + (zc[0].y + zc[1].y);
    tc::tmem_st32(taddr + c, v);
  }
  float4 all[kSplit];
  row_all(m, make_float4(mx, z, 0.f, 0.f), all);
  float b = all[0].x;
#pragma unroll
  for (int i = 1; i < kSplit; ++i) b = fmaxf(b, all[i].x);
  const float bref = b == -INFINITY ? 0.f : b;
  float Z = 0.f;
#pragma unroll
  for (int i = 0; i < kSplit; ++i) Z += __fmul_rn(all[i].y, exp2f(all[i].x - bref));
  const float beta = (Z > 0.f && row_id() < nv) ? bref + log2f(Z) : INFINITY;
  const float mref = mx == -INFINITY ? 0.f : mx;
  return make_float2(beta, exp2f(mref - beta));
}

// attention weights w_jk = 2^(u_jk - beta_j) of 32 columns from raw scores v
// (in place); empty columns and empty rows give 0
__device__ __forceinline__ void softmax_w(const Params& p, const Misc* m, int c, float beta,
                                          float* v) {
  const float a = p.inv_sqrt_d * 1.4426950408889634f;
#pragma unroll
  for (int q = 0; q < 32; q += 2) {
    const float2 u = fadd2(ffma2(make_float2(v[q], v[q + 1]), bc2(a), ld2(&m->cl[0][c + q])),
                           bc2(-beta));
    v[q] = exp2f(u.x);
    v[q + 1] = exp2f(u.y);
  }
}

// ------------------------------------------------------------------ forward
// Barriers: mb tensor-core products, wb the W tile (embedding weights, Wo),
// xb the projection weights.
template <bool MP>
__device__ bool fwd_atom(const Params& p, int atom, uint8_t* sm, Misc* m, uint32_t tb, Bar& mb,
                         Bar& wb, Bar& xb) {
  const int t = threadIdx.x, r = row_id(), pt = part_id();
  const uint32_t lo = lane_base();
  if (t == 0 && atom + (int)gridDim.x < p.n) {
    const int next = atom + (int)gridDim.x;
    prefetch_env(p, next);
    if (MP && p.lb > 0) tc::prefetch_l2(p.Gf32, (size_t)next * 32 * kW * 16, (size_t)32 * kW * 16);
  }
  atom_setup(p, atom, m);
  const int ngroups = (m->nvalid + 7) >> 3;
  if (ngroups == 0) {   // no neighbours: R~ = 0, so T = 0 and D = 0 (the fitting still runs)
    op_t* Drow = p.D + (size_t)atom * kW * p.m2;
    for (int i = t; i < kW * p.m2; i += kThreads) Drow[i] = f2op(0.f);
    for (int i = t; i < 4 * kW; i += kThreads) p.Tm[(size_t)atom * 4 * kW + i] = 0.f;
    __syncthreads();
    return true;
  }
  uint8_t* Gdst = p.Gst + (size_t)atom * (p.n_layers + 1) * kTile;
  if (!MP || p.lb == 0) {
    if (!embed_forward(p, sm, m, tb, mb, wb, xb)) return false;
    if (p.le > 0) load_qkv_weights(p, 0, sm, xb);   // H1, H2 tiles are free again
    __syncthreads();
    for (int i = t; i < ngroups * 2048 / 16; i += kThreads)
      reinterpret_cast<int4*>(Gdst)[i] = reinterpret_cast<const int4*>(sm + SM_G)[i];
  } else {   // message passing: the residual stream left by the previous launch
    load_qkv_weights(p, p.lb, sm, xb);
    const float4* src = reinterpret_cast<const float4*>(p.Gf32) + (size_t)atom * 32 * kW + r;
    for (int c = 32 * pt; c < kW; c += kStride) {
      float g[32];
#pragma unroll
      for (int q = 0; q < 32; q += 4) {
        const float4 v = src[(size_t)((c + q) >> 2) * kW];
        g[q] = v.x; g[q + 1] = v.y; g[q + 2] = v.z; g[q + 3] = v.w;
      }
      tc::tmem_st32(tb + lo + R2 + c, g);
    }
  }
  const bool valid = m->tj[r] >= 0;
  const float2 rj[3] = {make_float2(m->cl[1][r], m->cl[1][r]), make_float2(m->cl[2][r], m->cl[2][r]),
                        make_float2(m->cl[3][r], m->cl[3][r])};
  const int l_end = MP ? p.le : p.n_layers;
  for (int l = MP ? p.lb : 0; l < l_end; ++l) {
    if constexpr (MP) {
      // message: G' = G + U of the slot's neighbour, into R2 (FP32) and the G
      // tile (16-bit, also kept for the backward's recomputation)
      const int jr = r < p.nmax ? p.sel_j[(size_t)atom * p.nmax + r] : -1;
      const float* u = p.U + ((size_t)l * p.cap + (jr >= 0 ? jr : 0)) * kW;
      for (int c = 32 * pt; c < kW; c += kStride) {
        float g[32];
        tc::tmem_ld32(tb + lo + R2 + c, g);
        if (jr >= 0) {
#pragma unroll
          for (int q = 0; q < 32; q += 4) {
            const float4 v = *reinterpret_cast<const float4*>(u + c + q);
            g[q] += v.x; g[q + 1] += v.y; g[q + 2] += v.z; g[q + 3] += v.w;
          }
        }
        tc::tmem_st32(tb + lo + R2 + c, g);
        store32(sm + SM_G, r, c, kW, kW, g);
      }
      tc::fence_before_sync();
      __syncthreads();
      uint8_t* gp = p.Gpst + ((size_t)atom * p.n_layers + l) * kTile;
      for (int i = t; i < ngroups * 2048 / 16; i += kThreads)
        reinterpret_cast<int4*>(gp)[i] = reinterpret_cast<const int4*>(sm + SM_G)[i];
    }
    if (!qkv(p, sm, tb, mb, xb)) return false;
    bulk_load(wb, sm + SM_W, p.WoT + (size_t)l * kTile, kTile);  // lands during the heads
    MMA_GROUP(mb, p.status,
              mma_issue(tb + R3, kop(sm + SM_Q, kW), kop(sm + SM_K, kW), kW, kDH, false));
    for (int h = 0; h < p.heads; ++h) {
      const float2 st = softmax_beta_keep(p, m, tb + lo + R3);
      if (pt == 0) p.smx[(((size_t)atom * p.n_layers + l) * p.heads + h) * kW + r] = st.x;
      for (int c = 32 * pt; c < kW; c += kStride) {
        float v[32];
        if (c < m->nvalid) {
          tc::tmem_ld32(tb + lo + R3 + c, v);   // e_k = 2^(u_k - m)
#pragma unroll
          for (int q = 0; q < 32; q += 2) {
            const float2 w = fmul2(fmul2(make_float2(v[q], v[q + 1]), bc2(st.y)), gate2(rj, m, c + q));
            v[q] = w.x;
            v[q + 1] = w.y;
          }
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) v[q] = 0.f;
        }
        store32(sm + SM_P, r, c, kW, kW, v);
      }
      tc::fence_before_sync();
      // O_h = A V_h as two halves of the neighbour sum (R0 and R1, added at
      // the drain) and the next head's scores (R3 has been read), from three
      // issuing threads
      MMA_GROUP4(mb, p.status,
                 mma_issue(tb + R0 + h * kDH, kop(sm + SM_P, kW), mnop(sm + SM_V, kW, h * kDH), kDH,
                           kW / 2, false),
                 mma_issue(tb + R1 + h * kDH, kop(sm + SM_P, kW, kW / 2),
                           mnop(sm + SM_V, kW, h * kDH, kW / 2), kDH, kW / 2, false),
                 if (h + 1 < p.heads)
                   mma_issue(tb + R3, kop(sm + SM_Q, kW, (h + 1) * kDH),
                             kop(sm + SM_K, kW, (h + 1) * kDH), kW, kDH, false),
                 (void)0);
    }
    for (int c = 32 * pt; c < kW; c += kStride) {
      float v[32], u[32];
      tc::tmem_ld32(tb + lo + R0 + c, v);
      tc::tmem_ld32(tb + lo + R1 + c, u);
#pragma unroll
      for (int q = 0; q < 32; ++q) v[q] += u[q];
      store32(sm + SM_Q, r, c, kW, kW, v);
    }
    tc::fence_before_sync();
    if (!wb.wait(p.status)) return false;
    MMA_GROUP(mb, p.status, mma_issue(tb + R1, kop(sm + SM_Q, kW), kop(sm + SM_W, kW), kW, kW, false));
    // next layer's projections land in the free Q, K, V tiles during the LayerNorm
    if (l + 1 < l_end) load_qkv_weights(p, l + 1, sm, xb);
    // residual + LayerNorm over the row's real columns: the sum and the sum of
    // squares of z = G + Y + bo in one pass and one row exchange (z is 0 in
    // the padding columns), variance = mean(z^2) - mean(z)^2
    const float* bo = p.bo + l * kW;
    // real columns: every column with message passing (it needs m1 = 128)
    const int m1 = MP ? kW : p.m1;
    const float inv_m1 = MP ? 1.f / kW : p.inv_m1;
    float sum = 0.f, sq = 0.f;
    for (int c = 32 * pt; c < kW; c += kStride) {
      float g[32], y[32];
      tc::tmem_ld32(tb + lo + R2 + c, g);
      tc::tmem_ld32(tb + lo + R1 + c, y);
      float s4[4] = {0.f, 0.f, 0.f, 0.f}, q4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const float z = g[q] + y[q] + bo[c + q];
        s4[q & 3] += z;
        q4[q & 3] += z * z;
      }
      sum += (s4[0] + s4[1]) + (s4[2] + s4[3]);
      sq += (q4[0] + q4[1]) + (q4[2] + q4[3]);
    }
    {
      const float4 o = row_sum(m, make_float4(sum, sq, 0.f, 0.f));
      sum = o.x;
      sq = o.y;
    }
    const float mu = sum * inv_m1;
    const float var = fmaxf(sq * inv_m1 - mu * mu, 0.f);
    const float rs = valid ? rsqrtf(var + 1e-5f) : 0.f;
    for (int c = 32 * pt; c < kW; c += kStride) {
      float g[32], y[32];
      tc::tmem_ld32(tb + lo + R2 + c, g);
      tc::tmem_ld32(tb + lo + R1 + c, y);
#pragma unroll
      for (int q = 0; q < 32; ++q) g[q] = c + q < m1 ? (g[q] + y[q] + bo[c + q] - mu) * rs : 0.f;
      tc::tmem_st32(tb + lo + R2 + c, g);
      store32(sm + SM_G, r, c, kW, kW, g);
    }
    if (pt == 0) p.rstd[((size_t)atom * p.n_layers + l) * kW + r] = rs;
    tc::fence_before_sync();
    __syncthreads();
    uint8_t* dst = Gdst + (size_t)(l + 1) * kTile;
    for (int i = t; i < ngroups * 2048 / 16; i += kThreads)
      reinterpret_cast<int4*>(dst)[i] = reinterpret_cast<const int4*>(sm + SM_G)[i];
    if (MP && l + 1 < p.n_layers) {
      // atom channel: h_i += (1/Nmax) sum_r sw_r G[r][c].  Each warp sums its
      // 32 rows of its 32 columns by a butterfly (lane q ends with column
      // c + q), then the four row quarters are added in order.
      float v[32];
      tc::tmem_ld32(tb + lo + R2 + 32 * pt, v);
      const float swr = m->sw[r];
#pragma unroll
      for (int q = 0; q < 32; ++q) v[q] *= swr;
      const int lane = t & 31;
#pragma unroll
      for (int w = 16; w >= 1; w >>= 1) {
        const bool up = (lane & w) != 0;
#pragma unroll
        for (int q = 0; q < w; ++q) {
          const float send = up ? v[q] : v[q + w];
          const float keep = up ? v[q + w] : v[q];
          v[q] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
      }
      float* xs = reinterpret_cast<float*>(&m->xch[0][0]);   // [row quarter][column]
      xs[((t >> 5) & 3) * kW + 32 * pt + lane] = v[0];
      __syncthreads();
      if (pt == 0)
        p.hbuf[(size_t)atom * kW + r] += ((xs[r] + xs[kW + r]) + (xs[2 * kW + r] + xs[3 * kW + r])) * p.inv_nmax;
      __syncthreads();
    }
  }
  if (MP && p.le < p.n_layers) {   // message passing: the next launch continues from R2
    float4* dstf = reinterpret_cast<float4*>(p.Gf32) + (size_t)atom * 32 * kW + r;
    for (int c = 32 * pt; c < kW; c += kStride) {
      float g[32];
      tc::tmem_ld32(tb + lo + R2 + c, g);
#pragma unroll
      for (int q = 0; q < 32; q += 4)
        dstf[(size_t)((c + q) >> 2) * kW] = make_float4(g[q], g[q + 1], g[q + 2], g[q + 3]);
    }
    tc::fence_before_sync();
    __syncthreads();
    return true;
  }
  // descriptor: T[a][f] = (1/Nmax) sum_j R~[j][a] G[j][f]; feature f = row id,
  // neighbours j split between the parts of a row
  const int f = r;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int j = pt; j < m->nvalid; j += kSplit) {
    float gv = op2f(*reinterpret_cast<const op_t*>(sm + SM_G + tc::kmajor_off(j, f, kW)));
#pragma unroll
    for (int a = 0; a < 4; ++a) acc[a] += m->Rt[j][a] * gv;
  }
  {
    const float4 o = row_sum(m, make_float4(acc[0], acc[1], acc[2], acc[3]));
    acc[0] = o.x; acc[1] = o.y; acc[2] = o.z; acc[3] = o.w;
  }
  if (pt == 0) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      m->T[a][f] = acc[a] * p.inv_nmax;
      p.Tm[((size_t)atom * 4 + a) * kW + f] = acc[a] * p.inv_nmax;
    }
  }
  __syncthreads();
  op_t* Drow = p.D + (size_t)atom * kW * p.m2 + (size_t)f * p.m2;
  for (int q = pt; q < p.m2; q += kSplit) {
    float v = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) v += m->T[a][f] * m->T[a][q];
    Drow[q] = f2op(v);
  }
  __syncthreads();
  return true;
}

__device__ void kernel_prologue(Misc* m, uint32_t product_arrivals) {
  const int t = threadIdx.x, warp = t >> 5;
  if (t == 0) {
    tc::mbar_init(reinterpret_cast<uint64_t*>(&m->bar), product_arrivals);
    tc::mbar_init(reinterpret_cast<uint64_t*>(&m->wbar), 1);
    tc::mbar_init(reinterpret_cast<uint64_t*>(&m->pbar), 1);
    tc::mbar_init(reinterpret_cast<uint64_t*>(&m->xbar), 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(&m->tptr, 512);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
}

__device__ void kernel_epilogue(Misc* m) {
  tc::fence_before_sync();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(m->tptr, 512);
}

template <bool MP>
__global__ void __launch_bounds__(kThreads, 1) k_af_fwd(Params p) {
  extern __shared__ __align__(1024) uint8_t sm[];
  Misc* m = reinterpret_cast<Misc*>(sm + SM_MISC);
  kernel_prologue(m, 4);   // product groups with up to four issuers
  Bar mb{&m->bar, 0u, 4u}, wb{&m->wbar, 0u}, xb{&m->xbar, 0u};
  for (int atom = p.atom0 + blockIdx.x; atom < p.n; atom += gridDim.x)
    if (!fwd_atom<MP>(p, atom, sm, m, m->tptr, mb, wb, xb)) break;
  kernel_epilogue(m);
}

// ------------------------------------------------------------------ backward
// Adjoint of one atom: dE/dD (from the fitting kernel) back to g_ij.
// Barriers: mb tensor-core products, gb stored activation tiles, wb and xb
// weight tiles (xb also dE/dD and T at the start of an atom).
template <bool MP>
__device__ bool bwd_atom(const Params& p, int atom, uint8_t* sm, Misc* m, uint32_t tb, Bar& mb,
                         Bar& wb, Bar& gb, Bar& xb) {
  const int t = threadIdx.x, r = row_id(), pt = part_id();
  const uint32_t lo = lane_base();
  // dE/dD (into the P tile, FP32) and T arrive by bulk copy during the setup
  const int L = p.n_layers;
  const bool top = !MP || p.le == L;   // this launch starts at the descriptor
  tc::fence_async_smem();
  __syncthreads();
  if (t == 0 && top) {
    const uint32_t bd = kW * p.m2 * 4, bt = 4 * kW * 4;
    issue_copy(xb, sm + SM_P, p.dD + (size_t)atom * kW * p.m2, bd, bd + bt);
    issue_copy(xb, reinterpret_cast<uint8_t*>(&m->T[0][0]), p.Tm + (size_t)atom * 4 * kW, bt, 0);
  }
  atom_setup(p, atom, m);
  const int ngroups = (m->nvalid + 7) >> 3;
  const uint8_t* Gsrc = p.Gst + (size_t)atom * (L + 1) * kTile;
  const uint8_t* Gpsrc = MP ? p.Gpst + (size_t)atom * L * kTile : Gsrc;
  const bool valid = m->tj[r] >= 0;
  constexpr int DH = kDH;
  const int nv = m->nvalid;
  // load a stored G tile: real row groups by bulk copy, the rest zero
  auto load_G = [&](uint8_t* dst, int l, Bar& b) {
    zero_smem(dst + ngroups * 2048, kTile - ngroups * 2048);
    if (ngroups > 0) bulk_load(b, dst, Gsrc + (size_t)l * kTile, ngroups * 2048);
  };
  // ---- descriptor adjoint: dT[a][f] = sum_q dD[f][q] T[a][q] + sum_g dD[g][f] T[a][g]
  // (the second sum for f < m2 only); feature f = row id, the 128-term sum split
  if (top) {
    load_G(sm + SM_G, L, gb);   // the last layer's output, for dG_L below
    if (!xb.wait(p.status)) return false;
  }
  if (ngroups == 0) {   // no neighbours: no pair gradients (no copy was issued on gb)
    for (int i = t; i < p.nmax * 3; i += kThreads) p.g[(size_t)atom * p.nmax * 3 + i] = 0.f;
    __syncthreads();
    return true;
  }
  if (!top) {
    // message passing: dE/dG' of layer le and the accumulated sums, as the
    // previous launch left them (the cross-atom step ran in between)
    const float4* src = reinterpret_cast<const float4*>(p.dG32) + (size_t)atom * 32 * kW + r;
    for (int c = 32 * pt; c < kW; c += kStride) {
      float g[32];
#pragma unroll
      for (int q = 0; q < 32; q += 4) {
        const float4 v = src[(size_t)((c + q) >> 2) * kW];
        g[q] = v.x; g[q + 1] = v.y; g[q + 2] = v.z; g[q + 3] = v.w;
      }
      tc::tmem_st32(tb + lo + R2 + c, g);
    }
    if (pt == 0) {
      const float* a = p.accs + (size_t)atom * 8 * kW + r;
      for (int q = 0; q < 4; ++q) m->dRt[r][q] = a[q * kW];
      for (int q = 0; q < 3; ++q) m->drc[r][q] = a[(4 + q) * kW];
      m->dswa[r] = a[7 * kW];
      for (int q = 0; q < 3; ++q)
        *reinterpret_cast<op_t*>(m->rhb + tc::kmajor_off(q, r, kW)) = f2op(valid ? m->rh[r][q] : 0.f);
    }
    __syncthreads();
  } else {   // descriptor adjoint
  {
    const int f = r;
    const float* dDs = reinterpret_cast<const float*>(sm + SM_P);   // 128 x m2 FP32
    float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (pt == 0)
        for (int q = 0; q < p.m2; ++q) v[a] += dDs[f * p.m2 + q] * m->T[a][q];
      if (f < p.m2)
        for (int g = (kW / kSplit) * pt; g < (kW / kSplit) * (pt + 1); ++g)
          v[a] += dDs[g * p.m2 + f] * m->T[a][g];
    }
    const float4 o = row_sum(m, make_float4(v[0], v[1], v[2], v[3]));
    if (pt == 0) {
      m->dT[0][f] = o.x;
      m->dT[1][f] = o.y;
      m->dT[2][f] = o.z;
      m->dT[3][f] = o.w;
    }
  }
  if (ngroups > 0 && !gb.wait(p.status)) return false;
  __syncthreads();
  {
    float dr[4] = {0.f, 0.f, 0.f, 0.f};
    float rt[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) rt[a] = m->Rt[r][a];
    for (int c = 32 * pt; c < kW; c += kStride) {
      float g[32];
#pragma unroll
      for (int q = 0; q < 32; q += 8) load8(sm + SM_G, r, c + q, kW, g + q);
      float dg[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int f = c + q;
#pragma unroll
        for (int a = 0; a < 4; ++a) dr[a] += m->dT[a][f] * g[q];
        dg[q] = valid ? kGradScale * p.inv_nmax *
                            (m->dT[0][f] * rt[0] + m->dT[1][f] * rt[1] + m->dT[2][f] * rt[2] +
                             m->dT[3][f] * rt[3])
                      : 0.f;
      }
      tc::tmem_st32(tb + lo + R2 + c, dg);
    }
    const float4 o = row_sum(m, make_float4(dr[0], dr[1], dr[2], dr[3]));
    if (pt == 0) {
      m->dRt[r][0] = o.x * p.inv_nmax;
      m->dRt[r][1] = o.y * p.inv_nmax;
      m->dRt[r][2] = o.z * p.inv_nmax;
      m->dRt[r][3] = o.w * p.inv_nmax;
      m->dswa[r] = 0.f;
      m->drc[r][0] = m->drc[r][1] = m->drc[r][2] = 0.f;
      // gate column-sum operand: rows 0..2 = rh components of neighbour r (column r)
      for (int a = 0; a < 3; ++a)
        *reinterpret_cast<op_t*>(m->rhb + tc::kmajor_off(a, r, kW)) =
            f2op(valid ? m->rh[r][a] : 0.f);
    }
  }
  }
  const float2 rj[3] = {make_float2(m->cl[1][r], m->cl[1][r]), make_float2(m->cl[2][r], m->cl[2][r]),
                        make_float2(m->cl[3][r], m->cl[3][r])};
  for (int l = (MP ? p.le : L) - 1; l >= (MP ? p.lb : 0); --l) {
    // ---- loads of this layer, all in flight at once: the stored layer input
    // (G tile) and output (V tile) on gb, Wo^T (W tile) on wb, and the Q and
    // K weights (Q and K tiles, overwritten by the recomputed Q and K) on xb
    zero_smem(sm + SM_G + ngroups * 2048, kTile - ngroups * 2048);
    zero_smem(sm + SM_V + ngroups * 2048, kTile - ngroups * 2048);
    tc::fence_async_smem();
    __syncthreads();
    if (t == 0) {
      if (ngroups > 0) {
        issue_copy(gb, sm + SM_G, Gpsrc + (size_t)l * kTile, ngroups * 2048, 2 * ngroups * 2048);
        issue_copy(gb, sm + SM_V, Gsrc + (size_t)(l + 1) * kTile, ngroups * 2048, 0);
      }
      issue_copy(wb, sm + SM_W, p.WoR + (size_t)l * kTile, kTile, kTile);
      issue_copy(xb, sm + SM_Q, p.WqT + (size_t)l * kTile, kTile, 2 * kTile);
      issue_copy(xb, sm + SM_K, p.WkT + (size_t)l * kTile, kTile, 0);
    }
    // the layer's softmax normalisers (one per head), needed by the heads below
    // (with message passing read per head, which keeps the variant's live
    // state within its registers)
    float beta4[4];
    if constexpr (!MP) {
#pragma unroll
      for (int h = 0; h < 4; ++h) beta4[h] = p.smx[(((size_t)atom * L + l) * 4 + h) * kW + r];
    }
    if (ngroups > 0 && !gb.wait(p.status)) return false;
    if (MP && l + 1 < L) {
      // adjoint of h^{l+1} = h^l + (1/Nmax) sum_r sw_r G_{l+1}[r]: dG_{l+1}[r] +=
      // (sw_r / Nmax) dh, dE/dsw_r += (1/Nmax) G_{l+1}[r] . dh (G_{l+1} in the V tile)
      const float sc = m->sw[r] * p.inv_nmax;
      const float* dhr = p.hgrad + (size_t)atom * kW;
      float dot = 0.f;
      for (int c = 32 * pt; c < kW; c += kStride) {
        float a4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int h16 = 0; h16 < 32; h16 += 16) {   // 16 columns at a time (register budget)
          float dg[16], go[16];
          tc::tmem_ld16(tb + lo + R2 + c + h16, dg);
          load8(sm + SM_V, r, c + h16, kW, go);
          load8(sm + SM_V, r, c + h16 + 8, kW, go + 8);
#pragma unroll
          for (int q = 0; q < 16; q += 4) {
            const float4 d = *reinterpret_cast<const float4*>(dhr + c + h16 + q);
            dg[q] += sc * d.x; dg[q + 1] += sc * d.y; dg[q + 2] += sc * d.z; dg[q + 3] += sc * d.w;
            a4[0] += go[q] * d.x; a4[1] += go[q + 1] * d.y; a4[2] += go[q + 2] * d.z; a4[3] += go[q + 3] * d.w;
          }
          tc::tmem_st16(tb + lo + R2 + c + h16, dg);
        }
        dot += (a4[0] + a4[1]) + (a4[2] + a4[3]);
      }
      dot = row_sum(m, make_float4(dot, 0.f, 0.f, 0.f)).x;
      if (pt == 0 && valid) m->dswa[r] += dot * p.inv_nmax;
    }
    // ---- LayerNorm adjoint: dZ = rstd (dG - mean dG - Gout mean(dG Gout))
    {
      const float rs = p.rstd[((size_t)atom * L + l) * kW + r];
      float s1 = 0.f, s2 = 0.f;
      for (int c = 32 * pt; c < kW; c += kStride) {
        float dg[32], go[32];
        tc::tmem_ld32(tb + lo + R2 + c, dg);
#pragma unroll
        for (int q = 0; q < 32; q += 8) load8(sm + SM_V, r, c + q, kW, go + q);
        float a4[4] = {0.f, 0.f, 0.f, 0.f}, b4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          a4[q & 3] += dg[q];
          b4[q & 3] += dg[q] * go[q];
        }
        s1 += (a4[0] + a4[1]) + (a4[2] + a4[3]);
        s2 += (b4[0] + b4[1]) + (b4[2] + b4[3]);
      }
      const float4 o = row_sum(m, make_float4(s1, s2, 0.f, 0.f));
      const int m1 = MP ? kW : p.m1;   // message passing needs m1 = 128
      s1 = o.x * (MP ? 1.f / kW : p.inv_m1);
      s2 = o.y * (MP ? 1.f / kW : p.inv_m1);
      for (int c = 32 * pt; c < kW; c += kStride) {
        float dg[32], go[32];
        tc::tmem_ld32(tb + lo + R2 + c, dg);
#pragma unroll
        for (int q = 0; q < 32; q += 8) load8(sm + SM_V, r, c + q, kW, go + q);
#pragma unroll
        for (int q = 0; q < 32; ++q)
          dg[q] = valid && c + q < m1 ? rs * (dg[q] - s1 - go[q] * s2) : 0.f;
        tc::tmem_st32(tb + lo + R2 + c, dg);
        store32(sm + SM_P, r, c, kW, kW, dg);
      }
      tc::fence_before_sync();
    }
    // ---- dO = dZ Wo^T into R1; then Wv into the free W tile and dO (16-bit)
    // into the free P tile
    if (!wb.wait(p.status)) return false;
    MMA_GROUP(mb, p.status, mma_issue(tb + R1, kop(sm + SM_P, kW), kop(sm + SM_W, kW), kW, kW, false));
    bulk_load(wb, sm + SM_W, p.WvT + (size_t)l * kTile, kTile);
    for (int c = 32 * pt; c < kW; c += kStride) {
      float v[32];
      tc::tmem_ld32(tb + lo + R1 + c, v);
      store32(sm + SM_P, r, c, kW, kW, v);
    }
    tc::fence_before_sync();
    // ---- recompute Q, K, V in one product group, drained over their weights
    {
      const bool ok = xb.wait(p.status);
      if (!(wb.wait(p.status) && ok)) return false;
    }
    MMA_GROUP4(mb, p.status,
               mma_issue(tb + R0, kop(sm + SM_G, kW), kop(sm + SM_Q, kW), kW, kW, false),
               mma_issue(tb + R1, kop(sm + SM_G, kW), kop(sm + SM_K, kW), kW, kW, false),
               mma_issue(tb + R3, kop(sm + SM_G, kW), kop(sm + SM_W, kW), kW, kW, false), (void)0);
    {
      const uint32_t src[3] = {R0, R1, R3};
      uint8_t* tiles[3] = {sm + SM_Q, sm + SM_K, sm + SM_V};
#pragma unroll
      for (int q3 = 0; q3 < 3; ++q3)
        for (int c = 32 * pt; c < kW; c += kStride) {
          float v[32];
          tc::tmem_ld32(tb + lo + src[q3] + c, v);
          store32(tiles[q3], r, c, kW, kW, v);
        }
      tc::fence_before_sync();
    }
    // ---- heads.  Tiles: Q, K, V; dO in P; A, then the gate adjoint, in G;
    // dS in W
    MMA_GROUP(mb, p.status,   // scores of head 0; later heads' ride with the previous head
              mma_issue(tb + R3, kop(sm + SM_Q, kW), kop(sm + SM_K, kW), kW, DH, false));
    for (int h = 0; h < p.heads; ++h) {
      const int c0 = h * DH;
      const float st = MP ? p.smx[(((size_t)atom * L + l) * 4 + h) * kW + r]
                          : h == 0 ? beta4[0] : h == 1 ? beta4[1] : h == 2 ? beta4[2] : beta4[3];
      // w (kept in R3 for the adjoint below) and A = w * gate -> G tile
      for (int c = 32 * pt; c < kW; c += kStride) {
        float v[32];
        if (c < nv) {
          tc::tmem_ld32(tb + lo + R3 + c, v);
          softmax_w(p, m, c, st, v);
          tc::tmem_st32(tb + lo + R3 + c, v);
#pragma unroll
          for (int q = 0; q < 32; q += 2) {
            const float2 w = fmul2(make_float2(v[q], v[q + 1]), gate2(rj, m, c + q));
            v[q] = w.x;
            v[q + 1] = w.y;
          }
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) v[q] = 0.f;
        }
        store32(sm + SM_G, r, c, kW, kW, v);
      }
      tc::fence_before_sync();
      // dA = dO_h V_h^T (R1), dV_h = A^T dO_h (R0 + 2d), O_h = A V_h (R0, consumed
      // below before dQ_h overwrites it)
      MMA_GROUP4(mb, p.status,
                 mma_issue(tb + R1, kop(sm + SM_P, kW, c0), kop(sm + SM_V, kW, c0), kW, DH, false),
                 mma_issue(tb + R0 + 2 * DH, mnop(sm + SM_G, kW, 0), mnop(sm + SM_P, kW, c0), DH, kW,
                           false),
                 mma_issue(tb + R0, kop(sm + SM_G, kW), mnop(sm + SM_V, kW, c0), DH, kW, false), (void)0);
      // sum_k w_jk dw_jk = sum_k A_jk dA_jk = dO_j . O_j over this head's
      // columns; every part forms it whole (same order, same value)
      float wdw = 0.f;
      {
        float o[32];
        tc::tmem_ld32(tb + lo + R0, o);
        float a4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < DH; q += 8) {
          float g8[8];
          load8(sm + SM_P, r, c0 + q, kW, g8);
#pragma unroll
          for (int e = 0; e < 8; ++e) a4[e & 3] += g8[e] * o[q + e];
        }
        wdw = (a4[0] + a4[1]) + (a4[2] + a4[3]);
      }
      // softmax + gate adjoint for this row, 16 columns at a time
      for (int c = 32 * pt; c < kW; c += kStride) {
        if (c < nv) {
#pragma unroll
          for (int c16 = 0; c16 < 32; c16 += 16) {
            float s[16], da[16];
            tc::tmem_ld16x2(tb + lo + R3 + c + c16, s, tb + lo + R1 + c + c16, da);
#pragma unroll
            for (int q8 = 0; q8 < 16; q8 += 8) {
              float ds[8], x[8];
#pragma unroll
              for (int e = 0; e < 8; e += 2) {
                const int q = q8 + e;
                const float2 s2 = make_float2(s[q], s[q + 1]), da2 = make_float2(da[q], da[q + 1]);
                const float2 dw = fmul2(da2, gate2(rj, m, c + c16 + q));
                const float2 xx = fmul2(da2, s2);                       // gate adjoint dc_jk
                const float2 dd = fmul2(s2, fadd2(dw, bc2(-wdw)));      // dS = w (dw - sum w dw)
                x[e] = xx.x;
                x[e + 1] = xx.y;
                ds[e] = dd.x;
                ds[e + 1] = dd.y;
              }
              store8(sm + SM_W, r, c + c16 + q8, kW, ds);
              store8(sm + SM_G, r, c + c16 + q8, kW, x);
            }
          }
        } else {
          float z[32];
#pragma unroll
          for (int q = 0; q < 32; ++q) z[q] = 0.f;
          store32(sm + SM_W, r, c, kW, kW, z);
          store32(sm + SM_G, r, c, kW, kW, z);
        }
      }
      tc::fence_before_sync();
      // dQ_h = dS K_h, dK_h = dS^T Q_h (scaled at drain); column sums of dS
      // (ones) and of the gate adjoint weighted by rh_j (accumulated over
      // heads); row sums of the gate adjoint weighted by rh_k (R1, free once
      // dA has been read); the next head's scores (R3, w has been read)
      MMA_GROUP4(mb, p.status,
                 mma_issue(tb + R0, kop(sm + SM_W, kW), mnop(sm + SM_K, kW, c0), DH, kW, false),
                 mma_issue(tb + R0 + DH, mnop(sm + SM_W, kW, 0), mnop(sm + SM_Q, kW, c0), DH, kW, false),
                 mma_issue(tb + R0 + 112, mnop(sm + SM_W, kW, 0), kop(m->ones, kW), 16, kW, h > 0);
                 mma_issue(tb + R0 + 96, mnop(sm + SM_G, kW, 0), kop(m->rhb, kW), 16, kW, h > 0),
                 mma_issue(tb + R1, kop(sm + SM_G, kW), kop(m->rhb, kW), 16, kW, false);
                 if (h + 1 < p.heads)
                   mma_issue(tb + R3, kop(sm + SM_Q, kW, c0 + DH), kop(sm + SM_K, kW, c0 + DH), kW, DH,
                             false));
      // the gate adjoint's row part, sum_k dc_jk rh_k, joins the column part in drc
      if (pt == 0) {
        float v[8];
        tc::tmem_ld8(tb + lo + R1, v);
        m->drc[r][0] += v[0];
        m->drc[r][1] += v[1];
        m->drc[r][2] += v[2];
      }
      // write dQ_h, dK_h, dV_h (R0 columns [0,32), [32,64), [64,96)) over the
      // head's columns of Q, K, V; each part of a row takes 32 / kSplit columns
      {
        constexpr int kCw = 32 / kSplit;
        uint8_t* tiles[3] = {sm + SM_Q, sm + SM_K, sm + SM_V};
#pragma unroll
        for (int part = 0; part < 3; ++part) {
          float v[kCw];
          if constexpr (kCw == 16) tc::tmem_ld16(tb + lo + R0 + 32 * part + kCw * pt, v);
          else tc::tmem_ld8(tb + lo + R0 + 32 * part + kCw * pt, v);
          const float sc = part < 2 ? p.inv_sqrt_d : 1.f;
#pragma unroll
          for (int q = 0; q < kCw; ++q) v[q] *= sc;
#pragma unroll
          for (int q = 0; q < kCw; q += 8) store8(tiles[part], r, c0 + kCw * pt + q, kW, v + q);
        }
      }
      tc::fence_before_sync();
    }
    // column sums of this layer: row id k owns column k (warps of part 0)
    if (pt == 0) {
      float v[32];
      tc::tmem_ld32(tb + lo + R0 + 96, v);
      m->drc[r][0] += v[0];
      m->drc[r][1] += v[1];
      m->drc[r][2] += v[2];
      if (valid && m->sw[r] > 0.f) m->dswa[r] += v[16] / m->sw[r];
    }
    // ---- dG_in = dZ + dQ Wq^T + dK Wk^T + dV Wv^T, accumulated onto R2; the
    // three weights arrive together in the free W, G and P tiles
    tc::fence_async_smem();
    __syncthreads();
    if (t == 0) {
      issue_copy(wb, sm + SM_W, p.WqR + (size_t)l * kTile, kTile, kTile);
      issue_copy(xb, sm + SM_G, p.WkR + (size_t)l * kTile, kTile, 2 * kTile);
      issue_copy(xb, sm + SM_P, p.WvR + (size_t)l * kTile, kTile, 0);
    }
    {
      const bool ok = wb.wait(p.status);
      if (!(xb.wait(p.status) && ok)) return false;
    }
    MMA_GROUP(mb, p.status,
              mma_issue(tb + R2, kop(sm + SM_Q, kW), kop(sm + SM_W, kW), kW, kW, true);
              mma_issue(tb + R2, kop(sm + SM_K, kW), kop(sm + SM_G, kW), kW, kW, true);
              mma_issue(tb + R2, kop(sm + SM_V, kW), kop(sm + SM_P, kW), kW, kW, true));
  }
  if (MP && p.lb > 0) {
    // message passing: dE/dG' of layer lb and the sums go to the cross-atom
    // step and the next launch
    float4* dst = reinterpret_cast<float4*>(p.dG32) + (size_t)atom * 32 * kW + r;
    for (int c = 32 * pt; c < kW; c += kStride) {
      float g[32];
      tc::tmem_ld32(tb + lo + R2 + c, g);
#pragma unroll
      for (int q = 0; q < 32; q += 4)
        dst[(size_t)((c + q) >> 2) * kW] = make_float4(g[q], g[q + 1], g[q + 2], g[q + 3]);
    }
    if (pt == 0) {
      float* a = p.accs + (size_t)atom * 8 * kW + r;
      for (int q = 0; q < 4; ++q) a[q * kW] = m->dRt[r][q];
      for (int q = 0; q < 3; ++q) a[(4 + q) * kW] = m->drc[r][q];
      a[7 * kW] = m->dswa[r];
    }
    tc::fence_before_sync();
    __syncthreads();
    return true;
  }
  // ---- embedding adjoint: dG0 (R2) -> ds.  G0 lands in the G tile while H1
  // (Q tile) and H2 (K tile) are recomputed with weights through W and P.
  load_G(sm + SM_G, 0, gb);
  if (!embed_h2(p, sm, m, tb, mb, wb, xb, sm + SM_Q, sm + SM_K, sm + SM_W, sm + SM_P))
    return false;
  if (ngroups > 0 && !gb.wait(p.status)) return false;
  __syncthreads();
  for (int c = 32 * pt; c < kW; c += kStride) {  // da3 = dG0 (1 - G0^2) -> P tile
    float dg[32], g0[32];
    tc::tmem_ld32(tb + lo + R2 + c, dg);
#pragma unroll
    for (int q = 0; q < 32; q += 8) load8(sm + SM_G, r, c + q, kW, g0 + q);
#pragma unroll
    for (int q = 0; q < 32; ++q) dg[q] = valid ? dg[q] * (1.f - g0[q] * g0[q]) : 0.f;
    store32(sm + SM_P, r, c, kW, kW, dg);
  }
  tc::fence_before_sync();
  const int tj = m->tj[r];
  for (int c = 8 * pt; c < p.e2; c += 8 * kSplit) {
    float z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    store8(sm + SM_V, r, c, p.e2, z);
  }
  // da2 = (da3 W3^T) (1 - h2^2) -> V tile; weights through W and G
  {
    const uint32_t bytes = p.e2 * kW * 2;
    const bool ok = species_loop((unsigned)m->mask, p.W3R, bytes, bytes, sm + SM_W, sm + SM_G, wb,
                                 xb, p.status, [&](int sp, uint8_t* Wt) -> bool {
      MMA_GROUP(mb, p.status, mma_issue(tb + R1, kop(sm + SM_P, kW), kop(Wt, kW), p.e2, kW, false));
      const bool mine = tj == sp;
      if (__any_sync(0xffffffffu, mine)) {
        for (int c = 32 * pt; c < p.e2; c += kStride) {
          float v[32], h2[32] = {};
          tc::tmem_ld32(tb + lo + R1 + c, v);
          if (mine) {
#pragma unroll
            for (int q = 0; q < 32; q += 8)
              if (c + q < p.e2) load8(sm + SM_K, r, c + q, p.e2, h2 + q);
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] *= c + q < p.e2 ? 1.f - h2[q] * h2[q] : 0.f;
            store32(sm + SM_V, r, c, p.e2, p.e2, v);
          }
        }
      }
      tc::fence_before_sync();
      return true;
    });
    if (!ok) return false;
  }
  // da1 = (da2 W2^T) (1 - h1^2); ds = da1 . W1
  float ds_emb = 0.f;
  {
    const uint32_t bytes = p.e1 * p.e2 * 2;
    const bool ok = species_loop((unsigned)m->mask, p.W2R, bytes, bytes, sm + SM_W, sm + SM_G, wb,
                                 xb, p.status, [&](int sp, uint8_t* Wt) -> bool {
      MMA_GROUP(mb, p.status,
                mma_issue(tb + R1, kop(sm + SM_V, p.e2), kop(Wt, p.e2), p.e1, p.e2, false));
      const bool mine = tj == sp;
      if (__any_sync(0xffffffffu, mine)) {
        for (int c = 32 * pt; c < p.e1; c += kStride) {
          float v[32];
          tc::tmem_ld32(tb + lo + R1 + c, v);
          if (mine) {
#pragma unroll
            for (int q = 0; q < 32; q += 8) {
              if (c + q >= p.e1) break;
              float h8[8];
              load8(sm + SM_Q, r, c + q, p.e1, h8);   // h1 (16-bit copy from the H1 tile)
#pragma unroll
              for (int e = 0; e < 8; ++e)
                ds_emb += v[q + e] * (1.f - h8[e] * h8[e]) * p.W1[sp * p.e1 + c + q + e];
            }
          }
        }
      }
      tc::fence_before_sync();
      return true;
    });
    if (!ok) return false;
  }
  // ---- environment adjoint: g_j
  __syncthreads();
  {
    ds_emb = row_sum(m, make_float4(0.f, 0.f, 0.f, ds_emb)).w;
  }
  if (pt == 0 && r < p.nmax) {
    float* gout = p.g + ((size_t)atom * p.nmax + r) * 3;
    if (!valid) {
      gout[0] = gout[1] = gout[2] = 0.f;
    } else {
      const float d = m->d[r], s = m->s[r], sw = m->sw[r], dswr = m->dsw[r];
      const float* rr = m->rh[r];
      const float un = 1.f / kGradScale;   // the layer adjoints carry the seed scale
      float dst = m->dRt[r][0] + ds_emb * un;
      float dr[3];
      for (int a = 0; a < 3; ++a) {
        dst += m->dRt[r][1 + a] * rr[a];
        dr[a] = m->drc[r][a] * un + s * m->dRt[r][1 + a];
      }
      const float radial = dst * (dswr / d - sw / (d * d)) + m->dswa[r] * un * dswr;
      const float proj = dr[0] * rr[0] + dr[1] * rr[1] + dr[2] * rr[2];
      for (int a = 0; a < 3; ++a) gout[a] = radial * rr[a] + (dr[a] - proj * rr[a]) / d;
    }
  }
  __syncthreads();
  return true;
}

template <bool MP>
__global__ void __launch_bounds__(kThreads, 1) k_af_bwd(Params p) {
  extern __shared__ __align__(1024) uint8_t sm[];
  Misc* m = reinterpret_cast<Misc*>(sm + SM_MISC);
  kernel_prologue(m, 4);   // product groups with four issuers
  // constant operand: a ones row (column sums) and zero rows 3..15 of rhb
  zero_smem(m->ones, 16 * kW * 2);
  zero_smem(m->rhb, 16 * kW * 2);
  __syncthreads();
  if (threadIdx.x < kW)
    *reinterpret_cast<op_t*>(m->ones + tc::kmajor_off(0, threadIdx.x, kW)) = f2op(1.f);
  __syncthreads();
  Bar mb{&m->bar, 0u, 4u}, wb{&m->wbar, 0u}, gb{&m->pbar, 0u}, xb{&m->xbar, 0u};
  for (int atom = p.atom0 + blockIdx.x; atom < p.n; atom += gridDim.x)
    if (!bwd_atom<MP>(p, atom, sm, m, m->tptr, mb, wb, gb, xb)) break;
  kernel_epilogue(m);
}

// ================================================================== fitting
struct FitParams {
  int n_tiles, kd, f1, f2, f3, kc1, kc2;
  int kcw;                // one chunk over K = f1 (F2T, F1R), staged in the free Y2 + Y3 space
  const int4* tiles;      // {species, start, count, 0}
  const int* order;       // atoms grouped by species
  const op_t* D;          // [n][kd]
  // per species, chunked BF16 tiles (see host packing)
  const uint8_t *F1T, *F2T, *F3T, *F3R, *F2R, *F1R;
  size_t sF1T, sF2T, sF3T, sF3R, sF2R, sF1R;  // bytes per species
  const float *c1, *c2, *c3, *F4, *c4;
  double* atom_e;
  float* dD;              // [n][kd]
  int* status;
  int grad;               // 1: also dE/dD (the head that drives the forces); 0: energy only
  const unsigned char* seed;  // energy seed per atom (optional): the adjoint starts from it
};

constexpr int FT_Y1 = 0;
constexpr int FT_TILE = 128 * 256 * 2;  // room for K up to 256
constexpr int FT_Y2 = FT_TILE, FT_Y3 = 2 * FT_TILE, FT_CA = 3 * FT_TILE;
constexpr int FT_CB = FT_CA + 128 * 32 * 2;
constexpr int FT_MISC = FT_CB + 256 * 48 * 2;
constexpr int kSmemFit = FT_MISC + 64;

// acc(128 x N, tmem col0) = A(tile, Kx = K) * B(chunks of kc columns, N rows),
// each chunk staged in bbuf
__device__ bool fit_product(uint8_t* bbuf, const uint8_t* A, int K, const uint8_t* Bchunks, int N,
                            int kc, uint32_t tcol, Bar& mb, Bar& wb, int* status) {
  for (int k0 = 0; k0 < K; k0 += kc) {
    bulk_load(wb, bbuf, Bchunks + (size_t)(k0 / kc) * N * kc * 2, N * kc * 2);
    if (!wb.wait(status)) return false;
    MMA_GROUP(mb, status, mma_issue(tcol, kop(A, K, k0), kop(bbuf, kc), N, kc, k0 > 0));
  }
  return true;
}

__device__ bool fit_layer1(uint8_t* CA, uint8_t* CB, int kc, int N, bool acc, uint32_t tb, Bar& mb,
                           int* status) {
  MMA_GROUP(mb, status, mma_issue(tb, kop(CA, kc), kop(CB, kc), N, kc, acc));
  return true;
}

__global__ void __launch_bounds__(kFitThreads, 1) k_fit(FitParams p) {
  extern __shared__ __align__(1024) uint8_t sm[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(sm + FT_MISC);
  unsigned long long* wbar = reinterpret_cast<unsigned long long*>(sm + FT_MISC + 8);
  uint32_t* tptr = reinterpret_cast<uint32_t*>(sm + FT_MISC + 16);
  const int t = threadIdx.x, warp = t >> 5;
  const uint32_t lane_off = (uint32_t)(32 * warp) << 16;
  if (t == 0) {
    tc::mbar_init(reinterpret_cast<uint64_t*>(bar), 1);
    tc::mbar_init(reinterpret_cast<uint64_t*>(wbar), 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tptr, 512);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tb = *tptr;
  Bar mb{bar, 0u}, wb{wbar, 0u};
  bool ok = true;
  uint8_t *Y1 = sm + FT_Y1, *Y2 = sm + FT_Y2, *Y3 = sm + FT_Y3;
  for (int tile = blockIdx.x; tile < p.n_tiles && ok; tile += gridDim.x) {
    const int4 td = p.tiles[tile];
    const int sp = td.x;
    const int atom = t < td.z ? p.order[td.y + t] : -1;
    // ---- layer 1: D (gathered rows, K = kd in chunks of kc1) x F1; the
    // chunks' A and B tiles use the Y2 and Y3 space, free until layer 2
    uint8_t* CA1 = sm + FT_Y2;
    uint8_t* CB1 = CA1 + 128 * p.kc1 * 2;
    for (int k0 = 0; k0 < p.kd && ok; k0 += p.kc1) {
      for (int c = 0; c < p.kc1; c += 8) {
        uint4 u = make_uint4(0, 0, 0, 0);
        if (atom >= 0) u = *reinterpret_cast<const uint4*>(p.D + (size_t)atom * p.kd + k0 + c);
        *reinterpret_cast<uint4*>(CA1 + tc::kmajor_off(t, c, p.kc1)) = u;
      }
      bulk_load(wb, CB1, p.F1T + sp * p.sF1T + (size_t)(k0 / p.kc1) * p.f1 * p.kc1 * 2,
                p.f1 * p.kc1 * 2);
      ok = wb.wait(p.status) && fit_layer1(CA1, CB1, p.kc1, p.f1, k0 > 0, tb, mb, p.status);
    }
    if (!ok) break;
    // epilogue: y = tanh(acc + c) into a K-major tile
    auto epi_tanh = [&](int N, const float* bias, uint8_t* Y) {
      for (int c = 0; c < N; c += 32) {
        float v[32];
        tc::tmem_ld32(tb + lane_off + c, v);
        for (int q = 0; q < 32; ++q) v[q] = (c + q < N) ? tanhf(v[q] + bias[sp * N + c + q]) : 0.f;
        for (int q = 0; q < 32 && c + q < N; q += 8) store8(Y, t, c + q, N, v + q);
      }
    };
    epi_tanh(p.f1, p.c1, Y1);
    tc::fence_before_sync();
    // layer 2 in one chunk: its weights fill the Y2 + Y3 space, free until
    // the epilogue writes y2
    ok = fit_product(Y2, Y1, p.f1, p.F2T + sp * p.sF2T, p.f2, p.kcw, tb, mb, wb, p.status);
    if (!ok) break;
    epi_tanh(p.f2, p.c2, Y2);
    tc::fence_before_sync();
    ok = fit_product(sm + FT_CB, Y2, p.f2, p.F3T + sp * p.sF3T, p.f3, p.kc2, tb, mb, wb, p.status);
    if (!ok) break;
    // y3, energy (FP64 sum) and delta3 = seed F4 (1 - y3^2) into Y3
    {
      const float sd = p.seed && atom >= 0 && !p.seed[atom] ? 0.f : 1.f;
      double e = 0.0;
      for (int c = 0; c < p.f3; c += 32) {
        float v[32];
        tc::tmem_ld32(tb + lane_off + c, v);
        for (int q = 0; q < 32; ++q) {
          if (c + q >= p.f3) { v[q] = 0.f; continue; }
          float y = tanhf(v[q] + p.c3[sp * p.f3 + c + q]);
          float w4 = p.F4[sp * p.f3 + c + q];
          e += (double)y * (double)w4;
          v[q] = sd * w4 * (1.f - y * y);
        }
        for (int q = 0; q < 32 && c + q < p.f3; q += 8) store8(Y3, t, c + q, p.f3, v + q);
      }
      if (atom >= 0) p.atom_e[atom] = e + (double)p.c4[sp];
    }
    if (!p.grad) continue;
    // backward: delta2 = (delta3 F3^T) (1 - y2^2), delta1 = (delta2 F2^T) (1 - y1^2)
    auto epi_dtanh = [&](int N, uint8_t* Y) {
      for (int c = 0; c < N; c += 32) {
        float v[32];
        tc::tmem_ld32(tb + lane_off + c, v);
        for (int q = 0; q < 32 && c + q < N; q += 8) {
          float y[8];
          load8(Y, t, c + q, N, y);
          for (int u = 0; u < 8; ++u) y[u] = v[q + u] * (1.f - y[u] * y[u]);
          store8(Y, t, c + q, N, y);
        }
      }
    };
    ok = fit_product(sm + FT_CB, Y3, p.f3, p.F3R + sp * p.sF3R, p.f2, p.kc2, tb, mb, wb, p.status);
    if (!ok) break;
    epi_dtanh(p.f2, Y2);
    tc::fence_before_sync();
    ok = fit_product(sm + FT_CB, Y2, p.f2, p.F2R + sp * p.sF2R, p.f1, p.kc2, tb, mb, wb, p.status);
    if (!ok) break;
    epi_dtanh(p.f1, Y1);
    tc::fence_before_sync();
    // dE/dD = delta1 F1^T, 256 columns at a time, each in one chunk staged
    // in the Y2 + Y3 space (delta2 has been used)
    for (int nb = 0; nb < p.kd / 256 && ok; ++nb) {
      ok = fit_product(Y2, Y1, p.f1, p.F1R + sp * p.sF1R + (size_t)nb * 256 * p.f1 * 2, 256, p.kcw,
                       tb, mb, wb, p.status);
      if (!ok) break;
      for (int c = 0; c < 256; c += 32) {
        float v[32];
        tc::tmem_ld32(tb + lane_off + c, v);
        if (atom >= 0) {
          float4* dst = reinterpret_cast<float4*>(p.dD + (size_t)atom * p.kd + nb * 256 + c);
          for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
      }
      tc::fence_before_sync();
      __syncthreads();
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tb, 512);
}

// ================================================================== host side
static uint16_t f2bf(double x) {
#ifdef DP_FUSED_BF16
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
#else
  __half h = __float2half_rn((float)x);
  uint16_t u;
  memcpy(&u, &h, 2);
  return u;
#endif
}

// Append the K-major core-matrix tile of M (R x K, element (r, k) = get(r, k))
// to `out`, K split into chunks of kc columns (each chunk its own tile).
template <typename Get>
static void pack(std::vector<uint16_t>& out, int R, int K, int kc, Get get) {
  for (int k0 = 0; k0 < K; k0 += kc) {
    size_t base = out.size();
    out.resize(base + (size_t)R * kc, 0);
    for (int r = 0; r < R; ++r)
      for (int k = 0; k < kc; ++k) {
        size_t off = (((size_t)(r >> 3) * (kc >> 3)) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
        out[base + off] = f2bf(get(r, k0 + k));
      }
  }
}

class FusedAf : public Model {
 public:
  ~FusedAf() override {
    for (void* q : allocs_) cudaFree(q);
  }
  int run(const NbrView& nv, const int* types, double* atom_e, cudaStream_t st) override {
    return run_parts(nv, types, atom_e, st, 7);
  }
  int run_parts(const NbrView& nv, const int* types, double* atom_e, cudaStream_t st,
                int parts) override {
    return launch(nv, types, atom_e, st, parts, 0);
  }
  // The fitting kernel still runs over every atom (its species tiles span the
  // batch); outside [atom0, n) it reads stale descriptors and writes energies
  // and dE/dD that nothing reads before the next full evaluation.
  int run_range(const NbrView& nv, const int* types, double* atom_e, cudaStream_t st,
                int atom0) override {
    return launch(nv, types, atom_e, st, 7, atom0);
  }
  int launch(const NbrView& nv, const int* types, double* atom_e, cudaStream_t st, int parts,
             int atom0) {
    Params p = base_;
    p.sel_j = nv.sel_j;
    p.sel_r = nv.sel_r;
    p.types = types;
    if (m_.mp) atom0 = 0;   // every atom's previous layer feeds its neighbours
    p.atom0 = atom0;
    const int grid = std::max(1, std::min(n_ - atom0, sms_));
    const int L = m_.n_layers;
    int k = 0;
    if ((parts & 1) && m_.mp) {
      // one launch per layer; U = tanh(h Wm + bm) of every atom in between
      k_mp_init<float><<<ceil_div((long long)n_ * kW, 256), 256, 0, st>>>(n_, kW, types, mp_Wt_,
                                                                         p.hbuf);
      ++k;
      for (int l = 0; l < L; ++l) {
        Gemm<float> g = gemm_rowmajor<float>(n_, kW, kW, p.hbuf, kW, mp_Wm_[l], kW,
                                             mp_U_ + (size_t)l * cap_ * kW, kW);
        g.bias = mp_bm_[l];
        g.epi = 1;
        gemm(g, 1, st);
        Params q = p;
        q.lb = l;
        q.le = l + 1;
        k_af_fwd<true><<<grid, kThreads, kSmemAtom, st>>>(q);
        k += 2;
      }
    } else if (parts & 1) {
      k_af_fwd<false><<<grid, kThreads, kSmemAtom, st>>>(p);
      ++k;
    }
    if (parts & 2) {
      FitParams f = fit_;
      f.atom_e = atom_e;
      k_fit<<<std::min(fit_.n_tiles, sms_), kFitThreads, kSmemFit, st>>>(f);
      ++k;
      for (size_t h = 0; h < heads_fit_.size(); ++h) {   // further heads: energies only
        FitParams fh = heads_fit_[h];
        fh.n_tiles = fit_.n_tiles;
        fh.atom_e = head_e_ + h * (size_t)cap_;
        k_fit<<<std::min(fit_.n_tiles, sms_), kFitThreads, kSmemFit, st>>>(fh);
        ++k;
      }
    }
    if ((parts & 4) && m_.mp) {
      // one launch per layer, from the top; between them the message adjoint
      // dh += ((sum of dE/dG' over the slots naming j) (1 - U_j^2)) Wm^T
      cudaMemsetAsync(mp_dh_, 0, sizeof(float) * (size_t)n_ * kW, st);
      for (int l = L - 1; l >= 0; --l) {
        Params q = p;
        q.lb = l;
        q.le = l + 1;
        k_af_bwd<true><<<grid, kThreads, kSmemAtom, st>>>(q);
        ++k;
        if (l == 0) break;
        int warps = 4;
        while (warps > 1 && sizeof(int) * 2 * nv.cap * warps > 48 * 1024) --warps;
        k_mp_gather4<<<ceil_div(n_, warps), warps * 32, sizeof(int) * 2 * nv.cap * warps, st>>>(
            n_, m_.nmax, nv.cap, nv.skin, nv.skin_cnt, nv.mirror, nv.selpos,
            reinterpret_cast<const float4*>(p.dG32), mp_U_ + (size_t)l * cap_ * kW, mp_dq_);
        Gemm<float> g{};
        g.M = n_; g.N = kW; g.K = kW;
        g.A = mp_dq_; g.a_rm = kW; g.a_rk = 1;
        g.B = mp_Wm_[l]; g.b_rk = 1; g.b_rn = kW;
        g.C = mp_dh_; g.c_rm = kW; g.c_rn = 1; g.nb2 = 1; g.alpha = 1.f; g.beta = 1.f;
        gemm(g, 1, st);
        k += 2;
      }
    } else if (parts & 4) {
      k_af_bwd<false><<<grid, kThreads, kSmemAtom, st>>>(p);
      ++k;
    }
    return k;
  }
  const float* grad32() const override { return g_; }
  const double* head_energies() const override { return head_e_; }
  size_t bytes() const override { return bytes_; }
  // atoms grouped by species for the fitting kernel, tiles of <= 128 of one species
  bool set_atoms(int n, const int* types) override {
    if (n < 1 || n > cap_) return false;
    std::vector<int> order;
    std::vector<int4> tiles;
    for (int t = 0; t < m_.n_species; ++t) {
      int start = (int)order.size();
      for (int i = 0; i < n; ++i)
        if (types[i] == t) order.push_back(i);
      int cnt = (int)order.size() - start;
      for (int o = 0; o < cnt; o += 128) tiles.push_back(make_int4(t, start + o, std::min(128, cnt - o), 0));
    }
    if (cudaMemcpy(dorder_, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dtiles_, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return false;
    n_ = n;
    base_.n = n;
    fit_.n_tiles = (int)tiles.size();
    grid_ = std::min(n, sms_);
    return true;
  }
  void bind_flags(int* flags) override {
    base_.status = flags;
    fit_.status = flags;
  }
  bool set_energy_seed(const unsigned char* seed) override {
    fit_.seed = seed;
    return true;
  }

  bool init(const AfDims& m, const double* w, int n_atoms, const int* types, std::string* err);

 private:
  template <typename T>
  bool dalloc(T** p, size_t count, std::string* err) {
    size_t b = sizeof(T) * (count ? count : 1);
    cudaError_t e = cudaMalloc((void**)p, b);
    if (e != cudaSuccess) {
      *err = std::string("fused model: ") + cudaGetErrorString(e);
      cudaGetLastError();
      return false;
    }
    allocs_.push_back(*p);
    bytes_ += b;
    return true;
  }
  template <typename T>
  bool upload(T** p, const std::vector<T>& v, std::string* err) {
    if (!dalloc(p, v.size(), err)) return false;
    if (cudaMemcpy(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      *err = "fused model: weight upload failed";
      return false;
    }
    return true;
  }
  AfDims m_{};
  int n_ = 0, grid_ = 0, sms_ = 0, cap_ = 0;
  int4* dtiles_ = nullptr;
  int* dorder_ = nullptr;
  std::vector<FitParams> heads_fit_;   // fitting heads 1.. (energy only)
  double* head_e_ = nullptr;           // their atomic energies, [head - 1][cap_]
  Params base_{};
  FitParams fit_{};
  float* g_ = nullptr;
  // message passing (FP32): Wt [S][128], per layer Wm [128][128] and bm, U, dh, dq
  float* mp_Wt_ = nullptr;
  std::vector<float*> mp_Wm_, mp_bm_;
  float *mp_U_ = nullptr, *mp_dh_ = nullptr, *mp_dq_ = nullptr;
  std::vector<void*> allocs_;
  size_t bytes_ = 0;
};

bool FusedAf::init(const AfDims& m, const double* w, int n_atoms, const int* types, std::string* err) {
  m_ = m;
  n_ = n_atoms;
  const int S = m.n_species, L = m.n_layers, H = m.hidden;
  // Real widths (blob layout) and the widths the kernels run at: the embedding
  // widths are padded to multiples of 16 and m1 to 128 with zero weights and
  // biases, so every padded unit is tanh(0) = 0 and feeds nothing; the
  // LayerNorm takes its statistics over the m1 real columns only.
  const int E1r = m.e1, E2r = m.e2, M1 = m.m1;
  const int E1 = (E1r + 15) / 16 * 16, E2 = (E2r + 15) / 16 * 16;
  const int KD = kW * m.m2, KDr = M1 * m.m2;
  // ---- walk the blob
  size_t off = 0;
  auto at = [&](size_t o) { return w[o]; };
  std::vector<size_t> oW1(S), ob1(S), oW2(S), ob2(S), oW3(S), ob3(S);
  for (int t = 0; t < S; ++t) {
    oW1[t] = off; off += E1r;
    ob1[t] = off; off += E1r;
    oW2[t] = off; off += (size_t)E1r * E2r;
    ob2[t] = off; off += E2r;
    oW3[t] = off; off += (size_t)E2r * M1;
    ob3[t] = off; off += M1;
  }
  size_t oWt = 0;
  if (m.mp) { oWt = off; off += (size_t)S * kW; }
  std::vector<size_t> oq(L), ok(L), ov(L), oo(L), obo(L), oWm(L), obm(L);
  for (int l = 0; l < L; ++l) {
    oq[l] = off; off += (size_t)M1 * H;
    ok[l] = off; off += (size_t)M1 * H;
    ov[l] = off; off += (size_t)M1 * H;
    oo[l] = off; off += (size_t)H * M1;
    obo[l] = off; off += M1;
    if (m.mp) {
      oWm[l] = off; off += (size_t)kW * kW;
      obm[l] = off; off += kW;
    }
  }
  std::vector<size_t> oF1(S), oc1(S), oF2(S), oc2(S), oF3(S), oc3(S), oF4(S), oc4(S);
  for (int t = 0; t < S; ++t) {
    oF1[t] = off; off += (size_t)KDr * m.f1;
    oc1[t] = off; off += m.f1;
    oF2[t] = off; off += (size_t)m.f1 * m.f2;
    oc2[t] = off; off += m.f2;
    oF3[t] = off; off += (size_t)m.f2 * m.f3;
    oc3[t] = off; off += m.f3;
    oF4[t] = off; off += m.f3;
    oc4[t] = off; off += 1;
  }
  // ---- pack tiles
  std::vector<uint16_t> W2T, W3T, W2R, W3R, WqT, WkT, WvT, WoT, WqR, WkR, WvR, WoR;
  std::vector<float> W1, b1, b2, b3, bo;
  // weight (row, col) of a row-major (rows x cols) block at o, zero outside
  auto wz = [&](size_t o, int row, int col, int rows, int cols) {
    return row < rows && col < cols ? at(o + (size_t)row * cols + col) : 0.0;
  };
  for (int t = 0; t < S; ++t) {
    pack(W2T, E2, E1, E1, [&](int r, int k) { return wz(oW2[t], k, r, E1r, E2r); });
    pack(W3T, kW, E2, E2, [&](int r, int k) { return wz(oW3[t], k, r, E2r, M1); });
    pack(W2R, E1, E2, E2, [&](int r, int k) { return wz(oW2[t], r, k, E1r, E2r); });
    pack(W3R, E2, kW, kW, [&](int r, int k) { return wz(oW3[t], r, k, E2r, M1); });
    for (int k = 0; k < E1; ++k) {
      W1.push_back(k < E1r ? (float)at(oW1[t] + k) : 0.f);
      b1.push_back(k < E1r ? (float)at(ob1[t] + k) : 0.f);
    }
    for (int k = 0; k < E2; ++k) b2.push_back(k < E2r ? (float)at(ob2[t] + k) : 0.f);
    for (int k = 0; k < kW; ++k) b3.push_back(k < M1 ? (float)at(ob3[t] + k) : 0.f);
  }
  for (int l = 0; l < L; ++l) {
    pack(WqT, H, kW, kW, [&](int r, int k) { return wz(oq[l], k, r, M1, H); });
    pack(WkT, H, kW, kW, [&](int r, int k) { return wz(ok[l], k, r, M1, H); });
    pack(WvT, H, kW, kW, [&](int r, int k) { return wz(ov[l], k, r, M1, H); });
    pack(WoT, kW, H, H, [&](int r, int k) { return wz(oo[l], k, r, H, M1); });
    pack(WqR, kW, H, H, [&](int r, int k) { return wz(oq[l], r, k, M1, H); });
    pack(WkR, kW, H, H, [&](int r, int k) { return wz(ok[l], r, k, M1, H); });
    pack(WvR, kW, H, H, [&](int r, int k) { return wz(ov[l], r, k, M1, H); });
    pack(WoR, H, kW, kW, [&](int r, int k) { return wz(oo[l], r, k, H, M1); });
    for (int k = 0; k < kW; ++k) bo.push_back(k < M1 ? (float)at(obo[l] + k) : 0.f);
  }
  // fitting: chunk widths kc1 for K = KD (the A and B chunks of 128 x kc1
  // and f1 x kc1 fill the 128 KB of the Y2 and Y3 tiles at most), kc2 for K = f
  const int kc1 = 128;
  const int kc2 = (m.f1 % 48 == 0 && m.f2 % 48 == 0 && m.f3 % 48 == 0) ? 48 : 16;
  const int kcw = m.f1;   // f2 x f1 or 256 x f1 16-bit: at most 128 KB, the Y2 + Y3 space
  std::vector<uint16_t> F1T, F2T, F3T, F3R, F2R, F1R;
  std::vector<float> c1, c2, c3, F4, c4;
  for (int t = 0; t < S; ++t) {
    pack(F1T, m.f1, KD, kc1, [&](int r, int k) { return wz(oF1[t], k, r, KDr, m.f1); });
    pack(F2T, m.f2, m.f1, kcw, [&](int r, int k) { return at(oF2[t] + (size_t)k * m.f2 + r); });
    pack(F3T, m.f3, m.f2, kc2, [&](int r, int k) { return at(oF3[t] + (size_t)k * m.f3 + r); });
    pack(F3R, m.f2, m.f3, kc2, [&](int r, int k) { return at(oF3[t] + (size_t)r * m.f3 + k); });
    pack(F2R, m.f1, m.f2, kc2, [&](int r, int k) { return at(oF2[t] + (size_t)r * m.f2 + k); });
    for (int nb = 0; nb < KD / 256; ++nb)
      pack(F1R, 256, m.f1, kcw,
           [&](int r, int k) { return wz(oF1[t], nb * 256 + r, k, KDr, m.f1); });
    for (int k = 0; k < m.f1; ++k) c1.push_back((float)at(oc1[t] + k));
    for (int k = 0; k < m.f2; ++k) c2.push_back((float)at(oc2[t] + k));
    for (int k = 0; k < m.f3; ++k) {
      c3.push_back((float)at(oc3[t] + k));
      F4.push_back((float)at(oF4[t] + k));
    }
    c4.push_back((float)at(oc4[t]));
  }
  // further fitting heads (same layout, one block after another): forward only
  const int HF = m.fit_heads > 1 ? m.fit_heads : 1;
  const size_t fit_len = off - oF1[0];
  struct HeadTiles {
    std::vector<uint16_t> F1T, F2T, F3T;
    std::vector<float> c1, c2, c3, F4, c4;
  };
  std::vector<HeadTiles> extra(HF - 1);
  for (int h = 1; h < HF; ++h) {
    HeadTiles& X = extra[h - 1];
    const size_t sh = (size_t)h * fit_len;
    for (int t = 0; t < S; ++t) {
      pack(X.F1T, m.f1, KD, kc1, [&](int r, int k) { return wz(sh + oF1[t], k, r, KDr, m.f1); });
      pack(X.F2T, m.f2, m.f1, kcw, [&](int r, int k) { return at(sh + oF2[t] + (size_t)k * m.f2 + r); });
      pack(X.F3T, m.f3, m.f2, kc2, [&](int r, int k) { return at(sh + oF3[t] + (size_t)k * m.f3 + r); });
      for (int k = 0; k < m.f1; ++k) X.c1.push_back((float)at(sh + oc1[t] + k));
      for (int k = 0; k < m.f2; ++k) X.c2.push_back((float)at(sh + oc2[t] + k));
      for (int k = 0; k < m.f3; ++k) {
        X.c3.push_back((float)at(sh + oc3[t] + k));
        X.F4.push_back((float)at(sh + oF4[t] + k));
      }
      X.c4.push_back((float)at(sh + oc4[t]));
    }
  }
  Params& p = base_;
  p.n = n_atoms; p.nmax = m.nmax; p.e1 = E1; p.e2 = E2; p.m2 = m.m2; p.n_layers = L;
  p.m1 = M1; p.inv_m1 = 1.f / M1;
  p.heads = m.heads; p.dh = H / m.heads;
  p.rs = (float)m.rs; p.rc = (float)m.rc; p.inv_nmax = 1.f / m.nmax;
  p.inv_sqrt_d = 1.f / sqrtf((float)p.dh);
  uint16_t *dW2T, *dW3T, *dW2R, *dW3R, *dWqT, *dWkT, *dWvT, *dWoT, *dWqR, *dWkR, *dWvR, *dWoR;
  float *dW1, *db1, *db2, *db3, *dbo;
  bool good = upload(&dW2T, W2T, err) && upload(&dW3T, W3T, err) && upload(&dW2R, W2R, err) &&
              upload(&dW3R, W3R, err) && upload(&dW1, W1, err) && upload(&db1, b1, err) &&
              upload(&db2, b2, err) && upload(&db3, b3, err);
  if (good && L > 0)
    good = upload(&dWqT, WqT, err) && upload(&dWkT, WkT, err) && upload(&dWvT, WvT, err) &&
           upload(&dWoT, WoT, err) && upload(&dWqR, WqR, err) && upload(&dWkR, WkR, err) &&
           upload(&dWvR, WvR, err) && upload(&dWoR, WoR, err) && upload(&dbo, bo, err);
  if (!good) return false;
  p.W2T = (const uint8_t*)dW2T; p.W3T = (const uint8_t*)dW3T;
  p.W2R = (const uint8_t*)dW2R; p.W3R = (const uint8_t*)dW3R;
  if (L > 0) {
    p.WqT = (const uint8_t*)dWqT; p.WkT = (const uint8_t*)dWkT; p.WvT = (const uint8_t*)dWvT;
    p.WoT = (const uint8_t*)dWoT; p.WqR = (const uint8_t*)dWqR; p.WkR = (const uint8_t*)dWkR;
    p.WvR = (const uint8_t*)dWvR; p.WoR = (const uint8_t*)dWoR; p.bo = dbo;
  }
  p.W1 = dW1; p.b1 = db1; p.b2 = db2; p.b3 = db3;
  size_t N = n_atoms;
  if (!dalloc(&p.Gst, N * (L + 1) * kTile, err) || !dalloc(&p.rstd, N * (L > 0 ? L : 1) * kW, err) ||
      !dalloc(&p.smx, N * (L > 0 ? L : 1) * m.heads * kW, err) ||
      !dalloc(&p.D, N * KD, err) || !dalloc(&p.Tm, N * 4 * kW, err) ||
      !dalloc(&g_, N * m.nmax * 3, err) || !dalloc(&p.status, 1, err))
    return false;
  float* ddD;
  if (!dalloc(&ddD, N * KD, err)) return false;
  p.dD = ddD;
  p.g = g_;
  p.lb = 0;
  p.le = L;
  p.cap = n_atoms;
  p.mp = m.mp;
  if (m.mp && n_atoms > 500000) {   // the gather's 32-bit float4 indices of per-slot state
    *err = "fused message passing supports at most 500,000 atoms";
    return false;
  }
  if (m.mp) {   // message passing (m1 = 128): FP32 atom-channel weights and between-launch state
    std::vector<float> Wt(w + oWt, w + oWt + (size_t)S * kW);
    if (!upload(&mp_Wt_, Wt, err)) return false;
    mp_Wm_.resize(L);
    mp_bm_.resize(L);
    for (int l = 0; l < L; ++l) {
      std::vector<float> a(w + oWm[l], w + oWm[l] + (size_t)kW * kW), b(w + obm[l], w + obm[l] + kW);
      if (!upload(&mp_Wm_[l], a, err) || !upload(&mp_bm_[l], b, err)) return false;
    }
    float* U = nullptr;
    float* dh = nullptr;
    if (!dalloc(&p.Gpst, N * (L > 0 ? L : 1) * kTile, err) || !dalloc(&p.Gf32, N * kW * kW, err) ||
        !dalloc(&U, (size_t)(L > 0 ? L : 1) * N * kW, err) || !dalloc(&p.hbuf, N * kW, err) ||
        !dalloc(&p.dG32, N * kW * kW, err) || !dalloc(&dh, N * kW, err) ||
        !dalloc(&mp_dq_, N * kW, err) || !dalloc(&p.accs, N * kW * 8, err))
      return false;
    p.U = U;
    p.hgrad = dh;
    mp_U_ = U;
    mp_dh_ = dh;
  }
  cudaMemset(p.status, 0, sizeof(int));
  // fitting tiles (capacity for any atom set up to n_atoms): see set_atoms
  FitParams& f = fit_;
  f.kd = KD; f.f1 = m.f1; f.f2 = m.f2; f.f3 = m.f3;
  f.kc1 = kc1; f.kc2 = kc2; f.kcw = kcw;
  cap_ = n_atoms;
  if (!dalloc(&dtiles_, (size_t)n_atoms / 128 + S + 1, err) || !dalloc(&dorder_, (size_t)n_atoms, err))
    return false;
  uint16_t *dF1T, *dF2T, *dF3T, *dF3R, *dF2R, *dF1R;
  float *dc1, *dc2, *dc3, *dF4, *dc4;
  good = upload(&dF1T, F1T, err) &&
         upload(&dF2T, F2T, err) && upload(&dF3T, F3T, err) && upload(&dF3R, F3R, err) &&
         upload(&dF2R, F2R, err) && upload(&dF1R, F1R, err) && upload(&dc1, c1, err) &&
         upload(&dc2, c2, err) && upload(&dc3, c3, err) && upload(&dF4, F4, err) && upload(&dc4, c4, err);
  if (!good) return false;
  f.tiles = dtiles_; f.order = dorder_; f.D = p.D;
  f.F1T = (const uint8_t*)dF1T; f.F2T = (const uint8_t*)dF2T; f.F3T = (const uint8_t*)dF3T;
  f.F3R = (const uint8_t*)dF3R; f.F2R = (const uint8_t*)dF2R; f.F1R = (const uint8_t*)dF1R;
  f.sF1T = F1T.size() * 2 / S; f.sF2T = F2T.size() * 2 / S; f.sF3T = F3T.size() * 2 / S;
  f.sF3R = F3R.size() * 2 / S; f.sF2R = F2R.size() * 2 / S; f.sF1R = F1R.size() * 2 / S;
  f.c1 = dc1; f.c2 = dc2; f.c3 = dc3; f.F4 = dF4; f.c4 = dc4;
  f.dD = ddD;
  f.status = p.status;
  f.grad = 1;
  for (int h = 1; h < HF; ++h) {
    HeadTiles& X = extra[h - 1];
    FitParams fh = f;
    uint16_t *e1, *e2, *e3;
    float *v1, *v2, *v3, *v4, *v5;
    if (!(upload(&e1, X.F1T, err) && upload(&e2, X.F2T, err) && upload(&e3, X.F3T, err) &&
          upload(&v1, X.c1, err) && upload(&v2, X.c2, err) && upload(&v3, X.c3, err) &&
          upload(&v4, X.F4, err) && upload(&v5, X.c4, err)))
      return false;
    fh.F1T = (const uint8_t*)e1; fh.F2T = (const uint8_t*)e2; fh.F3T = (const uint8_t*)e3;
    fh.F3R = fh.F2R = fh.F1R = nullptr;
    fh.c1 = v1; fh.c2 = v2; fh.c3 = v3; fh.F4 = v4; fh.c4 = v5;
    fh.grad = 0;
    heads_fit_.push_back(fh);
  }
  if (HF > 1 && !dalloc(&head_e_, (size_t)(HF - 1) * n_atoms, err)) return false;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, dev);
  if (!set_atoms(n_atoms, types)) {
    *err = "fused model: fitting tiles upload failed";
    return false;
  }
  if (cudaFuncSetAttribute(k_af_fwd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemAtom) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_af_bwd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemAtom) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_af_fwd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemAtom) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_af_bwd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemAtom) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_fit, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemFit) !=
          cudaSuccess) {
    *err = "fused model: shared-memory configuration failed";
    return false;
  }
  return true;
}

}  // namespace fz

bool fused_af_supported(const AfDims& m, std::string* why) {
  if (m.m1 < 1 || m.m1 > 128 || m.hidden != 128) { *why = "fused path needs m1 <= 128 and hidden = 128"; return false; }
  if (m.mp && m.m1 != 128) { *why = "fused message passing needs m1 = 128"; return false; }
  if (m.heads != 4) { *why = "fused path needs 4 heads of width 32"; return false; }
  if (m.e1 < 1 || m.e2 < 1 || m.e1 > 64 || m.e2 > 128) { *why = "fused path needs e1 <= 64 and e2 <= 128"; return false; }
  if (m.nmax > 128) { *why = "fused path needs nmax <= 128"; return false; }
  if ((128 * m.m2) % 256) { *why = "fused path needs 128 * m2 to be a multiple of 256"; return false; }
  if (m.f1 % 16 || m.f2 % 16 || m.f3 % 16 || m.f1 > 256 || m.f2 > 256 || m.f3 > 256) { *why = "fused path needs fitting widths multiples of 16 and <= 256"; return false; }
  if (m.n_species > 32) { *why = "fused path supports at most 32 species"; return false; }
  return true;
}

Model* make_fused_af(const AfDims& m, const double* weights, int n_atoms, const int* types_host,
                     std::string* err) {
  if (!fused_af_supported(m, err)) return nullptr;
  auto* f = new fz::FusedAf();
  if (!f->init(m, weights, n_atoms, types_host, err)) {
    delete f;
    return nullptr;
  }
  return f;
}

}  // namespace dp
