// Tensor-core GEMM for FP32-stored operands: C = A B [+ bias] [+ beta C], then
// an optional epilogue (tanh, or times 1 - aux^2), with 16-bit operands (FP16,
// or BF16) and FP32 accumulation on tcgen05.  It serves the graph family's mixed form,
// whose matrix products are all of the shape (rows x K) (K x N) with K, N
// multiples of 16 up to 256 and rows = atoms or atom-slot pairs (millions).
//
// One CTA of 128 threads owns tiles of 128 rows (persistent over tiles): B is
// converted into shared memory once, each A tile is loaded with coalesced
// float4 reads, converted and stored in the core-matrix layout, multiplied
// into tensor memory (K/16 instructions of 128 x N x 16) and drained by
// thread = row through the epilogue.
#include <algorithm>

#include "common.cuh"
#include "gemm_tc.cuh"
#include "tc.cuh"

namespace dp {
namespace {

constexpr int kRows = 128;
constexpr int kStageLd = 20;
constexpr size_t kMaxSmemBlock = 232448;   // opt-in shared memory per block (static + dynamic)   // epilogue stage row stride (floats): 16-byte rows, conflict-free phases
constexpr long long kPollsTc = 1LL << 22;

__device__ __forceinline__ uint64_t desc_k(uint32_t base, int Kx, int k0) {
  return tc::make_desc(base + (uint32_t)((k0 >> 3) * 128), 128u, (uint32_t)((Kx >> 3) * 128));
}
__device__ __forceinline__ uint64_t desc_mn(uint32_t base, int Kx, int k0) {
  return tc::make_desc(base + (uint32_t)((k0 >> 3) * (Kx >> 3) * 128), (uint32_t)((Kx >> 3) * 128),
                       128u);
}

// four values rounded to the 16-bit operand type, as one 8-byte store
__device__ __forceinline__ uint2 pack4(int fp16, float a, float b, float c, float d) {
  return fp16 ? make_uint2(tc::pack_f16(a, b), tc::pack_f16(c, d))
              : make_uint2(tc::pack_bf16(a, b), tc::pack_bf16(c, d));
}

// four 16-bit values, loaded as raw bits, as FP32 (the conversion is kept
// apart from the load: the epilogue issues all of a block's loads first, and
// a conversion next to its load would make the warp wait for that load)
__device__ __forceinline__ float4 unpack4(int fp16, uint2 u) {
  float2 a, b;
  if (fp16) {
    a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
    b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  } else {
    a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
    b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
  }
  return make_float4(a.x, a.y, b.x, b.y);
}

// EPI: 3, 4 or 5 for those epilogues, 0 for the others (none, tanh, the
// 1 - aux^2 factor), so that each variant carries only its own epilogue
template <int EPI>
__global__ void __launch_bounds__(kRows) k_gemm_tc(GemmTc g, int tmem_cols) {
  extern __shared__ __align__(1024) uint8_t sm[];
  const int t = threadIdx.x, warp = t >> 5;
  const int brows = g.b_nk ? g.N : g.K, bcols = g.b_nk ? g.K : g.N;
  uint8_t* Bs = sm;
  uint8_t* As = sm + (((size_t)brows * bcols * 2 + 1023) & ~(size_t)1023);
  uint8_t* Al = As + (size_t)kRows * g.K * 2;   // remainder tile (split only)
  uint8_t* tail = g.split ? Al + (size_t)kRows * g.K * 2 : Al;
  uint64_t* bar = reinterpret_cast<uint64_t*>(tail);
  float* stage = reinterpret_cast<float*>(tail + 64);   // kRows x kStageLd
  __shared__ uint32_t tptr;
  if (t == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(&tptr, (uint32_t)tmem_cols);
    tc::tmem_relinquish();
  }
  // B once: stored rows x cols (K x N, or N x K when b_nk), row-major in global;
  // by float4 with eight reads in flight per thread when rows are 16-byte aligned
  const bool bvec = (bcols & 3) == 0 && (g.ldb & 3) == 0 &&
                    (reinterpret_cast<uintptr_t>(g.B) & 15) == 0;
  if (bvec) {
    const int cq = bcols >> 2, total4 = brows * cq;
    constexpr int kBLoads = 8;
    for (int base = 0; base < total4; base += kRows * kBLoads) {
      float4 v[kBLoads];
#pragma unroll
      for (int u = 0; u < kBLoads; ++u) {
        const int i = base + u * kRows + t;
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < total4) {
          const int r = i / cq, c = (i - r * cq) << 2;
          v[u] = *reinterpret_cast<const float4*>(g.B + (long long)r * g.ldb + c);
        }
      }
#pragma unroll
      for (int u = 0; u < kBLoads; ++u) {
        const int i = base + u * kRows + t;
        if (i >= total4) break;
        const int r = i / cq, c = (i - r * cq) << 2;
        uint2 w;
        if (g.fp16) {
          w.x = tc::pack_f16(v[u].x, v[u].y);
          w.y = tc::pack_f16(v[u].z, v[u].w);
        } else {
          w.x = tc::pack_bf16(v[u].x, v[u].y);
          w.y = tc::pack_bf16(v[u].z, v[u].w);
        }
        *reinterpret_cast<uint2*>(Bs + tc::kmajor_off(r, c, bcols)) = w;
      }
    }
  }
  for (int i = bvec ? brows * bcols : t; i < brows * bcols; i += kRows) {
    const int r = i / bcols, c = i - r * bcols;
    const float x = g.B[(long long)r * g.ldb + c];
    uint16_t h;
    if (g.fp16) {
      __half v = __float2half_rn(x);
      h = *reinterpret_cast<uint16_t*>(&v);
    } else {
      __nv_bfloat16 v = __float2bfloat16(x);
      h = *reinterpret_cast<uint16_t*>(&v);
    }
    *reinterpret_cast<uint16_t*>(Bs + tc::kmajor_off(r, c, bcols)) = h;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tb = tptr;
  const uint32_t lane_off = (uint32_t)(32 * warp) << 16;
  const int lane = t & 31;
  const uint32_t idesc = tc::idesc_f16(kRows, g.N, 0, g.b_nk ? 0 : 1, g.fp16 ? 0u : 1u);
  const uint32_t a_base = tc::smem_u32(As), al_base = tc::smem_u32(Al), b_base = tc::smem_u32(Bs);
  const int tiles = (g.M + kRows - 1) / kRows;
  const int k4 = g.K >> 2;
  // row of element i of an A tile: i / k4, a shift when k4 is a power of two
  const int k4s = (k4 & (k4 - 1)) == 0 ? __ffs(k4) - 1 : -1;
  uint32_t phase = 0;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long long m0 = (long long)tile * kRows;
    if (g.a16) {
      // A rows stored in 16 bits (the operand type): 16-byte chunks straight
      // into the core-matrix layout, eight reads in flight per thread
      constexpr int kLoads16 = 8;
      const int k8 = g.K >> 3, total16 = kRows * k8;
      for (int base = 0; base < total16; base += kRows * kLoads16) {
        uint4 v[kLoads16];
#pragma unroll
        for (int u = 0; u < kLoads16; ++u) {
          const int i = base + u * kRows + t;
          v[u] = make_uint4(0u, 0u, 0u, 0u);
          if (i < total16) {
            const int r = i / k8, c = (i - r * k8) << 3;
            const long long m = m0 + r;
            if (m < g.M) {
              const long long row = g.a_rows ? (long long)g.a_rows[m] : m;
              v[u] = *reinterpret_cast<const uint4*>(g.a16 + row * g.lda + c);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < kLoads16; ++u) {
          const int i = base + u * kRows + t;
          if (i >= total16) break;
          const int r = i / k8, c = (i - r * k8) << 3;
          *reinterpret_cast<uint4*>(As + tc::kmajor_off(r, c, g.K)) = v[u];
        }
      }
    }
    // A tile: 128 rows x K, coalesced float4 reads -> 16-bit core-matrix layout;
    // each thread issues kLoads reads before converting any, so that enough
    // bytes are in flight to keep HBM busy
    constexpr int kLoads = 16;
    const int total = g.a16 ? 0 : kRows * k4;
    for (int base = 0; base < total; base += kRows * kLoads) {
      float4 v[kLoads];
#pragma unroll
      for (int u = 0; u < kLoads; ++u) {
        const int i = base + u * kRows + t;
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < total) {
          const int r = k4s >= 0 ? i >> k4s : i / k4, c = (i - r * k4) << 2;
          const long long m = m0 + r;
          if (m < g.M) {
            const long long row = g.a_rows ? (long long)g.a_rows[m] : m;
            v[u] = *reinterpret_cast<const float4*>(g.A + row * g.lda + c);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kLoads; ++u) {
        const int i = base + u * kRows + t;
        if (i >= total) break;
        const int r = k4s >= 0 ? i >> k4s : i / k4, c = (i - r * k4) << 2;
        uint2 w;
        if (g.fp16) {
          w.x = tc::pack_f16(v[u].x, v[u].y);
          w.y = tc::pack_f16(v[u].z, v[u].w);
        } else {
          w.x = tc::pack_bf16(v[u].x, v[u].y);
          w.y = tc::pack_bf16(v[u].z, v[u].w);
        }
        const int off = tc::kmajor_off(r, c, g.K);
        *reinterpret_cast<uint2*>(As + off) = w;
        if (g.split) {   // remainder v - high, itself rounded to 16 bits
          const float2 h0 = g.fp16 ? __half22float2(*reinterpret_cast<const __half2*>(&w.x))
                                   : __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w.x));
          const float2 h1 = g.fp16 ? __half22float2(*reinterpret_cast<const __half2*>(&w.y))
                                   : __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w.y));
          uint2 lo;
          if (g.fp16) {
            lo.x = tc::pack_f16(v[u].x - h0.x, v[u].y - h0.y);
            lo.y = tc::pack_f16(v[u].z - h1.x, v[u].w - h1.y);
          } else {
            lo.x = tc::pack_bf16(v[u].x - h0.x, v[u].y - h0.y);
            lo.y = tc::pack_bf16(v[u].z - h1.x, v[u].w - h1.y);
          }
          *reinterpret_cast<uint2*>(Al + off) = lo;
        }
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) {
      for (int ks = 0; ks < g.K; ks += 16) {
        const uint64_t db = g.b_nk ? desc_k(b_base, g.K, ks) : desc_mn(b_base, g.N, ks);
        tc::mma_bf16(tb, desc_k(a_base, g.K, ks), db, idesc, ks > 0 ? 1u : 0u);
        if (g.split) tc::mma_bf16(tb, desc_k(al_base, g.K, ks), db, idesc, 1u);
      }
      tc::mma_commit(bar);
    }
    // The epilogue's row indices, read while the products run.  Thread
    // (warp w, lane) owns rows 32 w + lane / 4 + 8 u (u = 0..3) and, in every
    // 16-column block, the four columns from (lane mod 4) x 4.
    const int c4 = (lane & 3) << 2;
    long long rowu[4];   // row'(m) of each owned row, -1 beyond M
    long long xru[4];    // epi 4: row of e_in, v_out and sa
    int jnu[4];          // epi 3, 5: the slot's neighbour (-1: empty slot or beyond M)
    float fu[4];         // epi 5: inv_nmax sw of a kept slot; epi 4: sa of the row
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long m = m0 + 32 * warp + (lane >> 2) + 8 * u;
      rowu[u] = m < g.M ? (g.c_rows ? (long long)g.c_rows[m] : m) : -1;
      xru[u] = -1;
      if constexpr (EPI == 4)
        if (m < g.M) xru[u] = g.x_rows ? (long long)g.x_rows[m] : rowu[u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      jnu[u] = -1;
      fu[u] = 0.f;
      if constexpr (EPI == 3 || EPI == 5)
        if (rowu[u] >= 0) jnu[u] = g.sel_j[rowu[u]];
      if constexpr (EPI == 4)
        if (xru[u] >= 0) fu[u] = g.sa[xru[u]];
    }
    if constexpr (EPI == 5) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (jnu[u] >= 0) fu[u] = g.inv_nmax * g.sw[rowu[u]];
    }
    bool ok = true;
    if (t == 0) ok = tc::mbar_wait(bar, phase & 1u, kPollsTc);
    phase ^= 1u;
    ok = __syncthreads_and(ok) != 0;
    tc::fence_after_sync();
    if (!ok) {
      if (t == 0) atomicOr(g.status, kFlagTimeout);
      break;
    }
    // epilogue, 16 columns at a time: each warp reads its 32 accumulator rows
    // (thread = row) and turns them around through its shared-memory stage,
    // so that four neighbouring threads own one row's 16 columns and every
    // global access of the warp covers 8 rows x 64 contiguous bytes.  A
    // block's global operands of all four owned rows are requested before any
    // of them is used, so that their latencies overlap.
    float* st = stage + warp * 32 * kStageLd;
    float dacc[4] = {0.f, 0.f, 0.f, 0.f};   // epi 5: this thread's part of each row's dsw sum
    for (int c = 0; c < g.N; c += 16) {
      const int col = c + c4;
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      float4 o0[4], o1[4], o2[4], o3[4];
      uint2 e16r[4];   // 16-bit edge rows (g.e16), converted where used
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        o0[u] = o1[u] = o2[u] = o3[u] = z4;
        e16r[u] = make_uint2(0u, 0u);
        const long long row = rowu[u];
        if constexpr (EPI == 3) {        // Ai of the slot's atom, Bj of its neighbour, e_in
          if (jnu[u] >= 0) {
            o0[u] = *reinterpret_cast<const float4*>(g.Ai + (long long)((int)row / g.nmax) * g.ldc + col);
            o1[u] = *reinterpret_cast<const float4*>(g.Bj + (long long)jnu[u] * g.ldc + col);
            if (g.e16) e16r[u] = *reinterpret_cast<const uint2*>(g.e16 + row * g.ldc + col);
            else o2[u] = *reinterpret_cast<const float4*>(g.e_in + row * g.ldc + col);
          }
        } else if constexpr (EPI == 5) { // de, and on kept slots g_i, u_j, e_in
          if (row >= 0) o0[u] = *reinterpret_cast<const float4*>(g.C + row * g.ldc + col);
          if (jnu[u] >= 0) {
            o1[u] = *reinterpret_cast<const float4*>(g.dm + (long long)((int)row / g.nmax) * g.lddm + col);
            o2[u] = *reinterpret_cast<const float4*>(g.u + (long long)jnu[u] * g.ldc + col);
            if (g.e16) e16r[u] = *reinterpret_cast<const uint2*>(g.e16 + row * g.ldc + col);
            else o3[u] = *reinterpret_cast<const float4*>(g.e_in + row * g.ldc + col);
          }
        } else if constexpr (EPI == 4) { // e_in of the output row
          if (xru[u] >= 0) {
            if (g.e16) e16r[u] = *reinterpret_cast<const uint2*>(g.e16 + xru[u] * g.ldc + col);
            else o0[u] = *reinterpret_cast<const float4*>(g.e_in + xru[u] * g.ldc + col);
          }
        } else {                         // C (beta != 0), aux (epi 2)
          if (row >= 0) {
            if (g.beta != 0.f) o0[u] = *reinterpret_cast<const float4*>(g.C + row * g.ldc + col);
            if (g.epi == 2) o1[u] = *reinterpret_cast<const float4*>(g.aux + row * g.ldc + col);
          }
        }
      }
      float v[16];
      tc::tmem_ld16(tb + lane_off + (uint32_t)c, v);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4*>(st + lane * kStageLd + 4 * q) =
            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      __syncwarp();
      const float4 bv = g.bias ? *reinterpret_cast<const float4*>(g.bias + col) : z4;
      const float b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long row = rowu[u];
        if (row < 0) continue;
        const int rl = (lane >> 2) + 8 * u;
        const float4 acc = *reinterpret_cast<const float4*>(st + rl * kStageLd + c4);
        const float x[4] = {acc.x, acc.y, acc.z, acc.w};
        float4* Cp = reinterpret_cast<float4*>(g.C + row * g.ldc + col);
        if constexpr (EPI == 4) {   // angle output: t = tanh(acc + b), e_out = e_in + sa t
          const long long xr = xru[u];
          const float4 e = g.e16 ? unpack4(g.fp16, e16r[u]) : o0[u];
          const float sw = fu[u];
          float y[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) y[q] = tanhf(x[q] + b[q]);
          *Cp = make_float4(y[0], y[1], y[2], y[3]);
          if (g.o16)
            *reinterpret_cast<uint2*>(g.o16 + xr * g.ldc + col) =
                pack4(g.fp16, e.x + sw * y[0], e.y + sw * y[1], e.z + sw * y[2], e.w + sw * y[3]);
          else
            *reinterpret_cast<float4*>(g.v_out + xr * g.ldc + col) =
                make_float4(e.x + sw * y[0], e.y + sw * y[1], e.z + sw * y[2], e.w + sw * y[3]);
          continue;
        }
        if constexpr (EPI == 5) {   // edge adjoint and the message's adjoint on kept slots
          const float4 dv = o0[u];
          float y[4] = {dv.x + x[0], dv.y + x[1], dv.z + x[2], dv.w + x[3]};
          if (jnu[u] >= 0) {
            const float f = fu[u];
            const float4 gv = o1[u], uv = o2[u], ev = g.e16 ? unpack4(g.fp16, e16r[u]) : o3[u];
            const float gq[4] = {gv.x, gv.y, gv.z, gv.w}, uq[4] = {uv.x, uv.y, uv.z, uv.w},
                        eq[4] = {ev.x, ev.y, ev.z, ev.w};
            float xo[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              y[q] += f * gq[q] * uq[q];
              xo[q] = f * gq[q] * eq[q];
              dacc[u] += gq[q] * eq[q] * uq[q];
            }
            if (g.x16)
              *reinterpret_cast<uint2*>(g.x16 + row * g.ldc + col) = pack4(g.fp16, xo[0], xo[1], xo[2], xo[3]);
            else
              *reinterpret_cast<float4*>(g.x_out + row * g.ldc + col) = make_float4(xo[0], xo[1], xo[2], xo[3]);
          }
          *Cp = make_float4(y[0], y[1], y[2], y[3]);
          continue;
        }
        if constexpr (EPI == 3) {   // edge update: v = tanh(Ai + Bj + acc + b), e1 = e_in + v
          if (jnu[u] < 0) {
            if (g.v16) *reinterpret_cast<uint2*>(g.v16 + row * g.ldc + col) = make_uint2(0u, 0u);
            else *reinterpret_cast<float4*>(g.v_out + row * g.ldc + col) = make_float4(0.f, 0.f, 0.f, 0.f);
            if (g.o16) *reinterpret_cast<uint2*>(g.o16 + row * g.ldc + col) = make_uint2(0u, 0u);
            else *Cp = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
          }
          const float4 av = o0[u], bj = o1[u], e = g.e16 ? unpack4(g.fp16, e16r[u]) : o2[u];
          const float y0 = tanhf(av.x + bj.x + x[0] + b[0]);
          const float y1 = tanhf(av.y + bj.y + x[1] + b[1]);
          const float y2 = tanhf(av.z + bj.z + x[2] + b[2]);
          const float y3 = tanhf(av.w + bj.w + x[3] + b[3]);
          if (g.v16) *reinterpret_cast<uint2*>(g.v16 + row * g.ldc + col) = pack4(g.fp16, y0, y1, y2, y3);
          else *reinterpret_cast<float4*>(g.v_out + row * g.ldc + col) = make_float4(y0, y1, y2, y3);
          if (g.o16) *reinterpret_cast<uint2*>(g.o16 + row * g.ldc + col) = pack4(g.fp16, e.x + y0, e.y + y1, e.z + y2, e.w + y3);
          else *Cp = make_float4(e.x + y0, e.y + y1, e.z + y2, e.w + y3);
          continue;
        }
        const float cin[4] = {o0[u].x, o0[u].y, o0[u].z, o0[u].w};
        const float ax[4] = {o1[u].x, o1[u].y, o1[u].z, o1[u].w};
        float y[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float z = x[q] + b[q];
          if (g.beta != 0.f) z += g.beta * cin[q];
          if (g.epi == 1) {
            z = tanhf(z);
          } else if (g.epi == 2) {
            z *= 1.f - ax[q] * ax[q];
          }
          y[q] = z;
        }
        *Cp = make_float4(y[0], y[1], y[2], y[3]);
      }
      __syncwarp();   // the stage is rewritten by the next column block
    }
    if constexpr (EPI == 5) {   // each row's dsw sum over its four threads (lanes 4r .. 4r + 3), in a fixed order
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float v = dacc[u];
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        if ((lane & 3) == 0 && jnu[u] >= 0) g.dsw[rowu[u]] += g.inv_nmax * v;
      }
    }
    tc::fence_before_sync();
    __syncthreads();          // tensor memory and the A tile are reused by the next tile
    tc::fence_after_sync();
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tb, (uint32_t)tmem_cols);
}

int g_sms = 0;
size_t g_max_dyn = 0;   // dynamic shared memory the kernel may request

}  // namespace

bool gemm_tc_shape_ok(int N, int K) {
  return N >= 16 && N <= 256 && N % 16 == 0 && K >= 16 && K <= 256 && K % 16 == 0;
}

static size_t smem_of(const GemmTc& g) {
  const size_t b = ((size_t)g.N * g.K * 2 + 1023) & ~(size_t)1023;
  return b + (size_t)kRows * g.K * 2 * (g.split ? 2 : 1) + 64 + (size_t)kRows * kStageLd * 4;
}

bool gemm_tc_prepare(std::string* err) {
  if (g_sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      *err = "cannot query the device";
      return false;
    }
  }
  // up to the per-block limit less the static part (a split A that would not
  // fit falls back to one product)
  void (*const kernels[4])(GemmTc, int) = {k_gemm_tc<0>, k_gemm_tc<3>, k_gemm_tc<4>, k_gemm_tc<5>};
  size_t stat = 0;
  for (auto k : kernels) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) {
      *err = "tensor-core GEMM: cannot query the kernel";
      return false;
    }
    stat = std::max(stat, fa.sharedSizeBytes);
  }
  g_max_dyn = kMaxSmemBlock - stat;
  for (auto k : kernels)
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g_max_dyn) != cudaSuccess) {
      *err = "tensor-core GEMM cannot get its shared memory";
      return false;
    }
  return true;
}

void gemm_tc(const GemmTc& g0, cudaStream_t st) {
  if (g0.M <= 0) return;
  GemmTc g = g0;
  if (g.split && smem_of(g) > g_max_dyn) g.split = 0;
  if (g.a16) g.split = 0;   // a 16-bit A has no remainder to carry
  int cols = 32;
  while (cols < g.N) cols <<= 1;
  // at most 512 / cols CTAs may share an SM's tensor memory: pad the shared
  // memory request so that no more than that many fit on one SM
  const int per_sm = 512 / cols;
  const size_t floor_smem = 233472 / (size_t)(per_sm + 1) + 1;
  const size_t smem = std::max(smem_of(g), floor_smem);
  const int tiles = (g.M + kRows - 1) / kRows;
  const int grid = std::min(tiles, std::max(1, g_sms) * per_sm);
  switch (g.epi) {
    case 3: k_gemm_tc<3><<<grid, kRows, smem, st>>>(g, cols); break;
    case 4: k_gemm_tc<4><<<grid, kRows, smem, st>>>(g, cols); break;
    case 5: k_gemm_tc<5><<<grid, kRows, smem, st>>>(g, cols); break;
    default: k_gemm_tc<0><<<grid, kRows, smem, st>>>(g, cols); break;
  }
}

}  // namespace dp
