// Forces from pair gradients, FP64 energy/virial reductions and the
// velocity-Verlet integrator (paper Sec. II: MD integrates Newton's equations
// with a Verlet-type scheme; forces are -dE/dx).
//
// F_i = sum_p g_ip - sum_{(k,p'): slot p' of k is atom i} g_kp', with
// g = dE/dr_ij for r_ij = x_j - x_i.  The second sum is gathered, not
// scattered: each skin entry (i -> j) knows the index of its mirror entry
// (j -> i) in j's skin list, and selpos says which kept slot that is.  The
// second sum runs in skin-list order, which depends on when the list was last
// rebuilt, so it is accumulated exactly in 128-bit fixed point (2^-80
// resolution) and rounded once: no atomics, and the force does not depend on
// the rebuild schedule or on which other systems share the batch (bitwise
// reproducible).  With FP32 pair gradients the first sum and the per-atom
// virial are accumulated the same way, in integer arithmetic; with FP64 ones
// (the FP64 path) they are FP64 sums over the kept slots in their order.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace dp {


template <typename G>
__global__ void k_force_gather(int atom0, int n, int nmax, int cap, const int* __restrict__ sel_j,
                               const double* __restrict__ sel_r, const SkinEntry* __restrict__ skin,
                               const int* __restrict__ skin_cnt, const int* __restrict__ mirror,
                               const short* __restrict__ selpos, const G* __restrict__ g,
                               double* __restrict__ F, double* __restrict__ atom_vir) {
  int i = atom0 + (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  if constexpr (std::is_same<G, float>::value) {
    // FP32 pair gradients: both force sums and the virial's FP32 products
    // r_a g_b are accumulated exactly in 128-bit fixed point with integer
    // arithmetic (no FP64 pipe work per slot), and each total is rounded
    // once to FP64, by a lane of its own.
    __int128 acc[12];   // F (3), then the virial -sum r_a g_b (9)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = 0;
    bool bad = false;
    for (int p = lane; p < nmax; p += 32) {
      const size_t o = (size_t)i * nmax + p;
      if (sel_j[o] < 0) continue;
      const float gg[3] = {g[3 * o], g[3 * o + 1], g[3 * o + 2]};
      const float r[3] = {(float)sel_r[3 * o], (float)sel_r[3 * o + 1], (float)sel_r[3 * o + 2]};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        acc[a] = fixed_add(acc[a], to_fixed_f32(gg[a], &bad), &bad);
#pragma unroll
        for (int b = 0; b < 3; ++b)
          acc[3 + 3 * a + b] = fixed_add(acc[3 + 3 * a + b], -to_fixed_f32(r[a] * gg[b], &bad), &bad);
      }
    }
    // the mirrored gradients: four skin entries per lane go through each level
    // of the gather chain (mirror index and neighbour, its slot, its
    // gradient) together, so that their loads overlap
    const int cnt = skin_cnt[i];
    for (int c0 = lane; c0 < cnt; c0 += 4 * 32) {
      int mc[4], jn[4], ps[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + 32 * u;
        mc[u] = -1;
        jn[u] = 0;
        if (c < cnt) {
          const size_t o = (size_t)i * cap + c;
          mc[u] = mirror[o];
          jn[u] = skin[o].j;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) ps[u] = mc[u] >= 0 ? selpos[(size_t)jn[u] * cap + mc[u]] : -1;
      float gm[4][3];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const size_t q = (size_t)jn[u] * nmax + (ps[u] >= 0 ? ps[u] : 0);
#pragma unroll
        for (int a = 0; a < 3; ++a) gm[u][a] = ps[u] >= 0 ? g[3 * q + a] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (ps[u] >= 0)
#pragma unroll
          for (int a = 0; a < 3; ++a) acc[a] = fixed_add(acc[a], -to_fixed_f32(gm[u][a], &bad), &bad);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = warp_sum_fixed(acc[k], &bad);
    bad = __any_sync(0xffffffffu, bad);
    __int128 mine = acc[0];
#pragma unroll
    for (int k = 1; k < 12; ++k)
      if (lane == k) mine = acc[k];
    if (lane < 3) F[3 * i + lane] = bad ? quiet_nan() : from_fixed(mine);
    else if (lane < 12) atom_vir[9 * i + lane - 3] = from_fixed(mine);
    return;
  }
  double f[3] = {0, 0, 0};
  double vir[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int p = lane; p < nmax; p += 32) {
    size_t o = (size_t)i * nmax + p;
    if (sel_j[o] < 0) continue;
    double gg[3] = {(double)g[3 * o], (double)g[3 * o + 1], (double)g[3 * o + 2]};
    double r[3] = {sel_r[3 * o], sel_r[3 * o + 1], sel_r[3 * o + 2]};
    for (int a = 0; a < 3; ++a) {
      f[a] += gg[a];
      for (int b = 0; b < 3; ++b) vir[3 * a + b] -= r[a] * gg[b];
    }
  }
  __int128 fm[3] = {0, 0, 0};
  bool bad = false;
  int cnt = skin_cnt[i];
  for (int c = lane; c < cnt; c += 32) {
    size_t o = (size_t)i * cap + c;
    int mc = mirror[o];
    if (mc < 0) continue;
    int j = skin[o].j;
    int p = selpos[(size_t)j * cap + mc];
    if (p < 0) continue;
    size_t q = (size_t)j * nmax + p;
    for (int a = 0; a < 3; ++a) fm[a] = fixed_add(fm[a], to_fixed((double)g[3 * q + a], &bad), &bad);
  }
  for (int a = 0; a < 3; ++a) f[a] = warp_sum(f[a]);
  for (int a = 0; a < 3; ++a) fm[a] = warp_sum_fixed(fm[a], &bad);
  for (int a = 0; a < 9; ++a) vir[a] = warp_sum(vir[a]);
  bad = __any_sync(0xffffffffu, bad);
  if (lane == 0) {
    for (int a = 0; a < 3; ++a) F[3 * i + a] = bad ? quiet_nan() : f[a] - from_fixed(fm[a]);
    for (int a = 0; a < 9; ++a) atom_vir[9 * i + a] = vir[a];
  }
}

void launch_force_gather(const ForceArgs& a, cudaStream_t st) {
  int blocks = ceil_div((long long)(a.n - a.atom0) * 32, 256);
  if (blocks <= 0) return;
  if (a.g64)
    k_force_gather<double><<<blocks, 256, 0, st>>>(a.atom0, a.n, a.nmax, a.cap, a.sel_j, a.sel_r, a.skin,
                                                   a.skin_cnt, a.mirror, a.selpos, a.g64, a.F,
                                                   a.atom_vir);
  else
    k_force_gather<float><<<blocks, 256, 0, st>>>(a.atom0, a.n, a.nmax, a.cap, a.sel_j, a.sel_r, a.skin,
                                                  a.skin_cnt, a.mirror, a.selpos, a.g32, a.F,
                                                  a.atom_vir);
}

// Per system: E and the virial summed exactly in 128-bit fixed point
// (integer arithmetic, 2^-80 resolution) and rounded once to FP64, so the
// totals do not depend on the summation order.  Blocks of k_reduce_part take
// chunks of kReduceChunk atoms of one system and write the chunk's partial
// sums; k_reduce_final adds a system's partials (still exact).  A value that
// is not finite, or beyond the fixed-point range (|v| >= 2^46), and a sum
// that would leave it (|sum| >= 2^47, checked at every addition) raise the
// non-finite flag, as a non-finite force does.  With a DP group, atoms
// outside it contribute nothing (their energy is set to 0; they have no kept
// pairs, so no virial or force either).
constexpr int kReduceThreads = 256;
__global__ void __launch_bounds__(kReduceThreads) k_reduce_part(
    const int* __restrict__ sys_atom0, double* __restrict__ atom_e, const double* __restrict__ atom_vir,
    const double* __restrict__ F, int* __restrict__ flags, const unsigned char* __restrict__ grp,
    unsigned long long* __restrict__ part, int part_chunks) {
  const int s = blockIdx.y, chunk = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int a0 = sys_atom0[s], a1 = sys_atom0[s + 1];
  const long long lo = (long long)a0 + (long long)chunk * kReduceChunk;
  if (lo >= a1) return;   // beyond this system's atoms: no partial
  const int hi = lo + kReduceChunk < a1 ? (int)(lo + kReduceChunk) : a1;
  __shared__ unsigned long long sh[kReduceThreads / 32][10][2];
  __int128 acc[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) acc[q] = 0;
  bool bad = false;
  for (int i = (int)lo + threadIdx.x; i < hi; i += blockDim.x) {
    if (grp && !grp[i]) atom_e[i] = 0.0;
    acc[0] = fixed_add(acc[0], to_fixed_f64(atom_e[i], &bad), &bad);
#pragma unroll
    for (int q = 0; q < 9; ++q)
      acc[1 + q] = fixed_add(acc[1 + q], to_fixed_f64(atom_vir[9 * (size_t)i + q], &bad), &bad);
#pragma unroll
    for (int q = 0; q < 3; ++q)   // exponent all ones: infinite or NaN
      bad |= ((__double_as_longlong(F[3 * (size_t)i + q]) >> 52) & 0x7ff) == 0x7ff;
  }
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    const __int128 v = warp_sum_fixed(acc[q], &bad);
    if (lane == 0) {
      sh[warp][q][0] = (unsigned long long)v;
      sh[warp][q][1] = (unsigned long long)(v >> 64);
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, kFlagNonFinite);
  if (warp != 0) return;
  const int nw = blockDim.x >> 5;
  unsigned long long* out = part + ((size_t)s * part_chunks + chunk) * 20;
  bool over = false;
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    __int128 v = 0;
    if (lane < nw) v = (__int128)(((unsigned __int128)sh[lane][q][1] << 64) | sh[lane][q][0]);
    v = warp_sum_fixed(v, &over);
    if (lane == q) {
      out[2 * q] = (unsigned long long)v;
      out[2 * q + 1] = (unsigned long long)(v >> 64);
    }
  }
  if (__any_sync(0xffffffffu, over) && lane == 0) atomicOr(flags, kFlagNonFinite);
}
// one warp per system: lane q < 10 adds value q over the system's chunks
__global__ void k_reduce_final(const int* __restrict__ sys_atom0,
                               const unsigned long long* __restrict__ part, int part_chunks,
                               double* __restrict__ sys_e, double* __restrict__ sys_vir,
                               int* __restrict__ flags) {
  const int s = blockIdx.x, q = threadIdx.x;
  if (q >= 10) return;
  const int na = sys_atom0[s + 1] - sys_atom0[s];
  const int nch = (na + kReduceChunk - 1) / kReduceChunk;
  const unsigned long long* in = part + (size_t)s * part_chunks * 20;
  __int128 v = 0;
  bool over = false;
  for (int c = 0; c < nch; ++c)
    v = fixed_add(v, (__int128)(((unsigned __int128)in[20 * c + 2 * q + 1] << 64) | in[20 * c + 2 * q]),
                  &over);
  if (over) atomicOr(flags, kFlagNonFinite);
  const double r = over ? quiet_nan() : from_fixed(v);
  if (q == 0) sys_e[s] = r;
  else sys_vir[9 * s + q - 1] = r;
}

void launch_reduce(const ReduceArgs& a, cudaStream_t st) {
  const int chunks = std::max(1, (a.n + kReduceChunk - 1) / kReduceChunk);
  k_reduce_part<<<dim3(chunks, a.n_sys), kReduceThreads, 0, st>>>(
      a.sys_atom0, a.atom_e_out, a.atom_vir, a.F, a.flags, a.grp, a.part, a.part_chunks);
  k_reduce_final<<<a.n_sys, 32, 0, st>>>(a.sys_atom0, a.part, a.part_chunks, a.sys_e, a.sys_vir,
                                          a.flags);
}

// v += dt/2 F/m; x += dt v; request a neighbour rebuild when an atom moved
// more than skin/2 since the last one, or every rebuild_every steps
__global__ void k_kick_drift(int n, double dt, double* __restrict__ x, double* __restrict__ v,
                             const double* __restrict__ F, const double* __restrict__ minv,
                             const double* __restrict__ xref, double half_skin2,
                             int rebuild_every, long long* __restrict__ step,
                             int* __restrict__ flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    long long s = *step + 1;
    *step = s;
    if (rebuild_every > 0 && s % rebuild_every == 0) atomicOr(flags, kFlagRebuild);
  }
  if (i >= n) return;
  double d2 = 0;
  for (int a = 0; a < 3; ++a) {
    double vv = v[3 * i + a] + 0.5 * dt * F[3 * i + a] * minv[i];
    double xx = x[3 * i + a] + dt * vv;
    v[3 * i + a] = vv;
    x[3 * i + a] = xx;
    double dx = xx - xref[3 * i + a];
    d2 += dx * dx;
  }
  if (d2 > half_skin2) atomicOr(flags, kFlagRebuild);
}

// v += dt/2 F/m, and the atom's kinetic energy sum_a (m/2) v_a^2 (FP64,
// spread over the whole grid) for the step's record
__global__ void k_kick(int n, double dt, double* __restrict__ v, const double* __restrict__ F,
                       const double* __restrict__ minv, const double* __restrict__ mass,
                       double* __restrict__ ke) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double hm = 0.5 * mass[i];
  double k = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double vv = v[3 * i + a] + 0.5 * dt * F[3 * i + a] * minv[i];
    v[3 * i + a] = vv;
    k += hm * vv * vv;
  }
  ke[i] = k;
}

void launch_kick_drift(const MdArgs& a, cudaStream_t st) {
  k_kick_drift<<<ceil_div(a.n, 256), 256, 0, st>>>(a.n, a.dt, a.x, a.v, a.F, a.minv, a.xref,
                                                   a.half_skin2, a.rebuild_every, a.step, a.flags);
}

void launch_kick_final(const MdArgs& a, cudaStream_t st) {
  k_kick<<<ceil_div(a.n, 256), 256, 0, st>>>(a.n, a.dt, a.v, a.F, a.minv, a.mass, a.atom_ke);
}

// per system: {E_pot, E_kin} of the step just finished into trace[step - base - 1];
// E_kin is the exact fixed-point sum of the atoms' kinetic energies (from the
// final kick), rounded once
constexpr int kRecordThreads = 1024;
__global__ void __launch_bounds__(kRecordThreads) k_record(const int* __restrict__ sys_atom0,
                                                const double* __restrict__ ke, double inv_kappa,
                                                const double* __restrict__ sys_e,
                                                const long long* __restrict__ step,
                                                double* __restrict__ trace, int n_sys, int trace_len) {
  const int s = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int a0 = sys_atom0[s], a1 = sys_atom0[s + 1];
  __shared__ unsigned long long sh[kRecordThreads / 32][2];
  __int128 acc = 0;
  bool bad = false;
  // four loads in flight per thread (one SM runs the whole system)
  const int bd = blockDim.x;
  for (int i0 = a0 + threadIdx.x; i0 < a1; i0 += 4 * bd) {
    double k[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) k[u] = i0 + u * bd < a1 ? ke[i0 + u * bd] : 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u) acc = fixed_add(acc, to_fixed_f64(k[u], &bad), &bad);
  }
  acc = warp_sum_fixed(acc, &bad);
  bad = __syncthreads_or(bad) != 0;
  if (lane == 0) {
    sh[warp][0] = (unsigned long long)acc;
    sh[warp][1] = (unsigned long long)(acc >> 64);
  }
  __syncthreads();
  if (warp != 0) return;
  __int128 v = 0;
  if (lane < (int)(blockDim.x >> 5)) v = (__int128)(((unsigned __int128)sh[lane][1] << 64) | sh[lane][0]);
  v = warp_sum_fixed(v, &bad);
  bad = __any_sync(0xffffffffu, bad);
  if (lane == 0) {
    long long slot = step[0] - step[1] - 1;   // step[1] holds the base
    if (slot >= 0 && slot < trace_len) {
      trace[(slot * n_sys + s) * 2 + 0] = sys_e[s];
      trace[(slot * n_sys + s) * 2 + 1] = bad ? quiet_nan() : from_fixed(v) * inv_kappa;
    }
  }
}

void launch_record(const MdArgs& a, const double* sys_e, double* trace, int trace_len,
                   cudaStream_t st) {
  const double kappa = 1.602176634e-19 / (1.66053906660e-27 * 1e10);
  k_record<<<a.n_sys, kRecordThreads, 0, st>>>(a.sys_atom0, a.atom_ke, 1.0 / kappa, sys_e, a.step,
                                               trace, a.n_sys, trace_len);
}

__global__ void k_compare(long long count, const double* __restrict__ a,
                          const double* __restrict__ b, int* __restrict__ differs) {
  bool d = false;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    d |= __double_as_longlong(a[i]) != __double_as_longlong(b[i]);
  if (__any_sync(0xffffffffu, d) && (threadIdx.x & 31) == 0) atomicOr(differs, 1);
}

void launch_compare(long long count, const double* a, const double* b, int* differs,
                    cudaStream_t st) {
  const long long blocks = std::min<long long>(ceil_div(count, 256), 1184);
  if (blocks > 0) k_compare<<<(int)blocks, 256, 0, st>>>(count, a, b, differs);
}

// one block per (system, extra fitting head), fixed summation order
__global__ void __launch_bounds__(256) k_head_reduce(int heads, int n, const int* __restrict__ sys_atom0,
                                                     const double* __restrict__ head_e,
                                                     const unsigned char* __restrict__ grp,
                                                     double* __restrict__ out) {
  // the exact fixed-point sum of k_reduce, so that head 0's total equals E
  const int s = blockIdx.x, h = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int a0 = sys_atom0[s], a1 = sys_atom0[s + 1];
  __shared__ unsigned long long sh[8][2];
  __int128 acc = 0;
  bool bad = false;
  for (int i = a0 + threadIdx.x; i < a1; i += blockDim.x)
    if (!grp || grp[i]) acc = fixed_add(acc, to_fixed_f64(head_e[(size_t)h * n + i], &bad), &bad);
  acc = warp_sum_fixed(acc, &bad);
  bad = __syncthreads_or(bad) != 0;
  if (lane == 0) {
    sh[warp][0] = (unsigned long long)acc;
    sh[warp][1] = (unsigned long long)(acc >> 64);
  }
  __syncthreads();
  if (warp != 0) return;
  __int128 v = 0;
  if (lane < (int)(blockDim.x >> 5)) v = (__int128)(((unsigned __int128)sh[lane][1] << 64) | sh[lane][0]);
  v = warp_sum_fixed(v, &bad);
  bad = __any_sync(0xffffffffu, bad);
  if (lane == 0) out[(size_t)s * heads + h] = bad ? quiet_nan() : from_fixed(v);
}

void launch_head_reduce(int n_sys, int heads, int n, const int* sys_atom0, const double* head_e,
                        const unsigned char* grp, double* out, cudaStream_t st) {
  if (n_sys > 0 && heads > 0)
    k_head_reduce<<<dim3(n_sys, heads), 256, 0, st>>>(heads, n, sys_atom0, head_e, grp, out);
}

}  // namespace dp
