// Cell list, skin (Verlet) list and per-step neighbour selection.
//
// The model's neighbours of atom i are every periodic image (j, n) with
// 0 < |r_ij| < rc, r_ij = (w_j - w_i) + n*L (w = wrapped positions), and when
// there are more than nmax, the nmax smallest by (|r|^2, j, n) -- cutoff-based
// Verlet neighbour lists of the paper's Sec. II with the 0.6 nm cutoff of
// Sec. IV.  To keep the per-step cost O(N) the search runs in two stages:
//
//   rebuild (every few steps, or when an atom moved more than skin/2):
//     cell list over wrapped positions (cells >= rc + skin) -> skin list of all
//     (j, m) within rc + skin, m the image relative to unwrapped positions,
//     plus the "mirror" index of every entry in the partner's list;
//   every step:
//     exact FP64 distances of the skin entries with the current positions,
//     membership r^2 < rc^2 and rank by (r^2, j, n), keep rank < nmax.
//
// Distances are computed with explicitly rounded FP64 operations so that the
// selected set and its order are the same bits as a plain IEEE evaluation.
#include "common.cuh"
#include "kernels.cuh"

namespace dp {

// -------------------------------------------------------------- per atom wrap
// Non-finite or absurdly large coordinates are flagged and parked at the
// origin so that no later index computation sees them.
__global__ void k_wrap(int n, const double* __restrict__ x, const int* __restrict__ sys_of,
                       const SysInfo* __restrict__ sys, double* __restrict__ w,
                       int* __restrict__ fl, int* __restrict__ flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const SysInfo& S = sys[sys_of[i]];
  for (int a = 0; a < 3; ++a) {
    double f;
    double xv = x[3 * i + a];
    double wv = wrap_coord(xv, S.L[a], &f);
    if (!isfinite(xv) || !(fabs(f) < 1.0e8)) {
      atomicOr(flags, kFlagNonFinite);
      wv = 0.0;
      f = 0.0;
    }
    w[3 * i + a] = wv;
    fl[3 * i + a] = (int)f;
  }
}

// -------------------------------------------------------------- cells
__global__ void k_cell_clear(int ncell, int* __restrict__ cell_cnt, int* __restrict__ fill,
                             const int* __restrict__ flags) {
  if (!(*flags & kFlagRebuild)) return;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncell) {
    cell_cnt[c] = 0;
    fill[c] = 0;
  }
}

__device__ __forceinline__ int cell_coord(double w, double cs, int nc) {
  int k = (int)floor(w / cs);
  return k < 0 ? 0 : (k >= nc ? nc - 1 : k);
}

__global__ void k_cell_count(int n, const double* __restrict__ w, const int* __restrict__ sys_of,
                             const SysInfo* __restrict__ sys, int* __restrict__ cell_of,
                             int* __restrict__ cell_cnt, const int* __restrict__ flags) {
  if (!(*flags & kFlagRebuild)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const SysInfo& S = sys[sys_of[i]];
  if (!S.use_cells) {
    cell_of[i] = -1;
    return;
  }
  int k0 = cell_coord(w[3 * i + 0], S.cs[0], S.nc[0]);
  int k1 = cell_coord(w[3 * i + 1], S.cs[1], S.nc[1]);
  int k2 = cell_coord(w[3 * i + 2], S.cs[2], S.nc[2]);
  int c = S.cell0 + (k0 * S.nc[1] + k1) * S.nc[2] + k2;
  cell_of[i] = c;
  atomicAdd(&cell_cnt[c], 1);
}

// exclusive scan of the cell counts (one block; the cell count is small)
__global__ void k_cell_scan(int ncell, const int* __restrict__ cell_cnt,
                            int* __restrict__ cell_start, const int* __restrict__ flags) {
  if (!(*flags & kFlagRebuild)) return;
  __shared__ int part[1024];
  int t = threadIdx.x, nt = blockDim.x;
  int per = (ncell + nt - 1) / nt;
  int lo = t * per, hi = min(ncell, lo + per);
  int s = 0;
  for (int c = lo; c < hi; ++c) s += cell_cnt[c];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < nt; o <<= 1) {
    int v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = part[t] - s;
  for (int c = lo; c < hi; ++c) {
    cell_start[c] = run;
    run += cell_cnt[c];
  }
  if (t == nt - 1) cell_start[ncell] = part[nt - 1];
}

__global__ void k_cell_fill(int n, const int* __restrict__ cell_of,
                            const int* __restrict__ cell_start, int* __restrict__ fill,
                            int* __restrict__ cell_idx, const int* __restrict__ flags) {
  if (!(*flags & kFlagRebuild)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = cell_of[i];
  if (c < 0) return;
  cell_idx[cell_start[c] + atomicAdd(&fill[c], 1)] = i;
}

// ascending atom order inside every cell, so the skin lists come out in a
// fixed order whatever order the atomics above took
__global__ void k_cell_sort(int ncell, const int* __restrict__ cell_start,
                            int* __restrict__ cell_idx, const int* __restrict__ flags) {
  if (!(*flags & kFlagRebuild)) return;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  int lo = cell_start[c], hi = cell_start[c + 1];
  for (int a = lo + 1; a < hi; ++a) {
    int v = cell_idx[a];
    int b = a - 1;
    while (b >= lo && cell_idx[b] > v) {
      cell_idx[b + 1] = cell_idx[b];
      --b;
    }
    cell_idx[b + 1] = v;
  }
}

// -------------------------------------------------------------- skin lists
// One warp per atom.  Candidates (j, image) first pass a conservative FP32
// test, |r|^2 < (rskin + margin)^2 for the cell search or |r_a| < rskin +
// margin per axis for small boxes, where the margin is orders of magnitude
// above the FP32 rounding of coordinates of that size; the survivors go
// through a per-warp queue and are decided by the exact FP64 distance in
// batches of 32, so the (slow) FP64 work scales with the skin size rather
// than with the number of candidates.  Entries are appended through ballots
// in the order the candidates were queued, so the list is deterministic.
constexpr int kSkinWarps = 4;

// position of the k-th (from 0) set bit of m, -1 if there are fewer
__device__ __forceinline__ int nth_bit(unsigned m, int k) {
  for (int b = 0; b < 32; ++b)
    if ((m >> b) & 1u) {
      if (k == 0) return b;
      --k;
    }
  return -1;
}

__global__ void __launch_bounds__(32 * kSkinWarps)
k_skin_build(int n, const double* __restrict__ w, const int* __restrict__ fl,
             const int* __restrict__ sys_of, const SysInfo* __restrict__ sys,
             const int* __restrict__ cell_of, const int* __restrict__ cell_start,
             const int* __restrict__ cell_idx, double rskin, int cap,
             SkinEntry* __restrict__ skin, int* __restrict__ skin_cnt,
             int* __restrict__ flags) {
  if (!(*flags & kFlagRebuild)) return;
  __shared__ int4 queue_all[kSkinWarps][64];
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= n) return;
  int4* queue = queue_all[threadIdx.x >> 5];
  const unsigned lt = (1u << lane) - 1u;
  int i = warp;
  const SysInfo& S = sys[sys_of[i]];
  double wi[3] = {w[3 * i], w[3 * i + 1], w[3 * i + 2]};
  int fi[3] = {fl[3 * i], fl[3 * i + 1], fl[3 * i + 2]};
  const double r2cut = rskin * rskin;
  const float Lf[3] = {(float)S.L[0], (float)S.L[1], (float)S.L[2]};
  const float wif[3] = {(float)wi[0], (float)wi[1], (float)wi[2]};
  const float lim = (float)rskin + 1e-5f * (fmaxf(Lf[0], fmaxf(Lf[1], Lf[2])) + (float)rskin);
  const float lim2 = lim * lim;
  int cnt = 0, qn = 0;
  SkinEntry* out = skin + (size_t)i * cap;

  // exact decision for queue[0, k), then the rest moves to the front
  auto flush = [&](int k) {
    bool take = false;
    SkinEntry e;
    if (lane < k) {
      const int4 q = queue[lane];
      int nn[3] = {q.y, q.z, q.w};
      double r[3];
      double d2 = sep_exact(wi, w + 3 * q.x, nn, S.L, r);
      if (d2 < r2cut && d2 > 0.0) {
        take = true;
        e.j = q.x;
        e.mx = q.y - fl[3 * q.x + 0] + fi[0];
        e.my = q.z - fl[3 * q.x + 1] + fi[1];
        e.mz = q.w - fl[3 * q.x + 2] + fi[2];
      }
    }
    unsigned b = __ballot_sync(0xffffffffu, take);
    int pos = cnt + __popc(b & lt);
    if (take && pos < cap) out[pos] = e;
    cnt += __popc(b);
    const int rest = qn - k;
    int4 v = make_int4(0, 0, 0, 0);
    if (lane < rest) v = queue[k + lane];
    __syncwarp();
    if (lane < rest) queue[lane] = v;
    __syncwarp();
    qn = rest;
  };
  auto enqueue = [&](bool pass, int j, int nx, int ny, int nz) {
    unsigned b = __ballot_sync(0xffffffffu, pass);
    if (pass) queue[qn + __popc(b & lt)] = make_int4(j, nx, ny, nz);
    qn += __popc(b);
    __syncwarp();
    if (qn >= 32) flush(32);
  };

  if (S.use_cells) {
    int c = cell_of[i] - S.cell0;
    int k[3] = {c / (S.nc[1] * S.nc[2]), (c / S.nc[2]) % S.nc[1], c % S.nc[2]};
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          int q[3] = {k[0] + dx, k[1] + dy, k[2] + dz};
          int nn[3];
          for (int a = 0; a < 3; ++a) {
            nn[a] = 0;
            if (q[a] < 0) { q[a] += S.nc[a]; nn[a] = -1; }
            if (q[a] >= S.nc[a]) { q[a] -= S.nc[a]; nn[a] = 1; }
          }
          int cell = S.cell0 + (q[0] * S.nc[1] + q[1]) * S.nc[2] + q[2];
          int lo = cell_start[cell], hi = cell_start[cell + 1];
          for (int base = lo; base < hi; base += 32) {
            int s = base + lane;
            bool pass = false;
            int j = 0;
            if (s < hi) {
              j = cell_idx[s];
              float d2 = 0.f;
              for (int a = 0; a < 3; ++a) {
                const float r = ((float)w[3 * j + a] - wif[a]) + (float)nn[a] * Lf[a];
                d2 += r * r;
              }
              pass = d2 < lim2 && !(j == i && nn[0] == 0 && nn[1] == 0 && nn[2] == 0);
            }
            enqueue(pass, j, nn[0], nn[1], nn[2]);
          }
        }
  } else {
    // per lane one atom j; per axis the images with |r_a| < lim as a bit mask
    // (bit b: image b - nimg), then the lane's candidates in (x, y, z) order
    for (int base = 0; base < S.natom; base += 32) {
      const int jj = base + lane;
      const bool valid = jj < S.natom;
      const int j = S.atom0 + (valid ? jj : 0);
      unsigned m[3] = {0u, 0u, 0u};
      if (valid)
        for (int a = 0; a < 3; ++a) {
          const float t = (float)w[3 * j + a] - wif[a];
          for (int b = 0; b <= 2 * S.nimg[a]; ++b)
            if (fabsf(t + (float)(b - S.nimg[a]) * Lf[a]) < lim) m[a] |= 1u << b;
        }
      const int cy = __popc(m[1]), cz = __popc(m[2]);
      const int ncand = __popc(m[0]) * cy * cz;
      const int kmax = __reduce_max_sync(0xffffffffu, ncand);
      for (int q = 0; q < kmax; ++q) {
        bool pass = q < ncand;
        int nn[3] = {0, 0, 0};
        if (pass) {
          const int kk[3] = {q / (cy * cz), (q / cz) % cy, q % cz};
          for (int a = 0; a < 3; ++a) nn[a] = nth_bit(m[a], kk[a]) - S.nimg[a];
          pass = !(j == i && nn[0] == 0 && nn[1] == 0 && nn[2] == 0);
        }
        enqueue(pass, j, nn[0], nn[1], nn[2]);
      }
    }
  }
  if (qn > 0) flush(qn);
  if (lane == 0) {
    skin_cnt[i] = cnt < cap ? cnt : cap;
    if (cnt > cap) atomicOr(flags, kFlagOverflow);
  }
}

// mirror[i][c] = index c' in j's skin list of the entry (i, -m)
__global__ void k_mirror(int n, int cap, const SkinEntry* __restrict__ skin,
                         const int* __restrict__ skin_cnt, int* __restrict__ mirror,
                         int* __restrict__ flags) {
  if (!(*flags & kFlagRebuild)) return;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * cap) return;
  int i = (int)(t / cap), c = (int)(t % cap);
  if (c >= skin_cnt[i]) return;
  SkinEntry e = skin[t];
  const SkinEntry* other = skin + (size_t)e.j * cap;
  int cj = skin_cnt[e.j];
  int found = -1;
  for (int q = 0; q < cj; ++q) {
    SkinEntry o = other[q];
    if (o.j == i && o.mx == -e.mx && o.my == -e.my && o.mz == -e.mz) {
      found = q;
      break;
    }
  }
  mirror[t] = found;
  if (found < 0) atomicOr(flags, kFlagMirror);
}

__global__ void k_build_end(int n, const double* __restrict__ x, double* __restrict__ xref,
                            const int* __restrict__ flags) {
  if (!(*flags & kFlagRebuild)) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 3 * n) xref[i] = x[i];
}

__global__ void k_flag_clear(int* flags, int bits) {
  if (threadIdx.x == 0 && blockIdx.x == 0) atomicAnd(flags, ~bits);
}

__global__ void k_flag_set(int* flags, int bits) {
  if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(flags, bits);
}

// -------------------------------------------------------------- selection
// One warp per atom.  sel_* hold the kept neighbours in key order; selpos maps
// every skin entry to its slot (or -1).  With grp: pairs of members only, or
// (grp_centres) every pair whose centre is a member.
__global__ void k_select(int n, int cap, int nmax, double rc, const double* __restrict__ w,
                         const int* __restrict__ fl, const int* __restrict__ sys_of,
                         const SysInfo* __restrict__ sys, const SkinEntry* __restrict__ skin,
                         const int* __restrict__ skin_cnt, const unsigned char* __restrict__ grp,
                         int grp_centres, int* __restrict__ sel_j,
                         int* __restrict__ sel_img, double* __restrict__ sel_r,
                         short* __restrict__ selpos, int* __restrict__ n_in_rc) {
  extern __shared__ unsigned char smem_raw[];
  int wib = threadIdx.x >> 5;
  int lane = threadIdx.x & 31;
  int i = blockIdx.x * (blockDim.x >> 5) + wib;
  // per warp: cap x {d2, r[3]} doubles + cap x {j, n[3], c} ints
  double* sd2 = reinterpret_cast<double*>(smem_raw) + (size_t)wib * cap * 4;
  int* sint = reinterpret_cast<int*>(reinterpret_cast<double*>(smem_raw) + (size_t)(blockDim.x >> 5) * cap * 4) +
              (size_t)wib * cap * 5;
  if (i >= n) return;
  const SysInfo& S = sys[sys_of[i]];
  double wi[3] = {w[3 * i], w[3 * i + 1], w[3 * i + 2]};
  int fi[3] = {fl[3 * i], fl[3 * i + 1], fl[3 * i + 2]};
  int cnt = skin_cnt[i];
  const SkinEntry* lst = skin + (size_t)i * cap;
  short* sp = selpos + (size_t)i * cap;
  double rc2 = rc * rc;
  int k = 0;
  for (int base = 0; base < cnt; base += 32) {
    int c = base + lane;
    bool take = false;
    double r[3], d2 = 0;
    int nn[3] = {0, 0, 0};
    int j = 0;
    if (c < cnt) {
      SkinEntry e = lst[c];
      j = e.j;
      nn[0] = e.mx + fl[3 * j + 0] - fi[0];
      nn[1] = e.my + fl[3 * j + 1] - fi[1];
      nn[2] = e.mz + fl[3 * j + 2] - fi[2];
      d2 = sep_exact(wi, w + 3 * j, nn, S.L, r);
      take = d2 < rc2 && d2 > 0.0 && (!grp || (grp[i] && (grp_centres || grp[j])));
      sp[c] = -1;
    }
    unsigned b = __ballot_sync(0xffffffffu, take);
    if (take) {
      int q = k + __popc(b & ((1u << lane) - 1u));
      sd2[4 * q + 0] = d2;
      sd2[4 * q + 1] = r[0];
      sd2[4 * q + 2] = r[1];
      sd2[4 * q + 3] = r[2];
      sint[5 * q + 0] = j;
      sint[5 * q + 1] = nn[0];
      sint[5 * q + 2] = nn[1];
      sint[5 * q + 3] = nn[2];
      sint[5 * q + 4] = c;
    }
    k += __popc(b);
  }
  __syncwarp();
  if (lane == 0) n_in_rc[i] = k;
  // rank = the number of keys (d2, j, n) below the query's.  The count runs
  // on d2 alone (64-bit integer compares of the bit patterns, four keys per
  // step with their loads issued together); a query whose d2 equals another
  // key's is recounted with the full key, so the ranks are those of key_less.
  const long long* sbits = reinterpret_cast<const long long*>(sd2);
  for (int q = lane; q < k; q += 32) {
    const long long dqb = sbits[4 * q];
    int jq = sint[5 * q];
    const int* nq = sint + 5 * q + 1;
    int rank = 0, eq = 0;
    int p = 0;
    for (; p + 4 <= k; p += 4) {
      const long long d0 = sbits[4 * p], d1 = sbits[4 * p + 4], d2b = sbits[4 * p + 8],
                      d3 = sbits[4 * p + 12];
      rank += (d0 < dqb) + (d1 < dqb) + (d2b < dqb) + (d3 < dqb);
      eq += (d0 == dqb) + (d1 == dqb) + (d2b == dqb) + (d3 == dqb);
    }
    for (; p < k; ++p) {
      const long long d0 = sbits[4 * p];
      rank += d0 < dqb;
      eq += d0 == dqb;
    }
    if (eq > 1) {   // a tie besides the query itself
      const double dq = sd2[4 * q];
      rank = 0;
      for (int t = 0; t < k; ++t)
        rank += key_less(sd2[4 * t], sint[5 * t], sint + 5 * t + 1, dq, jq, nq) ? 1 : 0;
    }
    if (rank < nmax) {
      size_t o = (size_t)i * nmax + rank;
      sel_j[o] = jq;
      sel_img[3 * o + 0] = nq[0];
      sel_img[3 * o + 1] = nq[1];
      sel_img[3 * o + 2] = nq[2];
      sel_r[3 * o + 0] = sd2[4 * q + 1];
      sel_r[3 * o + 1] = sd2[4 * q + 2];
      sel_r[3 * o + 2] = sd2[4 * q + 3];
      sp[sint[5 * q + 4]] = (short)rank;
    }
  }
  for (int p = k + lane; p < nmax; p += 32) {
    size_t o = (size_t)i * nmax + p;
    sel_j[o] = -1;
    sel_img[3 * o + 0] = 0;
    sel_img[3 * o + 1] = 0;
    sel_img[3 * o + 2] = 0;
    sel_r[3 * o + 0] = 0.0;
    sel_r[3 * o + 1] = 0.0;
    sel_r[3 * o + 2] = 0.0;
  }
}

size_t select_smem_bytes(int cap, int warps) {
  return (size_t)warps * cap * (4 * sizeof(double) + 5 * sizeof(int));
}

// -------------------------------------------------------------- launchers
void launch_nlist_rebuild(const NlistArgs& a, cudaStream_t st) {
  int nb = ceil_div(a.n, 256);
  k_cell_clear<<<ceil_div(a.ncell > 0 ? a.ncell : 1, 256), 256, 0, st>>>(a.ncell, a.cell_cnt,
                                                                      a.cell_fill, a.flags);
  k_cell_count<<<nb, 256, 0, st>>>(a.n, a.w, a.sys_of, a.sys, a.cell_of, a.cell_cnt, a.flags);
  k_cell_scan<<<1, 1024, 0, st>>>(a.ncell, a.cell_cnt, a.cell_start, a.flags);
  k_cell_fill<<<nb, 256, 0, st>>>(a.n, a.cell_of, a.cell_start, a.cell_fill, a.cell_idx, a.flags);
  k_cell_sort<<<ceil_div(a.ncell > 0 ? a.ncell : 1, 128), 128, 0, st>>>(a.ncell, a.cell_start,
                                                                      a.cell_idx, a.flags);
  k_skin_build<<<ceil_div((long long)a.n, kSkinWarps), 32 * kSkinWarps, 0, st>>>(
      a.n, a.w, a.fl, a.sys_of, a.sys, a.cell_of, a.cell_start, a.cell_idx, a.rskin, a.cap, a.skin,
      a.skin_cnt, a.flags);
  k_mirror<<<ceil_div((long long)a.n * a.cap, 256), 256, 0, st>>>(a.n, a.cap, a.skin, a.skin_cnt,
                                                                 a.mirror, a.flags);
  k_build_end<<<ceil_div(3LL * a.n, 256), 256, 0, st>>>(a.n, a.x, a.xref, a.flags);
  k_flag_clear<<<1, 32, 0, st>>>(a.flags, kFlagRebuild);
}

int nlist_rebuild_kernels() { return 9; }

void launch_wrap(const NlistArgs& a, cudaStream_t st) {
  k_wrap<<<ceil_div(a.n, 256), 256, 0, st>>>(a.n, a.x, a.sys_of, a.sys, a.w, a.fl, a.flags);
}

static const size_t kSelectSmemMax = 200 * 1024;

int select_max_cap() { return (int)(kSelectSmemMax / select_smem_bytes(1, 1)); }

void launch_select(const NlistArgs& a, cudaStream_t st) {
  int warps = 4;
  while (warps > 1 && select_smem_bytes(a.cap, warps) > kSelectSmemMax) --warps;
  size_t sm = select_smem_bytes(a.cap, warps);
  k_select<<<ceil_div(a.n, warps), warps * 32, sm, st>>>(a.n, a.cap, a.nmax, a.rc, a.w, a.fl,
                                                         a.sys_of, a.sys, a.skin, a.skin_cnt,
                                                         a.grp, a.grp_centres, a.sel_j,
                                                         a.sel_img, a.sel_r,
                                                         a.selpos, a.n_in_rc);
}

void launch_flag_set(int* flags, int bits, cudaStream_t st) { k_flag_set<<<1, 32, 0, st>>>(flags, bits); }

cudaError_t nlist_configure() {
  // the largest shared-memory carve-out: each warp holds its atom's candidates
  // there, and more resident warps hide the latency of the FP64 distances
  cudaError_t e = cudaFuncSetAttribute(k_select, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kSelectSmemMax);
}

}  // namespace dp
