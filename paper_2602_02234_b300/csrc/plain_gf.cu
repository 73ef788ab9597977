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

template <typename T>
__global__ void k_init(int n, int nmax, int nd, int ed, const int* __restrict__ types,
                       const int* __restrict__ sel_j, const T* __restrict__ s,
                       const T* __restrict__ Wt, const T* __restrict__ we,
                       const T* __restrict__ be0, T* __restrict__ node, T* __restrict__ edge) {
  int i = blockIdx.x;
  for (int c = threadIdx.x; c < nd; c += blockDim.x) node[(size_t)i * nd + c] = Wt[types[i] * nd + c];
  for (int idx = threadIdx.x; idx < nmax * ed; idx += blockDim.x) {
    int p = idx / ed, c = idx % ed;
    size_t e = (size_t)i * nmax + p;
    edge[e * ed + c] = sel_j[e] >= 0 ? dtanh(s[e] * we[c] + be0[c]) : T(0);
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

__device__ __forceinline__ void legendre4(float c, float* P, float* dP) {
  P[0] = 1.f; P[1] = c; P[2] = 0.5f * (3.f * c * c - 1.f); P[3] = 0.5f * (5.f * c * c * c - 3.f * c);
  dP[0] = 0.f; dP[1] = 1.f; dP[2] = 3.f * c; dP[3] = 0.5f * (15.f * c * c - 3.f);
}
__device__ __forceinline__ void legendre4(double c, double* P, double* dP) {
  P[0] = 1.0; P[1] = c; P[2] = 0.5 * (3.0 * c * c - 1.0); P[3] = 0.5 * (5.0 * c * c * c - 3.0 * c);
  dP[0] = 0.0; dP[1] = 1.0; dP[2] = 3.0 * c; dP[3] = 0.5 * (15.0 * c * c - 3.0);
}

constexpr int kMaxNa = 64;

// number of angle slots of atom i (a prefix of the nearest-first list)
template <typename T>
__device__ int n_angle(const T* sa, long long base, int nmax, int na) {
  int k = 0;
  while (k < na && k < nmax && sa[base + k] > T(0)) ++k;
  return k;
}

// (c) forward: a_ip for the angle slots of one atom (block per atom).
// a_p[c] = sum_l Wphi[l][c] sum_k coef_pkl q_k[c] with coef_pkl = w_pk P_l(c_pk)
// (0 for k = p), the coefficients and the slots' q rows staged in shared memory.
// q and a hold the angle rows only: slot p < ca of atom i at row i ca + p
// (ca = min(na, nmax); rows p >= the atom's angle count get a = 0).
// Shared memory: na x na x 4 coefficients, Wphi by column (ed x 4), then
// (staged) na x ed of q.
template <typename T>
__global__ void k_angle(int nmax, int na, int ca, int ed, T inv_na, const T* __restrict__ sa,
                        const T* __restrict__ rh, const T* __restrict__ q,
                        const T* __restrict__ Wphi, T* __restrict__ a, int staged) {
  extern __shared__ unsigned char sm_raw[];
  T* coef = reinterpret_cast<T*>(sm_raw);  // na x na x 4
  T* W4 = coef + (size_t)na * na * 4;      // ed x 4: Wphi[l][c] at W4[4 c + l]
  int i = blockIdx.x;
  long long base = (long long)i * nmax;
  int nang = n_angle(sa, base, nmax, na);
  for (int idx = threadIdx.x; idx < 4 * ed; idx += blockDim.x) W4[idx] = Wphi[(idx & 3) * ed + (idx >> 2)];
  const long long abase = (long long)i * ca;   // this atom's first angle row
  const T* qs = q + abase * ed;
  if (staged) {
    T* st = W4 + (size_t)ed * 4;            // na x ed
    for (int idx = threadIdx.x; idx < nang * ed; idx += blockDim.x) st[idx] = qs[idx];
    qs = st;
  }
  for (int pk = threadIdx.x; pk < nang * nang; pk += blockDim.x) {
    int p = pk / nang, k = pk % nang;
    T P[4], dP[4];
    const T* rp = rh + 3 * (base + p);
    const T* rk = rh + 3 * (base + k);
    legendre4(rp[0] * rk[0] + rp[1] * rk[1] + rp[2] * rk[2], P, dP);
    T w = (p == k) ? T(0) : inv_na * sa[base + p] * sa[base + k];
    for (int l = 0; l < 4; ++l) coef[(p * nang + k) * 4 + l] = w * P[l];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < ca * ed; idx += blockDim.x) {
    int p = idx / ed, c = idx % ed;
    T out = T(0);
    if (p < nang) {
      T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
      for (int k = 0; k < nang; ++k) {
        const T qk = qs[k * ed + c];
        T cf[4];
        ld4(coef + (p * nang + k) * 4, cf);
        s0 += cf[0] * qk; s1 += cf[1] * qk; s2 += cf[2] * qk; s3 += cf[3] * qk;
      }
      T w[4];
      ld4(W4 + 4 * c, w);
      out = w[0] * s0 + w[1] * s1 + w[2] * s2 + w[3] * s3;
    }
    a[(abase + p) * ed + c] = out;
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

// (c) adjoint of a_ip: dq, and the switch / unit-vector terms; block per atom.
// Shared memory: the adjoints dcoef_pkl (na x na x 4); with mode >= 1 also the
// coefficients coef_pkl = w_pk P_l(c_pk) (0 for k = p), with mode 2 also the
// angle slots' da and q rows (na rows of ed, stored with stride ed + 1 so that
// threads on different rows of one column hit different banks).  Mode 0
// recomputes the coefficients per column (the host picks the largest mode
// that fits).  q, da and dq hold the angle rows only (row i ca + p).
template <typename T>
__global__ void k_angle_bwd(int nmax, int na, int ca, int ed, T inv_na, const T* __restrict__ sa,
                            const T* __restrict__ rh, const T* __restrict__ q,
                            const T* __restrict__ Wphi, const T* __restrict__ da,
                            T* __restrict__ dq, T* __restrict__ dsa_e, T* __restrict__ drh,
                            int mode) {
  extern __shared__ unsigned char sm_raw[];
  T* dcoef = reinterpret_cast<T*>(sm_raw);  // na x na x 4
  T* W4 = dcoef + (size_t)na * na * 4;      // ed x 4: Wphi[l][c] at W4[4 c + l]
  T* coef = W4 + (size_t)ed * 4;            // na x na x 4 (mode >= 1)
  int i = blockIdx.x;
  long long base = (long long)i * nmax;
  int nang = n_angle(sa, base, nmax, na);
  for (int idx = threadIdx.x; idx < 4 * ed; idx += blockDim.x) W4[idx] = Wphi[(idx & 3) * ed + (idx >> 2)];
  const long long abase = (long long)i * ca;   // this atom's first angle row
  const T* das = da + abase * ed;
  const T* qs = q + abase * ed;
  int ld = ed;
  if (mode == 2) {
    ld = ed + 1;
    T* s_da = coef + (size_t)na * na * 4;
    T* s_q = s_da + (size_t)na * ld;
    for (int idx = threadIdx.x; idx < nang * ed; idx += blockDim.x) {
      const int p = idx / ed, c = idx - p * ed;
      s_da[p * ld + c] = das[idx];
      s_q[p * ld + c] = qs[idx];
    }
    das = s_da;
    qs = s_q;
  }
  if (mode >= 1) {
    for (int pk = threadIdx.x; pk < nang * nang; pk += blockDim.x) {
      int p = pk / nang, k = pk % nang;
      T P[4], dP[4];
      const T* rp = rh + 3 * (base + p);
      const T* rk = rh + 3 * (base + k);
      legendre4(rp[0] * rk[0] + rp[1] * rk[1] + rp[2] * rk[2], P, dP);
      T w = (p == k) ? T(0) : inv_na * sa[base + p] * sa[base + k];
      for (int l = 0; l < 4; ++l) coef[pk * 4 + l] = w * P[l];
    }
  }
  __syncthreads();
  // dq_k[c] = sum_l Wphi[l][c] sum_p coef_pkl da_p[c]
  for (int idx = threadIdx.x; idx < ca * ed; idx += blockDim.x) {
    int k = idx / ed, c = idx % ed;
    T out = T(0);
    if (k < nang) {
      T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
      const T* rk = rh + 3 * (base + k);
      for (int p = 0; p < nang; ++p) {
        const T d = das[p * ld + c];
        T cf[4];
        if (mode >= 1) {
          ld4(coef + (p * nang + k) * 4, cf);
        } else {
          const T* rp = rh + 3 * (base + p);
          T P[4], dP[4];
          legendre4(rp[0] * rk[0] + rp[1] * rk[1] + rp[2] * rk[2], P, dP);
          const T w = (p == k) ? T(0) : inv_na * sa[base + p] * sa[base + k];
          for (int l = 0; l < 4; ++l) cf[l] = w * P[l];
        }
        s0 += cf[0] * d; s1 += cf[1] * d; s2 += cf[2] * d; s3 += cf[3] * d;
      }
      T w[4];
      ld4(W4 + 4 * c, w);
      out = w[0] * s0 + w[1] * s1 + w[2] * s2 + w[3] * s3;
    }
    dq[(abase + k) * ed + c] = out;
  }
  // dcoef_pkl = sum_c da_p[c] Wphi[l][c] q_k[c]  (one thread per (p, k))
  for (int pk = threadIdx.x; pk < nang * nang; pk += blockDim.x) {
    const int p = pk / nang, k = pk - p * nang;
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    if (p != k)
      for (int c = 0; c < ed; ++c) {
        const T x = das[p * ld + c] * qs[k * ld + c];
        T w[4];
        ld4(W4 + 4 * c, w);
        a0 += x * w[0];
        a1 += x * w[1];
        a2 += x * w[2];
        a3 += x * w[3];
      }
    dcoef[pk * 4 + 0] = a0;
    dcoef[pk * 4 + 1] = a1;
    dcoef[pk * 4 + 2] = a2;
    dcoef[pk * 4 + 3] = a3;
  }
  __syncthreads();
  // switch and unit-vector terms: one warp per angle slot p, lanes over the
  // partners k, then a fixed-order warp reduction
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int p = warp; p < nang; p += nw) {
    const T* rp = rh + 3 * (base + p);
    const T sp = sa[base + p];
    T dsp = T(0), dr[3] = {T(0), T(0), T(0)};
    for (int k = lane; k < nang; k += 32) {
      if (k == p) continue;
      const T* rk = rh + 3 * (base + k);
      T P[4], dP[4];
      legendre4(rp[0] * rk[0] + rp[1] * rk[1] + rp[2] * rk[2], P, dP);
      // p as the first index (dcoef_pk) and as the second (dcoef_kp)
      const T* d1 = dcoef + (p * nang + k) * 4;
      const T* d2 = dcoef + (k * nang + p) * 4;
      const T sk = sa[base + k];
      T dc = T(0);
      for (int l = 0; l < 4; ++l) {
        dsp += (d1[l] + d2[l]) * inv_na * sk * P[l];
        dc += (d1[l] + d2[l]) * inv_na * sp * sk * dP[l];
      }
      for (int a = 0; a < 3; ++a) dr[a] += dc * rk[a];
    }
    dsp = warp_sum(dsp);
    for (int a = 0; a < 3; ++a) dr[a] = warp_sum(dr[a]);
    if (lane == 0) {
      dsa_e[base + p] += dsp;
      for (int a = 0; a < 3; ++a) drh[3 * (base + p) + a] += dr[a];
    }
  }
}

// (b): dy = de1 (1 - v^2) on real slots
template <typename T>
__global__ void k_dtanh(long long n, const T* __restrict__ g, const T* __restrict__ y,
                        T* __restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = g[i] * (T(1) - y[i] * y[i]);
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

// (a) per slot: de += (1/nmax) sw dm_i * u_j;  X = (1/nmax) sw dm_i * e (for du_j);
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
  long long i = s / nmax;
  T acc = T(0);
  for (int c = lane; c < ed; c += 32) {
    if (j < 0) {
      X[s * ed + c] = T(0);
      continue;
    }
    T g = dm[i * ldm + c], ev = e[s * ed + c], uv = u[(long long)j * ed + c];
    de[s * ed + c] += inv_nmax * sw[s] * g * uv;
    X[s * ed + c] = inv_nmax * sw[s] * g * ev;
    acc += g * ev * uv;
  }
  acc = warp_sum(acc);
  if (lane == 0 && j >= 0) dsw_e[s] += inv_nmax * acc;
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

template <typename T>
__global__ void k_fill(long long n, T v, T* __restrict__ p) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// ------------------------------------------------------------------ host side
template <typename T>
class PlainGf : public Model {
 public:
  ~PlainGf() override {
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
          (reinterpret_cast<uintptr_t>(g.aux) & 15) == 0) {   // 16-byte rows of A, C, aux
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
        gemm_tc(t, st);
        return;
      }
    }
    gemm(g, 1, st);
  }
  // per atom j: the sum of x over every kept slot (i, p) whose neighbour is j,
  // in increasing (i, p) order whatever the skin list's order
  void gather_in(const NbrView& nv, const T* x, T* out, cudaStream_t st) {
    int warps = 4;
    while (warps > 1 && sizeof(int) * 2 * nv.cap * warps > 48 * 1024) --warps;
    k_mp_gather<T><<<ceil_div(n_, warps), warps * 32, sizeof(int) * 2 * nv.cap * warps, st>>>(
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
      t.status = flags_;
#ifdef DP_GF_BF16
      t.fp16 = 0;
#else
      t.fp16 = 1;
#endif
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
      t.status = flags_;
#ifdef DP_GF_BF16
      t.fp16 = 0;
#else
      t.fp16 = 1;
#endif
      gemm_tc(t, st);
      return true;
    } else {
      (void)l; (void)st;
      return false;
    }
  }
  bool tc_ = false;
  int* flags_ = nullptr;
  const unsigned char* seed_ = nullptr;   // energy seed (device, optional)
  // shared-memory variants of the angle kernels (see k_angle, k_angle_bwd)
  int angle_staged_ = 0, angle_mode_ = 0;
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
  for (int l = 0; l <= L && ok; ++l) ok = dalloc(&nn_[l], N * Nd, err) && dalloc(&ee_[l], P * Ed, err);
  for (int l = 0; l < L && ok; ++l)
    ok = dalloc(&hh_[l], N * Nd, err) && dalloc(&uu_[l], N * Ed, err) &&
         dalloc(&mm_[l], N * Ed, err) && dalloc(&vv_[l], P * Ed, err) && dalloc(&qq_[l], PA * Ed, err) &&
         dalloc(&tt_[l], PA * Ed, err);
  // the angle kernels stage as much as fits in 227 KB of shared memory
  const size_t kMaxSmem = 232448, na2 = (size_t)m.na * m.na * 4 * sizeof(T),
               w4 = (size_t)m.ed * 4 * sizeof(T),
               rowsz = (size_t)m.na * m.ed * sizeof(T), rowsz1 = (size_t)m.na * (m.ed + 1) * sizeof(T);
  angle_staged_ = na2 + w4 + rowsz <= kMaxSmem ? 1 : 0;
  angle_smem_ = na2 + w4 + (angle_staged_ ? rowsz : 0);
  angle_mode_ = 2 * na2 + w4 + 2 * rowsz1 <= kMaxSmem ? 2 : (2 * na2 + w4 <= kMaxSmem ? 1 : 0);
  angle_bwd_smem_ = na2 * (angle_mode_ >= 1 ? 2 : 1) + w4 + (angle_mode_ == 2 ? 2 * rowsz1 : 0);
  const int angle_smem = (int)angle_smem_, angle_bwd_smem = (int)angle_bwd_smem_;
  if (cudaFuncSetAttribute(k_angle<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, angle_smem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_angle_bwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, angle_bwd_smem) !=
          cudaSuccess) {
    *err = "graph model: angle kernels cannot get their shared memory";
    return false;
  }
  ok = ok && dalloc(&Ai_, N * Ed, err) && dalloc(&Bj_, N * Ed, err) && dalloc(&Ce_, P * Ed, err) &&
       dalloc(&aa_, PA * Ed, err) && dalloc(&y1_, N * m.f1, err) && dalloc(&y2_, N * m.f2, err) &&
       dalloc(&y3_, N * m.f3, err) && dalloc(&d1_, N * m.f1, err) && dalloc(&d2_, N * m.f2, err) &&
       dalloc(&d3_, N * m.f3, err) && dalloc(&dn_, N * Nd, err) && dalloc(&dn1_, N * Nd, err) &&
       dalloc(&de_, P * Ed, err) && dalloc(&dy_, P * Ed, err) &&
       dalloc(&dz_, PA * Ed, err) && dalloc(&da_, PA * Ed, err) && dalloc(&dq_, PA * Ed, err) &&
       dalloc(&du_, N * Ed, err) && dalloc(&dx_, N * Nd, err) && dalloc(&dnm_, N * (Nd + Ed), err) &&
       dalloc(&X_, P * Ed, err) && dalloc(&sdy_, N * Ed, err) && dalloc(&gat_, N * Ed, err) &&
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
  k_init<T><<<n, 128, 0, st>>>(n, NM, Nd, Ed, types, nv.sel_j, s_, Wt_, we_, be0_, nn_[0], ee_[0]);
  k += 2;
  const size_t angle_smem = angle_smem_, angle_bwd_smem = angle_bwd_smem_;
  const int ed_shift = (Ed & (Ed - 1)) == 0 ? __builtin_ctz((unsigned)Ed) : -1;
  for (int l = 0; l < L; ++l) {
    // (a)
    mm(gemm_rowmajor<T>(n, Ed, Nd, nn_[l], Nd, Wm_[l], Ed, uu_[l], Ed), st);
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
    {
      Gemm<T> g = gemm_rowmajor<T>((int)PA, Ed, Ed, ee_[l + 1], Ed, Wp_[l], Ed, qq_[l], Ed);
      g.a_rows = ang_rows_;
      mm(g, st);
    }
    k_angle<T><<<n, 256, angle_smem, st>>>(NM, NA, CA, Ed, inv_na, sa_, rh_, qq_[l], Wphi_[l], aa_,
                                           angle_staged_);
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
  // fitting
  for (int t = 0; t < S; ++t) {
    auto rg = fit_ranges_[t];
    if (rg.second == 0) continue;
    const int* rws = fit_rows_ + rg.first;
    Gemm<T> g = gemm_rowmajor<T>(rg.second, m.f1, Nd, nn_[L], Nd, F1_[t], m.f1, y1_, m.f1);
    g.a_rows = rws; g.c_rows = rws; g.bias = c1_[t]; g.epi = 1;
    mm(g, st);
    g = gemm_rowmajor<T>(rg.second, m.f2, m.f1, y1_, m.f1, F2_[t], m.f2, y2_, m.f2);
    g.a_rows = rws; g.c_rows = rws; g.bias = c2_[t]; g.epi = 1;
    mm(g, st);
    g = gemm_rowmajor<T>(rg.second, m.f3, m.f2, y2_, m.f2, F3_[t], m.f3, y3_, m.f3);
    g.a_rows = rws; g.c_rows = rws; g.bias = c3_[t]; g.epi = 1;
    mm(g, st);
    k += 3;
  }
  k_fit_out<T><<<ceil_div((long long)n * 32, 256), 256, 0, st>>>(n, m.f3, types, y3_, F4_, c4_, atom_e, d3_,
                                                                 seed_);
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
    mm(g, st);
    g.N = m.f1; g.K = m.f2; g.A = d2_; g.a_rm = m.f2; g.B = F2_[t]; g.b_rn = m.f2;
    g.C = d1_; g.c_rm = m.f1; g.aux = y1_;
    mm(g, st);
    g.N = Nd; g.K = m.f1; g.A = d1_; g.a_rm = m.f1; g.B = F1_[t]; g.b_rn = m.f1;
    g.C = dn_; g.c_rm = Nd; g.epi = 0; g.aux = nullptr;
    mm(g, st);
    k += 3;
  }
  // ---- adjoint through the layers
  k_fill<T><<<grid(PE), 256, 0, st>>>(PE, T(0), de_);
  k_fill<T><<<grid(P), 256, 0, st>>>(P, T(0), dsw_e_);
  k_fill<T><<<grid(P), 256, 0, st>>>(P, T(0), dsa_e_);
  k_fill<T><<<grid(3 * P), 256, 0, st>>>(3 * P, T(0), drh_);
  k += 5;
  for (int l = L - 1; l >= 0; --l) {
    // (c): de holds dE/de_{l+1}; it becomes dE/de1 in place (e_{l+1} = e1 + swa t)
    k_angle_out_bwd<T><<<grid(PA * 32), 256, 0, st>>>(PA, Ed, NM, CA, sa_, tt_[l], de_, dz_, dsa_e_);
    {  // da = dz Wq^T (angle rows)
      Gemm<T> g{};
      g.M = (int)PA; g.N = Ed; g.K = Ed;
      g.A = dz_; g.a_rm = Ed; g.a_rk = 1;
      g.B = Wq_[l]; g.b_rk = 1; g.b_rn = Ed;
      g.C = da_; g.c_rm = Ed; g.c_rn = 1; g.nb2 = 1; g.alpha = T(1);
      mm(g, st);
    }
    k_angle_bwd<T><<<n, 256, angle_bwd_smem, st>>>(NM, NA, CA, Ed, inv_na, sa_, rh_, qq_[l], Wphi_[l],
                                                   da_, dq_, dsa_e_, drh_, angle_mode_);
    {  // de1 = de + dq Wp^T, in place on the angle rows' slots (dq is 0 elsewhere)
      Gemm<T> g{};
      g.M = (int)PA; g.N = Ed; g.K = Ed;
      g.A = dq_; g.a_rm = Ed; g.a_rk = 1;
      g.B = Wp_[l]; g.b_rk = 1; g.b_rn = Ed;
      g.C = de_; g.c_rm = Ed; g.c_rn = 1; g.nb2 = 1; g.alpha = T(1); g.beta = T(1);
      g.c_rows = ang_rows_;
      mm(g, st);
    }
    // (b): de now holds dE/de1; it becomes dE/de_l (e1 = e_l + tanh(...))
    k_dtanh<T><<<grid(PE), 256, 0, st>>>(PE, de_, vv_[l], dy_);
    {  // de += dy Wc^T
      Gemm<T> g{};
      g.M = (int)P; g.N = Ed; g.K = Ed;
      g.A = dy_; g.a_rm = Ed; g.a_rk = 1;
      g.B = Wc_[l]; g.b_rk = 1; g.b_rn = Ed;
      g.C = de_; g.c_rm = Ed; g.c_rn = 1; g.nb2 = 1; g.alpha = T(1); g.beta = T(1);
      mm(g, st);
    }
    k_rowsum<T><<<n, 64, 0, st>>>(NM, Ed, dy_, sdy_);
    gather_in(nv, dy_, gat_, st);
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
    k_msg_bwd<T><<<grid(P * 32), 256, 0, st>>>(P, NM, Ed, Nd + Ed, inv_nmax, nv.sel_j, sw_, ee_[l],
                                               uu_[l], dnm_ + Nd, de_, X_, dsw_e_);
    gather_in(nv, X_, du_, st);
    {  // dn += du Wm^T
      Gemm<T> g{};
      g.M = n; g.N = Nd; g.K = Ed;
      g.A = du_; g.a_rm = Ed; g.a_rk = 1;
      g.B = Wm_[l]; g.b_rk = 1; g.b_rn = Ed;
      g.C = dn_; g.c_rm = Nd; g.c_rn = 1; g.nb2 = 1; g.alpha = T(1); g.beta = T(1);
      mm(g, st);
    }
    k += 18;
  }
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
