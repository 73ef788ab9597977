// Plain (unfused) attention-family potential: one simple kernel per operation,
// templated on FP32 / FP64.  It is the comparator of the fused BF16 path and
// the FP64 form used for tight parity on small systems.
//
// Model (paper Sec. II: DPA2's "repinit" embedding, "repformer" residual
// self-attention, "fitting-net"; the paper gives no formulas, this is the
// library's reading, identical in the fused path):
//   env:        sw(r) quintic switch rs..rc, s = sw/r, R~ = (s, s r^/1), r^ = r/|r|
//   embedding:  G = tanh(tanh(tanh(s W1 + b1) W2 + b2) W3 + b3), net of the
//               neighbour's species
//   attention:  per head S = Q K^T / sqrt(d), w_jk = sw_k e^{S_jk} / sum_k sw_k e^{S_jk},
//               A = w (r^_j . r^_k), O = A V;  G <- LN(G + O Wo + bo)
//   descriptor: T = R~^T G / Nmax (4 x M1), D = T^T T[:, :M2]
//   fitting:    e = tanh(tanh(tanh(D F1 + c1) F2 + c2) F3 + c3) F4 + c4, net of
//               the centre's species
// and the adjoint of every step, ending in g_ij = dE/dr_ij per neighbour slot.
// Atoms are processed in chunks so that activations for the backward pass fit
// in device memory; the model is atom-local, so chunks are independent.
#include <math.h>

#include <string>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "gemm.cuh"
#include "mp.cuh"
#include "model.h"

namespace dp {

// =========================================================================
// forward kernels
// =========================================================================
// environment of every neighbour slot; empty slots get zeros
template <typename T>
__global__ void k_env(int rows, int nmax, int atom0, const int* __restrict__ sel_j,
                      const double* __restrict__ sel_r, const int* __restrict__ types, T rs, T rc,
                      T* __restrict__ d, T* __restrict__ sw, T* __restrict__ dsw, T* __restrict__ s,
                      T* __restrict__ Rt, T* __restrict__ rh, int* __restrict__ tj) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= rows) return;
  long long gp = (long long)atom0 * nmax + p;
  int j = sel_j[gp];
  if (j < 0) {
    d[p] = T(1); sw[p] = T(0); dsw[p] = T(0); s[p] = T(0);
    for (int a = 0; a < 4; ++a) Rt[4 * p + a] = T(0);
    for (int a = 0; a < 3; ++a) rh[3 * p + a] = T(0);
    tj[p] = -1;
    return;
  }
  T r[3] = {(T)sel_r[3 * gp], (T)sel_r[3 * gp + 1], (T)sel_r[3 * gp + 2]};
  T dd = dsqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  T a, b;
  smooth_switch(dd, rs, rc, &a, &b);
  T ss = a / dd;
  d[p] = dd; sw[p] = a; dsw[p] = b; s[p] = ss;
  Rt[4 * p] = ss;
  for (int q = 0; q < 3; ++q) {
    rh[3 * p + q] = r[q] / dd;
    Rt[4 * p + 1 + q] = ss * r[q] / dd;
  }
  tj[p] = types[j];
}

// embedding MLP; 8 neighbour slots per 128-thread block; empty slots -> G = 0
template <typename T>
__global__ void k_embed(int rows, int e1, int e2, int m1, const T* __restrict__ s,
                        const int* __restrict__ tj, const T* __restrict__ W1,
                        const T* __restrict__ b1, const T* __restrict__ W2,
                        const T* __restrict__ b2, const T* __restrict__ W3,
                        const T* __restrict__ b3, T* __restrict__ h1, T* __restrict__ h2,
                        T* __restrict__ G) {
  constexpr int R = 8;
  extern __shared__ unsigned char sm_raw[];
  T* sh1 = reinterpret_cast<T*>(sm_raw);
  T* sh2 = sh1 + R * e1;
  __shared__ int st[R];
  __shared__ T ss[R];
  int p0 = blockIdx.x * R;
  if (threadIdx.x < R) {
    int p = p0 + threadIdx.x;
    st[threadIdx.x] = p < rows ? tj[p] : -1;
    ss[threadIdx.x] = p < rows ? s[p] : T(0);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < R * e1; idx += blockDim.x) {
    int r = idx / e1, k = idx % e1, t = st[r];
    T v = T(0);
    if (t >= 0) v = dtanh(ss[r] * W1[t * e1 + k] + b1[t * e1 + k]);
    sh1[idx] = v;
    if (p0 + r < rows) h1[(long long)(p0 + r) * e1 + k] = v;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < R * e2; idx += blockDim.x) {
    int r = idx / e2, f = idx % e2, t = st[r];
    T v = T(0);
    if (t >= 0) {
      T acc = b2[t * e2 + f];
      const T* w = W2 + (long long)t * e1 * e2;
      for (int k = 0; k < e1; ++k) acc += sh1[r * e1 + k] * w[k * e2 + f];
      v = dtanh(acc);
    }
    sh2[idx] = v;
    if (p0 + r < rows) h2[(long long)(p0 + r) * e2 + f] = v;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < R * m1; idx += blockDim.x) {
    int r = idx / m1, f = idx % m1, t = st[r];
    if (p0 + r >= rows) continue;
    T v = T(0);
    if (t >= 0) {
      T acc = b3[t * m1 + f];
      const T* w = W3 + (long long)t * e2 * m1;
      for (int k = 0; k < e2; ++k) acc += sh2[r * e2 + k] * w[k * m1 + f];
      v = dtanh(acc);
    }
    G[(long long)(p0 + r) * m1 + f] = v;
  }
}

// switch-weighted softmax and angular gate, one warp per (atom, head, row);
// S holds the scores on entry and A = w * gate on exit; P keeps e^S / Z
template <typename T>
__global__ void k_softmax(int na, int heads, int nmax, const T* __restrict__ sw,
                          const T* __restrict__ rh, const int* __restrict__ tj,
                          T* __restrict__ S, T* __restrict__ P) {
  long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  long long total = (long long)na * heads * nmax;
  if (wid >= total) return;
  int j = (int)(wid % nmax);
  long long ah = wid / nmax;
  int a = (int)(ah / heads);
  long long rowoff = ah * nmax * nmax + (long long)j * nmax;
  const T* swa = sw + (long long)a * nmax;
  const T* rha = rh + (long long)a * nmax * 3;
  bool rowvalid = tj[(long long)a * nmax + j] >= 0;
  T mx = T(-1e30);
  for (int k = lane; k < nmax; k += 32)
    if (tj[(long long)a * nmax + k] >= 0) mx = fmax(mx, S[rowoff + k]);
  mx = warp_max(mx);
  T z = T(0);
  for (int k = lane; k < nmax; k += 32)
    if (tj[(long long)a * nmax + k] >= 0) z += swa[k] * dexp(S[rowoff + k] - mx);
  z = warp_sum(z);
  T rhj[3] = {rha[3 * j], rha[3 * j + 1], rha[3 * j + 2]};
  for (int k = lane; k < nmax; k += 32) {
    T p = T(0), A = T(0);
    if (rowvalid && tj[(long long)a * nmax + k] >= 0 && z > T(0)) {
      p = dexp(S[rowoff + k] - mx) / z;
      T c = rhj[0] * rha[3 * k] + rhj[1] * rha[3 * k + 1] + rhj[2] * rha[3 * k + 2];
      A = swa[k] * p * c;
    }
    P[rowoff + k] = p;
    S[rowoff + k] = A;
  }
}

// residual + LayerNorm (gamma 1, beta 0, eps 1e-5), one warp per row
template <typename T>
__global__ void k_layernorm(int rows, int m1, const T* __restrict__ gin, const T* __restrict__ y,
                            const int* __restrict__ tj, T* __restrict__ gout,
                            T* __restrict__ rstd) {
  long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const T* gi = gin + row * m1;
  const T* yi = y + row * m1;
  T* go = gout + row * m1;
  if (tj[row] < 0) {
    for (int f = lane; f < m1; f += 32) go[f] = T(0);
    if (lane == 0) rstd[row] = T(0);
    return;
  }
  T sum = T(0);
  for (int f = lane; f < m1; f += 32) sum += gi[f] + yi[f];
  T mu = warp_sum(sum) / T(m1);
  T var = T(0);
  for (int f = lane; f < m1; f += 32) {
    T z = gi[f] + yi[f] - mu;
    var += z * z;
  }
  var = warp_sum(var) / T(m1);
  T rs = T(1) / dsqrt(var + T(1e-5));
  for (int f = lane; f < m1; f += 32) go[f] = (gi[f] + yi[f] - mu) * rs;
  if (lane == 0) rstd[row] = rs;
}

// descriptor: T = R~^T G / Nmax, D = T^T T[:, :m2]; one block per atom
template <typename T>
__global__ void k_descriptor(int nmax, int m1, int m2, const T* __restrict__ Rt,
                             const T* __restrict__ G, T* __restrict__ Tm, T* __restrict__ D) {
  extern __shared__ unsigned char sm_raw[];
  T* sT = reinterpret_cast<T*>(sm_raw);  // 4 x m1
  int a = blockIdx.x;
  const T* Ra = Rt + (long long)a * nmax * 4;
  const T* Ga = G + (long long)a * nmax * m1;
  T inv = T(1) / T(nmax);
  for (int f = threadIdx.x; f < m1; f += blockDim.x) {
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int j = 0; j < nmax; ++j) {
      T g = Ga[(long long)j * m1 + f];
      for (int q = 0; q < 4; ++q) acc[q] += Ra[4 * j + q] * g;
    }
    for (int q = 0; q < 4; ++q) {
      sT[q * m1 + f] = acc[q] * inv;
      Tm[(long long)a * 4 * m1 + q * m1 + f] = acc[q] * inv;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < m1 * m2; idx += blockDim.x) {
    int f = idx / m2, q = idx % m2;
    T v = T(0);
    for (int c = 0; c < 4; ++c) v += sT[c * m1 + f] * sT[c * m1 + q];
    D[(long long)a * m1 * m2 + idx] = v;
  }
}

// e_i = y3 . F4 + c4 in FP64, and delta3 = F4 * (1 - y3^2)
template <typename T>
__global__ void k_fit_out(int na, int f3, int atom0, const int* __restrict__ types,
                          const T* __restrict__ y3, const T* __restrict__ F4,
                          const T* __restrict__ c4, double* __restrict__ atom_e,
                          T* __restrict__ d3, const unsigned char* __restrict__ seed) {
  long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (wid >= na) return;
  int a = (int)wid;
  int t = types[atom0 + a];
  const T sd = seed && !seed[atom0 + a] ? T(0) : T(1);   // energy seed of the adjoint
  double acc = 0.0;
  for (int b = lane; b < f3; b += 32) {
    T y = y3[(long long)a * f3 + b];
    T w = F4[t * f3 + b];
    acc += (double)y * (double)w;
    d3[(long long)a * f3 + b] = sd * w * (T(1) - y * y);
  }
  acc = warp_sum(acc);
  if (lane == 0) atom_e[atom0 + a] = acc + (double)c4[t];
}

// energy only (further fitting heads): e_i = y3 . F4 + c4 in FP64
template <typename T>
__global__ void k_fit_energy(int na, int f3, int atom0, const int* __restrict__ types,
                             const T* __restrict__ y3, const T* __restrict__ F4,
                             const T* __restrict__ c4, double* __restrict__ atom_e) {
  long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (wid >= na) return;
  int a = (int)wid;
  int t = types[atom0 + a];
  double acc = 0.0;
  for (int b = lane; b < f3; b += 32) acc += (double)y3[(long long)a * f3 + b] * (double)F4[t * f3 + b];
  acc = warp_sum(acc);
  if (lane == 0) atom_e[atom0 + a] = acc + (double)c4[t];
}

// =========================================================================
// backward kernels
// =========================================================================
// dT from dD, then dR~ (4 per slot) and dG (m1 per slot); one block per atom
template <typename T>
__global__ void k_descriptor_bwd(int nmax, int m1, int m2, const T* __restrict__ Rt,
                                 const T* __restrict__ G, const T* __restrict__ Tm,
                                 const T* __restrict__ dD, T* __restrict__ dRt,
                                 T* __restrict__ dG) {
  extern __shared__ unsigned char sm_raw[];
  T* sT = reinterpret_cast<T*>(sm_raw);   // 4 x m1
  T* sdT = sT + 4 * m1;                   // 4 x m1
  int a = blockIdx.x;
  const T* dDa = dD + (long long)a * m1 * m2;
  for (int idx = threadIdx.x; idx < 4 * m1; idx += blockDim.x) sT[idx] = Tm[(long long)a * 4 * m1 + idx];
  __syncthreads();
  for (int idx = threadIdx.x; idx < 4 * m1; idx += blockDim.x) {
    int c = idx / m1, f = idx % m1;
    T v = T(0);
    for (int q = 0; q < m2; ++q) v += dDa[f * m2 + q] * sT[c * m1 + q];
    if (f < m2)
      for (int g = 0; g < m1; ++g) v += dDa[g * m2 + f] * sT[c * m1 + g];
    sdT[idx] = v;
  }
  __syncthreads();
  T inv = T(1) / T(nmax);
  const T* Ra = Rt + (long long)a * nmax * 4;
  const T* Ga = G + (long long)a * nmax * m1;
  for (int idx = threadIdx.x; idx < nmax * m1; idx += blockDim.x) {
    int j = idx / m1, f = idx % m1;
    T v = T(0);
    for (int c = 0; c < 4; ++c) v += sdT[c * m1 + f] * Ra[4 * j + c];
    dG[(long long)a * nmax * m1 + idx] = v * inv;
  }
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int jc = warp; jc < nmax * 4; jc += nw) {
    int j = jc >> 2, c = jc & 3;
    T v = T(0);
    for (int f = lane; f < m1; f += 32) v += sdT[c * m1 + f] * Ga[(long long)j * m1 + f];
    v = warp_sum(v);
    if (lane == 0) dRt[(long long)a * nmax * 4 + jc] = v * inv;
  }
}

// LayerNorm adjoint, one warp per row: dZ = rstd (dG - mean dG - Gout mean(dG Gout));
// writes dZ to both dz and dg (dg then accumulates the Q/K/V paths)
template <typename T>
__global__ void k_layernorm_bwd(int rows, int m1, const T* __restrict__ gout,
                                const T* __restrict__ rstd, const int* __restrict__ tj,
                                T* __restrict__ dg, T* __restrict__ dz) {
  long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (row >= rows) return;
  T* dgi = dg + row * m1;
  T* dzi = dz + row * m1;
  const T* go = gout + row * m1;
  if (tj[row] < 0) {
    for (int f = lane; f < m1; f += 32) {
      dgi[f] = T(0);
      dzi[f] = T(0);
    }
    return;
  }
  T s1 = T(0), s2 = T(0);
  for (int f = lane; f < m1; f += 32) {
    s1 += dgi[f];
    s2 += dgi[f] * go[f];
  }
  s1 = warp_sum(s1) / T(m1);
  s2 = warp_sum(s2) / T(m1);
  T rs = rstd[row];
  for (int f = lane; f < m1; f += 32) {
    T v = rs * (dgi[f] - s1 - go[f] * s2);
    dgi[f] = v;
    dzi[f] = v;
  }
}

// softmax + gate adjoint.  Block per atom, warp per row j, all heads.
// In:  dS holds dA = dO V^T;  P = e^S/Z.   Out: dS <- w (dw - sum w dw),
// S <- A = w * gate (for dV), dcg += dA * w (summed over heads), dsw += P rho.
template <typename T>
__global__ void k_softmax_bwd(int heads, int nmax, const T* __restrict__ sw,
                              const T* __restrict__ rh, const int* __restrict__ tj,
                              const T* __restrict__ P, T* __restrict__ S, T* __restrict__ dS,
                              T* __restrict__ dcg, T* __restrict__ dsw) {
  extern __shared__ unsigned char sm_raw[];
  T* sdsw = reinterpret_cast<T*>(sm_raw);  // warps x nmax partial sums
  int a = blockIdx.x;
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const T* swa = sw + (long long)a * nmax;
  const T* rha = rh + (long long)a * nmax * 3;
  const int* ta = tj + (long long)a * nmax;
  constexpr int KQ = 8;  // up to 256 neighbour slots
  T dsw_acc[KQ];
  for (int q = 0; q < KQ; ++q) dsw_acc[q] = T(0);
  for (int j = warp; j < nmax; j += nw) {
    if (ta[j] < 0) continue;
    T rhj[3] = {rha[3 * j], rha[3 * j + 1], rha[3 * j + 2]};
    T dc_acc[KQ];
    for (int q = 0; q < KQ; ++q) dc_acc[q] = T(0);
    for (int h = 0; h < heads; ++h) {
      long long off = ((long long)a * heads + h) * nmax * nmax + (long long)j * nmax;
      T wdw = T(0);
      T w_[KQ], dw_[KQ], dA_[KQ], p_[KQ];
      for (int q = 0; q < KQ; ++q) {
        int k = lane + 32 * q;
        w_[q] = dw_[q] = dA_[q] = p_[q] = T(0);
        if (k < nmax && ta[k] >= 0) {
          T c = rhj[0] * rha[3 * k] + rhj[1] * rha[3 * k + 1] + rhj[2] * rha[3 * k + 2];
          p_[q] = P[off + k];
          w_[q] = swa[k] * p_[q];
          dA_[q] = dS[off + k];
          dw_[q] = dA_[q] * c;
          wdw += w_[q] * dw_[q];
          S[off + k] = w_[q] * c;
        }
      }
      wdw = warp_sum(wdw);
      for (int q = 0; q < KQ; ++q) {
        int k = lane + 32 * q;
        if (k < nmax) {
          if (ta[k] >= 0) {
            T rho = dw_[q] - wdw;
            dS[off + k] = w_[q] * rho;
            dsw_acc[q] += p_[q] * rho;
            dc_acc[q] += dA_[q] * w_[q];
          } else {
            dS[off + k] = T(0);
            S[off + k] = T(0);
          }
        }
      }
    }
    for (int q = 0; q < KQ; ++q) {
      int k = lane + 32 * q;
      if (k < nmax) dcg[((long long)a * nmax + j) * nmax + k] += dc_acc[q];
    }
  }
  // rows of empty slots: zero their dS / A so the GEMMs below see zeros
  for (int j = warp; j < nmax; j += nw) {
    if (ta[j] >= 0) continue;
    for (int h = 0; h < heads; ++h) {
      long long off = ((long long)a * heads + h) * nmax * nmax + (long long)j * nmax;
      for (int k = lane; k < nmax; k += 32) {
        dS[off + k] = T(0);
        S[off + k] = T(0);
      }
    }
  }
  for (int q = 0; q < KQ; ++q) {
    int k = lane + 32 * q;
    if (k < nmax) sdsw[warp * nmax + k] = dsw_acc[q];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nmax; k += blockDim.x) {
    T v = T(0);
    for (int q = 0; q < nw; ++q) v += sdsw[q * nmax + k];
    dsw[(long long)a * nmax + k] += v;
  }
}

// embedding adjoint: ds per slot (one warp per slot)
template <typename T>
__global__ void k_embed_bwd(int rows, int e1, int e2, int m1, const int* __restrict__ tj,
                            const T* __restrict__ W1, const T* __restrict__ W2,
                            const T* __restrict__ W3, const T* __restrict__ h1,
                            const T* __restrict__ h2, const T* __restrict__ G0,
                            const T* __restrict__ dG, T* __restrict__ ds) {
  extern __shared__ unsigned char sm_raw[];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  T* buf = reinterpret_cast<T*>(sm_raw) + (size_t)warp * (m1 + e2);
  T* da3 = buf;
  T* da2 = buf + m1;
  long long p = (long long)blockIdx.x * nw + warp;
  if (p >= rows) return;
  int t = tj[p];
  if (t < 0) {
    if (lane == 0) ds[p] = T(0);
    return;
  }
  for (int f = lane; f < m1; f += 32) {
    T g = G0[p * m1 + f];
    da3[f] = dG[p * m1 + f] * (T(1) - g * g);
  }
  __syncwarp();
  const T* w3 = W3 + (long long)t * e2 * m1;
  for (int k = 0; k < e2; ++k) {
    T v = T(0);
    for (int f = lane; f < m1; f += 32) v += da3[f] * w3[k * m1 + f];
    v = warp_sum(v);
    if (lane == 0) {
      T h = h2[p * e2 + k];
      da2[k] = v * (T(1) - h * h);
    }
  }
  __syncwarp();
  const T* w2 = W2 + (long long)t * e1 * e2;
  T acc = T(0);
  for (int k = lane; k < e1; k += 32) {
    T v = T(0);
    for (int f = 0; f < e2; ++f) v += da2[f] * w2[k * e2 + f];
    T h = h1[p * e1 + k];
    acc += v * (T(1) - h * h) * W1[t * e1 + k];
  }
  acc = warp_sum(acc);
  if (lane == 0) ds[p] = acc;
}

// environment + gate adjoint -> g = dE/dr per slot (one warp per slot)
template <typename T>
__global__ void k_env_bwd(int rows, int nmax, int atom0, const T* __restrict__ d,
                          const T* __restrict__ sw, const T* __restrict__ dswdr,
                          const T* __restrict__ s, const T* __restrict__ rh,
                          const int* __restrict__ tj, const T* __restrict__ dRt,
                          const T* __restrict__ ds_emb, const T* __restrict__ dsw_att,
                          const T* __restrict__ dcg, T* __restrict__ g) {
  long long p = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (p >= rows) return;
  long long gp = (long long)atom0 * nmax + p;
  if (tj[p] < 0) {
    if (lane < 3) g[3 * gp + lane] = T(0);
    return;
  }
  long long a = p / nmax;
  int j = (int)(p % nmax);
  const T* rha = rh + a * nmax * 3;
  const T* dca = dcg + a * nmax * nmax;
  T dr[3] = {T(0), T(0), T(0)};
  for (int k = lane; k < nmax; k += 32) {
    T c = dca[(long long)j * nmax + k] + dca[(long long)k * nmax + j];
    for (int q = 0; q < 3; ++q) dr[q] += c * rha[3 * k + q];
  }
  for (int q = 0; q < 3; ++q) dr[q] = warp_sum(dr[q]);
  if (lane != 0) return;
  T rr[3] = {rh[3 * p], rh[3 * p + 1], rh[3 * p + 2]};
  T dd = d[p], sv = s[p];
  T dst = dRt[4 * p] + ds_emb[p];
  for (int q = 0; q < 3; ++q) {
    dst += dRt[4 * p + 1 + q] * rr[q];
    dr[q] += sv * dRt[4 * p + 1 + q];
  }
  T radial = dst * (dswdr[p] / dd - sw[p] / (dd * dd)) + dsw_att[p] * dswdr[p];
  T proj = dr[0] * rr[0] + dr[1] * rr[1] + dr[2] * rr[2];
  for (int q = 0; q < 3; ++q) g[3 * gp + q] = radial * rr[q] + (dr[q] - proj * rr[q]) / dd;
}

template <typename T>
__global__ void k_zero(long long n, T* __restrict__ p) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = T(0);
}

// =========================================================================
// message passing between atoms (atom channel h, width m1; one chunk holds
// every atom so that a layer finishes for all atoms before the next starts)
// =========================================================================
// G'_ip = G_ip + U_{j(p)} for kept slots; empty slots copy G (one warp per slot)
template <typename T>
__global__ void k_mp_add(long long rows, int m1, const int* __restrict__ sel_j,
                         const T* __restrict__ G, const T* __restrict__ U, T* __restrict__ Gp) {
  const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const int j = sel_j[row];
  const T* g = G + row * m1;
  T* o = Gp + row * m1;
  if (j < 0) {
    for (int f = lane; f < m1; f += 32) o[f] = g[f];
  } else {
    const T* u = U + (long long)j * m1;
    for (int f = lane; f < m1; f += 32) o[f] = g[f] + u[f];
  }
}

// h_i += (1/Nmax) sum_p sw_ip G_ip, slots in increasing order
template <typename T>
__global__ void k_mp_pool(int n, int nmax, int m1, T inv_nmax, const T* __restrict__ sw,
                          const T* __restrict__ G, T* __restrict__ h) {
  long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)n * m1) return;
  const long long i = q / m1;
  const int f = (int)(q % m1);
  T acc = T(0);
  for (int p = 0; p < nmax; ++p) acc += sw[i * nmax + p] * G[(i * nmax + p) * m1 + f];
  h[q] += acc * inv_nmax;
}

// adjoint of the pool for kept slots: dG_ip += (sw_ip / Nmax) dh_i and
// dE/dsw_ip += (1/Nmax) G_ip . dh_i (one warp per slot, fixed reduction tree)
template <typename T>
__global__ void k_mp_pool_bwd(long long rows, int nmax, int m1, T inv_nmax,
                              const int* __restrict__ sel_j, const T* __restrict__ sw,
                              const T* __restrict__ G, const T* __restrict__ dh, T* __restrict__ dG,
                              T* __restrict__ dsw) {
  const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= rows || sel_j[row] < 0) return;
  const long long i = row / nmax;
  const T sc = sw[row] * inv_nmax;
  T dot = T(0);
  for (int f = lane; f < m1; f += 32) {
    const T d = dh[i * m1 + f];
    dG[row * m1 + f] += sc * d;
    dot += G[row * m1 + f] * d;
  }
  for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
  if (lane == 0) dsw[row] += dot * inv_nmax;
}

// =========================================================================
// host side
// =========================================================================
template <typename T>
struct PlainAf {
  AfDims m;
  int n_atoms = 0, chunk = 0;
  // weights
  T *eW1, *eb1, *eW2, *eb2, *eW3, *eb3;  // species stacked
  std::vector<T*> Wqkv, Wo, bo;           // per layer; Wqkv is [m1][3H]
  std::vector<T*> F1, c1, F2, c2, F3, c3; // per head and species: [h * S + t]
  std::vector<T*> F4, c4;                 // per head, species stacked [S][f3], [S]
  double* head_e = nullptr;               // heads 1..: atomic energies [h - 1][n_atoms]
  // message passing: species rows of h^0, per layer Wm [m1][m1] and bm; atom
  // channel h, its adjoint dh, dq, per layer U = tanh(h Wm + bm), G' buffer
  T* Wt = nullptr;
  std::vector<T*> Wm, bm, U;
  T *hbuf = nullptr, *dh = nullptr, *dq = nullptr, *Gp = nullptr;
  const unsigned char* seed = nullptr;     // energy seed (device, optional)
  // per-chunk activations
  T *d, *sw, *dsw, *s, *Rt, *rh;
  int* tj;
  T *h1, *h2;
  std::vector<T*> G, QKV, Pm, rstd;
  T *O, *Zb, *SA, *SdA, *Tm, *D, *y1, *y2, *y3;
  T *dD, *dRt, *dG, *dZ, *dO, *dQKV, *dsw_att, *dcg, *ds, *d3, *d2, *d1;
  T* g;  // all atoms: n x nmax x 3
  // fitting row groups: per chunk, per species: local atom indices
  int* fit_rows;
  std::vector<std::vector<std::pair<int, int>>> fit_ranges;  // [chunk][species] -> (offset, count)
  std::vector<void*> allocs;
  size_t bytes = 0;
  int kernels_per_call = 0;

  template <typename U>
  cudaError_t alloc(U** p, size_t count) {
    size_t b = sizeof(U) * (count > 0 ? count : 1);
    cudaError_t e = cudaMalloc((void**)p, b);
    if (e == cudaSuccess) {
      allocs.push_back((void*)*p);
      bytes += b;
    }
    return e;
  }
  ~PlainAf() {
    for (void* p : allocs) cudaFree(p);
  }
};

template <typename T>
static cudaError_t upload(PlainAf<T>* P, T** dst, const std::vector<double>& src) {
  cudaError_t e = P->alloc(dst, src.size());
  if (e != cudaSuccess) return e;
  std::vector<T> tmp(src.begin(), src.end());
  return cudaMemcpy(*dst, tmp.data(), sizeof(T) * tmp.size(), cudaMemcpyHostToDevice);
}

template <typename T>
static void* create_impl(const AfDims& m, const double* w, int n_atoms, const int* types_host,
                         size_t mem_budget, std::string* err, size_t* bytes_out) {
  auto* P = new PlainAf<T>();
  P->m = m;
  P->n_atoms = n_atoms;
  const int S = m.n_species, L = m.n_layers, M1 = m.m1, M2 = m.m2, H = m.hidden;
  const int NH = m.heads, NM = m.nmax, E1 = m.e1, E2 = m.e2;
  // ---- weights: walk the blob in its documented order
  size_t off = 0;
  auto take = [&](size_t cnt) {
    std::vector<double> v(w + off, w + off + cnt);
    off += cnt;
    return v;
  };
  std::vector<double> eW1, eb1, eW2, eb2, eW3, eb3;
  for (int t = 0; t < S; ++t) {
    auto a = take(E1); eW1.insert(eW1.end(), a.begin(), a.end());
    a = take(E1); eb1.insert(eb1.end(), a.begin(), a.end());
    a = take((size_t)E1 * E2); eW2.insert(eW2.end(), a.begin(), a.end());
    a = take(E2); eb2.insert(eb2.end(), a.begin(), a.end());
    a = take((size_t)E2 * M1); eW3.insert(eW3.end(), a.begin(), a.end());
    a = take(M1); eb3.insert(eb3.end(), a.begin(), a.end());
  }
  cudaError_t e = cudaSuccess;
#define CK(x)                                                     \
  do {                                                            \
    e = (x);                                                      \
    if (e != cudaSuccess) {                                       \
      *err = std::string("plain model setup: ") + cudaGetErrorString(e); \
      delete P;                                                   \
      return nullptr;                                             \
    }                                                             \
  } while (0)
  CK(upload(P, &P->eW1, eW1)); CK(upload(P, &P->eb1, eb1));
  CK(upload(P, &P->eW2, eW2)); CK(upload(P, &P->eb2, eb2));
  CK(upload(P, &P->eW3, eW3)); CK(upload(P, &P->eb3, eb3));
  if (m.mp) CK(upload(P, &P->Wt, take((size_t)S * M1)));
  P->Wqkv.resize(L); P->Wo.resize(L); P->bo.resize(L);
  if (m.mp) { P->Wm.resize(L); P->bm.resize(L); P->U.resize(L); }
  for (int l = 0; l < L; ++l) {
    auto q = take((size_t)M1 * H), k = take((size_t)M1 * H), v = take((size_t)M1 * H);
    std::vector<double> qkv((size_t)M1 * 3 * H);
    for (int f = 0; f < M1; ++f)
      for (int c = 0; c < H; ++c) {
        qkv[(size_t)f * 3 * H + c] = q[(size_t)f * H + c];
        qkv[(size_t)f * 3 * H + H + c] = k[(size_t)f * H + c];
        qkv[(size_t)f * 3 * H + 2 * H + c] = v[(size_t)f * H + c];
      }
    CK(upload(P, &P->Wqkv[l], qkv));
    CK(upload(P, &P->Wo[l], take((size_t)H * M1)));
    CK(upload(P, &P->bo[l], take(M1)));
    if (m.mp) {
      CK(upload(P, &P->Wm[l], take((size_t)M1 * M1)));
      CK(upload(P, &P->bm[l], take(M1)));
    }
  }
  const int HF = m.fit_heads > 1 ? m.fit_heads : 1;
  P->F1.resize(HF * S); P->c1.resize(HF * S); P->F2.resize(HF * S); P->c2.resize(HF * S);
  P->F3.resize(HF * S); P->c3.resize(HF * S); P->F4.resize(HF); P->c4.resize(HF);
  for (int h = 0; h < HF; ++h) {      // fitting nets of head 0, 1, ... in blob order
    std::vector<double> F4, c4;
    for (int t = 0; t < S; ++t) {
      const int q = h * S + t;
      CK(upload(P, &P->F1[q], take((size_t)M1 * M2 * m.f1)));
      CK(upload(P, &P->c1[q], take(m.f1)));
      CK(upload(P, &P->F2[q], take((size_t)m.f1 * m.f2)));
      CK(upload(P, &P->c2[q], take(m.f2)));
      CK(upload(P, &P->F3[q], take((size_t)m.f2 * m.f3)));
      CK(upload(P, &P->c3[q], take(m.f3)));
      auto a = take(m.f3); F4.insert(F4.end(), a.begin(), a.end());
      a = take(1); c4.insert(c4.end(), a.begin(), a.end());
    }
    CK(upload(P, &P->F4[h], F4)); CK(upload(P, &P->c4[h], c4));
  }
  if (HF > 1) CK(P->alloc(&P->head_e, (size_t)(HF - 1) * n_atoms));

  // ---- chunk size from the activation footprint per atom
  size_t per_atom = sizeof(T) * ((size_t)NM * (4 + 4 + 3 + E1 + E2) + (size_t)(L + 1) * NM * M1 +
                                 (size_t)L * NM * 3 * H + (size_t)L * NH * NM * NM + (size_t)L * NM +
                                 (size_t)NM * (H + M1) + 2 * (size_t)NH * NM * NM + 4 * M1 +
                                 (size_t)M1 * M2 + 3 * (size_t)m.f1 + 3 * (size_t)m.f2 +
                                 2 * (size_t)m.f3 + (size_t)M1 * M2 + 4 * (size_t)NM +
                                 3 * (size_t)NM * M1 + (size_t)NM * H + (size_t)NM * 3 * H +
                                 (size_t)NM + (size_t)NM * NM + (size_t)NM) +
                      sizeof(int) * NM;
  size_t budget = mem_budget ? mem_budget : ((size_t)16 << 30);
  long long ch = (long long)(budget / per_atom);
  if (ch < 1) ch = 1;
  if (ch > n_atoms) ch = n_atoms;
  if (ch < 1) ch = 1;
  if (m.mp) ch = n_atoms;       // a layer needs every atom's previous layer
  int C = (int)ch;
  P->chunk = C;
  size_t rows = (size_t)C * NM;
  CK(P->alloc(&P->d, rows)); CK(P->alloc(&P->sw, rows)); CK(P->alloc(&P->dsw, rows));
  CK(P->alloc(&P->s, rows)); CK(P->alloc(&P->Rt, 4 * rows)); CK(P->alloc(&P->rh, 3 * rows));
  CK(P->alloc(&P->tj, rows));
  CK(P->alloc(&P->h1, rows * E1)); CK(P->alloc(&P->h2, rows * E2));
  P->G.resize(L + 1); P->QKV.resize(L); P->Pm.resize(L); P->rstd.resize(L);
  for (int l = 0; l <= L; ++l) CK(P->alloc(&P->G[l], rows * M1));
  for (int l = 0; l < L; ++l) {
    CK(P->alloc(&P->QKV[l], rows * 3 * H));
    CK(P->alloc(&P->Pm[l], (size_t)C * NH * NM * NM));
    CK(P->alloc(&P->rstd[l], rows));
  }
  CK(P->alloc(&P->O, rows * H)); CK(P->alloc(&P->Zb, rows * M1));
  CK(P->alloc(&P->SA, (size_t)C * NH * NM * NM)); CK(P->alloc(&P->SdA, (size_t)C * NH * NM * NM));
  CK(P->alloc(&P->Tm, (size_t)C * 4 * M1)); CK(P->alloc(&P->D, (size_t)C * M1 * M2));
  CK(P->alloc(&P->y1, (size_t)C * m.f1)); CK(P->alloc(&P->y2, (size_t)C * m.f2));
  CK(P->alloc(&P->y3, (size_t)C * m.f3));
  CK(P->alloc(&P->d1, (size_t)C * m.f1)); CK(P->alloc(&P->d2, (size_t)C * m.f2));
  CK(P->alloc(&P->d3, (size_t)C * m.f3));
  CK(P->alloc(&P->dD, (size_t)C * M1 * M2)); CK(P->alloc(&P->dRt, 4 * rows));
  CK(P->alloc(&P->dG, rows * M1)); CK(P->alloc(&P->dZ, rows * M1)); CK(P->alloc(&P->dO, rows * H));
  CK(P->alloc(&P->dQKV, rows * 3 * H)); CK(P->alloc(&P->dsw_att, rows));
  CK(P->alloc(&P->dcg, (size_t)C * NM * NM)); CK(P->alloc(&P->ds, rows));
  CK(P->alloc(&P->g, (size_t)n_atoms * NM * 3));
  if (m.mp) {
    const size_t na = (size_t)n_atoms * M1;
    CK(P->alloc(&P->hbuf, na)); CK(P->alloc(&P->dh, na)); CK(P->alloc(&P->dq, na));
    CK(P->alloc(&P->Gp, rows * M1));
    for (int l = 0; l < L; ++l) CK(P->alloc(&P->U[l], na));
  }
  // ---- fitting row groups (atoms of one species inside one chunk)
  int nch = (n_atoms + C - 1) / C;
  std::vector<int> rowsv;
  P->fit_ranges.assign(nch, std::vector<std::pair<int, int>>(S));
  for (int c = 0; c < nch; ++c) {
    int a0 = c * C, a1 = std::min(n_atoms, a0 + C);
    for (int t = 0; t < S; ++t) {
      int start = (int)rowsv.size();
      for (int a = a0; a < a1; ++a)
        if (types_host[a] == t) rowsv.push_back(a - a0);
      P->fit_ranges[c][t] = {start, (int)rowsv.size() - start};
    }
  }
  CK(P->alloc(&P->fit_rows, rowsv.size()));
  if (!rowsv.empty())
    CK(cudaMemcpy(P->fit_rows, rowsv.data(), sizeof(int) * rowsv.size(), cudaMemcpyHostToDevice));
#undef CK
  *bytes_out = P->bytes;
  return P;
}

template <typename T>
static int run_impl(PlainAf<T>* P, const NbrView& nv, const int* types, double* atom_e,
                    cudaStream_t st) {
  const int* sel_j = nv.sel_j;
  const double* sel_r = nv.sel_r;
  const AfDims& m = P->m;
  const int S = m.n_species, L = m.n_layers, M1 = m.m1, M2 = m.m2, H = m.hidden;
  const int NH = m.heads, NM = m.nmax, E1 = m.e1, E2 = m.e2, DH = H / NH;
  const T inv_sqrt_d = T(1) / (T)sqrt((double)DH);
  int launches = 0;
  for (int c = 0, a0 = 0; a0 < P->n_atoms; ++c, a0 += P->chunk) {
    int na = std::min(P->chunk, P->n_atoms - a0);
    int rows = na * NM;
    // ---------------- forward
    k_env<T><<<ceil_div(rows, 128), 128, 0, st>>>(rows, NM, a0, sel_j, sel_r, types, (T)m.rs,
                                                  (T)m.rc, P->d, P->sw, P->dsw, P->s, P->Rt,
                                                  P->rh, P->tj);
    k_embed<T><<<ceil_div(rows, 8), 128, sizeof(T) * 8 * (E1 + E2), st>>>(
        rows, E1, E2, M1, P->s, P->tj, P->eW1, P->eb1, P->eW2, P->eb2, P->eW3, P->eb3, P->h1,
        P->h2, P->G[0]);
    launches += 2;
    const T inv_nm = T(1) / (T)NM;
    const long long nm1 = (long long)na * M1;
    if (m.mp) {
      k_mp_init<T><<<ceil_div(nm1, 256), 256, 0, st>>>(na, M1, types, P->Wt, P->hbuf);
      launches += 1;
    }
    for (int l = 0; l < L; ++l) {
      T* QKV = P->QKV[l];
      const T* gin = P->G[l];
      if (m.mp) {   // U = tanh(h Wm + bm); G' = G + U of each slot's neighbour
        Gemm<T> g = gemm_rowmajor<T>(na, M1, M1, P->hbuf, M1, P->Wm[l], M1, P->U[l], M1);
        g.bias = P->bm[l];
        g.epi = 1;
        gemm(g, 1, st);
        k_mp_add<T><<<ceil_div((long long)rows * 32, 256), 256, 0, st>>>(
            rows, M1, sel_j + (long long)a0 * NM, P->G[l], P->U[l], P->Gp);
        gin = P->Gp;
        launches += 2;
      }
      gemm(gemm_rowmajor<T>(rows, 3 * H, M1, gin, M1, P->Wqkv[l], 3 * H, QKV, 3 * H), 1, st);
      {  // S = Q K^T / sqrt(d), per (atom, head)
        Gemm<T> g{};
        g.M = NM; g.N = NM; g.K = DH;
        g.A = QKV; g.a_rm = 3 * H; g.a_rk = 1; g.a_b1 = (long long)NM * 3 * H; g.a_b2 = DH;
        g.B = QKV + H; g.b_rk = 1; g.b_rn = 3 * H; g.b_b1 = (long long)NM * 3 * H; g.b_b2 = DH;
        g.C = P->SA; g.c_rm = NM; g.c_rn = 1; g.c_b1 = (long long)NH * NM * NM; g.c_b2 = (long long)NM * NM;
        g.nb2 = NH; g.alpha = inv_sqrt_d; g.beta = T(0);
        gemm(g, (long long)na * NH, st);
      }
      k_softmax<T><<<ceil_div((long long)na * NH * NM * 32, 256), 256, 0, st>>>(
          na, NH, NM, P->sw, P->rh, P->tj, P->SA, P->Pm[l]);
      {  // O = A V
        Gemm<T> g{};
        g.M = NM; g.N = DH; g.K = NM;
        g.A = P->SA; g.a_rm = NM; g.a_rk = 1; g.a_b1 = (long long)NH * NM * NM; g.a_b2 = (long long)NM * NM;
        g.B = QKV + 2 * H; g.b_rk = 3 * H; g.b_rn = 1; g.b_b1 = (long long)NM * 3 * H; g.b_b2 = DH;
        g.C = P->O; g.c_rm = H; g.c_rn = 1; g.c_b1 = (long long)NM * H; g.c_b2 = DH;
        g.nb2 = NH; g.alpha = T(1); g.beta = T(0);
        gemm(g, (long long)na * NH, st);
      }
      {
        Gemm<T> g = gemm_rowmajor<T>(rows, M1, H, P->O, H, P->Wo[l], M1, P->Zb, M1);
        g.bias = P->bo[l];
        gemm(g, 1, st);
      }
      k_layernorm<T><<<ceil_div((long long)rows * 32, 256), 256, 0, st>>>(
          rows, M1, gin, P->Zb, P->tj, P->G[l + 1], P->rstd[l]);
      launches += 6;
      if (m.mp && l + 1 < L) {   // h += (1/Nmax) sum_p sw_p G^{l+1}_p
        k_mp_pool<T><<<ceil_div(nm1, 256), 256, 0, st>>>(na, NM, M1, inv_nm, P->sw, P->G[l + 1],
                                                         P->hbuf);
        launches += 1;
      }
    }
    k_descriptor<T><<<na, 128, sizeof(T) * 4 * M1, st>>>(NM, M1, M2, P->Rt, P->G[L], P->Tm, P->D);
    launches += 1;
    for (int t = 0; t < S; ++t) {
      auto rg = P->fit_ranges[c][t];
      if (rg.second == 0) continue;
      const int* rws = P->fit_rows + rg.first;
      Gemm<T> g = gemm_rowmajor<T>(rg.second, m.f1, M1 * M2, P->D, M1 * M2, P->F1[t], m.f1, P->y1, m.f1);
      g.a_rows = rws; g.c_rows = rws; g.bias = P->c1[t]; g.epi = 1;
      gemm(g, 1, st);
      g = gemm_rowmajor<T>(rg.second, m.f2, m.f1, P->y1, m.f1, P->F2[t], m.f2, P->y2, m.f2);
      g.a_rows = rws; g.c_rows = rws; g.bias = P->c2[t]; g.epi = 1;
      gemm(g, 1, st);
      g = gemm_rowmajor<T>(rg.second, m.f3, m.f2, P->y2, m.f2, P->F3[t], m.f3, P->y3, m.f3);
      g.a_rows = rws; g.c_rows = rws; g.bias = P->c3[t]; g.epi = 1;
      gemm(g, 1, st);
      launches += 3;
    }
    k_fit_out<T><<<ceil_div((long long)na * 32, 256), 256, 0, st>>>(na, m.f3, a0, types, P->y3,
                                                                     P->F4[0], P->c4[0], atom_e, P->d3, P->seed);
    launches += 1;
    // ---------------- backward
    for (int t = 0; t < S; ++t) {
      auto rg = P->fit_ranges[c][t];
      if (rg.second == 0) continue;
      const int* rws = P->fit_rows + rg.first;
      // d2 = (d3 F3^T) * (1 - y2^2)
      Gemm<T> g{};
      g.M = rg.second; g.N = m.f2; g.K = m.f3;
      g.A = P->d3; g.a_rm = m.f3; g.a_rk = 1;
      g.B = P->F3[t]; g.b_rk = 1; g.b_rn = m.f3;
      g.C = P->d2; g.c_rm = m.f2; g.c_rn = 1; g.nb2 = 1;
      g.a_rows = rws; g.c_rows = rws; g.alpha = T(1); g.epi = 2; g.aux = P->y2;
      gemm(g, 1, st);
      g.N = m.f1; g.K = m.f2;
      g.A = P->d2; g.a_rm = m.f2;
      g.B = P->F2[t]; g.b_rn = m.f2;
      g.C = P->d1; g.c_rm = m.f1; g.aux = P->y1;
      gemm(g, 1, st);
      g.N = M1 * M2; g.K = m.f1;
      g.A = P->d1; g.a_rm = m.f1;
      g.B = P->F1[t]; g.b_rn = m.f1;
      g.C = P->dD; g.c_rm = M1 * M2; g.epi = 0; g.aux = nullptr;
      gemm(g, 1, st);
      launches += 3;
    }
    k_descriptor_bwd<T><<<na, 256, sizeof(T) * 8 * M1, st>>>(NM, M1, M2, P->Rt, P->G[L], P->Tm,
                                                            P->dD, P->dRt, P->dG);
    k_zero<T><<<ceil_div((long long)na * NM * NM, 256), 256, 0, st>>>((long long)na * NM * NM, P->dcg);
    k_zero<T><<<ceil_div(rows, 256), 256, 0, st>>>(rows, P->dsw_att);
    launches += 3;
    if (m.mp) {
      k_zero<T><<<ceil_div(nm1, 256), 256, 0, st>>>(nm1, P->dh);
      launches += 1;
    }
    for (int l = L - 1; l >= 0; --l) {
      T* QKV = P->QKV[l];
      if (m.mp && l + 1 < L) {   // adjoint of h^{l+1} = h^l + pool(G^{l+1})
        k_mp_pool_bwd<T><<<ceil_div((long long)rows * 32, 256), 256, 0, st>>>(
            rows, NM, M1, inv_nm, sel_j + (long long)a0 * NM, P->sw, P->G[l + 1], P->dh, P->dG,
            P->dsw_att);
        launches += 1;
      }
      k_layernorm_bwd<T><<<ceil_div((long long)rows * 32, 256), 256, 0, st>>>(
          rows, M1, P->G[l + 1], P->rstd[l], P->tj, P->dG, P->dZ);
      {  // dO = dZ Wo^T
        Gemm<T> g{};
        g.M = rows; g.N = H; g.K = M1;
        g.A = P->dZ; g.a_rm = M1; g.a_rk = 1;
        g.B = P->Wo[l]; g.b_rk = 1; g.b_rn = M1;
        g.C = P->dO; g.c_rm = H; g.c_rn = 1; g.nb2 = 1; g.alpha = T(1);
        gemm(g, 1, st);
      }
      {  // dA = dO_h V_h^T
        Gemm<T> g{};
        g.M = NM; g.N = NM; g.K = DH;
        g.A = P->dO; g.a_rm = H; g.a_rk = 1; g.a_b1 = (long long)NM * H; g.a_b2 = DH;
        g.B = QKV + 2 * H; g.b_rk = 1; g.b_rn = 3 * H; g.b_b1 = (long long)NM * 3 * H; g.b_b2 = DH;
        g.C = P->SdA; g.c_rm = NM; g.c_rn = 1; g.c_b1 = (long long)NH * NM * NM; g.c_b2 = (long long)NM * NM;
        g.nb2 = NH; g.alpha = T(1);
        gemm(g, (long long)na * NH, st);
      }
      k_softmax_bwd<T><<<na, 256, sizeof(T) * 8 * NM, st>>>(NH, NM, P->sw, P->rh, P->tj, P->Pm[l],
                                                         P->SA, P->SdA, P->dcg, P->dsw_att);
      {  // dV = A^T dO_h
        Gemm<T> g{};
        g.M = NM; g.N = DH; g.K = NM;
        g.A = P->SA; g.a_rm = 1; g.a_rk = NM; g.a_b1 = (long long)NH * NM * NM; g.a_b2 = (long long)NM * NM;
        g.B = P->dO; g.b_rk = H; g.b_rn = 1; g.b_b1 = (long long)NM * H; g.b_b2 = DH;
        g.C = P->dQKV + 2 * H; g.c_rm = 3 * H; g.c_rn = 1; g.c_b1 = (long long)NM * 3 * H; g.c_b2 = DH;
        g.nb2 = NH; g.alpha = T(1);
        gemm(g, (long long)na * NH, st);
      }
      {  // dQ = dS K_h / sqrt(d)
        Gemm<T> g{};
        g.M = NM; g.N = DH; g.K = NM;
        g.A = P->SdA; g.a_rm = NM; g.a_rk = 1; g.a_b1 = (long long)NH * NM * NM; g.a_b2 = (long long)NM * NM;
        g.B = QKV + H; g.b_rk = 3 * H; g.b_rn = 1; g.b_b1 = (long long)NM * 3 * H; g.b_b2 = DH;
        g.C = P->dQKV; g.c_rm = 3 * H; g.c_rn = 1; g.c_b1 = (long long)NM * 3 * H; g.c_b2 = DH;
        g.nb2 = NH; g.alpha = inv_sqrt_d;
        gemm(g, (long long)na * NH, st);
      }
      {  // dK = dS^T Q_h / sqrt(d)
        Gemm<T> g{};
        g.M = NM; g.N = DH; g.K = NM;
        g.A = P->SdA; g.a_rm = 1; g.a_rk = NM; g.a_b1 = (long long)NH * NM * NM; g.a_b2 = (long long)NM * NM;
        g.B = QKV; g.b_rk = 3 * H; g.b_rn = 1; g.b_b1 = (long long)NM * 3 * H; g.b_b2 = DH;
        g.C = P->dQKV + H; g.c_rm = 3 * H; g.c_rn = 1; g.c_b1 = (long long)NM * 3 * H; g.c_b2 = DH;
        g.nb2 = NH; g.alpha = inv_sqrt_d;
        gemm(g, (long long)na * NH, st);
      }
      {  // dG = dZ + dQKV Wqkv^T
        Gemm<T> g{};
        g.M = rows; g.N = M1; g.K = 3 * H;
        g.A = P->dQKV; g.a_rm = 3 * H; g.a_rk = 1;
        g.B = P->Wqkv[l]; g.b_rk = 1; g.b_rn = 3 * H;
        g.C = P->dG; g.c_rm = M1; g.c_rn = 1; g.nb2 = 1; g.alpha = T(1); g.beta = T(1);
        gemm(g, 1, st);
      }
      launches += 8;
      if (m.mp) {   // G' = G + U_{j(p)}: dh^l += ((sum of dG' naming j) (1 - U^2)) Wm^T
        int warps = 4;
        while (warps > 1 && sizeof(int) * 2 * nv.cap * warps > 48 * 1024) --warps;
        k_mp_gather<T><<<ceil_div(na, warps), warps * 32, sizeof(int) * 2 * nv.cap * warps, st>>>(
            na, NM, NM, M1, nv.cap, nv.skin, nv.skin_cnt, nv.mirror, nv.selpos, P->dG, P->U[l], P->dq);
        Gemm<T> g{};
        g.M = na; g.N = M1; g.K = M1;
        g.A = P->dq; g.a_rm = M1; g.a_rk = 1;
        g.B = P->Wm[l]; g.b_rk = 1; g.b_rn = M1;
        g.C = P->dh; g.c_rm = M1; g.c_rn = 1; g.nb2 = 1; g.alpha = T(1); g.beta = T(1);
        gemm(g, 1, st);
        launches += 2;
      }
    }
    {
      const int warps = 4;
      size_t sm = sizeof(T) * warps * (M1 + E2);
      k_embed_bwd<T><<<ceil_div(rows, warps), warps * 32, sm, st>>>(
          rows, E1, E2, M1, P->tj, P->eW1, P->eW2, P->eW3, P->h1, P->h2, P->G[0], P->dG, P->ds);
    }
    k_env_bwd<T><<<ceil_div((long long)rows * 32, 256), 256, 0, st>>>(
        rows, NM, a0, P->d, P->sw, P->dsw, P->s, P->rh, P->tj, P->dRt, P->ds, P->dsw_att, P->dcg,
        P->g);
    launches += 2;
    // further fitting heads on the same descriptor: energies only
    for (int h = 1; h < (int)P->F4.size(); ++h) {
      for (int t = 0; t < S; ++t) {
        auto rg = P->fit_ranges[c][t];
        if (rg.second == 0) continue;
        const int* rws = P->fit_rows + rg.first;
        const int q = h * S + t;
        Gemm<T> g = gemm_rowmajor<T>(rg.second, m.f1, M1 * M2, P->D, M1 * M2, P->F1[q], m.f1, P->y1, m.f1);
        g.a_rows = rws; g.c_rows = rws; g.bias = P->c1[q]; g.epi = 1;
        gemm(g, 1, st);
        g = gemm_rowmajor<T>(rg.second, m.f2, m.f1, P->y1, m.f1, P->F2[q], m.f2, P->y2, m.f2);
        g.a_rows = rws; g.c_rows = rws; g.bias = P->c2[q]; g.epi = 1;
        gemm(g, 1, st);
        g = gemm_rowmajor<T>(rg.second, m.f3, m.f2, P->y2, m.f2, P->F3[q], m.f3, P->y3, m.f3);
        g.a_rows = rws; g.c_rows = rws; g.bias = P->c3[q]; g.epi = 1;
        gemm(g, 1, st);
        launches += 3;
      }
      k_fit_energy<T><<<ceil_div((long long)na * 32, 256), 256, 0, st>>>(
          na, m.f3, a0, types, P->y3, P->F4[h], P->c4[h], P->head_e + (size_t)(h - 1) * P->n_atoms);
      launches += 1;
    }
  }
  P->kernels_per_call = launches;
  return 0;
}

// ------------------------------------------------------------------ Model
template <typename T>
class PlainAfModel : public Model {
 public:
  explicit PlainAfModel(PlainAf<T>* p) : p_(p) {}
  ~PlainAfModel() override { delete p_; }
  int run(const NbrView& nv, const int* types, double* atom_e, cudaStream_t st) override {
    run_impl(p_, nv, types, atom_e, st);
    return p_->kernels_per_call;
  }
  const float* grad32() const override { return grad_as<float>(); }
  const double* grad64() const override { return grad_as<double>(); }
  const double* head_energies() const override { return p_->head_e; }
  bool set_energy_seed(const unsigned char* seed) override {
    p_->seed = seed;
    return true;
  }
  size_t bytes() const override { return p_->bytes; }

 private:
  template <typename U>
  const U* grad_as() const {
    if constexpr (std::is_same<T, U>::value) return p_->g;
    else return nullptr;
  }
  PlainAf<T>* p_;
};

Model* make_plain_af(const AfDims& m, bool f64, const double* weights, int n_atoms,
                     const int* types_host, size_t mem_budget, std::string* err) {
  if (m.nmax > 256) {
    *err = "plain attention model supports nmax <= 256";
    return nullptr;
  }
  size_t bytes = 0;
  if (f64) {
    auto* p = (PlainAf<double>*)create_impl<double>(m, weights, n_atoms, types_host, mem_budget, err, &bytes);
    return p ? new PlainAfModel<double>(p) : nullptr;
  }
  auto* p = (PlainAf<float>*)create_impl<float>(m, weights, n_atoms, types_host, mem_budget, err, &bytes);
  return p ? new PlainAfModel<float>(p) : nullptr;
}

}  // namespace dp
