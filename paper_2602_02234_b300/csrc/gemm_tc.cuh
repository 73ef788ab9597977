// Tensor-core GEMM over FP32-stored operands (16-bit products, FP16 or BF16,
// FP32 accumulation), used by the graph family's mixed-precision form.
#pragma once

#include <stdint.h>

#include <string>

#include <cuda_runtime.h>

namespace dp {

// C(m, n) = sum_k A(m, k) B(k, n) [+ bias(n)] [+ beta C(m, n)], then epi:
// 0 none, 1 tanh, 2 times (1 - aux(m, n)^2) with aux laid out like C, or
// 3 the graph family's edge update for row m = slot (i, p) of atom i = m / nmax
// with neighbour j = sel_j[m]: v = tanh(Ai(i, n) + Bj(j, n) + acc + bias(n)),
// v_out(m, n) = v and C(m, n) = e_in(m, n) + v (both 0 for an empty slot);
// Ai, Bj, e_in, v_out laid out like C, c_rows and beta unused; or 4 the angle
// channel's output: C(m, n) = t = tanh(acc + bias(n)) and
// v_out(x, n) = e_in(x, n) + sa[x] t at row x = x_rows ? x_rows[m] : row'(m)
// (e_in, v_out with C's ldc; e_in may equal v_out); or 5, below.
//   A(m, k) = A[row(m) * lda + k], row(m) = a_rows ? a_rows[m] : m; A 16-byte
//             aligned, lda a multiple of 4
//   B(k, n) = B[k * ldb + n]  (b_nk = 0)  or  B[n * ldb + k]  (b_nk = 1)
//   C(m, n) = C[row'(m) * ldc + n], row'(m) = c_rows ? c_rows[m] : m; C, aux,
//             bias (and Ai, Bj, e_in, v_out) 16-byte aligned, ldc a multiple of
//             4 (the epilogue moves float4s)
// N and K multiples of 16, at most 256.  A timed-out wait sets kFlagTimeout
// in *status.
struct GemmTc {
  int M, N, K;
  const float* A;
  long long lda;
  const int* a_rows;
  const float* B;
  long long ldb;
  int b_nk;
  float* C;
  long long ldc;
  const int* c_rows;
  const float* bias;
  float beta;
  int epi;
  const float* aux;
  int fp16;        // operands rounded to FP16 (1) or BF16 (0)
  int split;       // 1: A as a 16-bit high part plus a 16-bit remainder, two
                   // products per K step (A's rounding error ~2^-22 instead of 2^-11)
  int* status;
  // epi 3 and 4
  const int* sel_j;
  int nmax;
  const float *Ai, *Bj, *e_in, *sa;
  float* v_out;
  const int* x_rows;   // epi 4: row of e_in, v_out and sa for m (optional)
  // epi 5 (the graph family's edge adjoint with the message's, C = de, beta 1):
  // for row m = slot (i, p), i = m / nmax, j = sel_j[m]: C += acc, and on kept
  // slots C += f g_i u_j, x_out = f g_i e_in, dsw[m] += inv_nmax sum_n g_i e_in
  // u_j with f = inv_nmax sw[m] and g_i row i of dm (stride lddm); u, e_in,
  // x_out laid out like C
  const float *sw, *dm, *u;
  long long lddm;
  float *x_out, *dsw;
  float inv_nmax;
  // 16-bit storage in the operand type (FP16, or BF16 when fp16 = 0) instead
  // of FP32, where set: A (a16, lda in elements, a multiple of 8, 16-byte
  // aligned rows; no split), epi 3's v_out (v16) and epi 5's x_out (x16),
  // both laid out like C
  const uint16_t* a16;
  uint16_t *v16, *x16;
  // the edge state in 16 bits (the operand type), where set: e16 replaces
  // e_in (epi 3, 4, 5), and o16 receives epi 3's C (e1, C itself unused) or
  // epi 4's v_out (e_{l+1}; o16 may equal e16), all laid out like C
  const uint16_t* e16;
  uint16_t* o16;
};

bool gemm_tc_shape_ok(int N, int K);
// once per process (device attributes, shared-memory limit)
bool gemm_tc_prepare(std::string* err);
void gemm_tc(const GemmTc& g, cudaStream_t st);

}  // namespace dp
