/*
 * FP64 CPU oracle of the attention family with cross-atom message passing --
 * TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's
 * CPU-baseline leg).  Plain loops in double precision; every stage runs over
 * all atoms before the next starts (OpenMP over atoms inside a stage).
 *
 * The paper (Sec. II) names DPA2's "repformer" layers, and Sec. III states
 * that DPA2 needs the atoms within L x rc of a subdomain, i.e. its L layers
 * pass information between neighbouring atoms; it prints no formula.  The
 * reading computed here adds an atom channel to the attention family of
 * af_oracle.c (same environment, embedding, attention layer, descriptor and
 * fitting, same neighbour lists):
 *
 *   atom channel (width M1):  h^0_i = Wt[t_i]
 *   layer l = 0 .. L-1, every atom before any atom's layer l+1:
 *     U_j      = tanh(h^l_j Wm_l + bm_l)
 *     G'_ip    = G^l_ip + U_{j(p)}                 (each kept neighbour slot p)
 *     G^{l+1}_i = attention layer l of the base model applied to G'_i
 *     h^{l+1}_i = h^l_i + (1/Nmax) sum_p sw_ip G^{l+1}_ip     (only l+1 < L)
 *   descriptor and fitting from G^L as in the base model; E = sum_i e_i.
 *
 * h^l_j depends on the atoms within l neighbour hops of j, so e_i depends on
 * the atoms within L hops of i: the L x rc halo.  With Wm = 0 and bm = 0 the
 * model is the base model exactly (U = 0).
 *
 * Gradient by hand in reverse order: the attention layer's adjoint is the
 * base model's; the message adds dU_j = sum over slots (i, p) naming j of
 * dG'_ip, then dh^l_j += (dU_j * (1 - U_j^2)) Wm_l^T; the atom-channel update
 * adds (sw_ip / Nmax) dh^{l+1}_i to dG^{l+1}_ip and (1/Nmax) G^{l+1}_ip . dh^{l+1}_i
 * to dE/dsw_ip.  Forces and virial from g_ip = dE/dr_ip as in the base model.
 *
 * Weight blob (row-major W[in][out], W before b):
 *    for t < S: embedding W1[1][e1] b1 W2[e1][e2] b2 W3[e2][M1] b3
 *    Wt[S][M1]
 *    for l < L: Wq[M1][H] Wk[M1][H] Wv[M1][H] Wo[H][M1] bo[M1] Wm[M1][M1] bm[M1]
 *    for t < S: fitting W1[M1*M2][f1] b1 W2[f1][f2] b2 W3[f2][f3] b3 W4[f3][1] b4[1]
 */
#include "oracle_common.h"

#ifdef _OPENMP
#include <omp.h>
#endif

#define AMP_MAXS 16
#define AMP_MAXL 16

typedef struct {
  int n_species, e1, e2, m1, m2, n_layers, hidden, heads, f1, f2, f3, nmax;
  double rc, rs;
} amp_model;

typedef struct {
  const double *eW1[AMP_MAXS], *eb1[AMP_MAXS], *eW2[AMP_MAXS], *eb2[AMP_MAXS], *eW3[AMP_MAXS],
      *eb3[AMP_MAXS];
  const double* Wt;
  const double *Wq[AMP_MAXL], *Wk[AMP_MAXL], *Wv[AMP_MAXL], *Wo[AMP_MAXL], *bo[AMP_MAXL],
      *Wm[AMP_MAXL], *bm[AMP_MAXL];
  const double *fW1[AMP_MAXS], *fb1[AMP_MAXS], *fW2[AMP_MAXS], *fb2[AMP_MAXS], *fW3[AMP_MAXS],
      *fb3[AMP_MAXS], *fW4[AMP_MAXS], *fb4[AMP_MAXS];
} amp_weights;

static void amp_model_from(const int32_t* i, const double* f, amp_model* m) {
  m->n_species = i[0];
  m->e1 = i[1];
  m->e2 = i[2];
  m->m1 = i[3];
  m->m2 = i[4];
  m->n_layers = i[5];
  m->hidden = i[6];
  m->heads = i[7];
  m->f1 = i[8];
  m->f2 = i[9];
  m->f3 = i[10];
  m->nmax = i[11];
  m->rc = f[0];
  m->rs = f[1];
}

static int amp_check(const amp_model* m) {
  if (m->n_species < 1 || m->n_species > AMP_MAXS) return -1;
  if (m->n_layers < 0 || m->n_layers > AMP_MAXL) return -1;
  if (m->heads < 1 || m->hidden % m->heads) return -1;
  if (m->m2 > m->m1 || m->nmax < 1) return -1;
  if (!(m->rs < m->rc)) return -1;
  return 0;
}

/* Walks the blob in its documented order; with W == NULL only counts. */
static size_t amp_bind(const amp_model* m, const double* base, amp_weights* W) {
  size_t off = 0;
  const int S = m->n_species, M1 = m->m1, H = m->hidden;
#define TAKE(dst, cnt)                       \
  do {                                       \
    if (W) (dst) = base + off;               \
    off += (size_t)(cnt);                    \
  } while (0)
  amp_weights dummy;
  if (!W) W = &dummy, base = NULL;
  for (int t = 0; t < S; ++t) {
    TAKE(W->eW1[t], m->e1);
    TAKE(W->eb1[t], m->e1);
    TAKE(W->eW2[t], m->e1 * m->e2);
    TAKE(W->eb2[t], m->e2);
    TAKE(W->eW3[t], m->e2 * M1);
    TAKE(W->eb3[t], M1);
  }
  TAKE(W->Wt, S * M1);
  for (int l = 0; l < m->n_layers; ++l) {
    TAKE(W->Wq[l], M1 * H);
    TAKE(W->Wk[l], M1 * H);
    TAKE(W->Wv[l], M1 * H);
    TAKE(W->Wo[l], H * M1);
    TAKE(W->bo[l], M1);
    TAKE(W->Wm[l], M1 * M1);
    TAKE(W->bm[l], M1);
  }
  for (int t = 0; t < S; ++t) {
    TAKE(W->fW1[t], (size_t)M1 * m->m2 * m->f1);
    TAKE(W->fb1[t], m->f1);
    TAKE(W->fW2[t], m->f1 * m->f2);
    TAKE(W->fb2[t], m->f2);
    TAKE(W->fW3[t], m->f2 * m->f3);
    TAKE(W->fb3[t], m->f3);
    TAKE(W->fW4[t], m->f3);
    TAKE(W->fb4[t], 1);
  }
#undef TAKE
  return off;
}

long long oracle_afmp_weight_count(const int32_t* idims, const double* fdims) {
  amp_model m;
  amp_model_from(idims, fdims, &m);
  if (amp_check(&m)) return -1;
  return (long long)amp_bind(&m, NULL, NULL);
}

/* Offset of Wt (kind 0, a ignored), Wm of layer a (kind 1) or bm of layer a
 * (kind 2), for tests that set or clear the message weights. */
long long oracle_afmp_weight_offset(const int32_t* idims, const double* fdims, int kind, int a) {
  amp_model m;
  amp_model_from(idims, fdims, &m);
  if (amp_check(&m)) return -1;
  const long long S = m.n_species, M1 = m.m1, H = m.hidden, E1 = m.e1, E2 = m.e2;
  const long long wt = S * (E1 + E1 + E1 * E2 + E2 + E2 * M1 + M1);
  const long long layer = 3 * M1 * H + H * M1 + M1 + M1 * M1 + M1;
  if (kind == 0) return wt;
  if (a < 0 || a >= m.n_layers) return -1;
  const long long wm = wt + S * M1 + a * layer + 3 * M1 * H + H * M1 + M1;
  if (kind == 1) return wm;
  if (kind == 2) return wm + M1 * M1;
  return -1;
}

/* Everything one centre atom keeps between the stages. */
typedef struct {
  int nn;
  onbr* v;
  double *d, *sw, *dsw, *s, *Rt, *rh, *cg;
  double *h1, *h2;
  double** G;                                  /* L + 1 arrays of nn x M1 */
  double **Q, **K, **V, **P, **Wa, **rstd;     /* per layer */
  double* Gin;                                 /* G' of the current layer */
  double *dG, *dRt, *dsw_att, *dcg;
  double e;
} amp_atom;

static double* z_alloc(size_t n) { return (double*)calloc(n > 0 ? n : 1, sizeof(double)); }

static void amp_env_embed(const amp_model* m, const amp_weights* W, const int32_t* types,
                          amp_atom* a) {
  const int R = a->nn > 0 ? a->nn : 1, M1 = m->m1, E1 = m->e1, E2 = m->e2, L = m->n_layers;
  a->d = z_alloc(R); a->sw = z_alloc(R); a->dsw = z_alloc(R); a->s = z_alloc(R);
  a->Rt = z_alloc(4 * R); a->rh = z_alloc(3 * R); a->cg = z_alloc((size_t)R * R);
  a->h1 = z_alloc((size_t)R * E1); a->h2 = z_alloc((size_t)R * E2);
  a->G = (double**)calloc(L + 1, sizeof(double*));
  for (int l = 0; l <= L; ++l) a->G[l] = z_alloc((size_t)R * M1);
  for (int j = 0; j < a->nn; ++j) {
    a->d[j] = sqrt(a->v[j].d2);
    oswitch(a->d[j], m->rs, m->rc, &a->sw[j], &a->dsw[j]);
    a->s[j] = a->sw[j] / a->d[j];
    for (int c = 0; c < 3; ++c) a->rh[3 * j + c] = a->v[j].r[c] / a->d[j];
    a->Rt[4 * j] = a->s[j];
    for (int c = 0; c < 3; ++c) a->Rt[4 * j + 1 + c] = a->s[j] * a->rh[3 * j + c];
  }
  for (int j = 0; j < a->nn; ++j)
    for (int k = 0; k < a->nn; ++k)
      a->cg[j * R + k] = a->rh[3 * j] * a->rh[3 * k] + a->rh[3 * j + 1] * a->rh[3 * k + 1] +
                         a->rh[3 * j + 2] * a->rh[3 * k + 2];
  for (int j = 0; j < a->nn; ++j) {
    const int t = types[a->v[j].j];
    for (int k = 0; k < E1; ++k) a->h1[j * E1 + k] = tanh(a->s[j] * W->eW1[t][k] + W->eb1[t][k]);
    for (int f = 0; f < E2; ++f) {
      double acc = W->eb2[t][f];
      for (int k = 0; k < E1; ++k) acc += a->h1[j * E1 + k] * W->eW2[t][k * E2 + f];
      a->h2[j * E2 + f] = tanh(acc);
    }
    for (int f = 0; f < M1; ++f) {
      double acc = W->eb3[t][f];
      for (int k = 0; k < E2; ++k) acc += a->h2[j * E2 + k] * W->eW3[t][k * M1 + f];
      a->G[0][j * M1 + f] = tanh(acc);
    }
  }
  const size_t RH = (size_t)R * m->hidden, RR = (size_t)R * R;
  const int LL = L > 0 ? L : 1;
  a->Q = (double**)calloc(LL, sizeof(double*)); a->K = (double**)calloc(LL, sizeof(double*));
  a->V = (double**)calloc(LL, sizeof(double*)); a->P = (double**)calloc(LL, sizeof(double*));
  a->Wa = (double**)calloc(LL, sizeof(double*)); a->rstd = (double**)calloc(LL, sizeof(double*));
  for (int l = 0; l < L; ++l) {
    a->Q[l] = z_alloc(RH); a->K[l] = z_alloc(RH); a->V[l] = z_alloc(RH);
    a->P[l] = z_alloc((size_t)m->heads * RR); a->Wa[l] = z_alloc((size_t)m->heads * RR);
    a->rstd[l] = z_alloc(R);
  }
  a->Gin = z_alloc((size_t)R * M1);
  a->dG = z_alloc((size_t)R * M1); a->dRt = z_alloc(4 * R);
  a->dsw_att = z_alloc(R); a->dcg = z_alloc(RR);
}

static void amp_free(amp_atom* a, int L) {
  free(a->v);
  free(a->d); free(a->sw); free(a->dsw); free(a->s); free(a->Rt); free(a->rh); free(a->cg);
  free(a->h1); free(a->h2);
  for (int l = 0; l <= L; ++l) free(a->G[l]);
  for (int l = 0; l < L; ++l) {
    free(a->Q[l]); free(a->K[l]); free(a->V[l]); free(a->P[l]); free(a->Wa[l]); free(a->rstd[l]);
  }
  free(a->G); free(a->Q); free(a->K); free(a->V); free(a->P); free(a->Wa); free(a->rstd);
  free(a->Gin); free(a->dG); free(a->dRt); free(a->dsw_att); free(a->dcg);
}

/* Attention layer l on a->Gin (G'), written to a->G[l + 1]. */
static void amp_layer_fwd(const amp_model* m, const amp_weights* W, int l, amp_atom* a) {
  const int nn = a->nn, R = nn > 0 ? nn : 1, M1 = m->m1, H = m->hidden, NH = m->heads;
  const int DH = H / NH;
  const double inv_sqrt_d = 1.0 / sqrt((double)DH);
  const size_t RR = (size_t)R * R;
  const double* gin = a->Gin;
  double *Q = a->Q[l], *K = a->K[l], *V = a->V[l];
  for (int j = 0; j < nn; ++j)
    for (int c = 0; c < H; ++c) {
      double q = 0, k = 0, v = 0;
      for (int f = 0; f < M1; ++f) {
        q += gin[j * M1 + f] * W->Wq[l][f * H + c];
        k += gin[j * M1 + f] * W->Wk[l][f * H + c];
        v += gin[j * M1 + f] * W->Wv[l][f * H + c];
      }
      Q[j * H + c] = q;
      K[j * H + c] = k;
      V[j * H + c] = v;
    }
  double* O = z_alloc((size_t)R * H);
  for (int h = 0; h < NH; ++h) {
    double* Ph = a->P[l] + (size_t)h * RR;
    double* Wh = a->Wa[l] + (size_t)h * RR;
    for (int j = 0; j < nn; ++j) {
      double mx = -INFINITY;
      for (int k = 0; k < nn; ++k) {
        double sc = 0;
        for (int c = 0; c < DH; ++c) sc += Q[j * H + h * DH + c] * K[k * H + h * DH + c];
        sc *= inv_sqrt_d;
        Ph[j * R + k] = sc;
        if (sc > mx) mx = sc;
      }
      double z = 0;
      for (int k = 0; k < nn; ++k) {
        Ph[j * R + k] = exp(Ph[j * R + k] - mx);
        z += a->sw[k] * Ph[j * R + k];
      }
      for (int k = 0; k < nn; ++k) {
        Ph[j * R + k] = z > 0 ? Ph[j * R + k] / z : 0.0;
        Wh[j * R + k] = a->sw[k] * Ph[j * R + k];
      }
      for (int c = 0; c < DH; ++c) {
        double o = 0;
        for (int k = 0; k < nn; ++k) o += Wh[j * R + k] * a->cg[j * R + k] * V[k * H + h * DH + c];
        O[j * H + h * DH + c] = o;
      }
    }
  }
  double* Z = z_alloc(M1);
  for (int j = 0; j < nn; ++j) {
    double mu = 0;
    for (int f = 0; f < M1; ++f) {
      double y = W->bo[l][f];
      for (int c = 0; c < H; ++c) y += O[j * H + c] * W->Wo[l][c * M1 + f];
      Z[f] = gin[j * M1 + f] + y;
      mu += Z[f];
    }
    mu /= M1;
    double var = 0;
    for (int f = 0; f < M1; ++f) var += (Z[f] - mu) * (Z[f] - mu);
    var /= M1;
    a->rstd[l][j] = 1.0 / sqrt(var + 1e-5);
    for (int f = 0; f < M1; ++f) a->G[l + 1][j * M1 + f] = (Z[f] - mu) * a->rstd[l][j];
  }
  free(O);
  free(Z);
}

/* Descriptor and fitting from G^L: e_i, then seed * de_i/dG^L into a->dG and
 * seed * de_i/dR~ into a->dRt. */
static void amp_fit(const amp_model* m, const amp_weights* W, int ti, double seed, amp_atom* a) {
  const int nn = a->nn, M1 = m->m1, M2 = m->m2, L = m->n_layers;
  const int F1 = m->f1, F2 = m->f2, F3 = m->f3, ND = M1 * M2;
  const double inv_nmax = 1.0 / (double)m->nmax;
  const double* Gf = a->G[L];
  double* T = z_alloc(4 * (size_t)M1);
  for (int c = 0; c < 4; ++c)
    for (int f = 0; f < M1; ++f) {
      double acc = 0;
      for (int j = 0; j < nn; ++j) acc += a->Rt[4 * j + c] * Gf[j * M1 + f];
      T[c * M1 + f] = acc * inv_nmax;
    }
  double* D = z_alloc(ND);
  for (int f = 0; f < M1; ++f)
    for (int q = 0; q < M2; ++q) {
      double acc = 0;
      for (int c = 0; c < 4; ++c) acc += T[c * M1 + f] * T[c * M1 + q];
      D[f * M2 + q] = acc;
    }
  double *y1 = z_alloc(F1), *y2 = z_alloc(F2), *y3 = z_alloc(F3);
  for (int b = 0; b < F1; ++b) {
    double acc = W->fb1[ti][b];
    for (int c = 0; c < ND; ++c) acc += D[c] * W->fW1[ti][(size_t)c * F1 + b];
    y1[b] = tanh(acc);
  }
  for (int b = 0; b < F2; ++b) {
    double acc = W->fb2[ti][b];
    for (int c = 0; c < F1; ++c) acc += y1[c] * W->fW2[ti][c * F2 + b];
    y2[b] = tanh(acc);
  }
  for (int b = 0; b < F3; ++b) {
    double acc = W->fb3[ti][b];
    for (int c = 0; c < F2; ++c) acc += y2[c] * W->fW3[ti][c * F3 + b];
    y3[b] = tanh(acc);
  }
  double e = W->fb4[ti][0];
  for (int c = 0; c < F3; ++c) e += y3[c] * W->fW4[ti][c];
  a->e = e;
  /* backward */
  double *l3 = z_alloc(F3), *l2 = z_alloc(F2), *l1 = z_alloc(F1), *dD = z_alloc(ND);
  for (int b = 0; b < F3; ++b) l3[b] = seed * W->fW4[ti][b] * (1.0 - y3[b] * y3[b]);
  for (int c = 0; c < F2; ++c) {
    double acc = 0;
    for (int b = 0; b < F3; ++b) acc += W->fW3[ti][c * F3 + b] * l3[b];
    l2[c] = acc * (1.0 - y2[c] * y2[c]);
  }
  for (int c = 0; c < F1; ++c) {
    double acc = 0;
    for (int b = 0; b < F2; ++b) acc += W->fW2[ti][c * F2 + b] * l2[b];
    l1[c] = acc * (1.0 - y1[c] * y1[c]);
  }
  for (int c = 0; c < ND; ++c) {
    double acc = 0;
    for (int b = 0; b < F1; ++b) acc += W->fW1[ti][(size_t)c * F1 + b] * l1[b];
    dD[c] = acc;
  }
  double* dT = z_alloc(4 * (size_t)M1);
  for (int c = 0; c < 4; ++c)
    for (int f = 0; f < M1; ++f) {
      double acc = 0;
      for (int q = 0; q < M2; ++q) acc += dD[f * M2 + q] * T[c * M1 + q];
      dT[c * M1 + f] += acc;
    }
  for (int c = 0; c < 4; ++c)
    for (int q = 0; q < M2; ++q) {
      double acc = 0;
      for (int f = 0; f < M1; ++f) acc += dD[f * M2 + q] * T[c * M1 + f];
      dT[c * M1 + q] += acc;
    }
  for (int j = 0; j < nn; ++j) {
    for (int c = 0; c < 4; ++c) {
      double acc = 0;
      for (int f = 0; f < M1; ++f) acc += dT[c * M1 + f] * Gf[j * M1 + f];
      a->dRt[4 * j + c] = acc * inv_nmax;
    }
    for (int f = 0; f < M1; ++f) {
      double acc = 0;
      for (int c = 0; c < 4; ++c) acc += dT[c * M1 + f] * a->Rt[4 * j + c];
      a->dG[j * M1 + f] = acc * inv_nmax;
    }
  }
  free(T); free(D); free(y1); free(y2); free(y3);
  free(l3); free(l2); free(l1); free(dD); free(dT);
}

/* Adjoint of attention layer l: a->dG holds dE/dG^{l+1} on entry and
 * dE/dG' (the layer's input) on return; dE/dsw and dE/dc accumulate. */
static void amp_layer_bwd(const amp_model* m, const amp_weights* W, int l, amp_atom* a) {
  const int nn = a->nn, R = nn > 0 ? nn : 1, M1 = m->m1, H = m->hidden, NH = m->heads;
  const int DH = H / NH;
  const double inv_sqrt_d = 1.0 / sqrt((double)DH);
  const size_t RH = (size_t)R * H, RR = (size_t)R * R;
  const double* gout = a->G[l + 1];
  double* dG = a->dG;
  double* dZ = z_alloc((size_t)R * M1);
  double *dO = z_alloc(RH), *dQ = z_alloc(RH), *dK = z_alloc(RH), *dV = z_alloc(RH);
  double *dA = z_alloc(R), *rho = z_alloc(R);
  for (int j = 0; j < nn; ++j) {   /* LayerNorm */
    double m1v = 0, m2v = 0;
    for (int f = 0; f < M1; ++f) {
      m1v += dG[j * M1 + f];
      m2v += dG[j * M1 + f] * gout[j * M1 + f];
    }
    m1v /= M1;
    m2v /= M1;
    for (int f = 0; f < M1; ++f)
      dZ[j * M1 + f] = a->rstd[l][j] * (dG[j * M1 + f] - m1v - gout[j * M1 + f] * m2v);
  }
  for (int j = 0; j < nn; ++j)       /* Z = G' + O Wo + bo */
    for (int c = 0; c < H; ++c) {
      double acc = 0;
      for (int f = 0; f < M1; ++f) acc += dZ[j * M1 + f] * W->Wo[l][c * M1 + f];
      dO[j * H + c] = acc;
    }
  const double *Q = a->Q[l], *K = a->K[l], *V = a->V[l];
  for (int h = 0; h < NH; ++h) {
    const double* Ph = a->P[l] + (size_t)h * RR;
    const double* Wh = a->Wa[l] + (size_t)h * RR;
    for (int j = 0; j < nn; ++j) {
      double wdw = 0;
      for (int k = 0; k < nn; ++k) {
        double da = 0;
        for (int c = 0; c < DH; ++c) da += dO[j * H + h * DH + c] * V[k * H + h * DH + c];
        dA[k] = da;
        for (int c = 0; c < DH; ++c)
          dV[k * H + h * DH + c] += Wh[j * R + k] * a->cg[j * R + k] * dO[j * H + h * DH + c];
        a->dcg[j * R + k] += da * Wh[j * R + k];
        const double dw = da * a->cg[j * R + k];
        rho[k] = dw;
        wdw += Wh[j * R + k] * dw;
      }
      for (int k = 0; k < nn; ++k) {
        rho[k] -= wdw;
        const double dS = Wh[j * R + k] * rho[k];
        a->dsw_att[k] += Ph[j * R + k] * rho[k];
        for (int c = 0; c < DH; ++c) {
          dQ[j * H + h * DH + c] += dS * K[k * H + h * DH + c] * inv_sqrt_d;
          dK[k * H + h * DH + c] += dS * Q[j * H + h * DH + c] * inv_sqrt_d;
        }
      }
    }
  }
  for (int j = 0; j < nn; ++j)
    for (int f = 0; f < M1; ++f) {
      double acc = dZ[j * M1 + f];
      for (int c = 0; c < H; ++c)
        acc += dQ[j * H + c] * W->Wq[l][f * H + c] + dK[j * H + c] * W->Wk[l][f * H + c] +
               dV[j * H + c] * W->Wv[l][f * H + c];
      dG[j * M1 + f] = acc;
    }
  free(dZ); free(dO); free(dQ); free(dK); free(dV); free(dA); free(rho);
}

/* Embedding, gate and environment adjoints: a->dG = dE/dG^0 -> g (nn x 3). */
static void amp_env_bwd(const amp_model* m, const amp_weights* W, const int32_t* types,
                        amp_atom* a, double* g) {
  const int nn = a->nn, R = nn > 0 ? nn : 1, M1 = m->m1, E1 = m->e1, E2 = m->e2;
  double *ds = z_alloc(R), *da2 = z_alloc(E2), *da1 = z_alloc(E1), *drh = z_alloc(3 * (size_t)R);
  for (int j = 0; j < nn; ++j) {
    const int t = types[a->v[j].j];
    for (int k = 0; k < E2; ++k) {
      double acc = 0;
      for (int f = 0; f < M1; ++f) {
        const double g0 = a->G[0][j * M1 + f];
        acc += a->dG[j * M1 + f] * (1.0 - g0 * g0) * W->eW3[t][k * M1 + f];
      }
      da2[k] = acc * (1.0 - a->h2[j * E2 + k] * a->h2[j * E2 + k]);
    }
    double acc1 = 0;
    for (int k = 0; k < E1; ++k) {
      double acc = 0;
      for (int f = 0; f < E2; ++f) acc += da2[f] * W->eW2[t][k * E2 + f];
      da1[k] = acc * (1.0 - a->h1[j * E1 + k] * a->h1[j * E1 + k]);
      acc1 += da1[k] * W->eW1[t][k];
    }
    ds[j] = acc1;
  }
  for (int j = 0; j < nn; ++j)
    for (int k = 0; k < nn; ++k)
      for (int c = 0; c < 3; ++c) {
        drh[3 * j + c] += a->dcg[j * R + k] * a->rh[3 * k + c];
        drh[3 * k + c] += a->dcg[j * R + k] * a->rh[3 * j + c];
      }
  for (int j = 0; j < nn; ++j) {
    double dst = a->dRt[4 * j] + ds[j];
    double dr3[3];
    for (int c = 0; c < 3; ++c) {
      dst += a->dRt[4 * j + 1 + c] * a->rh[3 * j + c];
      dr3[c] = drh[3 * j + c] + a->s[j] * a->dRt[4 * j + 1 + c];
    }
    const double d = a->d[j], sw = a->sw[j], dsw = a->dsw[j];
    const double radial = dst * (dsw / d - sw / (d * d)) + a->dsw_att[j] * dsw;
    const double proj = dr3[0] * a->rh[3 * j] + dr3[1] * a->rh[3 * j + 1] + dr3[2] * a->rh[3 * j + 2];
    for (int c = 0; c < 3; ++c)
      g[3 * j + c] = radial * a->rh[3 * j + c] + (dr3[c] - proj * a->rh[3 * j + c]) / d;
  }
  free(ds); free(da2); free(da1); free(drh);
}

static void owrap_all_mp(int n, const double* x, const double* L, double* w) {
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < 3; ++c) w[3 * i + c] = owrap(x[3 * i + c], L[c]);
}

/* E = sum_i seed_i e_i (seed NULL: all ones), its forces -dE/dx (n x 3) and
 * virial (3 x 3, row-major), and the atomic energies e_i; every output but
 * `energy` is nullable.  Sums run in atom order.  Returns -1 for an invalid
 * model.  A seed of 0 makes an atom a ghost: it is a centre (its neighbours'
 * features need it) but its energy is not counted. */
static int afmp_compute(const int32_t* idims, const double* fdims, const double* weights, int n,
                        const int32_t* types, const double* x, const double* box, int nthreads,
                        const double* seed, double* energy, double* atom_e, double* forces,
                        double* virial) {
  amp_model m;
  amp_weights W;
  amp_model_from(idims, fdims, &m);
  if (amp_check(&m)) return -1;
  amp_bind(&m, weights, &W);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  const int L = m.n_layers, M1 = m.m1;
  const double inv_nmax = 1.0 / (double)m.nmax;
  double* w = z_alloc(3 * (size_t)n);
  owrap_all_mp(n, x, box, w);
  ocells cells;
  const int have = ocells_build(&cells, n, w, box, m.rc);
  amp_atom* at = (amp_atom*)calloc(n > 0 ? n : 1, sizeof(amp_atom));
  /* neighbours, environment, embedding */
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < n; ++i) {
    onbr* v;
    const int c = have ? onbrs_cells(&cells, i, w, box, m.rc, &v) : onbrs_brute(i, n, w, box, m.rc, &v);
    at[i].nn = c < m.nmax ? c : m.nmax;
    at[i].v = v;
    amp_env_embed(&m, &W, types, &at[i]);
  }
  /* layers, synchronous over atoms */
  double* h = z_alloc((size_t)n * M1);
  double** U = (double**)calloc(L > 0 ? L : 1, sizeof(double*));
  for (int i = 0; i < n; ++i)
    for (int f = 0; f < M1; ++f) h[(size_t)i * M1 + f] = W.Wt[types[i] * M1 + f];
  for (int l = 0; l < L; ++l) {
    U[l] = z_alloc((size_t)n * M1);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
      for (int f = 0; f < M1; ++f) {
        double acc = W.bm[l][f];
        for (int c = 0; c < M1; ++c) acc += h[(size_t)i * M1 + c] * W.Wm[l][c * M1 + f];
        U[l][(size_t)i * M1 + f] = tanh(acc);
      }
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n; ++i) {
      amp_atom* a = &at[i];
      for (int p = 0; p < a->nn; ++p)
        for (int f = 0; f < M1; ++f)
          a->Gin[p * M1 + f] = a->G[l][p * M1 + f] + U[l][(size_t)a->v[p].j * M1 + f];
      amp_layer_fwd(&m, &W, l, a);
    }
    if (l + 1 < L) {
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) {
        const amp_atom* a = &at[i];
        for (int f = 0; f < M1; ++f) {
          double acc = 0;
          for (int p = 0; p < a->nn; ++p) acc += a->sw[p] * a->G[l + 1][p * M1 + f];
          h[(size_t)i * M1 + f] += acc * inv_nmax;
        }
      }
    }
  }
  /* energies, then the adjoint in reverse */
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < n; ++i) amp_fit(&m, &W, types[i], seed ? seed[i] : 1.0, &at[i]);
  double* dh = z_alloc((size_t)n * M1);     /* dE/dh^{l+1}, then dE/dh^l */
  double* dU = z_alloc((size_t)n * M1);
  for (int l = L - 1; l >= 0; --l) {
    if (l + 1 < L) {                          /* h^{l+1} = h^l + pool(G^{l+1}) */
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) {
        amp_atom* a = &at[i];
        for (int p = 0; p < a->nn; ++p) {
          double dot = 0;
          for (int f = 0; f < M1; ++f) {
            a->dG[p * M1 + f] += a->sw[p] * inv_nmax * dh[(size_t)i * M1 + f];
            dot += a->G[l + 1][p * M1 + f] * dh[(size_t)i * M1 + f];
          }
          a->dsw_att[p] += dot * inv_nmax;
        }
      }
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n; ++i) amp_layer_bwd(&m, &W, l, &at[i]);
    memset(dU, 0, sizeof(double) * (size_t)n * M1);
    for (int i = 0; i < n; ++i)               /* G' = G + U_{j(p)} */
      for (int p = 0; p < at[i].nn; ++p)
        for (int f = 0; f < M1; ++f) dU[(size_t)at[i].v[p].j * M1 + f] += at[i].dG[p * M1 + f];
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n; ++j) {
      double* q = dU + (size_t)j * M1;
      for (int c = 0; c < M1; ++c) {
        const double u = U[l][(size_t)j * M1 + c];
        q[c] *= 1.0 - u * u;
      }
      for (int f = 0; f < M1; ++f) {
        double acc = 0;
        for (int c = 0; c < M1; ++c) acc += q[c] * W.Wm[l][f * M1 + c];
        dh[(size_t)j * M1 + f] += acc;
      }
    }
  }
  /* pair gradients, forces, virial */
  double* pg = z_alloc((size_t)n * m.nmax * 3);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < n; ++i) amp_env_bwd(&m, &W, types, &at[i], pg + (size_t)i * m.nmax * 3);
  double E = 0, vir[9] = {0};
  if (forces) memset(forces, 0, sizeof(double) * 3 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    E += seed ? seed[i] * at[i].e : at[i].e;
    if (atom_e) atom_e[i] = at[i].e;
    for (int p = 0; p < at[i].nn; ++p) {
      const double* g = pg + ((size_t)i * m.nmax + p) * 3;
      const int j = at[i].v[p].j;
      if (forces)
        for (int c = 0; c < 3; ++c) {
          forces[3 * i + c] += g[c];
          forces[3 * (size_t)j + c] -= g[c];
        }
      for (int c = 0; c < 3; ++c)
        for (int b = 0; b < 3; ++b) vir[3 * c + b] -= at[i].v[p].r[c] * g[b];
    }
  }
  if (energy) *energy = E;
  if (virial) memcpy(virial, vir, sizeof vir);
  for (int i = 0; i < n; ++i) amp_free(&at[i], L);
  for (int l = 0; l < L; ++l) free(U[l]);
  free(U); free(at); free(h); free(dh); free(dU); free(pg); free(w);
  if (have) ocells_free(&cells);
  return 0;
}

int oracle_afmp_compute(const int32_t* idims, const double* fdims, const double* weights, int n,
                        const int32_t* types, const double* x, const double* box, int nthreads,
                        double* energy, double* atom_e, double* forces, double* virial) {
  return afmp_compute(idims, fdims, weights, n, types, x, box, nthreads, NULL, energy, atom_e,
                      forces, virial);
}

int oracle_afmp_compute_seeded(const int32_t* idims, const double* fdims, const double* weights,
                               int n, const int32_t* types, const double* x, const double* box,
                               int nthreads, const double* seed, double* energy, double* atom_e,
                               double* forces, double* virial) {
  return afmp_compute(idims, fdims, weights, n, types, x, box, nthreads, seed, energy, atom_e,
                      forces, virial);
}
