/*
 * FP64 CPU oracle of the attention-family deep potential -- TEST
 * INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's CPU-baseline
 * leg).  Plain loops in double precision, one centre atom at a time, OpenMP
 * over centre atoms; no blocking or fusion.
 *
 * The paper (Sec. II) names the DPA2 stages -- a "repinit" embedding MLP, a
 * "repformer" stack of residual self-attention layers and a per-atom
 * "fitting-net" MLP giving atomic energies -- but prints no formula.  The
 * model computed here is a reading written out in full:
 *
 *  Neighbours (Sec. II, cutoff-based Verlet lists; cutoff 0.6 nm, Sec. IV):
 *    all (j, n) with 0 < |r_ij| < rc, r_ij = (w_j - w_i) + n*L, w wrapped
 *    positions; when more than Nmax, the Nmax smallest by (|r|^2, j, n).
 *  Switch: sw(r) = 1 (r < rs), u^3(-6u^2+15u-10)+1 (rs <= r < rc), 0 beyond,
 *    u = (r-rs)/(rc-rs).  s = sw/r, R~_j = (s, s x/r, s y/r, s z/r),
 *    unit vector rh_j = r/|r|.
 *  Embedding (one net per neighbour species t_j):
 *    G_j = tanh(tanh(tanh(s_j W1 + b1) W2 + b2) W3 + b3).
 *  Attention layer (hidden H = heads*d, no Q/K/V biases), per head:
 *    S_jk = Q_j.K_k / sqrt(d); w_jk = sw_k exp(S_jk) / sum_k' sw_k' exp(S_jk');
 *    A_jk = w_jk (rh_j . rh_k); O = A V; then
 *    G <- LayerNorm(G + concat_h(O) Wo + bo) with eps 1e-5, gamma 1, beta 0.
 *  Descriptor: T = (1/Nmax) R~^T G (4 x M1); D = T^T T[:, :M2] (M1 x M2, row-major).
 *  Fitting (one net per centre species t_i):
 *    e_i = tanh(tanh(tanh(D W1 + b1) W2 + b2) W3 + b3) W4 + b4;  E = sum_i e_i.
 *  Gradient: g_ij = dE/dr_ij by hand (reverse order of the above);
 *    F_i = sum_j g_ij - sum_{k: i in nl(k)} g_ki;  virial X_ab = -sum r_a g_b.
 *
 * Weight blob (row-major W[in][out], W before b):
 *    for t < S: embedding W1[1][e1] b1 W2[e1][e2] b2 W3[e2][M1] b3
 *    for l < L: Wq[M1][H] Wk[M1][H] Wv[M1][H] Wo[H][M1] bo[M1]
 *    for t < S: fitting W1[M1*M2][f1] b1 W2[f1][f2] b2 W3[f2][f3] b3 W4[f3][1] b4[1]
 */
#include "oracle_common.h"

#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OAF_MAXS 16
#define OAF_MAXL 16

typedef struct {
  int n_species, e1, e2, m1, m2, n_layers, hidden, heads, f1, f2, f3, nmax;
  double rc, rs;
} oaf_model;

typedef struct {
  const double *eW1[OAF_MAXS], *eb1[OAF_MAXS], *eW2[OAF_MAXS], *eb2[OAF_MAXS], *eW3[OAF_MAXS],
      *eb3[OAF_MAXS];
  const double *Wq[OAF_MAXL], *Wk[OAF_MAXL], *Wv[OAF_MAXL], *Wo[OAF_MAXL], *bo[OAF_MAXL];
  const double *fW1[OAF_MAXS], *fb1[OAF_MAXS], *fW2[OAF_MAXS], *fb2[OAF_MAXS], *fW3[OAF_MAXS],
      *fb3[OAF_MAXS], *fW4[OAF_MAXS], *fb4[OAF_MAXS];
} oaf_weights;

static void oaf_model_from(const int32_t* idims, const double* fdims, oaf_model* m) {
  m->n_species = idims[0];
  m->e1 = idims[1];
  m->e2 = idims[2];
  m->m1 = idims[3];
  m->m2 = idims[4];
  m->n_layers = idims[5];
  m->hidden = idims[6];
  m->heads = idims[7];
  m->f1 = idims[8];
  m->f2 = idims[9];
  m->f3 = idims[10];
  m->nmax = idims[11];
  m->rc = fdims[0];
  m->rs = fdims[1];
}

/* Offsets (in doubles) of every block of the blob, in its fixed order. */
typedef struct {
  size_t eW1[OAF_MAXS], eb1[OAF_MAXS], eW2[OAF_MAXS], eb2[OAF_MAXS], eW3[OAF_MAXS], eb3[OAF_MAXS];
  size_t Wq[OAF_MAXL], Wk[OAF_MAXL], Wv[OAF_MAXL], Wo[OAF_MAXL], bo[OAF_MAXL];
  size_t fW1[OAF_MAXS], fb1[OAF_MAXS], fW2[OAF_MAXS], fb2[OAF_MAXS], fW3[OAF_MAXS],
      fb3[OAF_MAXS], fW4[OAF_MAXS], fb4[OAF_MAXS];
  size_t total;
} oaf_offsets;

static void oaf_offsets_of(const oaf_model* m, oaf_offsets* o) {
  size_t off = 0;
#define TAKE(dst, cnt) do { (dst) = off; off += (size_t)(cnt); } while (0)
  for (int t = 0; t < m->n_species; ++t) {
    TAKE(o->eW1[t], m->e1);
    TAKE(o->eb1[t], m->e1);
    TAKE(o->eW2[t], m->e1 * m->e2);
    TAKE(o->eb2[t], m->e2);
    TAKE(o->eW3[t], m->e2 * m->m1);
    TAKE(o->eb3[t], m->m1);
  }
  for (int l = 0; l < m->n_layers; ++l) {
    TAKE(o->Wq[l], m->m1 * m->hidden);
    TAKE(o->Wk[l], m->m1 * m->hidden);
    TAKE(o->Wv[l], m->m1 * m->hidden);
    TAKE(o->Wo[l], m->hidden * m->m1);
    TAKE(o->bo[l], m->m1);
  }
  for (int t = 0; t < m->n_species; ++t) {
    TAKE(o->fW1[t], (size_t)m->m1 * m->m2 * m->f1);
    TAKE(o->fb1[t], m->f1);
    TAKE(o->fW2[t], m->f1 * m->f2);
    TAKE(o->fb2[t], m->f2);
    TAKE(o->fW3[t], m->f2 * m->f3);
    TAKE(o->fb3[t], m->f3);
    TAKE(o->fW4[t], m->f3);
    TAKE(o->fb4[t], 1);
  }
#undef TAKE
  o->total = off;
}

static void oaf_bind(const oaf_model* m, const double* base, oaf_weights* w) {
  oaf_offsets o;
  oaf_offsets_of(m, &o);
  for (int t = 0; t < m->n_species; ++t) {
    w->eW1[t] = base + o.eW1[t]; w->eb1[t] = base + o.eb1[t];
    w->eW2[t] = base + o.eW2[t]; w->eb2[t] = base + o.eb2[t];
    w->eW3[t] = base + o.eW3[t]; w->eb3[t] = base + o.eb3[t];
    w->fW1[t] = base + o.fW1[t]; w->fb1[t] = base + o.fb1[t];
    w->fW2[t] = base + o.fW2[t]; w->fb2[t] = base + o.fb2[t];
    w->fW3[t] = base + o.fW3[t]; w->fb3[t] = base + o.fb3[t];
    w->fW4[t] = base + o.fW4[t]; w->fb4[t] = base + o.fb4[t];
  }
  for (int l = 0; l < m->n_layers; ++l) {
    w->Wq[l] = base + o.Wq[l]; w->Wk[l] = base + o.Wk[l]; w->Wv[l] = base + o.Wv[l];
    w->Wo[l] = base + o.Wo[l]; w->bo[l] = base + o.bo[l];
  }
}

static int oaf_check(const oaf_model* m) {
  if (m->n_species < 1 || m->n_species > OAF_MAXS) return -1;
  if (m->n_layers < 0 || m->n_layers > OAF_MAXL) return -1;
  if (m->heads < 1 || m->hidden % m->heads) return -1;
  if (m->m2 > m->m1 || m->nmax < 1) return -1;
  if (!(m->rs < m->rc)) return -1;
  return 0;
}

/* Number of doubles in the weight blob, or -1 for an invalid model. */
long long oracle_af_weight_count(const int32_t* idims, const double* fdims) {
  oaf_model m;
  oaf_offsets o;
  oaf_model_from(idims, fdims, &m);
  if (oaf_check(&m)) return -1;
  oaf_offsets_of(&m, &o);
  return (long long)o.total;
}

/* Offset of one block, for tests that edit single weights: kind 0..5 =
 * embedding W1 b1 W2 b2 W3 b3 of species a; 10..14 = Wq Wk Wv Wo bo of layer a;
 * 20..27 = fitting W1 b1 W2 b2 W3 b3 W4 b4 of species a. */
long long oracle_af_weight_offset(const int32_t* idims, const double* fdims, int kind, int a) {
  oaf_model m;
  oaf_offsets o;
  oaf_model_from(idims, fdims, &m);
  if (oaf_check(&m) || a < 0) return -1;
  oaf_offsets_of(&m, &o);
  int S = m.n_species, L = m.n_layers;
  switch (kind) {
    case 0: return a < S ? (long long)o.eW1[a] : -1;
    case 1: return a < S ? (long long)o.eb1[a] : -1;
    case 2: return a < S ? (long long)o.eW2[a] : -1;
    case 3: return a < S ? (long long)o.eb2[a] : -1;
    case 4: return a < S ? (long long)o.eW3[a] : -1;
    case 5: return a < S ? (long long)o.eb3[a] : -1;
    case 10: return a < L ? (long long)o.Wq[a] : -1;
    case 11: return a < L ? (long long)o.Wk[a] : -1;
    case 12: return a < L ? (long long)o.Wv[a] : -1;
    case 13: return a < L ? (long long)o.Wo[a] : -1;
    case 14: return a < L ? (long long)o.bo[a] : -1;
    case 20: return a < S ? (long long)o.fW1[a] : -1;
    case 21: return a < S ? (long long)o.fb1[a] : -1;
    case 22: return a < S ? (long long)o.fW2[a] : -1;
    case 23: return a < S ? (long long)o.fb2[a] : -1;
    case 24: return a < S ? (long long)o.fW3[a] : -1;
    case 25: return a < S ? (long long)o.fb3[a] : -1;
    case 26: return a < S ? (long long)o.fW4[a] : -1;
    case 27: return a < S ? (long long)o.fb4[a] : -1;
    default: return -1;
  }
}

/* ------------------------------------------------------------------------ */
/* one centre atom: energy e_i and g_j = dE/dr_j for its nn neighbours        */
/* ------------------------------------------------------------------------ */
static double oaf_atom(const oaf_model* m, const oaf_weights* W, const int32_t* types, int ti,
                       int nn, const onbr* nb, double* g, double* D_out) {
  const int M1 = m->m1, M2 = m->m2, H = m->hidden, NH = m->heads, DH = H / NH;
  const int E1 = m->e1, E2 = m->e2, L = m->n_layers;
  const double inv_nmax = 1.0 / (double)m->nmax;
  const double inv_sqrt_d = 1.0 / sqrt((double)DH);
  const int R = nn > 0 ? nn : 1;

  /* environment */
  double* d = calloc(R, sizeof(double));
  double* sw = calloc(R, sizeof(double));
  double* dsw = calloc(R, sizeof(double));
  double* s = calloc(R, sizeof(double));
  double* Rt = calloc(4 * R, sizeof(double));
  double* rh = calloc(3 * R, sizeof(double));
  for (int j = 0; j < nn; ++j) {
    d[j] = sqrt(nb[j].d2);
    oswitch(d[j], m->rs, m->rc, &sw[j], &dsw[j]);
    s[j] = sw[j] / d[j];
    for (int a = 0; a < 3; ++a) rh[3 * j + a] = nb[j].r[a] / d[j];
    Rt[4 * j + 0] = s[j];
    for (int a = 0; a < 3; ++a) Rt[4 * j + 1 + a] = s[j] * rh[3 * j + a];
  }

  /* embedding */
  double* h1 = calloc((size_t)R * E1, sizeof(double));
  double* h2 = calloc((size_t)R * E2, sizeof(double));
  double** G = calloc(L + 1, sizeof(double*));
  for (int l = 0; l <= L; ++l) G[l] = calloc((size_t)R * M1, sizeof(double));
  for (int j = 0; j < nn; ++j) {
    int t = types[nb[j].j];
    for (int k = 0; k < E1; ++k) h1[j * E1 + k] = tanh(s[j] * W->eW1[t][k] + W->eb1[t][k]);
    for (int f = 0; f < E2; ++f) {
      double acc = W->eb2[t][f];
      for (int k = 0; k < E1; ++k) acc += h1[j * E1 + k] * W->eW2[t][k * E2 + f];
      h2[j * E2 + f] = tanh(acc);
    }
    for (int f = 0; f < M1; ++f) {
      double acc = W->eb3[t][f];
      for (int k = 0; k < E2; ++k) acc += h2[j * E2 + k] * W->eW3[t][k * M1 + f];
      G[0][j * M1 + f] = tanh(acc);
    }
  }

  /* attention layers, activations kept for the backward pass */
  size_t RH = (size_t)R * H, RR = (size_t)R * R;
  double** Q = calloc(L > 0 ? L : 1, sizeof(double*));
  double** K = calloc(L > 0 ? L : 1, sizeof(double*));
  double** V = calloc(L > 0 ? L : 1, sizeof(double*));
  double** P = calloc(L > 0 ? L : 1, sizeof(double*));  /* exp(S-m)/Z per head */
  double** Wt = calloc(L > 0 ? L : 1, sizeof(double*)); /* w = sw_k * P */
  double** rstd = calloc(L > 0 ? L : 1, sizeof(double*));
  double* cg = calloc(RR, sizeof(double)); /* gate rh_j . rh_k */
  for (int j = 0; j < nn; ++j)
    for (int k = 0; k < nn; ++k)
      cg[j * R + k] = rh[3 * j] * rh[3 * k] + rh[3 * j + 1] * rh[3 * k + 1] +
                      rh[3 * j + 2] * rh[3 * k + 2];
  double* Obuf = calloc(RH, sizeof(double));
  double* Zbuf = calloc((size_t)R * M1, sizeof(double));
  for (int l = 0; l < L; ++l) {
    const double *gin = G[l];
    Q[l] = calloc(RH, sizeof(double));
    K[l] = calloc(RH, sizeof(double));
    V[l] = calloc(RH, sizeof(double));
    P[l] = calloc((size_t)NH * RR, sizeof(double));
    Wt[l] = calloc((size_t)NH * RR, sizeof(double));
    rstd[l] = calloc(R, sizeof(double));
    for (int j = 0; j < nn; ++j)
      for (int c = 0; c < H; ++c) {
        double q = 0, k = 0, v = 0;
        for (int f = 0; f < M1; ++f) {
          q += gin[j * M1 + f] * W->Wq[l][f * H + c];
          k += gin[j * M1 + f] * W->Wk[l][f * H + c];
          v += gin[j * M1 + f] * W->Wv[l][f * H + c];
        }
        Q[l][j * H + c] = q;
        K[l][j * H + c] = k;
        V[l][j * H + c] = v;
      }
    memset(Obuf, 0, RH * sizeof(double));
    for (int h = 0; h < NH; ++h) {
      double* Ph = P[l] + (size_t)h * RR;
      double* Wh = Wt[l] + (size_t)h * RR;
      for (int j = 0; j < nn; ++j) {
        double mx = -INFINITY;
        for (int k = 0; k < nn; ++k) {
          double sc = 0;
          for (int c = 0; c < DH; ++c) sc += Q[l][j * H + h * DH + c] * K[l][k * H + h * DH + c];
          sc *= inv_sqrt_d;
          Ph[j * R + k] = sc;
          if (sc > mx) mx = sc;
        }
        double z = 0;
        for (int k = 0; k < nn; ++k) {
          Ph[j * R + k] = exp(Ph[j * R + k] - mx);
          z += sw[k] * Ph[j * R + k];
        }
        for (int k = 0; k < nn; ++k) {
          Ph[j * R + k] = z > 0 ? Ph[j * R + k] / z : 0.0;
          Wh[j * R + k] = sw[k] * Ph[j * R + k];
        }
        for (int c = 0; c < DH; ++c) {
          double o = 0;
          for (int k = 0; k < nn; ++k) o += Wh[j * R + k] * cg[j * R + k] * V[l][k * H + h * DH + c];
          Obuf[j * H + h * DH + c] = o;
        }
      }
    }
    for (int j = 0; j < nn; ++j) {
      double mu = 0;
      for (int f = 0; f < M1; ++f) {
        double y = W->bo[l][f];
        for (int c = 0; c < H; ++c) y += Obuf[j * H + c] * W->Wo[l][c * M1 + f];
        Zbuf[j * M1 + f] = gin[j * M1 + f] + y;
        mu += Zbuf[j * M1 + f];
      }
      mu /= M1;
      double var = 0;
      for (int f = 0; f < M1; ++f) var += (Zbuf[j * M1 + f] - mu) * (Zbuf[j * M1 + f] - mu);
      var /= M1;
      rstd[l][j] = 1.0 / sqrt(var + 1e-5);
      for (int f = 0; f < M1; ++f) G[l + 1][j * M1 + f] = (Zbuf[j * M1 + f] - mu) * rstd[l][j];
    }
  }
  const double* Gf = G[L];

  /* descriptor */
  double* T = calloc(4 * (size_t)M1, sizeof(double));
  for (int a = 0; a < 4; ++a)
    for (int f = 0; f < M1; ++f) {
      double acc = 0;
      for (int j = 0; j < nn; ++j) acc += Rt[4 * j + a] * Gf[j * M1 + f];
      T[a * M1 + f] = acc * inv_nmax;
    }
  double* D = calloc((size_t)M1 * M2, sizeof(double));
  for (int f = 0; f < M1; ++f)
    for (int q = 0; q < M2; ++q) {
      double acc = 0;
      for (int a = 0; a < 4; ++a) acc += T[a * M1 + f] * T[a * M1 + q];
      D[f * M2 + q] = acc;
    }
  if (D_out) memcpy(D_out, D, sizeof(double) * M1 * M2);

  /* fitting */
  int t_i = types[ti];
  const int F1 = m->f1, F2 = m->f2, F3 = m->f3, ND = M1 * M2;
  double* y1 = calloc(F1, sizeof(double));
  double* y2 = calloc(F2, sizeof(double));
  double* y3 = calloc(F3, sizeof(double));
  for (int b = 0; b < F1; ++b) {
    double acc = W->fb1[t_i][b];
    for (int a = 0; a < ND; ++a) acc += D[a] * W->fW1[t_i][(size_t)a * F1 + b];
    y1[b] = tanh(acc);
  }
  for (int b = 0; b < F2; ++b) {
    double acc = W->fb2[t_i][b];
    for (int a = 0; a < F1; ++a) acc += y1[a] * W->fW2[t_i][a * F2 + b];
    y2[b] = tanh(acc);
  }
  for (int b = 0; b < F3; ++b) {
    double acc = W->fb3[t_i][b];
    for (int a = 0; a < F2; ++a) acc += y2[a] * W->fW3[t_i][a * F3 + b];
    y3[b] = tanh(acc);
  }
  double e = W->fb4[t_i][0];
  for (int a = 0; a < F3; ++a) e += y3[a] * W->fW4[t_i][a];

  /* ---------------- backward ---------------- */
  if (g) {
    double* dl3 = calloc(F3, sizeof(double));
    double* dl2 = calloc(F2, sizeof(double));
    double* dl1 = calloc(F1, sizeof(double));
    double* dD = calloc(ND, sizeof(double));
    for (int b = 0; b < F3; ++b) dl3[b] = W->fW4[t_i][b] * (1.0 - y3[b] * y3[b]);
    for (int a = 0; a < F2; ++a) {
      double acc = 0;
      for (int b = 0; b < F3; ++b) acc += W->fW3[t_i][a * F3 + b] * dl3[b];
      dl2[a] = acc * (1.0 - y2[a] * y2[a]);
    }
    for (int a = 0; a < F1; ++a) {
      double acc = 0;
      for (int b = 0; b < F2; ++b) acc += W->fW2[t_i][a * F2 + b] * dl2[b];
      dl1[a] = acc * (1.0 - y1[a] * y1[a]);
    }
    for (int a = 0; a < ND; ++a) {
      double acc = 0;
      for (int b = 0; b < F1; ++b) acc += W->fW1[t_i][(size_t)a * F1 + b] * dl1[b];
      dD[a] = acc;
    }
    /* D[f][q] = sum_a T[a][f] T[a][q] */
    double* dT = calloc(4 * (size_t)M1, sizeof(double));
    for (int a = 0; a < 4; ++a)
      for (int f = 0; f < M1; ++f) {
        double acc = 0;
        for (int q = 0; q < M2; ++q) acc += dD[f * M2 + q] * T[a * M1 + q];
        dT[a * M1 + f] += acc;
      }
    for (int a = 0; a < 4; ++a)
      for (int q = 0; q < M2; ++q) {
        double acc = 0;
        for (int f = 0; f < M1; ++f) acc += dD[f * M2 + q] * T[a * M1 + f];
        dT[a * M1 + q] += acc;
      }
    /* T = (1/Nmax) R~^T G */
    double* dRt = calloc(4 * (size_t)R, sizeof(double));
    double* dG = calloc((size_t)R * M1, sizeof(double));
    for (int j = 0; j < nn; ++j) {
      for (int a = 0; a < 4; ++a) {
        double acc = 0;
        for (int f = 0; f < M1; ++f) acc += dT[a * M1 + f] * Gf[j * M1 + f];
        dRt[4 * j + a] = acc * inv_nmax;
      }
      for (int f = 0; f < M1; ++f) {
        double acc = 0;
        for (int a = 0; a < 4; ++a) acc += dT[a * M1 + f] * Rt[4 * j + a];
        dG[j * M1 + f] = acc * inv_nmax;
      }
    }
    /* attention layers in reverse */
    double* dsw_att = calloc(R, sizeof(double));
    double* dcg = calloc(RR, sizeof(double));
    double* dZ = calloc((size_t)R * M1, sizeof(double));
    double* dO = calloc(RH, sizeof(double));
    double* dQ = calloc(RH, sizeof(double));
    double* dK = calloc(RH, sizeof(double));
    double* dV = calloc(RH, sizeof(double));
    double* dA = calloc(R, sizeof(double));
    double* rho = calloc(R, sizeof(double));
    for (int l = L - 1; l >= 0; --l) {
      const double* gout = G[l + 1];
      /* LayerNorm: dZ = rstd (dG - mean(dG) - Gout mean(dG Gout)) */
      for (int j = 0; j < nn; ++j) {
        double m1v = 0, m2v = 0;
        for (int f = 0; f < M1; ++f) {
          m1v += dG[j * M1 + f];
          m2v += dG[j * M1 + f] * gout[j * M1 + f];
        }
        m1v /= M1;
        m2v /= M1;
        for (int f = 0; f < M1; ++f)
          dZ[j * M1 + f] = rstd[l][j] * (dG[j * M1 + f] - m1v - gout[j * M1 + f] * m2v);
      }
      /* Z = G_in + O Wo + bo */
      for (int j = 0; j < nn; ++j)
        for (int c = 0; c < H; ++c) {
          double acc = 0;
          for (int f = 0; f < M1; ++f) acc += dZ[j * M1 + f] * W->Wo[l][c * M1 + f];
          dO[j * H + c] = acc;
        }
      memset(dQ, 0, RH * sizeof(double));
      memset(dK, 0, RH * sizeof(double));
      memset(dV, 0, RH * sizeof(double));
      for (int h = 0; h < NH; ++h) {
        const double* Ph = P[l] + (size_t)h * RR;
        const double* Wh = Wt[l] + (size_t)h * RR;
        for (int j = 0; j < nn; ++j) {
          /* O_j = sum_k w_jk c_jk V_k */
          double wdw = 0;
          for (int k = 0; k < nn; ++k) {
            double da = 0;
            for (int c = 0; c < DH; ++c) da += dO[j * H + h * DH + c] * V[l][k * H + h * DH + c];
            dA[k] = da;
            for (int c = 0; c < DH; ++c)
              dV[k * H + h * DH + c] += Wh[j * R + k] * cg[j * R + k] * dO[j * H + h * DH + c];
            dcg[j * R + k] += da * Wh[j * R + k];
            double dw = da * cg[j * R + k];
            rho[k] = dw;
            wdw += Wh[j * R + k] * dw;
          }
          for (int k = 0; k < nn; ++k) {
            rho[k] -= wdw;
            double dS = Wh[j * R + k] * rho[k];
            dsw_att[k] += Ph[j * R + k] * rho[k];
            for (int c = 0; c < DH; ++c) {
              dQ[j * H + h * DH + c] += dS * K[l][k * H + h * DH + c] * inv_sqrt_d;
              dK[k * H + h * DH + c] += dS * Q[l][j * H + h * DH + c] * inv_sqrt_d;
            }
          }
        }
      }
      /* Q = G Wq, K = G Wk, V = G Wv; residual path adds dZ */
      for (int j = 0; j < nn; ++j)
        for (int f = 0; f < M1; ++f) {
          double acc = dZ[j * M1 + f];
          for (int c = 0; c < H; ++c)
            acc += dQ[j * H + c] * W->Wq[l][f * H + c] + dK[j * H + c] * W->Wk[l][f * H + c] +
                   dV[j * H + c] * W->Wv[l][f * H + c];
          dG[j * M1 + f] = acc;
        }
    }
    /* embedding backward: ds_j */
    double* ds = calloc(R, sizeof(double));
    double* da2 = calloc(E2, sizeof(double));
    double* da1 = calloc(E1, sizeof(double));
    for (int j = 0; j < nn; ++j) {
      int t = types[nb[j].j];
      for (int k = 0; k < E2; ++k) {
        double acc = 0;
        for (int f = 0; f < M1; ++f) {
          double g0 = G[0][j * M1 + f];
          acc += dG[j * M1 + f] * (1.0 - g0 * g0) * W->eW3[t][k * M1 + f];
        }
        da2[k] = acc * (1.0 - h2[j * E2 + k] * h2[j * E2 + k]);
      }
      double acc1 = 0;
      for (int k = 0; k < E1; ++k) {
        double acc = 0;
        for (int f = 0; f < E2; ++f) acc += da2[f] * W->eW2[t][k * E2 + f];
        da1[k] = acc * (1.0 - h1[j * E1 + k] * h1[j * E1 + k]);
        acc1 += da1[k] * W->eW1[t][k];
      }
      ds[j] = acc1;
    }
    /* gate backward: c_jk = rh_j . rh_k */
    double* drh = calloc(3 * (size_t)R, sizeof(double));
    for (int j = 0; j < nn; ++j)
      for (int k = 0; k < nn; ++k)
        for (int a = 0; a < 3; ++a) {
          drh[3 * j + a] += dcg[j * R + k] * rh[3 * k + a];
          drh[3 * k + a] += dcg[j * R + k] * rh[3 * j + a];
        }
    /* environment backward */
    for (int j = 0; j < nn; ++j) {
      double dst = dRt[4 * j] + ds[j];
      double dr3[3];
      for (int a = 0; a < 3; ++a) {
        dst += dRt[4 * j + 1 + a] * rh[3 * j + a];
        dr3[a] = drh[3 * j + a] + s[j] * dRt[4 * j + 1 + a];
      }
      double radial = dst * (dsw[j] / d[j] - sw[j] / (d[j] * d[j])) + dsw_att[j] * dsw[j];
      double proj = dr3[0] * rh[3 * j] + dr3[1] * rh[3 * j + 1] + dr3[2] * rh[3 * j + 2];
      for (int a = 0; a < 3; ++a)
        g[3 * j + a] = radial * rh[3 * j + a] + (dr3[a] - proj * rh[3 * j + a]) / d[j];
    }
    free(dl3); free(dl2); free(dl1); free(dD); free(dT); free(dRt); free(dG);
    free(dsw_att); free(dcg); free(dZ); free(dO); free(dQ); free(dK); free(dV); free(dA);
    free(rho); free(ds); free(da2); free(da1); free(drh);
  }

  free(d); free(sw); free(dsw); free(s); free(Rt); free(rh); free(h1); free(h2);
  for (int l = 0; l <= L; ++l) free(G[l]);
  for (int l = 0; l < L; ++l) {
    free(Q[l]); free(K[l]); free(V[l]); free(P[l]); free(Wt[l]); free(rstd[l]);
  }
  free(G); free(Q); free(K); free(V); free(P); free(Wt); free(rstd);
  free(cg); free(Obuf); free(Zbuf); free(T); free(D); free(y1); free(y2); free(y3);
  return e;
}

/* ------------------------------------------------------------------------ */
/* system-level entry points                                                */
/* ------------------------------------------------------------------------ */
static void owrap_all(int n, const double* x, const double* L, double* w) {
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) w[3 * i + a] = owrap(x[3 * i + a], L[a]);
}

/* Neighbour lists of `nc` centre atoms (brute force when use_cells == 0 or
 * the box has fewer than 3 cells of edge rc per direction).  Per centre:
 * total count within rc, and the first nmax entries (j, n) in key order.
 * Unused slots get j = -1. */
int oracle_neighbours(int n, const double* x, const double* box, double rc, int nmax,
                      int nc, const int32_t* centres, int use_cells, int32_t* cnt_in_range,
                      int32_t* nbr_j, int32_t* nbr_img, double* nbr_r) {
  double* w = malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
  owrap_all(n, x, box, w);
  ocells cells;
  int have = use_cells ? ocells_build(&cells, n, w, box, rc) : 0;
#pragma omp parallel for schedule(dynamic, 4)
  for (int q = 0; q < nc; ++q) {
    int i = centres[q];
    onbr* v;
    int c = have ? onbrs_cells(&cells, i, w, box, rc, &v) : onbrs_brute(i, n, w, box, rc, &v);
    cnt_in_range[q] = c;
    for (int k = 0; k < nmax; ++k) {
      size_t o = (size_t)q * nmax + k;
      if (k < c) {
        nbr_j[o] = v[k].j;
        for (int a = 0; a < 3; ++a) {
          nbr_img[3 * o + a] = v[k].n[a];
          if (nbr_r) nbr_r[3 * o + a] = v[k].r[a];
        }
      } else {
        nbr_j[o] = -1;
        for (int a = 0; a < 3; ++a) {
          nbr_img[3 * o + a] = 0;
          if (nbr_r) nbr_r[3 * o + a] = 0.0;
        }
      }
    }
    free(v);
  }
  if (have) ocells_free(&cells);
  free(w);
  return 0;
}

/* Atomic energies and per-pair gradients of `nc` centre atoms.
 * pair_g: nc x nmax x 3 (zero beyond the neighbour count); pair_j: nc x nmax
 * (-1 beyond); desc (nullable): nc x M1*M2.  nthreads <= 0 keeps the default. */
int oracle_af_atoms(const int32_t* idims, const double* fdims, const double* weights, int n,
                    const int32_t* types, const double* x, const double* box, int nc,
                    const int32_t* centres, int nthreads, double* atom_e, double* pair_g,
                    int32_t* pair_j, int32_t* pair_img, double* desc) {
  oaf_model m;
  oaf_weights W;
  oaf_model_from(idims, fdims, &m);
  if (oaf_check(&m)) return -1;
  oaf_bind(&m, weights, &W);
  double* w = malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
  owrap_all(n, x, box, w);
  ocells cells;
  int have = ocells_build(&cells, n, w, box, m.rc);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  size_t ND = (size_t)m.m1 * m.m2;
#pragma omp parallel for schedule(dynamic, 1)
  for (int q = 0; q < nc; ++q) {
    int i = centres[q];
    onbr* v;
    int c = have ? onbrs_cells(&cells, i, w, box, m.rc, &v) : onbrs_brute(i, n, w, box, m.rc, &v);
    int nn = c < m.nmax ? c : m.nmax;
    double* g = pair_g ? pair_g + (size_t)q * m.nmax * 3 : NULL;
    if (g) memset(g, 0, sizeof(double) * m.nmax * 3);
    double e = oaf_atom(&m, &W, types, i, nn, v, g, desc ? desc + (size_t)q * ND : NULL);
    if (atom_e) atom_e[q] = e;
    for (int k = 0; k < m.nmax; ++k) {
      size_t o = (size_t)q * m.nmax + k;
      if (pair_j) pair_j[o] = k < nn ? v[k].j : -1;
      if (pair_img)
        for (int a = 0; a < 3; ++a) pair_img[3 * o + a] = k < nn ? v[k].n[a] : 0;
    }
    free(v);
  }
  if (have) ocells_free(&cells);
  free(w);
  return 0;
}

/* Whole-system energy, forces (n x 3) and virial (3 x 3, row-major), plus
 * atomic energies (nullable).  Sums run in atom order. */
int oracle_af_compute(const int32_t* idims, const double* fdims, const double* weights, int n,
                      const int32_t* types, const double* x, const double* box, int nthreads,
                      double* energy, double* atom_e, double* forces, double* virial) {
  oaf_model m;
  oaf_model_from(idims, fdims, &m);
  if (oaf_check(&m)) return -1;
  int32_t* cen = malloc(sizeof(int32_t) * (n > 0 ? n : 1));
  for (int i = 0; i < n; ++i) cen[i] = i;
  size_t P = (size_t)n * m.nmax;
  double* ae = malloc(sizeof(double) * (n > 0 ? n : 1));
  double* pg = malloc(sizeof(double) * 3 * (P > 0 ? P : 1));
  int32_t* pj = malloc(sizeof(int32_t) * (P > 0 ? P : 1));
  int32_t* pim = malloc(sizeof(int32_t) * 3 * (P > 0 ? P : 1));
  int rc = oracle_af_atoms(idims, fdims, weights, n, types, x, box, n, cen, nthreads, ae, pg, pj,
                           pim, NULL);
  if (rc) goto out;
  double E = 0;
  for (int i = 0; i < n; ++i) E += ae[i];
  if (energy) *energy = E;
  if (atom_e) memcpy(atom_e, ae, sizeof(double) * n);
  if (forces) memset(forces, 0, sizeof(double) * 3 * n);
  double vir[9] = {0};
  double* w = malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
  owrap_all(n, x, box, w);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < m.nmax; ++k) {
      size_t o = (size_t)i * m.nmax + k;
      int j = pj[o];
      if (j < 0) continue;
      double r[3], d2;
      int nn[3] = {pim[3 * o], pim[3 * o + 1], pim[3 * o + 2]};
      osep(w + 3 * i, w + 3 * j, nn, box, r, &d2);
      const double* g = pg + 3 * o;
      if (forces)
        for (int a = 0; a < 3; ++a) {
          forces[3 * i + a] += g[a];
          forces[3 * j + a] -= g[a];
        }
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) vir[3 * a + b] -= r[a] * g[b];
    }
  if (virial) memcpy(virial, vir, sizeof vir);
  free(w);
out:
  free(cen); free(ae); free(pg); free(pj); free(pim);
  return rc;
}

/* eV/(A amu) -> A/fs^2, from CODATA e and amu. */
static double okappa(void) { return 1.602176634e-19 / (1.66053906660e-27 * 1e10); }

/* Velocity-Verlet NVE: v += dt/2 F/m; x += dt v; F(x); v += dt/2 F/m.
 * x, v (n x 3) are updated in place; epot/ekin (nullable) get one entry per
 * step, after the step.  masses: per species (amu). */
int oracle_af_md(const int32_t* idims, const double* fdims, const double* weights, int n,
                 const int32_t* types, const double* masses, const double* box, double* x,
                 double* v, int n_steps, double dt, int nthreads, double* epot, double* ekin) {
  double kap = okappa();
  double* F = malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
  double E;
  int rc = oracle_af_compute(idims, fdims, weights, n, types, x, box, nthreads, &E, NULL, F, NULL);
  if (rc) { free(F); return rc; }
  for (int s = 0; s < n_steps; ++s) {
    for (int i = 0; i < n; ++i) {
      double im = kap / masses[types[i]];
      for (int a = 0; a < 3; ++a) {
        v[3 * i + a] += 0.5 * dt * F[3 * i + a] * im;
        x[3 * i + a] += dt * v[3 * i + a];
      }
    }
    rc = oracle_af_compute(idims, fdims, weights, n, types, x, box, nthreads, &E, NULL, F, NULL);
    if (rc) break;
    double k = 0;
    for (int i = 0; i < n; ++i) {
      double im = kap / masses[types[i]];
      for (int a = 0; a < 3; ++a) {
        v[3 * i + a] += 0.5 * dt * F[3 * i + a] * im;
        k += 0.5 * masses[types[i]] * v[3 * i + a] * v[3 * i + a];
      }
    }
    if (epot) epot[s] = E;
    if (ekin) ekin[s] = k / kap;
  }
  free(F);
  return rc;
}

/* The switch function alone, for its closed-form pins. */
void oracle_switch(double r, double rs, double rc, double* sw, double* dsw) {
  oswitch(r, rs, rc, sw, dsw);
}
