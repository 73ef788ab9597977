/*
 * FP64 CPU oracle of the graph-family deep potential -- TEST INFRASTRUCTURE
 * ONLY (tests, the smoke check and the benchmark's CPU-baseline leg).
 *
 * The paper (Sec. II) describes DPA3 only as a graph neural network with a
 * "Line Graph Series" that carries bond, angle and dihedral representations,
 * followed by the per-atom fitting net; it prints no formula.  The model
 * computed here is a reading written out in full (the dihedral channel is not
 * included):
 *
 *   edges:  the attention family's neighbour list (nearest nmax within rc)
 *   angles: for centre i, the slots p of its list with |r_ip| < rca, at most
 *           na of them (the nearest ones)
 *   init:   n_i = W_type[t_i] (node, width Nd); e_ip = tanh(s_ip w_e + b_e)
 *           (edge, width Ed), s = sw(r)/r with the switch of (rs, rc)
 *   layer:  (a) u_j = n_j Wm; m_i = (1/nmax) sum_p sw_ip (e_ip * u_j(p));
 *               n_i <- n_i + tanh([n_i, m_i] Wn + bn)
 *           (b) e_ip <- e_ip + tanh(n_i Wa + n_j Wb + e_ip Wc + be)   (new n)
 *           (c) q_ik = e_ik Wp;  for p in the angle list of i:
 *               a_ip = sum_l Wphi[l] * (1/na) sum_{k != p} swa_ip swa_ik P_l(c_pk) q_ik,
 *               c_pk = rh_ip . rh_ik, P_l Legendre (l = 0..3), swa the switch
 *               of (rsa, rca); then e_ip <- e_ip + swa_ip tanh(a_ip Wq + bq)
 *               (all a computed before any update)
 *   energy: e_i = fitting_{t_i}(n_i) as in the attention family; E = sum e_i
 *   gradient: by hand in reverse order; F and the virial from g = dE/dr_ip.
 *
 * Weight blob (row-major W[in][out], W before b):
 *   W_type[S][Nd], w_e[1][Ed], b_e[Ed],
 *   for l < L: Wm[Nd][Ed] Wn[Nd+Ed][Nd] bn[Nd] Wa[Nd][Ed] Wb[Nd][Ed] Wc[Ed][Ed]
 *              be[Ed] Wp[Ed][Ed] Wphi[4][Ed] Wq[Ed][Ed] bq[Ed],
 *   for t < S: fitting F1[Nd][f1] c1 F2[f1][f2] c2 F3[f2][f3] c3 F4[f3][1] c4[1]
 */
#include "oracle_common.h"

#ifdef _OPENMP
#include <omp.h>
#endif

#define OGF_MAXS 16
#define OGF_MAXL 16

typedef struct {
  int n_species, nd, ed, n_layers, f1, f2, f3, nmax, na;
  double rc, rs, rca, rsa;
} ogf_model;

typedef struct {
  size_t Wt, we, be0;
  size_t Wm[OGF_MAXL], Wn[OGF_MAXL], bn[OGF_MAXL], Wa[OGF_MAXL], Wb[OGF_MAXL], Wc[OGF_MAXL],
      be[OGF_MAXL], Wp[OGF_MAXL], Wphi[OGF_MAXL], Wq[OGF_MAXL], bq[OGF_MAXL];
  size_t F1[OGF_MAXS], c1[OGF_MAXS], F2[OGF_MAXS], c2[OGF_MAXS], F3[OGF_MAXS], c3[OGF_MAXS],
      F4[OGF_MAXS], c4[OGF_MAXS];
  size_t total;
} ogf_offsets;

static void ogf_model_from(const int32_t* i, const double* f, ogf_model* m) {
  m->n_species = i[0];
  m->nd = i[1];
  m->ed = i[2];
  m->n_layers = i[3];
  m->f1 = i[4];
  m->f2 = i[5];
  m->f3 = i[6];
  m->nmax = i[7];
  m->na = i[8];
  m->rc = f[0];
  m->rs = f[1];
  m->rca = f[2];
  m->rsa = f[3];
}

static int ogf_check(const ogf_model* m) {
  if (m->n_species < 1 || m->n_species > OGF_MAXS) return -1;
  if (m->n_layers < 0 || m->n_layers > OGF_MAXL) return -1;
  if (m->nd < 1 || m->ed < 1 || m->nmax < 1 || m->na < 1) return -1;
  if (!(m->rs < m->rc) || !(m->rsa < m->rca) || m->rca > m->rc) return -1;
  return 0;
}

static void ogf_offsets_of(const ogf_model* m, ogf_offsets* o) {
  size_t off = 0;
  const size_t Nd = m->nd, Ed = m->ed;
#define TAKE(dst, cnt) do { (dst) = off; off += (size_t)(cnt); } while (0)
  TAKE(o->Wt, (size_t)m->n_species * Nd);
  TAKE(o->we, Ed);
  TAKE(o->be0, Ed);
  for (int l = 0; l < m->n_layers; ++l) {
    TAKE(o->Wm[l], Nd * Ed);
    TAKE(o->Wn[l], (Nd + Ed) * Nd);
    TAKE(o->bn[l], Nd);
    TAKE(o->Wa[l], Nd * Ed);
    TAKE(o->Wb[l], Nd * Ed);
    TAKE(o->Wc[l], Ed * Ed);
    TAKE(o->be[l], Ed);
    TAKE(o->Wp[l], Ed * Ed);
    TAKE(o->Wphi[l], 4 * Ed);
    TAKE(o->Wq[l], Ed * Ed);
    TAKE(o->bq[l], Ed);
  }
  for (int t = 0; t < m->n_species; ++t) {
    TAKE(o->F1[t], Nd * m->f1);
    TAKE(o->c1[t], m->f1);
    TAKE(o->F2[t], (size_t)m->f1 * m->f2);
    TAKE(o->c2[t], m->f2);
    TAKE(o->F3[t], (size_t)m->f2 * m->f3);
    TAKE(o->c3[t], m->f3);
    TAKE(o->F4[t], m->f3);
    TAKE(o->c4[t], 1);
  }
#undef TAKE
  o->total = off;
}

long long oracle_gf_weight_count(const int32_t* idims, const double* fdims) {
  ogf_model m;
  ogf_offsets o;
  ogf_model_from(idims, fdims, &m);
  if (ogf_check(&m)) return -1;
  ogf_offsets_of(&m, &o);
  return (long long)o.total;
}

/* kind: 0 W_type, 1 w_e, 2 b_e; 10..20 = Wm Wn bn Wa Wb Wc be Wp Wphi Wq bq of
 * layer a; 30..37 = fitting F1 c1 F2 c2 F3 c3 F4 c4 of species a. */
long long oracle_gf_weight_offset(const int32_t* idims, const double* fdims, int kind, int a) {
  ogf_model m;
  ogf_offsets o;
  ogf_model_from(idims, fdims, &m);
  if (ogf_check(&m) || a < 0) return -1;
  ogf_offsets_of(&m, &o);
  const int L = m.n_layers, S = m.n_species;
  switch (kind) {
    case 0: return (long long)o.Wt;
    case 1: return (long long)o.we;
    case 2: return (long long)o.be0;
    case 10: return a < L ? (long long)o.Wm[a] : -1;
    case 11: return a < L ? (long long)o.Wn[a] : -1;
    case 12: return a < L ? (long long)o.bn[a] : -1;
    case 13: return a < L ? (long long)o.Wa[a] : -1;
    case 14: return a < L ? (long long)o.Wb[a] : -1;
    case 15: return a < L ? (long long)o.Wc[a] : -1;
    case 16: return a < L ? (long long)o.be[a] : -1;
    case 17: return a < L ? (long long)o.Wp[a] : -1;
    case 18: return a < L ? (long long)o.Wphi[a] : -1;
    case 19: return a < L ? (long long)o.Wq[a] : -1;
    case 20: return a < L ? (long long)o.bq[a] : -1;
    case 30: return a < S ? (long long)o.F1[a] : -1;
    case 31: return a < S ? (long long)o.c1[a] : -1;
    case 32: return a < S ? (long long)o.F2[a] : -1;
    case 33: return a < S ? (long long)o.c2[a] : -1;
    case 34: return a < S ? (long long)o.F3[a] : -1;
    case 35: return a < S ? (long long)o.c3[a] : -1;
    case 36: return a < S ? (long long)o.F4[a] : -1;
    case 37: return a < S ? (long long)o.c4[a] : -1;
    default: return -1;
  }
}

/* Legendre polynomials P_0..P_3 and their derivatives at c */
static void olegendre(double c, double* P, double* dP) {
  P[0] = 1.0;
  P[1] = c;
  P[2] = 0.5 * (3.0 * c * c - 1.0);
  P[3] = 0.5 * (5.0 * c * c * c - 3.0 * c);
  dP[0] = 0.0;
  dP[1] = 1.0;
  dP[2] = 3.0 * c;
  dP[3] = 0.5 * (15.0 * c * c - 3.0);
}

/* y[out] = x[in] W[in][out] (+= when acc) */
static void ovecmat(const double* x, const double* W, int in, int out, double* y, int acc) {
  for (int c = 0; c < out; ++c) {
    double s = acc ? y[c] : 0.0;
    for (int a = 0; a < in; ++a) s += x[a] * W[(size_t)a * out + c];
    y[c] = s;
  }
}
/* y[in] += dy[out] W^T */
static void ovecmatT(const double* dy, const double* W, int in, int out, double* y) {
  for (int a = 0; a < in; ++a) {
    double s = 0.0;
    for (int c = 0; c < out; ++c) s += dy[c] * W[(size_t)a * out + c];
    y[a] += s;
  }
}

/* E = sum_i seed_i e_i (seed NULL: all ones), atomic energies e_i, forces
 * -dE/dx and virial.  A seed of 0 makes an atom a ghost: its features are
 * computed (its neighbours need them) but its energy is not counted. */
static int gf_compute(const int32_t* idims, const double* fdims, const double* w, int n,
                      const int32_t* types, const double* x, const double* box, int nthreads,
                      const double* seed, double* energy, double* atom_e, double* forces,
                      double* virial) {
  ogf_model m;
  ogf_offsets o;
  ogf_model_from(idims, fdims, &m);
  if (ogf_check(&m)) return -1;
  ogf_offsets_of(&m, &o);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  const int Nd = m.nd, Ed = m.ed, L = m.n_layers, NM = m.nmax, NA = m.na;
  const size_t N = n > 0 ? n : 1;
  const double inv_nmax = 1.0 / NM, inv_na = 1.0 / NA;

  /* ---- neighbours (nearest nmax within rc), geometry per edge */
  double* wr = malloc(sizeof(double) * 3 * N);
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) wr[3 * i + a] = owrap(x[3 * i + a], box[a]);
  ocells cells;
  int have = ocells_build(&cells, n, wr, box, m.rc);
  int* cnt = calloc(N, sizeof(int));
  int* nang = calloc(N, sizeof(int));
  int* nbj = malloc(sizeof(int) * N * NM);
  double* rv = calloc(N * NM * 3, sizeof(double));
  double* dd = calloc(N * NM, sizeof(double));
  double *sw = calloc(N * NM, sizeof(double)), *dsw = calloc(N * NM, sizeof(double));
  double *sa = calloc(N * NM, sizeof(double)), *dsa = calloc(N * NM, sizeof(double));
  double* sv = calloc(N * NM, sizeof(double));
  double* rh = calloc(N * NM * 3, sizeof(double));
#pragma omp parallel for schedule(dynamic, 4)
  for (int i = 0; i < n; ++i) {
    onbr* v;
    int c = have ? onbrs_cells(&cells, i, wr, box, m.rc, &v) : onbrs_brute(i, n, wr, box, m.rc, &v);
    int k = c < NM ? c : NM;
    cnt[i] = k;
    int na = 0;
    for (int p = 0; p < NM; ++p) {
      size_t e = (size_t)i * NM + p;
      nbj[e] = p < k ? v[p].j : -1;
      if (p >= k) continue;
      double d = sqrt(v[p].d2);
      dd[e] = d;
      for (int a = 0; a < 3; ++a) {
        rv[3 * e + a] = v[p].r[a];
        rh[3 * e + a] = v[p].r[a] / d;
      }
      oswitch(d, m.rs, m.rc, &sw[e], &dsw[e]);
      sv[e] = sw[e] / d;
      if (d < m.rca && na < NA) {
        oswitch(d, m.rsa, m.rca, &sa[e], &dsa[e]);
        ++na;
      }
    }
    nang[i] = na;  /* the angle slots are 0 .. na-1 (nearest first) */
    free(v);
  }
  if (have) ocells_free(&cells);

  /* ---- forward, keeping every layer's states */
  const size_t EN = N * NM * Ed;
  double** nn = malloc(sizeof(double*) * (L + 1));   /* n at layer input / final */
  double** n1 = malloc(sizeof(double*) * (L > 0 ? L : 1));  /* n after (a) */
  double** ee = malloc(sizeof(double*) * (L + 1));   /* e at layer input / final */
  double** e1 = malloc(sizeof(double*) * (L > 0 ? L : 1));  /* e after (b) */
  double** hh = malloc(sizeof(double*) * (L > 0 ? L : 1));  /* tanh of (a) */
  double** mm = malloc(sizeof(double*) * (L > 0 ? L : 1));  /* messages m_i */
  double** vv = malloc(sizeof(double*) * (L > 0 ? L : 1));  /* tanh of (b) */
  double** qq = malloc(sizeof(double*) * (L > 0 ? L : 1));  /* q = e1 Wp */
  double** tt = malloc(sizeof(double*) * (L > 0 ? L : 1));  /* tanh of (c) */
  double** uu = malloc(sizeof(double*) * (L > 0 ? L : 1));  /* u = n Wm */
  for (int l = 0; l <= L; ++l) {
    nn[l] = calloc(N * Nd, sizeof(double));
    ee[l] = calloc(EN, sizeof(double));
  }
  for (int l = 0; l < L; ++l) {
    n1[l] = calloc(N * Nd, sizeof(double));
    e1[l] = calloc(EN, sizeof(double));
    hh[l] = calloc(N * Nd, sizeof(double));
    mm[l] = calloc(N * Ed, sizeof(double));
    vv[l] = calloc(EN, sizeof(double));
    qq[l] = calloc(EN, sizeof(double));
    tt[l] = calloc(EN, sizeof(double));
    uu[l] = calloc(N * Ed, sizeof(double));
  }
  for (int i = 0; i < n; ++i) {
    for (int c = 0; c < Nd; ++c) nn[0][(size_t)i * Nd + c] = w[o.Wt + (size_t)types[i] * Nd + c];
    for (int p = 0; p < cnt[i]; ++p) {
      size_t e = (size_t)i * NM + p;
      for (int c = 0; c < Ed; ++c) ee[0][e * Ed + c] = tanh(sv[e] * w[o.we + c] + w[o.be0 + c]);
    }
  }
  double* xin = malloc(sizeof(double) * (Nd + Ed));
  for (int l = 0; l < L; ++l) {
    const double *Wm = w + o.Wm[l], *Wn = w + o.Wn[l], *bn = w + o.bn[l], *Wa = w + o.Wa[l],
                 *Wb = w + o.Wb[l], *Wc = w + o.Wc[l], *be = w + o.be[l], *Wp = w + o.Wp[l],
                 *Wphi = w + o.Wphi[l], *Wq = w + o.Wq[l], *bq = w + o.bq[l];
    /* (a) */
    for (int j = 0; j < n; ++j) ovecmat(nn[l] + (size_t)j * Nd, Wm, Nd, Ed, uu[l] + (size_t)j * Ed, 0);
    for (int i = 0; i < n; ++i) {
      double* mi = mm[l] + (size_t)i * Ed;
      for (int p = 0; p < cnt[i]; ++p) {
        size_t e = (size_t)i * NM + p;
        const double* uj = uu[l] + (size_t)nbj[e] * Ed;
        for (int c = 0; c < Ed; ++c) mi[c] += inv_nmax * sw[e] * ee[l][e * Ed + c] * uj[c];
      }
      memcpy(xin, nn[l] + (size_t)i * Nd, sizeof(double) * Nd);
      memcpy(xin + Nd, mi, sizeof(double) * Ed);
      double* hi = hh[l] + (size_t)i * Nd;
      ovecmat(xin, Wn, Nd + Ed, Nd, hi, 0);
      for (int c = 0; c < Nd; ++c) {
        hi[c] = tanh(hi[c] + bn[c]);
        n1[l][(size_t)i * Nd + c] = nn[l][(size_t)i * Nd + c] + hi[c];
      }
    }
    /* (b) */
    double* tmp = malloc(sizeof(double) * Ed);
    for (int i = 0; i < n; ++i)
      for (int p = 0; p < cnt[i]; ++p) {
        size_t e = (size_t)i * NM + p;
        const double* ni = n1[l] + (size_t)i * Nd;
        const double* nj = n1[l] + (size_t)nbj[e] * Nd;
        ovecmat(ni, Wa, Nd, Ed, tmp, 0);
        ovecmat(nj, Wb, Nd, Ed, tmp, 1);
        ovecmat(ee[l] + e * Ed, Wc, Ed, Ed, tmp, 1);
        for (int c = 0; c < Ed; ++c) {
          double v = tanh(tmp[c] + be[c]);
          vv[l][e * Ed + c] = v;
          e1[l][e * Ed + c] = ee[l][e * Ed + c] + v;
        }
      }
    /* (c) */
    memcpy(ee[l + 1], e1[l], sizeof(double) * EN);
    for (int i = 0; i < n; ++i) {
      for (int k = 0; k < nang[i]; ++k) {
        size_t e = (size_t)i * NM + k;
        ovecmat(e1[l] + e * Ed, Wp, Ed, Ed, qq[l] + e * Ed, 0);
      }
      for (int p = 0; p < nang[i]; ++p) {
        size_t ep = (size_t)i * NM + p;
        double* a = calloc(Ed, sizeof(double));
        for (int k = 0; k < nang[i]; ++k) {
          if (k == p) continue;
          size_t ek = (size_t)i * NM + k;
          double cpk = rh[3 * ep] * rh[3 * ek] + rh[3 * ep + 1] * rh[3 * ek + 1] + rh[3 * ep + 2] * rh[3 * ek + 2];
          double P[4], dP[4];
          olegendre(cpk, P, dP);
          for (int ll = 0; ll < 4; ++ll) {
            double coef = inv_na * sa[ep] * sa[ek] * P[ll];
            for (int c = 0; c < Ed; ++c) a[c] += Wphi[ll * Ed + c] * coef * qq[l][ek * Ed + c];
          }
        }
        ovecmat(a, Wq, Ed, Ed, tmp, 0);
        for (int c = 0; c < Ed; ++c) {
          double t = tanh(tmp[c] + bq[c]);
          tt[l][ep * Ed + c] = t;
          ee[l + 1][ep * Ed + c] = e1[l][ep * Ed + c] + sa[ep] * t;
        }
        free(a);
      }
    }
    free(tmp);
    memcpy(nn[l + 1], n1[l], sizeof(double) * N * Nd);
  }

  /* ---- fitting forward and backward per atom */
  double* dn = calloc(N * Nd, sizeof(double));
  double* ae = calloc(N, sizeof(double));
  const int F1 = m.f1, F2 = m.f2, F3 = m.f3;
  for (int i = 0; i < n; ++i) {
    int t = types[i];
    const double* xi = nn[L] + (size_t)i * Nd;
    double* y1 = malloc(sizeof(double) * F1);
    double* y2 = malloc(sizeof(double) * F2);
    double* y3 = malloc(sizeof(double) * F3);
    ovecmat(xi, w + o.F1[t], Nd, F1, y1, 0);
    for (int b = 0; b < F1; ++b) y1[b] = tanh(y1[b] + w[o.c1[t] + b]);
    ovecmat(y1, w + o.F2[t], F1, F2, y2, 0);
    for (int b = 0; b < F2; ++b) y2[b] = tanh(y2[b] + w[o.c2[t] + b]);
    ovecmat(y2, w + o.F3[t], F2, F3, y3, 0);
    double e = w[o.c4[t]];
    for (int b = 0; b < F3; ++b) {
      y3[b] = tanh(y3[b] + w[o.c3[t] + b]);
      e += y3[b] * w[o.F4[t] + b];
    }
    ae[i] = e;
    double* d3 = malloc(sizeof(double) * F3);
    double* d2 = calloc(F2, sizeof(double));
    double* d1 = calloc(F1, sizeof(double));
    const double sd = seed ? seed[i] : 1.0;
    for (int b = 0; b < F3; ++b) d3[b] = sd * w[o.F4[t] + b] * (1.0 - y3[b] * y3[b]);
    ovecmatT(d3, w + o.F3[t], F2, F3, d2);
    for (int b = 0; b < F2; ++b) d2[b] *= 1.0 - y2[b] * y2[b];
    ovecmatT(d2, w + o.F2[t], F1, F2, d1);
    for (int b = 0; b < F1; ++b) d1[b] *= 1.0 - y1[b] * y1[b];
    ovecmatT(d1, w + o.F1[t], Nd, F1, dn + (size_t)i * Nd);
    free(y1); free(y2); free(y3); free(d3); free(d2); free(d1);
  }
  double E = 0.0;
  for (int i = 0; i < n; ++i) E += seed ? seed[i] * ae[i] : ae[i];
  if (energy) *energy = E;
  if (atom_e) memcpy(atom_e, ae, sizeof(double) * n);

  /* ---- backward through the layers */
  double* de = calloc(EN, sizeof(double));      /* d/d e (current layer output) */
  double* dsw_e = calloc(N * NM, sizeof(double));
  double* dsa_e = calloc(N * NM, sizeof(double));
  double* drh = calloc(N * NM * 3, sizeof(double));
  double* tmp = malloc(sizeof(double) * (Nd + Ed));
  double* dn1 = calloc(N * Nd, sizeof(double));
  double* de1 = calloc(EN, sizeof(double));
  double* du = calloc(N * Ed, sizeof(double));
  double* dq = calloc(EN, sizeof(double));
  double* dz = malloc(sizeof(double) * Ed);
  double* da = malloc(sizeof(double) * Ed);
  double* dy = malloc(sizeof(double) * Ed);
  double* dx = malloc(sizeof(double) * Nd);
  for (int l = L - 1; l >= 0; --l) {
    const double *Wm = w + o.Wm[l], *Wn = w + o.Wn[l], *Wa = w + o.Wa[l], *Wb = w + o.Wb[l],
                 *Wc = w + o.Wc[l], *Wp = w + o.Wp[l], *Wphi = w + o.Wphi[l], *Wq = w + o.Wq[l];
    /* (c): e_out = e1 + swa tanh(a Wq + bq) on angle slots */
    memcpy(de1, de, sizeof(double) * EN);
    memset(dq, 0, sizeof(double) * EN);
    for (int i = 0; i < n; ++i) {
      for (int p = 0; p < nang[i]; ++p) {
        size_t ep = (size_t)i * NM + p;
        double dsa_acc = 0.0;
        for (int c = 0; c < Ed; ++c) {
          double t = tt[l][ep * Ed + c];
          dsa_acc += de[ep * Ed + c] * t;
          dz[c] = de[ep * Ed + c] * sa[ep] * (1.0 - t * t);
        }
        dsa_e[ep] += dsa_acc;
        memset(da, 0, sizeof(double) * Ed);
        ovecmatT(dz, Wq, Ed, Ed, da);
        for (int k = 0; k < nang[i]; ++k) {
          if (k == p) continue;
          size_t ek = (size_t)i * NM + k;
          double cpk = rh[3 * ep] * rh[3 * ek] + rh[3 * ep + 1] * rh[3 * ek + 1] + rh[3 * ep + 2] * rh[3 * ek + 2];
          double P[4], dP[4];
          olegendre(cpk, P, dP);
          for (int ll = 0; ll < 4; ++ll) {
            double base = inv_na * sa[ep] * sa[ek];
            double dcoef = 0.0;
            for (int c = 0; c < Ed; ++c) {
              double wq = Wphi[ll * Ed + c] * qq[l][ek * Ed + c];
              dcoef += da[c] * wq;
              dq[ek * Ed + c] += da[c] * Wphi[ll * Ed + c] * base * P[ll];
            }
            dsa_e[ep] += dcoef * inv_na * sa[ek] * P[ll];
            dsa_e[ek] += dcoef * inv_na * sa[ep] * P[ll];
            double dc = dcoef * base * dP[ll];
            for (int a3 = 0; a3 < 3; ++a3) {
              drh[3 * ep + a3] += dc * rh[3 * ek + a3];
              drh[3 * ek + a3] += dc * rh[3 * ep + a3];
            }
          }
        }
      }
      for (int k = 0; k < nang[i]; ++k) {
        size_t ek = (size_t)i * NM + k;
        ovecmatT(dq + ek * Ed, Wp, Ed, Ed, de1 + ek * Ed);
      }
    }
    /* (b): e1 = e + tanh(n1_i Wa + n1_j Wb + e Wc + be) */
    memcpy(dn1, dn, sizeof(double) * N * Nd);
    memcpy(de, de1, sizeof(double) * EN);
    for (int i = 0; i < n; ++i)
      for (int p = 0; p < cnt[i]; ++p) {
        size_t e = (size_t)i * NM + p;
        for (int c = 0; c < Ed; ++c) {
          double v = vv[l][e * Ed + c];
          dy[c] = de1[e * Ed + c] * (1.0 - v * v);
        }
        ovecmatT(dy, Wa, Nd, Ed, dn1 + (size_t)i * Nd);
        ovecmatT(dy, Wb, Nd, Ed, dn1 + (size_t)nbj[e] * Nd);
        ovecmatT(dy, Wc, Ed, Ed, de + e * Ed);
      }
    /* (a): n1 = n + tanh([n, m] Wn + bn), m_i = (1/nmax) sum sw e (n_j Wm) */
    memcpy(dn, dn1, sizeof(double) * N * Nd);
    memset(du, 0, sizeof(double) * N * Ed);
    for (int i = 0; i < n; ++i) {
      const double* hi = hh[l] + (size_t)i * Nd;
      for (int c = 0; c < Nd; ++c) dx[c] = dn1[(size_t)i * Nd + c] * (1.0 - hi[c] * hi[c]);
      memset(tmp, 0, sizeof(double) * (Nd + Ed));
      ovecmatT(dx, Wn, Nd + Ed, Nd, tmp);
      for (int c = 0; c < Nd; ++c) dn[(size_t)i * Nd + c] += tmp[c];
      const double* dm = tmp + Nd;
      for (int p = 0; p < cnt[i]; ++p) {
        size_t e = (size_t)i * NM + p;
        int j = nbj[e];
        const double* uj = uu[l] + (size_t)j * Ed;
        double acc = 0.0;
        for (int c = 0; c < Ed; ++c) {
          de[e * Ed + c] += inv_nmax * sw[e] * dm[c] * uj[c];
          du[(size_t)j * Ed + c] += inv_nmax * sw[e] * dm[c] * ee[l][e * Ed + c];
          acc += dm[c] * ee[l][e * Ed + c] * uj[c];
        }
        dsw_e[e] += inv_nmax * acc;
      }
    }
    for (int j = 0; j < n; ++j) ovecmatT(du + (size_t)j * Ed, Wm, Nd, Ed, dn + (size_t)j * Nd);
  }
  /* ---- edge init e = tanh(s w_e + b_e), then g per edge */
  double* vir = calloc(9, sizeof(double));
  if (forces) memset(forces, 0, sizeof(double) * 3 * n);
  for (int i = 0; i < n; ++i)
    for (int p = 0; p < cnt[i]; ++p) {
      size_t e = (size_t)i * NM + p;
      double ds = 0.0;
      for (int c = 0; c < Ed; ++c) {
        double e0 = ee[0][e * Ed + c];
        ds += de[e * Ed + c] * (1.0 - e0 * e0) * w[o.we + c];
      }
      double d = dd[e];
      double radial = ds * (dsw[e] / d - sw[e] / (d * d)) + dsw_e[e] * dsw[e] + dsa_e[e] * dsa[e];
      const double* r = rh + 3 * e;
      double proj = drh[3 * e] * r[0] + drh[3 * e + 1] * r[1] + drh[3 * e + 2] * r[2];
      double g[3];
      for (int a = 0; a < 3; ++a) g[a] = radial * r[a] + (drh[3 * e + a] - proj * r[a]) / d;
      int j = nbj[e];
      if (forces)
        for (int a = 0; a < 3; ++a) {
          forces[3 * i + a] += g[a];
          forces[3 * j + a] -= g[a];
        }
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) vir[3 * a + b] -= rv[3 * e + a] * g[b];
    }
  if (virial) memcpy(virial, vir, sizeof(double) * 9);

  free(vir); free(tmp); free(dn1); free(de1); free(du); free(dq); free(dz); free(da); free(dy);
  free(dx); free(de); free(dsw_e); free(dsa_e); free(drh); free(dn); free(ae); free(xin);
  for (int l = 0; l <= L; ++l) { free(nn[l]); free(ee[l]); }
  for (int l = 0; l < L; ++l) {
    free(n1[l]); free(e1[l]); free(hh[l]); free(mm[l]); free(vv[l]); free(qq[l]); free(tt[l]);
    free(uu[l]);
  }
  free(nn); free(n1); free(ee); free(e1); free(hh); free(mm); free(vv); free(qq); free(tt); free(uu);
  free(wr); free(cnt); free(nang); free(nbj); free(rv); free(dd); free(sw); free(dsw); free(sa);
  free(dsa); free(sv); free(rh);
  return 0;
}

int oracle_gf_compute(const int32_t* idims, const double* fdims, const double* w, int n,
                      const int32_t* types, const double* x, const double* box, int nthreads,
                      double* energy, double* atom_e, double* forces, double* virial) {
  return gf_compute(idims, fdims, w, n, types, x, box, nthreads, NULL, energy, atom_e, forces,
                    virial);
}

int oracle_gf_compute_seeded(const int32_t* idims, const double* fdims, const double* w, int n,
                             const int32_t* types, const double* x, const double* box,
                             int nthreads, const double* seed, double* energy, double* atom_e,
                             double* forces, double* virial) {
  return gf_compute(idims, fdims, w, n, types, x, box, nthreads, seed, energy, atom_e, forces,
                    virial);
}
