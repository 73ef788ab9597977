// Runtime of libdp: context, device buffers, neighbour-list maintenance, the
// CUDA-graph-captured MD step, and the C ABI declared in include/dp.h.
//
// The paper (Sec. III) couples an MD engine to the deep-potential library
// through a C++ interface that passes atom data in and forces out; its
// characterisation (Sec. V-B, Table II) finds thousands of kernel launches per
// MD step and recommends CUDA graphs.  Here every dp_step is one graph launch
// whose nodes are the library's own kernels; positions, velocities and
// neighbour lists stay resident on the device between steps.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "model.h"

using namespace dp;

struct dp_ctx {
  dp_model_desc desc{};
  AfDims af{};
  int n = 0;
  int n_sys = 1;
  double box[3] = {0, 0, 0};
  double rskin = 0, skin = 0;
  int rebuild_every = 10;
  int cap = 0;
  int ncell = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::string err;
  size_t bytes = 0;
  std::vector<void*> allocs;
  std::vector<int> types_host;
  std::vector<double> mass_species;
  bool have_masses = false;
  // device state
  double *x = nullptr, *v = nullptr, *F = nullptr, *xref = nullptr, *w = nullptr;
  double *minv = nullptr, *mass = nullptr;
  int* fl = nullptr;
  int* types = nullptr;
  int* sys_of = nullptr;
  int* sys_atom0 = nullptr;
  SysInfo* sys = nullptr;
  int *cell_of = nullptr, *cell_cnt = nullptr, *cell_fill = nullptr, *cell_start = nullptr,
      *cell_idx = nullptr;
  SkinEntry* skin_list = nullptr;
  int *skin_cnt = nullptr, *mirror = nullptr;
  short* selpos = nullptr;
  int *sel_j = nullptr, *sel_img = nullptr, *n_in_rc = nullptr;
  double* sel_r = nullptr;
  double *atom_e = nullptr, *atom_vir = nullptr, *sys_e = nullptr, *sys_vir = nullptr;
  int* flags = nullptr;
  long long* step = nullptr;   // [0] step counter, [1] trace base
  double* trace = nullptr;
  int trace_len = 0;
  // skin-list buffers are reallocated when the capacity grows
  std::vector<void*> skin_allocs;
  // network
  Model* model = nullptr;
  // graph of one MD step
  cudaGraphExec_t graph = nullptr;
  double graph_dt = 0;
  int graph_trace_len = 0;
  bool forces_valid = false;
  int kernels_compute = 0, kernels_step = 0;
};

static thread_local std::string g_init_error;

static int fail(dp_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  else g_init_error = msg;
  return code;
}

static int cuda_fail(dp_ctx* c, cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(c, DP_ERR_OOM, std::string(where) + ": out of device memory");
  }
  return fail(c, DP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(c, expr, where)                        \
  do {                                                  \
    cudaError_t e__ = (expr);                           \
    if (e__ != cudaSuccess) return cuda_fail(c, e__, where); \
  } while (0)

template <typename T>
static cudaError_t dalloc(dp_ctx* c, T** p, size_t count, std::vector<void*>* list = nullptr) {
  size_t b = sizeof(T) * (count > 0 ? count : 1);
  cudaError_t e = cudaMalloc((void**)p, b);
  if (e == cudaSuccess) {
    (list ? list : &c->allocs)->push_back((void*)*p);
    c->bytes += b;
    e = cudaMemsetAsync(*p, 0, b, c->st);
  }
  return e;
}

// ------------------------------------------------------------------ validation
static int check_desc(const dp_model_desc* d, std::string* why) {
  if (!d) { *why = "desc is NULL"; return -1; }
  if (d->family != DP_FAMILY_ATTENTION && d->family != DP_FAMILY_GRAPH) { *why = "unknown family"; return -1; }
  if (d->n_species < 1 || d->n_species > 64) { *why = "n_species must be 1..64"; return -1; }
  if (d->nmax < 1 || d->nmax > 256) { *why = "nmax must be 1..256"; return -1; }
  if (!(d->rcut > 0) || !(d->rcut_smth >= 0) || !(d->rcut_smth < d->rcut)) { *why = "need 0 <= rcut_smth < rcut"; return -1; }
  if (d->f1 < 1 || d->f2 < 1 || d->f3 < 1) { *why = "fitting widths must be positive"; return -1; }
  if (d->family == DP_FAMILY_ATTENTION) {
    if (d->e1 < 1 || d->e2 < 1 || d->m1 < 1 || d->m2 < 1 || d->m2 > d->m1) { *why = "embedding sizes invalid (need m2 <= m1)"; return -1; }
    if (d->n_layers < 0 || d->n_layers > 16) { *why = "n_layers must be 0..16"; return -1; }
    if (d->n_layers > 0 && (d->heads < 1 || d->hidden < 1 || d->hidden % d->heads)) { *why = "hidden must be a multiple of heads"; return -1; }
  }
  if (d->precision < DP_PREC_PLAIN_F64 || d->precision > DP_PREC_FUSED_BF16) { *why = "unknown precision"; return -1; }
  return 0;
}

extern "C" int dp_weight_count(const dp_model_desc* d, size_t* n) {
  std::string why;
  if (!n) return fail(nullptr, DP_ERR_ARG, "n is NULL");
  if (check_desc(d, &why)) return fail(nullptr, DP_ERR_ARG, why);
  if (d->family == DP_FAMILY_GRAPH) return fail(nullptr, DP_ERR_UNSUPPORTED, "graph family not available in this build");
  size_t S = d->n_species, E1 = d->e1, E2 = d->e2, M1 = d->m1, M2 = d->m2, H = d->hidden;
  size_t t = S * (E1 + E1 + E1 * E2 + E2 + E2 * M1 + M1);
  t += (size_t)d->n_layers * (3 * M1 * H + H * M1 + M1);
  t += S * (M1 * M2 * d->f1 + d->f1 + (size_t)d->f1 * d->f2 + d->f2 + (size_t)d->f2 * d->f3 + d->f3 + d->f3 + 1);
  *n = t;
  return DP_OK;
}

// ------------------------------------------------------------------ systems
static void make_sysinfo(const double* L, double rskin, int atom0, int natom, int cell0,
                         SysInfo* s, int* ncell) {
  memset(s, 0, sizeof *s);
  s->atom0 = atom0;
  s->natom = natom;
  s->cell0 = cell0;
  s->use_cells = 1;
  for (int a = 0; a < 3; ++a) {
    s->L[a] = L[a];
    s->nc[a] = (int)floor(L[a] / rskin);
    if (s->nc[a] < 3) s->use_cells = 0;
    s->nimg[a] = (int)ceil(rskin / L[a]) + 1;
  }
  if (s->use_cells) {
    for (int a = 0; a < 3; ++a) s->cs[a] = L[a] / s->nc[a];
    *ncell = s->nc[0] * s->nc[1] * s->nc[2];
  } else {
    for (int a = 0; a < 3; ++a) { s->nc[a] = 1; s->cs[a] = L[a]; }
    *ncell = 0;
  }
}

static int alloc_skin(dp_ctx* c, int cap) {
  if (cap > select_max_cap())
    return fail(c, DP_ERR_NLIST_OVERFLOW,
                "more than " + std::to_string(select_max_cap()) + " atoms within rc + skin of one atom");
  for (void* p : c->skin_allocs) cudaFree(p);
  c->skin_allocs.clear();
  c->cap = cap;
  size_t e = (size_t)c->n * cap;
  CUDA_TRY(c, dalloc(c, &c->skin_list, e, &c->skin_allocs), "skin list");
  CUDA_TRY(c, dalloc(c, &c->mirror, e, &c->skin_allocs), "skin mirror");
  CUDA_TRY(c, dalloc(c, &c->selpos, e, &c->skin_allocs), "skin selpos");
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return DP_OK;
}

static NlistArgs nlist_args(dp_ctx* c) {
  NlistArgs a{};
  a.n = c->n; a.ncell = c->ncell; a.cap = c->cap; a.nmax = c->desc.nmax;
  a.rc = c->desc.rcut; a.rskin = c->rskin;
  a.x = c->x; a.xref = c->xref; a.w = c->w; a.fl = c->fl;
  a.sys_of = c->sys_of; a.sys = c->sys;
  a.cell_of = c->cell_of; a.cell_cnt = c->cell_cnt; a.cell_fill = c->cell_fill;
  a.cell_start = c->cell_start; a.cell_idx = c->cell_idx;
  a.skin = c->skin_list; a.skin_cnt = c->skin_cnt; a.mirror = c->mirror;
  a.sel_j = c->sel_j; a.sel_img = c->sel_img; a.sel_r = c->sel_r; a.selpos = c->selpos;
  a.n_in_rc = c->n_in_rc; a.flags = c->flags;
  return a;
}

static MdArgs md_args(dp_ctx* c, double dt) {
  MdArgs m{};
  m.n = c->n; m.dt = dt; m.x = c->x; m.v = c->v; m.F = c->F; m.minv = c->minv; m.mass = c->mass;
  m.xref = c->xref; m.half_skin2 = 0.25 * c->skin * c->skin; m.rebuild_every = c->rebuild_every;
  m.step = c->step; m.flags = c->flags; m.n_sys = c->n_sys; m.sys_atom0 = c->sys_atom0;
  m.sys_of = c->sys_of;
  return m;
}

// One evaluation on the stream: neighbours (rebuild if flagged), model, forces,
// reductions.  Returns the number of kernels it launched.
static int enqueue_compute(dp_ctx* c) {
  NlistArgs na = nlist_args(c);
  int k = 0;
  launch_wrap(na, c->st); ++k;
  launch_nlist_rebuild(na, c->st); k += nlist_rebuild_kernels();
  launch_select(na, c->st); ++k;
  ForceArgs fa{};
  fa.n = c->n; fa.nmax = c->desc.nmax; fa.cap = c->cap; fa.sel_j = c->sel_j; fa.sel_r = c->sel_r;
  fa.skin = c->skin_list; fa.skin_cnt = c->skin_cnt; fa.mirror = c->mirror; fa.selpos = c->selpos;
  fa.F = c->F; fa.atom_vir = c->atom_vir;
  k += c->model->run(c->sel_j, c->sel_r, c->types, c->atom_e, c->st);
  fa.g32 = c->model->grad32();
  fa.g64 = c->model->grad64();
  launch_force_gather(fa, c->st); ++k;
  ReduceArgs ra{};
  ra.n_sys = c->n_sys; ra.sys_atom0 = c->sys_atom0; ra.atom_e = c->atom_e; ra.atom_vir = c->atom_vir;
  ra.F = c->F; ra.sys_e = c->sys_e; ra.sys_vir = c->sys_vir; ra.flags = c->flags;
  launch_reduce(ra, c->st); ++k;
  return k;
}

static int read_flags(dp_ctx* c, int* out) {
  CUDA_TRY(c, cudaMemcpyAsync(out, c->flags, sizeof(int), cudaMemcpyDeviceToHost, c->st), "flags");
  CUDA_TRY(c, cudaStreamSynchronize(c->st), "synchronize");
  return DP_OK;
}

static int clear_flags(dp_ctx* c, int bits) {
  launch_flag_set(c->flags, 0, c->st);
  (void)bits;
  int zero = 0;
  CUDA_TRY(c, cudaMemcpyAsync(c->flags, &zero, sizeof(int), cudaMemcpyHostToDevice, c->st), "flags");
  CUDA_TRY(c, cudaStreamSynchronize(c->st), "synchronize");
  return DP_OK;
}

// Evaluate at the resident positions with a fresh neighbour build; grows the
// skin capacity and retries on overflow.
static int compute_now(dp_ctx* c) {
  for (int attempt = 0; attempt < 4; ++attempt) {
    int rc = clear_flags(c, ~0);
    if (rc) return rc;
    launch_flag_set(c->flags, kFlagRebuild, c->st);
    c->kernels_compute = enqueue_compute(c) + 1;
    CUDA_TRY(c, cudaGetLastError(), "launch");
    int fl = 0;
    rc = read_flags(c, &fl);
    if (rc) return rc;
    if (fl & kFlagOverflow) {
      rc = alloc_skin(c, c->cap * 2);
      if (rc) return rc;
      continue;
    }
    if (fl & kFlagMirror) return fail(c, DP_ERR_CUDA, "internal error: neighbour mirror missing");
    if (fl & kFlagNonFinite) return fail(c, DP_ERR_NONFINITE, "coordinates, energy or forces are not finite");
    c->forces_valid = true;
    return DP_OK;
  }
  return fail(c, DP_ERR_NLIST_OVERFLOW, "neighbour skin list kept overflowing");
}

static int copy_in(dp_ctx* c, double* dst, const double* src, size_t count, int ptr_kind) {
  CUDA_TRY(c, cudaMemcpyAsync(dst, src, sizeof(double) * count,
                              ptr_kind == DP_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              c->st), "copy in");
  return DP_OK;
}

static int copy_out(dp_ctx* c, double* dst, const double* src, size_t count, int ptr_kind) {
  CUDA_TRY(c, cudaMemcpyAsync(dst, src, sizeof(double) * count,
                              ptr_kind == DP_PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              c->st), "copy out");
  return DP_OK;
}

// ------------------------------------------------------------------ C ABI
extern "C" int dp_init(dp_ctx** out, const dp_model_desc* desc, int n_atoms, const int32_t* types,
                       const double* masses, const double* box, const double* weights,
                       size_t n_weights, void* cuda_stream) {
  if (!out) return fail(nullptr, DP_ERR_ARG, "out is NULL");
  *out = nullptr;
  std::string why;
  if (check_desc(desc, &why)) return fail(nullptr, DP_ERR_ARG, why);
  if (n_atoms < 1) return fail(nullptr, DP_ERR_ARG, "n_atoms must be >= 1");
  if (!types || !box || !weights) return fail(nullptr, DP_ERR_ARG, "types, box and weights are required");
  size_t want = 0;
  dp_weight_count(desc, &want);
  if (n_weights != want)
    return fail(nullptr, DP_ERR_ARG, "weight blob has " + std::to_string(n_weights) + " values, model needs " + std::to_string(want));
  for (int a = 0; a < 3; ++a)
    if (!(box[a] > 0) || !isfinite(box[a])) return fail(nullptr, DP_ERR_ARG, "box lengths must be positive");
  for (int i = 0; i < n_atoms; ++i)
    if (types[i] < 0 || types[i] >= desc->n_species) return fail(nullptr, DP_ERR_ARG, "atom " + std::to_string(i) + " has a species outside 0..n_species-1");
  for (size_t q = 0; q < n_weights; ++q)
    if (!isfinite(weights[q])) return fail(nullptr, DP_ERR_ARG, "weights contain a non-finite value");
  AfDims afd{desc->n_species, desc->e1, desc->e2, desc->m1, desc->m2, desc->n_layers,
             desc->hidden, desc->heads, desc->f1, desc->f2, desc->f3, desc->nmax,
             desc->rcut, desc->rcut_smth};
  if (desc->family == DP_FAMILY_GRAPH)
    return fail(nullptr, DP_ERR_UNSUPPORTED, "graph family not available in this build");
  if (desc->precision == DP_PREC_FUSED_BF16 && !fused_af_supported(afd, &why))
    return fail(nullptr, DP_ERR_UNSUPPORTED, why);

  dp_ctx* c = new dp_ctx();
  c->desc = *desc;
  c->n = n_atoms;
  c->skin = desc->skin > 0 ? desc->skin : 1.0;
  c->rebuild_every = desc->rebuild_every > 0 ? desc->rebuild_every : 10;
  c->rskin = desc->rcut + c->skin;
  for (int a = 0; a < 3; ++a) c->box[a] = box[a];
  c->types_host.assign(types, types + n_atoms);
  c->af = afd;
  if (masses) {
    c->have_masses = true;
    c->mass_species.assign(masses, masses + desc->n_species);
    for (double m : c->mass_species)
      if (!(m > 0)) { delete c; return fail(nullptr, DP_ERR_ARG, "masses must be positive"); }
  }
  int rc = DP_OK;
  auto bail = [&](int code) {
    g_init_error = c->err;
    dp_free(c);
    return code;
  };
  if (cuda_stream) {
    c->st = (cudaStream_t)cuda_stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) { cuda_fail(c, e, "stream"); return bail(c->err.find("memory") != std::string::npos ? DP_ERR_OOM : DP_ERR_CUDA); }
    c->own_stream = true;
  }
  static bool configured = false;
  if (!configured) {
    nlist_configure();
    configured = true;
  }
  // systems: a single system here
  SysInfo si;
  make_sysinfo(box, c->rskin, 0, n_atoms, 0, &si, &c->ncell);
  double rho = n_atoms / (box[0] * box[1] * box[2]);
  double expect = 4.0 / 3.0 * M_PI * c->rskin * c->rskin * c->rskin * rho;
  int cap = (int)std::min<double>((double)n_atoms * 27.0 + 32.0, 2.0 * expect + 32.0);
  cap = std::max(64, ((cap + 31) / 32) * 32);
  std::vector<int> sys_of(n_atoms, 0), atom0 = {0, n_atoms};
  std::vector<double> minv(n_atoms, 0.0), mass(n_atoms, 0.0);
  const double kappa = 1.602176634e-19 / (1.66053906660e-27 * 1e10);
  if (c->have_masses)
    for (int i = 0; i < n_atoms; ++i) {
      mass[i] = c->mass_species[types[i]];
      minv[i] = kappa / mass[i];
    }
#define TRY(expr, where) do { cudaError_t e__ = (expr); if (e__ != cudaSuccess) { rc = cuda_fail(c, e__, where); return bail(rc); } } while (0)
  size_t N = n_atoms;
  TRY(dalloc(c, &c->x, 3 * N), "x");
  TRY(dalloc(c, &c->v, 3 * N), "v");
  TRY(dalloc(c, &c->F, 3 * N), "F");
  TRY(dalloc(c, &c->xref, 3 * N), "xref");
  TRY(dalloc(c, &c->w, 3 * N), "w");
  TRY(dalloc(c, &c->fl, 3 * N), "fl");
  TRY(dalloc(c, &c->minv, N), "minv");
  TRY(dalloc(c, &c->mass, N), "mass");
  TRY(dalloc(c, &c->types, N), "types");
  TRY(dalloc(c, &c->sys_of, N), "sys_of");
  TRY(dalloc(c, &c->sys_atom0, 2), "sys_atom0");
  TRY(dalloc(c, &c->sys, 1), "sys");
  TRY(dalloc(c, &c->cell_of, N), "cells");
  TRY(dalloc(c, &c->cell_cnt, c->ncell + 1), "cells");
  TRY(dalloc(c, &c->cell_fill, c->ncell + 1), "cells");
  TRY(dalloc(c, &c->cell_start, c->ncell + 1), "cells");
  TRY(dalloc(c, &c->cell_idx, N), "cells");
  TRY(dalloc(c, &c->skin_cnt, N), "skin");
  TRY(dalloc(c, &c->sel_j, N * desc->nmax), "sel");
  TRY(dalloc(c, &c->sel_img, 3 * N * desc->nmax), "sel");
  TRY(dalloc(c, &c->sel_r, 3 * N * desc->nmax), "sel");
  TRY(dalloc(c, &c->n_in_rc, N), "sel");
  TRY(dalloc(c, &c->atom_e, N), "energies");
  TRY(dalloc(c, &c->atom_vir, 9 * N), "virials");
  TRY(dalloc(c, &c->sys_e, 1), "energies");
  TRY(dalloc(c, &c->sys_vir, 9), "virials");
  TRY(dalloc(c, &c->flags, 1), "flags");
  TRY(dalloc(c, &c->step, 2), "step");
  TRY(cudaMemcpyAsync(c->types, types, sizeof(int) * N, cudaMemcpyHostToDevice, c->st), "upload");
  TRY(cudaMemcpyAsync(c->sys_of, sys_of.data(), sizeof(int) * N, cudaMemcpyHostToDevice, c->st), "upload");
  TRY(cudaMemcpyAsync(c->sys_atom0, atom0.data(), sizeof(int) * 2, cudaMemcpyHostToDevice, c->st), "upload");
  TRY(cudaMemcpyAsync(c->sys, &si, sizeof si, cudaMemcpyHostToDevice, c->st), "upload");
  TRY(cudaMemcpyAsync(c->minv, minv.data(), sizeof(double) * N, cudaMemcpyHostToDevice, c->st), "upload");
  TRY(cudaMemcpyAsync(c->mass, mass.data(), sizeof(double) * N, cudaMemcpyHostToDevice, c->st), "upload");
  TRY(cudaStreamSynchronize(c->st), "upload");
#undef TRY
  rc = alloc_skin(c, cap);
  if (rc) return bail(rc);
  if (desc->precision == DP_PREC_FUSED_BF16)
    c->model = make_fused_af(c->af, weights, n_atoms, types, &c->err);
  else
    c->model = make_plain_af(c->af, desc->precision == DP_PREC_PLAIN_F64, weights, n_atoms, types,
                             0, &c->err);
  if (!c->model) return bail(c->err.find("memory") != std::string::npos ? DP_ERR_OOM : DP_ERR_CUDA);
  c->bytes += c->model->bytes();
  *out = c;
  return DP_OK;
}

extern "C" int dp_compute(dp_ctx* c, const double* coords, double* energy, double* forces,
                          double* virial, int ptr_kind) {
  if (!c) return fail(nullptr, DP_ERR_ARG, "ctx is NULL");
  if (!coords) return fail(c, DP_ERR_ARG, "coords is NULL");
  int rc = copy_in(c, c->x, coords, 3 * (size_t)c->n, ptr_kind);
  if (rc) return rc;
  rc = compute_now(c);
  if (rc) return rc;
  if (energy) {
    if (ptr_kind == DP_PTR_DEVICE) rc = copy_out(c, energy, c->sys_e, 1, ptr_kind);
    else CUDA_TRY(c, cudaMemcpyAsync(energy, c->sys_e, sizeof(double), cudaMemcpyDeviceToHost, c->st), "energy");
  }
  if (!rc && forces) rc = copy_out(c, forces, c->F, 3 * (size_t)c->n, ptr_kind);
  if (!rc && virial) rc = copy_out(c, virial, c->sys_vir, 9, ptr_kind);
  if (rc) return rc;
  CUDA_TRY(c, cudaStreamSynchronize(c->st), "synchronize");
  return DP_OK;
}

static int build_step_graph(dp_ctx* c, double dt, int trace_len) {
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  if (trace_len > c->trace_len) {
    if (c->trace) cudaFree(c->trace);
    c->trace = nullptr;
    CUDA_TRY(c, cudaMalloc(&c->trace, sizeof(double) * 2 * c->n_sys * trace_len), "trace");
    c->trace_len = trace_len;
  }
  MdArgs m = md_args(c, dt);
  cudaGraph_t g;
  CUDA_TRY(c, cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal), "capture");
  launch_kick_drift(m, c->st);
  int k = 1 + enqueue_compute(c);
  launch_kick_final(m, c->st);
  launch_record(m, c->sys_e, c->trace, c->trace_len, c->st);
  k += 2;
  cudaError_t e = cudaStreamEndCapture(c->st, &g);
  if (e != cudaSuccess) return cuda_fail(c, e, "capture");
  e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
  c->graph_dt = dt;
  c->graph_trace_len = c->trace_len;
  c->kernels_step = k;
  return DP_OK;
}

extern "C" int dp_step(dp_ctx* c, int n_steps, double dt_fs, double* coords_io, double* vel_io,
                       double* energies_out, int ptr_kind) {
  if (!c) return fail(nullptr, DP_ERR_ARG, "ctx is NULL");
  if (n_steps < 0) return fail(c, DP_ERR_ARG, "n_steps must be >= 0");
  if (!(dt_fs > 0) || !isfinite(dt_fs)) return fail(c, DP_ERR_ARG, "dt must be positive");
  if (!c->have_masses) return fail(c, DP_ERR_ARG, "dp_step needs masses at dp_init");
  int rc = DP_OK;
  if (coords_io) {
    rc = copy_in(c, c->x, coords_io, 3 * (size_t)c->n, ptr_kind);
    if (rc) return rc;
    c->forces_valid = false;
  }
  if (vel_io) {
    rc = copy_in(c, c->v, vel_io, 3 * (size_t)c->n, ptr_kind);
    if (rc) return rc;
  }
  if (n_steps == 0) return DP_OK;
  // checkpoint for a retry after a neighbour-capacity overflow
  std::vector<double> x0(3 * (size_t)c->n), v0(3 * (size_t)c->n);
  long long step0[2];
  for (int attempt = 0; attempt < 4; ++attempt) {
    if (!c->forces_valid) {
      rc = compute_now(c);
      if (rc) return rc;
    }
    CUDA_TRY(c, cudaMemcpyAsync(x0.data(), c->x, sizeof(double) * x0.size(), cudaMemcpyDeviceToHost, c->st), "checkpoint");
    CUDA_TRY(c, cudaMemcpyAsync(v0.data(), c->v, sizeof(double) * v0.size(), cudaMemcpyDeviceToHost, c->st), "checkpoint");
    CUDA_TRY(c, cudaMemcpyAsync(step0, c->step, sizeof step0, cudaMemcpyDeviceToHost, c->st), "checkpoint");
    CUDA_TRY(c, cudaStreamSynchronize(c->st), "checkpoint");
    step0[1] = step0[0];
    CUDA_TRY(c, cudaMemcpyAsync(c->step, step0, sizeof step0, cudaMemcpyHostToDevice, c->st), "step base");
    int tl = energies_out ? n_steps : 1;
    if (!c->graph || c->graph_dt != dt_fs || c->graph_trace_len < tl) {
      rc = build_step_graph(c, dt_fs, std::max(tl, c->trace_len));
      if (rc) return rc;
    }
    for (int s = 0; s < n_steps; ++s) CUDA_TRY(c, cudaGraphLaunch(c->graph, c->st), "graph launch");
    int fl = 0;
    rc = read_flags(c, &fl);
    if (rc) return rc;
    if (fl & kFlagOverflow) {
      rc = alloc_skin(c, c->cap * 2);
      if (rc) return rc;
      CUDA_TRY(c, cudaMemcpyAsync(c->x, x0.data(), sizeof(double) * x0.size(), cudaMemcpyHostToDevice, c->st), "restore");
      CUDA_TRY(c, cudaMemcpyAsync(c->v, v0.data(), sizeof(double) * v0.size(), cudaMemcpyHostToDevice, c->st), "restore");
      step0[1] = 0;
      CUDA_TRY(c, cudaMemcpyAsync(c->step, step0, sizeof step0, cudaMemcpyHostToDevice, c->st), "restore");
      c->forces_valid = false;
      continue;
    }
    if (fl & kFlagMirror) return fail(c, DP_ERR_CUDA, "internal error: neighbour mirror missing");
    if (fl & kFlagNonFinite) return fail(c, DP_ERR_NONFINITE, "energy or forces are not finite");
    if (energies_out) {
      if (ptr_kind == DP_PTR_DEVICE)
        CUDA_TRY(c, cudaMemcpyAsync(energies_out, c->trace, sizeof(double) * 2 * n_steps, cudaMemcpyDeviceToDevice, c->st), "trace");
      else
        CUDA_TRY(c, cudaMemcpyAsync(energies_out, c->trace, sizeof(double) * 2 * n_steps, cudaMemcpyDeviceToHost, c->st), "trace");
    }
    if (coords_io) {
      rc = copy_out(c, coords_io, c->x, 3 * (size_t)c->n, ptr_kind);
      if (rc) return rc;
    }
    if (vel_io) {
      rc = copy_out(c, vel_io, c->v, 3 * (size_t)c->n, ptr_kind);
      if (rc) return rc;
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->st), "synchronize");
    return DP_OK;
  }
  return fail(c, DP_ERR_NLIST_OVERFLOW, "neighbour skin list kept overflowing");
}

extern "C" int dp_get_state(dp_ctx* c, double* coords, double* vel, long long* step, int ptr_kind) {
  if (!c) return fail(nullptr, DP_ERR_ARG, "ctx is NULL");
  int rc = DP_OK;
  if (coords) rc = copy_out(c, coords, c->x, 3 * (size_t)c->n, ptr_kind);
  if (!rc && vel) rc = copy_out(c, vel, c->v, 3 * (size_t)c->n, ptr_kind);
  if (rc) return rc;
  if (step) CUDA_TRY(c, cudaMemcpyAsync(step, c->step, sizeof(long long), cudaMemcpyDeviceToHost, c->st), "step");
  CUDA_TRY(c, cudaStreamSynchronize(c->st), "synchronize");
  return DP_OK;
}

extern "C" int dp_set_state(dp_ctx* c, const double* coords, const double* vel, long long step,
                            int ptr_kind) {
  if (!c) return fail(nullptr, DP_ERR_ARG, "ctx is NULL");
  int rc = DP_OK;
  if (coords) {
    rc = copy_in(c, c->x, coords, 3 * (size_t)c->n, ptr_kind);
    c->forces_valid = false;
  }
  if (!rc && vel) rc = copy_in(c, c->v, vel, 3 * (size_t)c->n, ptr_kind);
  if (rc) return rc;
  long long s2[2] = {step, step};
  CUDA_TRY(c, cudaMemcpyAsync(c->step, s2, sizeof s2, cudaMemcpyHostToDevice, c->st), "step");
  CUDA_TRY(c, cudaStreamSynchronize(c->st), "synchronize");
  return DP_OK;
}

extern "C" int dp_get_neighbours(dp_ctx* c, int32_t* nbr_j, int32_t* nbr_img, int32_t* n_in_rc) {
  if (!c) return fail(nullptr, DP_ERR_ARG, "ctx is NULL");
  size_t P = (size_t)c->n * c->desc.nmax;
  if (nbr_j) CUDA_TRY(c, cudaMemcpyAsync(nbr_j, c->sel_j, sizeof(int) * P, cudaMemcpyDeviceToHost, c->st), "nbr");
  if (nbr_img) CUDA_TRY(c, cudaMemcpyAsync(nbr_img, c->sel_img, sizeof(int) * 3 * P, cudaMemcpyDeviceToHost, c->st), "nbr");
  if (n_in_rc) CUDA_TRY(c, cudaMemcpyAsync(n_in_rc, c->n_in_rc, sizeof(int) * c->n, cudaMemcpyDeviceToHost, c->st), "nbr");
  CUDA_TRY(c, cudaStreamSynchronize(c->st), "synchronize");
  return DP_OK;
}

extern "C" int dp_get_atom_energies(dp_ctx* c, double* atom_e) {
  if (!c || !atom_e) return fail(c, DP_ERR_ARG, "NULL argument");
  CUDA_TRY(c, cudaMemcpyAsync(atom_e, c->atom_e, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->st), "atom energies");
  CUDA_TRY(c, cudaStreamSynchronize(c->st), "synchronize");
  return DP_OK;
}

extern "C" int dp_enqueue_network(dp_ctx* c, int reps) {
  if (!c) return fail(nullptr, DP_ERR_ARG, "ctx is NULL");
  if (reps < 0) return fail(c, DP_ERR_ARG, "reps must be >= 0");
  if (!c->forces_valid) return fail(c, DP_ERR_ARG, "no resident neighbour lists: call dp_compute first");
  for (int r = 0; r < reps; ++r) c->model->run(c->sel_j, c->sel_r, c->types, c->atom_e, c->st);
  CUDA_TRY(c, cudaGetLastError(), "launch");
  return DP_OK;
}

extern "C" int dp_kernels_per_step(dp_ctx* c, int* n_compute, int* n_step) {
  if (!c) return fail(nullptr, DP_ERR_ARG, "ctx is NULL");
  if (n_compute) *n_compute = c->kernels_compute;
  if (n_step) *n_step = c->kernels_step;
  return DP_OK;
}

extern "C" int dp_device_bytes(dp_ctx* c, size_t* bytes) {
  if (!c || !bytes) return fail(c, DP_ERR_ARG, "NULL argument");
  *bytes = c->bytes;
  return DP_OK;
}

extern "C" void dp_free(dp_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->trace) cudaFree(c->trace);
  delete c->model;
  for (void* p : c->skin_allocs) cudaFree(p);
  for (void* p : c->allocs) cudaFree(p);
  if (c->own_stream && c->st) cudaStreamDestroy(c->st);
  delete c;
}

extern "C" const char* dp_last_error(const dp_ctx* c) {
  if (!c) return g_init_error.c_str();
  return c->err.c_str();
}
