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
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

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
  int ncell = 0, ncell_cap = 0;
  int n_cap = 0, sys_cap = 1;
  std::vector<double> boxes;
  std::vector<void*> cell_allocs;
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
  double* xin = nullptr;      // staging for uploaded coordinates
  double* head_sys_e = nullptr;  // energies of fitting heads 1.. per system: [sys][head - 1]
  unsigned char* grp = nullptr;  // DP group (1 = member), used when use_grp
  bool use_grp = false;
  // what grp marks: 0 DP group members (dp_set_group), 1 centres
  // (dp_set_centres), 2 the atoms whose energy counts (dp_set_energy_seed)
  int grp_mode = 0;
  int* differs = nullptr;     // compare result
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
  double* atom_ke = nullptr;   // kinetic energy per atom (final kick -> record)
  unsigned long long* red_part = nullptr;   // per-chunk partial sums of the system reduction
  int red_chunks = 1;
  int* flags = nullptr;
  long long* step = nullptr;   // [0] step counter, [1] trace base
  // dp_step's checkpoint for a retry after a neighbour-capacity overflow
  double *xck = nullptr, *vck = nullptr;
  long long* stepck = nullptr;
  double* trace = nullptr;
  int trace_len = 0;
  size_t trace_elems = 0;
  // skin-list buffers are reallocated when the capacity grows
  std::vector<void*> skin_allocs;
  // network
  Model* model = nullptr;
  // graph of one MD step
  cudaGraphExec_t graph = nullptr;
  double graph_dt = 0;
  int graph_trace_len = 0;
  bool forces_valid = false;
  // atoms [0, valid_below) already hold forces for their current positions
  // (systems carried over by a serving repack); the next compute evaluates
  // only the rest
  int valid_below = 0;
  bool graph_stale = false;   // batch changed: recapture, update the executable
  int kernels_compute = 0, kernels_step = 0;
};

static thread_local std::string g_init_error;
struct dp_server;
extern "C" void dp_server_free(dp_server* s);

// NVTX range around an ABI call or an MD step (visible in Nsight timelines;
// no cost without a profiler attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

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
  } else {
    if (d->node_dim < 1 || d->edge_dim < 1) { *why = "node_dim and edge_dim must be positive"; return -1; }
    if (d->n_gnn_layers < 0 || d->n_gnn_layers > 16) { *why = "n_gnn_layers must be 0..16"; return -1; }
    if (d->angle_nmax < 1 || d->angle_nmax > 64) { *why = "angle_nmax must be 1..64"; return -1; }
    if (!(d->angle_rcut_smth >= 0) || !(d->angle_rcut_smth < d->angle_rcut) || d->angle_rcut > d->rcut) { *why = "need 0 <= angle_rcut_smth < angle_rcut <= rcut"; return -1; }
  }
  if (d->precision < DP_PREC_PLAIN_F64 || d->precision > DP_PREC_FUSED) { *why = "unknown precision"; return -1; }
  if (d->fit_heads < 0 || d->fit_heads > 16) { *why = "fit_heads must be 0..16"; return -1; }
  if (d->fit_heads > 1 && d->family != DP_FAMILY_ATTENTION) { *why = "fitting heads are an attention-family option"; return -1; }
  if (d->message_passing != 0 && d->message_passing != 1) { *why = "message_passing must be 0 or 1"; return -1; }
  if (d->message_passing && d->family != DP_FAMILY_ATTENTION) { *why = "message passing is an attention-family option"; return -1; }
  if (d->message_passing && d->fit_heads > 1) { *why = "message passing takes one fitting head"; return -1; }
  return 0;
}

static GfDims gf_dims(const dp_model_desc* d) {
  return GfDims{d->n_species, d->node_dim, d->edge_dim, d->n_gnn_layers, d->f1, d->f2, d->f3,
                d->nmax, d->angle_nmax, d->rcut, d->rcut_smth, d->angle_rcut, d->angle_rcut_smth};
}

extern "C" int dp_weight_count(const dp_model_desc* d, size_t* n) {
  std::string why;
  if (!n) return fail(nullptr, DP_ERR_ARG, "n is NULL");
  if (check_desc(d, &why)) return fail(nullptr, DP_ERR_ARG, why);
  if (d->family == DP_FAMILY_GRAPH) {
    *n = gf_weight_count(gf_dims(d));
    return DP_OK;
  }
  size_t S = d->n_species, E1 = d->e1, E2 = d->e2, M1 = d->m1, M2 = d->m2, H = d->hidden;
  size_t t = S * (E1 + E1 + E1 * E2 + E2 + E2 * M1 + M1);
  t += (size_t)d->n_layers * (3 * M1 * H + H * M1 + M1);
  if (d->message_passing) t += S * M1 + (size_t)d->n_layers * (M1 * M1 + M1);
  const size_t heads = d->fit_heads > 1 ? d->fit_heads : 1;
  t += heads * S * (M1 * M2 * d->f1 + d->f1 + (size_t)d->f1 * d->f2 + d->f2 + (size_t)d->f2 * d->f3 + d->f3 + d->f3 + 1);
  *n = t;
  return DP_OK;
}

// ------------------------------------------------------------------ systems
// the small-box search keeps the images -nimg..nimg of an axis in one 32-bit mask
constexpr int kMaxImages = 15;

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
  a.grp = c->use_grp && c->grp_mode != 2 ? c->grp : nullptr;   // an energy seed keeps every pair
  a.grp_centres = c->grp_mode == 1 ? 1 : 0;
  a.sys_of = c->sys_of; a.sys = c->sys;
  a.cell_of = c->cell_of; a.cell_cnt = c->cell_cnt; a.cell_fill = c->cell_fill;
  a.cell_start = c->cell_start; a.cell_idx = c->cell_idx;
  a.skin = c->skin_list; a.skin_cnt = c->skin_cnt; a.mirror = c->mirror;
  a.sel_j = c->sel_j; a.sel_img = c->sel_img; a.sel_r = c->sel_r; a.selpos = c->selpos;
  a.n_in_rc = c->n_in_rc; a.flags = c->flags;
  return a;
}

static NbrView nbr_view(dp_ctx* c) {
  return NbrView{c->sel_j, c->sel_r, c->skin_list, c->skin_cnt, c->mirror, c->selpos, c->cap};
}

static MdArgs md_args(dp_ctx* c, double dt) {
  MdArgs m{};
  m.n = c->n; m.dt = dt; m.x = c->x; m.v = c->v; m.F = c->F; m.minv = c->minv; m.mass = c->mass;
  m.xref = c->xref; m.half_skin2 = 0.25 * c->skin * c->skin; m.rebuild_every = c->rebuild_every;
  m.step = c->step; m.flags = c->flags; m.n_sys = c->n_sys; m.sys_atom0 = c->sys_atom0;
  m.sys_of = c->sys_of; m.atom_ke = c->atom_ke;
  return m;
}

// One evaluation on the stream: neighbours (rebuild if flagged), model, forces,
// reductions.  With atom0 > 0 only atoms [atom0, n) get energies and forces
// (their systems must not reach below atom0) and the per-system reduction is
// skipped.  Returns the number of kernels it launched.
static int enqueue_compute(dp_ctx* c, int atom0 = 0) {
  NlistArgs na = nlist_args(c);
  int k = 0;
  launch_wrap(na, c->st); ++k;
  launch_nlist_rebuild(na, c->st); k += nlist_rebuild_kernels();
  launch_select(na, c->st); ++k;
  ForceArgs fa{};
  fa.n = c->n; fa.nmax = c->desc.nmax; fa.cap = c->cap; fa.sel_j = c->sel_j; fa.sel_r = c->sel_r;
  fa.skin = c->skin_list; fa.skin_cnt = c->skin_cnt; fa.mirror = c->mirror; fa.selpos = c->selpos;
  fa.F = c->F; fa.atom_vir = c->atom_vir;
  fa.atom0 = atom0;
  if (atom0 > 0) k += c->model->run_range(nbr_view(c), c->types, c->atom_e, c->st, atom0);
  else k += c->model->run(nbr_view(c), c->types, c->atom_e, c->st);
  fa.g32 = c->model->grad32();
  fa.g64 = c->model->grad64();
  launch_force_gather(fa, c->st); ++k;
  if (atom0 > 0) return k;
  if (c->head_sys_e && c->model->head_energies()) {
    launch_head_reduce(c->n_sys, c->af.fit_heads - 1, c->n_cap, c->sys_atom0,
                       c->model->head_energies(), c->use_grp ? c->grp : nullptr, c->head_sys_e,
                       c->st);
    ++k;
  }
  ReduceArgs ra{};
  ra.n_sys = c->n_sys; ra.sys_atom0 = c->sys_atom0; ra.atom_e = c->atom_e; ra.atom_vir = c->atom_vir;
  ra.n = c->n; ra.part = c->red_part; ra.part_chunks = c->red_chunks;
  ra.F = c->F; ra.sys_e = c->sys_e; ra.sys_vir = c->sys_vir; ra.flags = c->flags;
  ra.atom_e_out = c->atom_e;
  ra.grp = c->use_grp ? c->grp : nullptr;
  launch_reduce(ra, c->st); k += 2;
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
  const int atom0 = c->valid_below < c->n ? c->valid_below : 0;
  for (int attempt = 0; attempt < 4; ++attempt) {
    int rc = clear_flags(c, ~0);
    if (rc) return rc;
    launch_flag_set(c->flags, kFlagRebuild, c->st);
    c->kernels_compute = enqueue_compute(c, atom0) + 1;
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
    if (fl & kFlagTimeout) return fail(c, DP_ERR_TIMEOUT, "a device-side wait gave up");
    if (fl & kFlagNonFinite) return fail(c, DP_ERR_NONFINITE, "coordinates, energy or forces are not finite");
    c->forces_valid = true;
    c->valid_below = 0;
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
// Weight blob and model sizes check shared by every constructor.
static int check_model(const dp_model_desc* desc, const double* weights, size_t n_weights,
                       const double* masses, AfDims* afd) {
  std::string why;
  if (check_desc(desc, &why)) return fail(nullptr, DP_ERR_ARG, why);
  if (!weights) return fail(nullptr, DP_ERR_ARG, "weights are required");
  size_t want = 0;
  dp_weight_count(desc, &want);
  if (n_weights != want)
    return fail(nullptr, DP_ERR_ARG, "weight blob has " + std::to_string(n_weights) + " values, model needs " + std::to_string(want));
  for (size_t q = 0; q < n_weights; ++q)
    if (!isfinite(weights[q])) return fail(nullptr, DP_ERR_ARG, "weights contain a non-finite value");
  if (masses)
    for (int t = 0; t < desc->n_species; ++t)
      if (!(masses[t] > 0)) return fail(nullptr, DP_ERR_ARG, "masses must be positive");
  *afd = AfDims{desc->n_species, desc->e1, desc->e2, desc->m1, desc->m2, desc->n_layers,
                desc->hidden, desc->heads, desc->f1, desc->f2, desc->f3, desc->nmax,
                desc->rcut, desc->rcut_smth, desc->fit_heads > 1 ? desc->fit_heads : 1,
                desc->message_passing};

  if (desc->family == DP_FAMILY_ATTENTION && desc->precision == DP_PREC_FUSED &&
      !fused_af_supported(*afd, &why))
    return fail(nullptr, DP_ERR_UNSUPPORTED, why);
  if (desc->family == DP_FAMILY_GRAPH && desc->precision == DP_PREC_FUSED &&
      !gf_mixed_supported(gf_dims(desc), &why))
    return fail(nullptr, DP_ERR_UNSUPPORTED, why);
  return DP_OK;
}

// A context with room for n_cap atoms in up to sys_cap systems.  The model is
// built for model_types (n_cap atoms); skin lists start at `cap` per atom.
static int ctx_create(dp_ctx** out, const dp_model_desc* desc, const double* masses,
                      const double* weights, void* cuda_stream, int n_cap, int sys_cap,
                      const int* model_types, int cap, const AfDims& afd) {
  dp_ctx* c = new dp_ctx();
  c->desc = *desc;
  c->n = n_cap;
  c->n_cap = n_cap;
  c->sys_cap = sys_cap;
  c->skin = desc->skin > 0 ? desc->skin : 1.0;
  c->rebuild_every = desc->rebuild_every > 0 ? desc->rebuild_every : 10;
  c->rskin = desc->rcut + c->skin;
  c->af = afd;
  if (masses) {
    c->have_masses = true;
    c->mass_species.assign(masses, masses + desc->n_species);
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
    if (e != cudaSuccess) { cuda_fail(c, e, "stream"); return bail(DP_ERR_CUDA); }
    c->own_stream = true;
  }
  static bool configured = false;
  if (!configured) {
    nlist_configure();
    configured = true;
  }
#define TRY(expr, where) do { cudaError_t e__ = (expr); if (e__ != cudaSuccess) { rc = cuda_fail(c, e__, where); return bail(rc); } } while (0)
  size_t N = n_cap, S = sys_cap;
  TRY(dalloc(c, &c->x, 3 * N), "x");
  TRY(dalloc(c, &c->v, 3 * N), "v");
  TRY(dalloc(c, &c->F, 3 * N), "F");
  TRY(dalloc(c, &c->xin, 3 * N), "xin");
  TRY(dalloc(c, &c->xck, 3 * N), "checkpoint");
  TRY(dalloc(c, &c->vck, 3 * N), "checkpoint");
  TRY(dalloc(c, &c->stepck, 1), "checkpoint");
  TRY(dalloc(c, &c->differs, 1), "differs");
  TRY(dalloc(c, &c->xref, 3 * N), "xref");
  TRY(dalloc(c, &c->w, 3 * N), "w");
  TRY(dalloc(c, &c->fl, 3 * N), "fl");
  TRY(dalloc(c, &c->minv, N), "minv");
  TRY(dalloc(c, &c->mass, N), "mass");
  TRY(dalloc(c, &c->types, N), "types");
  TRY(dalloc(c, &c->sys_of, N), "sys_of");
  TRY(dalloc(c, &c->sys_atom0, S + 1), "sys_atom0");
  TRY(dalloc(c, &c->sys, S), "sys");
  TRY(dalloc(c, &c->cell_of, N), "cells");
  TRY(dalloc(c, &c->cell_idx, N), "cells");
  TRY(dalloc(c, &c->skin_cnt, N), "skin");
  TRY(dalloc(c, &c->sel_j, N * desc->nmax), "sel");
  TRY(dalloc(c, &c->sel_img, 3 * N * desc->nmax), "sel");
  TRY(dalloc(c, &c->sel_r, 3 * N * desc->nmax), "sel");
  TRY(dalloc(c, &c->n_in_rc, N), "sel");
  TRY(dalloc(c, &c->atom_e, N), "energies");
  TRY(dalloc(c, &c->atom_vir, 9 * N), "virials");
  TRY(dalloc(c, &c->atom_ke, N), "kinetic energies");
  c->red_chunks = (int)((N + kReduceChunk - 1) / kReduceChunk);
  TRY(dalloc(c, &c->red_part, S * (size_t)c->red_chunks * 20), "reductions");
  TRY(dalloc(c, &c->sys_e, S), "energies");
  if (c->af.fit_heads > 1) TRY(dalloc(c, &c->head_sys_e, S * (c->af.fit_heads - 1)), "energies");
  TRY(dalloc(c, &c->sys_vir, 9 * S), "virials");
  TRY(dalloc(c, &c->flags, 1), "flags");
  TRY(dalloc(c, &c->step, 2), "step");
#undef TRY
  rc = alloc_skin(c, cap);
  if (rc) return bail(rc);
  if (desc->family == DP_FAMILY_GRAPH)
    c->model = make_plain_gf(gf_dims(desc), desc->precision == DP_PREC_PLAIN_F64,
                             desc->precision == DP_PREC_FUSED, weights, n_cap, model_types, &c->err);
  else if (desc->precision == DP_PREC_FUSED)
    c->model = make_fused_af(c->af, weights, n_cap, model_types, &c->err);
  else
    c->model = make_plain_af(c->af, desc->precision == DP_PREC_PLAIN_F64, weights, n_cap,
                             model_types, 0, &c->err);
  if (!c->model) return bail(c->err.find("memory") != std::string::npos ? DP_ERR_OOM : DP_ERR_CUDA);
  c->bytes += c->model->bytes();
  c->model->bind_flags(c->flags);
  *out = c;
  return DP_OK;
}

// Pack n_sys systems (atom counts natoms[], boxes[3*s], species types[] of all
// atoms in order) into the context; neighbour lists and forces become stale.
static int ctx_set_systems(dp_ctx* c, int n_sys, const int* natoms, const double* boxes,
                           const int* types) {
  int n = 0;
  for (int s = 0; s < n_sys; ++s) n += natoms[s];
  if (n_sys < 1 || n_sys > c->sys_cap || n < 1 || n > c->n_cap)
    return fail(c, DP_ERR_ARG, "batch exceeds the context's capacity");
  std::vector<SysInfo> si(n_sys);
  std::vector<int> sys_of(n), atom0(n_sys + 1, 0);
  int ncell = 0;
  for (int s = 0, a0 = 0; s < n_sys; ++s) {
    int nc = 0;
    make_sysinfo(boxes + 3 * s, c->rskin, a0, natoms[s], ncell, &si[s], &nc);
    if (std::max(si[s].nimg[0], std::max(si[s].nimg[1], si[s].nimg[2])) > kMaxImages)
      return fail(c, DP_ERR_ARG, "a box edge is shorter than (rc + skin) / 14");
    ncell += nc;
    for (int i = 0; i < natoms[s]; ++i) sys_of[a0 + i] = s;
    a0 += natoms[s];
    atom0[s + 1] = a0;
  }
  if (ncell + 1 > c->ncell_cap) {
    for (void* q : c->cell_allocs) cudaFree(q);
    c->cell_allocs.clear();
    int cap = std::max(ncell + 1, 2 * c->ncell_cap);
    CUDA_TRY(c, dalloc(c, &c->cell_cnt, cap, &c->cell_allocs), "cells");
    CUDA_TRY(c, dalloc(c, &c->cell_fill, cap, &c->cell_allocs), "cells");
    CUDA_TRY(c, dalloc(c, &c->cell_start, cap, &c->cell_allocs), "cells");
    c->ncell_cap = cap;
  }
  std::vector<double> minv(n, 0.0), mass(n, 0.0);
  const double kappa = 1.602176634e-19 / (1.66053906660e-27 * 1e10);
  if (c->have_masses)
    for (int i = 0; i < n; ++i) {
      mass[i] = c->mass_species[types[i]];
      minv[i] = kappa / mass[i];
    }
  CUDA_TRY(c, cudaMemcpyAsync(c->types, types, sizeof(int) * n, cudaMemcpyHostToDevice, c->st), "upload");
  CUDA_TRY(c, cudaMemcpyAsync(c->sys_of, sys_of.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->st), "upload");
  CUDA_TRY(c, cudaMemcpyAsync(c->sys_atom0, atom0.data(), sizeof(int) * (n_sys + 1), cudaMemcpyHostToDevice, c->st), "upload");
  CUDA_TRY(c, cudaMemcpyAsync(c->sys, si.data(), sizeof(SysInfo) * n_sys, cudaMemcpyHostToDevice, c->st), "upload");
  CUDA_TRY(c, cudaMemcpyAsync(c->minv, minv.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->st), "upload");
  CUDA_TRY(c, cudaMemcpyAsync(c->mass, mass.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->st), "upload");
  CUDA_TRY(c, cudaStreamSynchronize(c->st), "upload");
  bool same_types = c->n == n && c->types_host.size() == (size_t)n &&
                    std::equal(types, types + n, c->types_host.begin());
  if (!same_types && !c->model->set_atoms(n, types))
    return fail(c, DP_ERR_UNSUPPORTED, "this model cannot change its atom set");
  c->types_host.assign(types, types + n);
  c->n = n;
  c->n_sys = n_sys;
  c->ncell = ncell;
  c->boxes.assign(boxes, boxes + 3 * n_sys);
  for (int a = 0; a < 3; ++a) c->box[a] = boxes[a];
  c->graph_stale = true;
  c->forces_valid = false;
  c->valid_below = 0;
  return DP_OK;
}

// skin-list capacity per atom from the number density
static int skin_capacity(double rskin, double rho, int n_atoms) {
  double expect = 4.0 / 3.0 * M_PI * rskin * rskin * rskin * rho;
  int cap = (int)std::min<double>((double)n_atoms * 27.0 + 32.0, 2.0 * expect + 32.0);
  return std::max(64, ((cap + 31) / 32) * 32);
}

extern "C" int dp_init(dp_ctx** out, const dp_model_desc* desc, int n_atoms, const int32_t* types,
                       const double* masses, const double* box, const double* weights,
                       size_t n_weights, void* cuda_stream) {
  if (!out) return fail(nullptr, DP_ERR_ARG, "out is NULL");
  *out = nullptr;
  AfDims afd{};
  int rc = check_model(desc, weights, n_weights, masses, &afd);
  if (rc) return rc;
  if (n_atoms < 1) return fail(nullptr, DP_ERR_ARG, "n_atoms must be >= 1");
  if (!types || !box) return fail(nullptr, DP_ERR_ARG, "types and box are required");
  for (int a = 0; a < 3; ++a)
    if (!(box[a] > 0) || !isfinite(box[a])) return fail(nullptr, DP_ERR_ARG, "box lengths must be positive");
  for (int i = 0; i < n_atoms; ++i)
    if (types[i] < 0 || types[i] >= desc->n_species) return fail(nullptr, DP_ERR_ARG, "atom " + std::to_string(i) + " has a species outside 0..n_species-1");
  const double rskin = desc->rcut + (desc->skin > 0 ? desc->skin : 1.0);
  int cap = skin_capacity(rskin, n_atoms / (box[0] * box[1] * box[2]), n_atoms);
  dp_ctx* c = nullptr;
  rc = ctx_create(&c, desc, masses, weights, cuda_stream, n_atoms, 1, types, cap, afd);
  if (rc) return rc;
  c->types_host.assign(types, types + n_atoms);
  rc = ctx_set_systems(c, 1, &n_atoms, box, types);
  if (rc) {
    g_init_error = c->err;
    dp_free(c);
    return rc;
  }
  *out = c;
  return DP_OK;
}

extern "C" int dp_compute(dp_ctx* c, const double* coords, double* energy, double* forces,
                          double* virial, int ptr_kind) {
  NvtxRange nvtx("dp_compute");
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

// Capture one MD step; an existing executable graph of the same shape is
// updated in place (cheaper than a new instantiation after a batch change).
static int build_step_graph(dp_ctx* c, double dt, int trace_len) {
  const size_t need = (size_t)2 * c->n_sys * trace_len;
  if (need > c->trace_elems) {
    if (c->trace) cudaFree(c->trace);
    c->trace = nullptr;
    CUDA_TRY(c, cudaMalloc(&c->trace, sizeof(double) * need), "trace");
    c->trace_elems = need;
  }
  c->trace_len = trace_len;
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
  bool updated = false;
  if (c->graph) {
    cudaGraphExecUpdateResultInfo info{};
    updated = cudaGraphExecUpdate(c->graph, g, &info) == cudaSuccess;
    if (!updated) {
      cudaGetLastError();
      cudaGraphExecDestroy(c->graph);
      c->graph = nullptr;
    }
  }
  if (!updated) e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
  c->graph_stale = false;
  c->graph_dt = dt;
  c->graph_trace_len = c->trace_len;
  c->kernels_step = k;
  return DP_OK;
}

extern "C" int dp_get_head_energies(dp_ctx* c, double* out) {
  if (!c) return fail(nullptr, DP_ERR_ARG, "ctx is NULL");
  if (!out) return fail(c, DP_ERR_ARG, "out is NULL");
  if (!c->forces_valid) return fail(c, DP_ERR_ARG, "no evaluation at the resident positions yet");
  const int k = c->desc.family == DP_FAMILY_GRAPH ? 1 : std::max(1, c->af.fit_heads);
  std::vector<double> e0(c->n_sys), eh((size_t)c->n_sys * (k > 1 ? k - 1 : 0));
  CUDA_TRY(c, cudaMemcpyAsync(e0.data(), c->sys_e, sizeof(double) * c->n_sys, cudaMemcpyDeviceToHost, c->st), "energies");
  if (k > 1)
    CUDA_TRY(c, cudaMemcpyAsync(eh.data(), c->head_sys_e, sizeof(double) * eh.size(), cudaMemcpyDeviceToHost, c->st), "energies");
  CUDA_TRY(c, cudaStreamSynchronize(c->st), "synchronize");
  for (int s = 0; s < c->n_sys; ++s) {
    out[(size_t)s * k] = e0[s];
    for (int h = 1; h < k; ++h) out[(size_t)s * k + h] = eh[(size_t)s * (k - 1) + h - 1];
  }
  return DP_OK;
}

static int set_mask(dp_ctx* c, const unsigned char* mask, int mode) {
  if (c->n_sys != 1) return fail(c, DP_ERR_UNSUPPORTED, "a group needs a single-system context");
  if (mask) {
    if (!c->grp) CUDA_TRY(c, dalloc(c, &c->grp, (size_t)c->n_cap), "group");
    std::vector<unsigned char> g(c->n);
    for (int i = 0; i < c->n; ++i) g[i] = mask[i] ? 1 : 0;
    CUDA_TRY(c, cudaMemcpyAsync(c->grp, g.data(), c->n, cudaMemcpyHostToDevice, c->st), "group");
    CUDA_TRY(c, cudaStreamSynchronize(c->st), "group");
  }
  const bool seeded = mask != nullptr && mode == 2;
  if (!c->model->set_energy_seed(seeded ? c->grp : nullptr) && seeded)
    return fail(c, DP_ERR_UNSUPPORTED, "this model takes no energy seed");
  c->use_grp = mask != nullptr;
  c->grp_mode = mask != nullptr ? mode : 0;
  c->forces_valid = false;
  c->valid_below = 0;
  c->graph_stale = true;
  return DP_OK;
}

// DP group (the paper's NNPot atom group): only pairs of members are
// neighbours and only members carry energy; NULL restores every atom.
extern "C" int dp_set_group(dp_ctx* c, const unsigned char* mask) {
  if (!c) return fail(nullptr, DP_ERR_ARG, "ctx is NULL");
  return set_mask(c, mask, 0);
}

// Centres of a domain-decomposed subdomain: only marked atoms are centres and
// carry energy, every atom is a neighbour; NULL restores every atom.
extern "C" int dp_set_centres(dp_ctx* c, const unsigned char* mask) {
  if (!c) return fail(nullptr, DP_ERR_ARG, "ctx is NULL");
  if (mask && (c->desc.family != DP_FAMILY_ATTENTION || c->desc.message_passing))
    return fail(c, DP_ERR_UNSUPPORTED,
                "a centres mask needs an atom-local model (ghosts of layer-coupled models evaluate as centres)");
  return set_mask(c, mask, 1);
}

// Energy seed of a subdomain of a layer-coupled model: every atom evaluates as
// a centre, only marked atoms carry energy and seed the adjoint; NULL
// restores every atom.
extern "C" int dp_set_energy_seed(dp_ctx* c, const unsigned char* mask) {
  if (!c) return fail(nullptr, DP_ERR_ARG, "ctx is NULL");
  return set_mask(c, mask, 2);
}

extern "C" int dp_step(dp_ctx* c, int n_steps, double dt_fs, double* coords_io, double* vel_io,
                       double* energies_out, int ptr_kind) {
  NvtxRange nvtx("dp_step");
  if (!c) return fail(nullptr, DP_ERR_ARG, "ctx is NULL");
  if (n_steps < 0) return fail(c, DP_ERR_ARG, "n_steps must be >= 0");
  if (!(dt_fs > 0) || !isfinite(dt_fs)) return fail(c, DP_ERR_ARG, "dt must be positive");
  if (!c->have_masses) return fail(c, DP_ERR_ARG, "dp_step needs masses at dp_init");
  int rc = DP_OK;
  if (coords_io) {
    if (c->forces_valid) {
      // coordinates identical (bit for bit) to the resident ones keep the
      // resident forces: a caller that hands back what the last step returned
      // pays for one evaluation per step, not two
      rc = copy_in(c, c->xin, coords_io, 3 * (size_t)c->n, ptr_kind);
      if (rc) return rc;
      CUDA_TRY(c, cudaMemsetAsync(c->differs, 0, sizeof(int), c->st), "compare");
      launch_compare(3 * (long long)c->n, c->xin, c->x, c->differs, c->st);
      int differs = 1;
      CUDA_TRY(c, cudaMemcpyAsync(&differs, c->differs, sizeof(int), cudaMemcpyDeviceToHost, c->st), "compare");
      CUDA_TRY(c, cudaStreamSynchronize(c->st), "compare");
      if (differs) {
        CUDA_TRY(c, cudaMemcpyAsync(c->x, c->xin, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToDevice, c->st), "copy in");
        c->forces_valid = false;
      }
    } else {
      rc = copy_in(c, c->x, coords_io, 3 * (size_t)c->n, ptr_kind);
      if (rc) return rc;
    }
  }
  if (vel_io) {
    rc = copy_in(c, c->v, vel_io, 3 * (size_t)c->n, ptr_kind);
    if (rc) return rc;
  }
  if (n_steps == 0) return DP_OK;
  // checkpoint (on the device, no host round trip) for a retry after a
  // neighbour-capacity overflow; the trace base is the step counter at entry
  const size_t nb = sizeof(double) * 3 * (size_t)c->n;
  for (int attempt = 0; attempt < 4; ++attempt) {
    if (!c->forces_valid) {
      rc = compute_now(c);
      if (rc) return rc;
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->xck, c->x, nb, cudaMemcpyDeviceToDevice, c->st), "checkpoint");
    CUDA_TRY(c, cudaMemcpyAsync(c->vck, c->v, nb, cudaMemcpyDeviceToDevice, c->st), "checkpoint");
    CUDA_TRY(c, cudaMemcpyAsync(c->stepck, c->step, sizeof(long long), cudaMemcpyDeviceToDevice, c->st), "checkpoint");
    CUDA_TRY(c, cudaMemcpyAsync(c->step + 1, c->step, sizeof(long long), cudaMemcpyDeviceToDevice, c->st), "step base");
    int tl = energies_out ? n_steps : 1;
    if (!c->graph || c->graph_stale || c->graph_dt != dt_fs || c->graph_trace_len < tl) {
      rc = build_step_graph(c, dt_fs, std::max(tl, c->trace_len));
      if (rc) return rc;
    }
    for (int s = 0; s < n_steps; ++s) {
      NvtxRange step("md step");
      CUDA_TRY(c, cudaGraphLaunch(c->graph, c->st), "graph launch");
    }
    int fl = 0;
    rc = read_flags(c, &fl);
    if (rc) return rc;
    if (fl & kFlagOverflow) {
      rc = alloc_skin(c, c->cap * 2);
      if (rc) return rc;
      CUDA_TRY(c, cudaMemcpyAsync(c->x, c->xck, nb, cudaMemcpyDeviceToDevice, c->st), "restore");
      CUDA_TRY(c, cudaMemcpyAsync(c->v, c->vck, nb, cudaMemcpyDeviceToDevice, c->st), "restore");
      CUDA_TRY(c, cudaMemcpyAsync(c->step, c->stepck, sizeof(long long), cudaMemcpyDeviceToDevice, c->st), "restore");
      c->forces_valid = false;
      continue;
    }
    if (fl & kFlagMirror) return fail(c, DP_ERR_CUDA, "internal error: neighbour mirror missing");
    if (fl & kFlagTimeout) return fail(c, DP_ERR_TIMEOUT, "a device-side wait gave up");
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

extern "C" int dp_enqueue_network(dp_ctx* c, int reps, int parts) {
  if (!c) return fail(nullptr, DP_ERR_ARG, "ctx is NULL");
  if (reps < 0) return fail(c, DP_ERR_ARG, "reps must be >= 0");
  if (!c->forces_valid) return fail(c, DP_ERR_ARG, "no resident neighbour lists: call dp_compute first");
  for (int r = 0; r < reps; ++r)
    c->model->run_parts(nbr_view(c), c->types, c->atom_e, c->st, parts ? parts : ~0);
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
  for (void* p : c->cell_allocs) cudaFree(p);
  for (void* p : c->allocs) cudaFree(p);
  if (c->own_stream && c->st) cudaStreamDestroy(c->st);
  delete c;
}

extern "C" const char* dp_last_error(const dp_ctx* c) {
  if (!c) return g_init_error.c_str();
  return c->err.c_str();
}

// ===================================================================== serving
// Continuous batching of independent systems (paper Sec. V-C finds memory the
// limiting resource for DPA models; here requests are admitted as slots and
// device memory free up).  All resident systems advance together: one tick =
// one velocity-Verlet step of every system in one CUDA-graph launch over the
// packed batch.  Requests are admitted first-in first-out when a slot is free
// and the atoms fit the memory-sized capacity; finished ones leave at the end
// of their last tick, and the batch is repacked before the next one.

struct ServerReq {
  uint64_t id = 0;
  int n = 0;
  double box[3] = {0, 0, 0};
  std::vector<int> types;
  std::vector<double> x, v;
  std::vector<double> trace;  // {E_pot, E_kin} per step
  int steps_total = 0, steps_done = 0;
  int state = 0;              // 0 queued, 1 running, 2 done
  long long tick_submit = 0, tick_admit = -1, tick_done = -1;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int offset = -1;            // first atom in the current batch
};

struct dp_server {
  dp_ctx* ctx = nullptr;
  double dt = 0.5;
  int max_slots = 0;
  int n_cap = 0;
  uint64_t next_id = 1;
  std::map<uint64_t, ServerReq> reqs;
  std::deque<uint64_t> queue;
  std::vector<uint64_t> active;       // batch order
  bool dirty = false;
  long long ticks = 0, atom_steps = 0;
  int atoms_in_use = 0, max_active = 0, max_atoms_seen = 0;
  long long waits_for_memory = 0, waits_for_slot = 0;
  std::vector<double> tick_ms;
  double busy_ms = 0;
  double* stage_x = nullptr;
  double* stage_v = nullptr;
  double* stage_f = nullptr;
  std::string err;
};

static thread_local std::string g_server_error;

static double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// bytes of device memory one atom needs in a fused context (skin capacity cap)
static size_t bytes_per_atom(const dp_model_desc* d, int cap) {
  size_t nm = d->nmax, L = d->n_layers;
  size_t ctx = 120 + 12 + 16 + 24 + 4 * nm + 12 * nm + 24 * nm + 8 + 72 + (size_t)cap * 22 + 48 + 48;
  size_t model = (L + 1) * 32768 + L * 512 + 128 * (size_t)d->m2 * 6 + 2048 + 12 * nm + 8;
  if (d->fit_heads > 1) model += 8 * (size_t)(d->fit_heads - 1);
  // message passing: post-message tiles, FP32 stream and dE/dG', U, h, dh, dq, sums
  if (d->message_passing) model += L * 32768 + 2 * 65536 + L * 512 + 3 * 512 + 4096;
  return ctx + model;
}

extern "C" int dp_server_create(dp_server** out, const dp_model_desc* desc, const double* masses,
                                const double* weights, size_t n_weights, int max_slots,
                                long long max_atoms, size_t mem_budget, double dt_fs,
                                void* cuda_stream) {
  if (!out) { g_server_error = "out is NULL"; return DP_ERR_ARG; }
  *out = nullptr;
  AfDims afd{};
  int rc = check_model(desc, weights, n_weights, masses, &afd);
  if (rc) { g_server_error = g_init_error; return rc; }
  if (desc->family != DP_FAMILY_ATTENTION || desc->precision != DP_PREC_FUSED) {
    g_server_error = "the server batches the fused attention-family model";
    return DP_ERR_UNSUPPORTED;
  }
  if (!masses) { g_server_error = "masses are required"; return DP_ERR_ARG; }
  if (max_slots < 1 || !(dt_fs > 0)) { g_server_error = "need max_slots >= 1 and dt > 0"; return DP_ERR_ARG; }
  // capacity: atoms that fit the memory budget (default: 80 % of free memory)
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    g_server_error = "cudaMemGetInfo failed";
    return DP_ERR_CUDA;
  }
  size_t budget = mem_budget ? mem_budget : (size_t)(0.8 * (double)free_b);
  const double rskin = desc->rcut + (desc->skin > 0 ? desc->skin : 1.0);
  int cap = skin_capacity(rskin, 0.1, 1 << 20);
  size_t fixed = (size_t)256 << 20;  // weights, tiles and per-system tables
  if (budget <= fixed) { g_server_error = "memory budget too small"; return DP_ERR_OOM; }
  long long n_cap = (long long)((budget - fixed) / bytes_per_atom(desc, cap));
  if (max_atoms > 0 && max_atoms < n_cap) n_cap = max_atoms;
  if (desc->message_passing && n_cap > 500000) n_cap = 500000;   // the fused form's limit
  if (n_cap < 1) { g_server_error = "memory budget too small"; return DP_ERR_OOM; }
  if (n_cap > (1 << 30)) n_cap = 1 << 30;
  std::vector<int> types0((size_t)n_cap, 0);
  dp_ctx* c = nullptr;
  rc = ctx_create(&c, desc, masses, weights, cuda_stream, (int)n_cap, max_slots, types0.data(), cap,
                  afd);
  if (rc) { g_server_error = g_init_error; return rc; }
  dp_server* s = new dp_server();
  s->ctx = c;
  s->dt = dt_fs;
  s->max_slots = max_slots;
  s->n_cap = (int)n_cap;
  if (cudaMalloc(&s->stage_x, sizeof(double) * 3 * n_cap) != cudaSuccess ||
      cudaMalloc(&s->stage_v, sizeof(double) * 3 * n_cap) != cudaSuccess ||
      cudaMalloc(&s->stage_f, sizeof(double) * 3 * n_cap) != cudaSuccess) {
    g_server_error = "out of device memory for the staging buffers";
    dp_server_free(s);
    return DP_ERR_OOM;
  }
  *out = s;
  return DP_OK;
}

extern "C" int dp_server_capacity(dp_server* s, int* max_atoms, int* max_slots) {
  if (!s) return DP_ERR_ARG;
  if (max_atoms) *max_atoms = s->n_cap;
  if (max_slots) *max_slots = s->max_slots;
  return DP_OK;
}

extern "C" int dp_server_submit(dp_server* s, int n_atoms, const int32_t* types,
                                const double* box, const double* coords, const double* vel,
                                int n_steps, uint64_t* req_id) {
  if (!s || !types || !box || !coords || !vel || !req_id || n_steps < 1 || n_atoms < 1) {
    if (s) s->err = "invalid argument";
    return DP_ERR_ARG;
  }
  if (n_atoms > s->n_cap) {
    s->err = "system larger than the server's memory capacity";
    return DP_ERR_OOM;
  }
  for (int i = 0; i < n_atoms; ++i)
    if (types[i] < 0 || types[i] >= s->ctx->desc.n_species) {
      s->err = "species out of range";
      return DP_ERR_ARG;
    }
  ServerReq r;
  r.id = s->next_id++;
  r.n = n_atoms;
  for (int a = 0; a < 3; ++a) r.box[a] = box[a];
  r.types.assign(types, types + n_atoms);
  r.x.assign(coords, coords + 3 * (size_t)n_atoms);
  r.v.assign(vel, vel + 3 * (size_t)n_atoms);
  r.steps_total = n_steps;
  r.tick_submit = s->ticks;
  r.t_submit = now_ms();
  *req_id = r.id;
  s->queue.push_back(r.id);
  s->reqs.emplace(r.id, std::move(r));
  return DP_OK;
}

// Rebuild the packed batch from the active requests: retained systems keep
// their device state (copied through the staging buffers), new ones are
// uploaded from the host.
// Pack the active systems contiguously: the ones already running first, in
// their order, carrying positions, velocities and forces (still valid: a
// system's forces depend on its own atoms only), then the newly admitted ones.
// Only the new systems need a force evaluation before the next step.
static int server_repack(dp_server* s) {
  dp_ctx* c = s->ctx;
  std::vector<int> natoms, types;
  std::vector<double> boxes;
  std::vector<uint64_t> order;
  for (int pass = 0; pass < 2; ++pass)
    for (uint64_t id : s->active)
      if ((s->reqs[id].offset >= 0) == (pass == 0)) order.push_back(id);
  s->active.swap(order);
  int off = 0, carried = 0;
  for (uint64_t id : s->active) {
    ServerReq& r = s->reqs[id];
    const size_t b = sizeof(double) * 3 * r.n;
    if (r.offset >= 0) {
      CUDA_TRY(c, cudaMemcpyAsync(s->stage_x + 3 * off, c->x + 3 * r.offset, b, cudaMemcpyDeviceToDevice, c->st), "repack");
      CUDA_TRY(c, cudaMemcpyAsync(s->stage_v + 3 * off, c->v + 3 * r.offset, b, cudaMemcpyDeviceToDevice, c->st), "repack");
      if (c->forces_valid)
        CUDA_TRY(c, cudaMemcpyAsync(s->stage_f + 3 * off, c->F + 3 * r.offset, b, cudaMemcpyDeviceToDevice, c->st), "repack");
      carried = off + r.n;
    } else {
      CUDA_TRY(c, cudaMemcpyAsync(s->stage_x + 3 * off, r.x.data(), b, cudaMemcpyHostToDevice, c->st), "repack");
      CUDA_TRY(c, cudaMemcpyAsync(s->stage_v + 3 * off, r.v.data(), b, cudaMemcpyHostToDevice, c->st), "repack");
    }
    natoms.push_back(r.n);
    boxes.insert(boxes.end(), r.box, r.box + 3);
    types.insert(types.end(), r.types.begin(), r.types.end());
    r.offset = off;
    off += r.n;
  }
  s->atoms_in_use = off;
  if (off == 0) {
    s->dirty = false;
    return DP_OK;
  }
  const bool keep_forces = c->forces_valid && carried > 0;
  CUDA_TRY(c, cudaMemcpyAsync(c->x, s->stage_x, sizeof(double) * 3 * off, cudaMemcpyDeviceToDevice, c->st), "repack");
  CUDA_TRY(c, cudaMemcpyAsync(c->v, s->stage_v, sizeof(double) * 3 * off, cudaMemcpyDeviceToDevice, c->st), "repack");
  if (keep_forces)
    CUDA_TRY(c, cudaMemcpyAsync(c->F, s->stage_f, sizeof(double) * 3 * carried, cudaMemcpyDeviceToDevice, c->st), "repack");
  int rc = ctx_set_systems(c, (int)natoms.size(), natoms.data(), boxes.data(), types.data());
  if (rc) return rc;
  if (keep_forces) {
    if (carried == off) {      // departures only: no evaluation, rebuild the lists next step
      launch_flag_set(c->flags, kFlagRebuild, c->st);
      c->forces_valid = true;
    } else {
      c->valid_below = carried;
    }
  }
  s->dirty = false;
  return DP_OK;
}

extern "C" int dp_server_tick(dp_server* s, int* n_active, int* n_queued) {
  NvtxRange nvtx("dp_server_tick");
  if (!s) return DP_ERR_ARG;
  dp_ctx* c = s->ctx;
  const double t0 = now_ms();
  // admission, first in first out
  while (!s->queue.empty()) {
    ServerReq& r = s->reqs[s->queue.front()];
    if ((int)s->active.size() >= s->max_slots) { ++s->waits_for_slot; break; }
    int in_use = 0;
    for (uint64_t id : s->active) in_use += s->reqs[id].n;
    if (in_use + r.n > s->n_cap) { ++s->waits_for_memory; break; }
    r.state = 1;
    r.tick_admit = s->ticks;
    r.t_admit = now_ms();
    r.offset = -1;
    s->active.push_back(r.id);
    s->queue.pop_front();
    s->dirty = true;
  }
  if (s->dirty) {
    int rc = server_repack(s);
    if (rc) { s->err = c->err; return rc; }
  }
  if (!s->active.empty()) {
    int rc = DP_OK;
    if (!c->forces_valid) rc = compute_now(c);
    if (rc) { s->err = c->err; return rc; }
    long long st[2];
    for (int attempt = 0; attempt < 4; ++attempt) {
      CUDA_TRY(c, cudaMemcpyAsync(st, c->step, sizeof st, cudaMemcpyDeviceToHost, c->st), "tick");
      CUDA_TRY(c, cudaStreamSynchronize(c->st), "tick");
      st[1] = st[0];
      CUDA_TRY(c, cudaMemcpyAsync(c->step, st, sizeof st, cudaMemcpyHostToDevice, c->st), "tick");
      CUDA_TRY(c, cudaMemcpyAsync(s->stage_x, c->x, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToDevice, c->st), "tick");
      CUDA_TRY(c, cudaMemcpyAsync(s->stage_v, c->v, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToDevice, c->st), "tick");
      if (!c->graph || c->graph_stale || c->graph_dt != s->dt || c->graph_trace_len < 1) {
        rc = build_step_graph(c, s->dt, std::max(1, c->trace_len));
        if (rc) { s->err = c->err; return rc; }
      }
      CUDA_TRY(c, cudaGraphLaunch(c->graph, c->st), "tick");
      int fl = 0;
      rc = read_flags(c, &fl);
      if (rc) { s->err = c->err; return rc; }
      if (fl & kFlagOverflow) {  // grow the skin lists and redo the step
        rc = alloc_skin(c, c->cap * 2);
        if (rc) { s->err = c->err; return rc; }
        CUDA_TRY(c, cudaMemcpyAsync(c->x, s->stage_x, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToDevice, c->st), "tick");
        CUDA_TRY(c, cudaMemcpyAsync(c->v, s->stage_v, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToDevice, c->st), "tick");
        st[1] = 0;
        CUDA_TRY(c, cudaMemcpyAsync(c->step, st, sizeof st, cudaMemcpyHostToDevice, c->st), "tick");
        c->forces_valid = false;
        rc = compute_now(c);
        if (rc) { s->err = c->err; return rc; }
        continue;
      }
      if (fl & kFlagTimeout) { s->err = "a device-side wait gave up"; return DP_ERR_TIMEOUT; }
      if (fl & kFlagNonFinite) { s->err = "energy or forces are not finite"; return DP_ERR_NONFINITE; }
      break;
    }
    std::vector<double> tr(2 * s->active.size());
    CUDA_TRY(c, cudaMemcpyAsync(tr.data(), c->trace, sizeof(double) * tr.size(), cudaMemcpyDeviceToHost, c->st), "tick");
    CUDA_TRY(c, cudaStreamSynchronize(c->st), "tick");
    ++s->ticks;
    s->atom_steps += c->n;
    s->max_active = std::max(s->max_active, (int)s->active.size());
    s->max_atoms_seen = std::max(s->max_atoms_seen, c->n);
    std::vector<uint64_t> still;
    for (size_t k = 0; k < s->active.size(); ++k) {
      ServerReq& r = s->reqs[s->active[k]];
      r.trace.push_back(tr[2 * k]);
      r.trace.push_back(tr[2 * k + 1]);
      if (++r.steps_done == r.steps_total) {
        const size_t b = sizeof(double) * 3 * r.n;
        CUDA_TRY(c, cudaMemcpyAsync(r.x.data(), c->x + 3 * r.offset, b, cudaMemcpyDeviceToHost, c->st), "results");
        CUDA_TRY(c, cudaMemcpyAsync(r.v.data(), c->v + 3 * r.offset, b, cudaMemcpyDeviceToHost, c->st), "results");
        r.state = 2;
        r.tick_done = s->ticks;
        s->dirty = true;
      } else {
        still.push_back(r.id);
      }
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->st), "results");
    const double t1 = now_ms();
    for (size_t k = 0; k < s->active.size(); ++k) {
      ServerReq& r = s->reqs[s->active[k]];
      if (r.state == 2) r.t_done = t1;
    }
    s->active.swap(still);
    s->tick_ms.push_back(t1 - t0);
    s->busy_ms += t1 - t0;
  }
  if (n_active) *n_active = (int)s->active.size();
  if (n_queued) *n_queued = (int)s->queue.size();
  return DP_OK;
}

extern "C" int dp_server_poll(dp_server* s, uint64_t req_id, int* state, double* coords,
                              double* vel, double* energies, double* latency_ms) {
  if (!s) return DP_ERR_ARG;
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) { s->err = "unknown request"; return DP_ERR_ARG; }
  ServerReq& r = it->second;
  if (state) *state = r.state;
  if (r.state != 2) return DP_OK;
  if (coords) memcpy(coords, r.x.data(), sizeof(double) * r.x.size());
  if (vel) memcpy(vel, r.v.data(), sizeof(double) * r.v.size());
  if (energies) memcpy(energies, r.trace.data(), sizeof(double) * r.trace.size());
  if (latency_ms) {
    latency_ms[0] = r.t_done - r.t_submit;
    latency_ms[1] = r.t_admit - r.t_submit;
    latency_ms[2] = (double)r.tick_admit;
    latency_ms[3] = (double)r.tick_done;
  }
  return DP_OK;
}

extern "C" int dp_server_stats(dp_server* s, double* out, int n_out) {
  if (!s || !out) return DP_ERR_ARG;
  std::vector<double> t = s->tick_ms;
  std::sort(t.begin(), t.end());
  auto pct = [&](double q) {
    if (t.empty()) return 0.0;
    size_t k = (size_t)std::min<double>((double)t.size() - 1, std::ceil(q * (double)t.size()) - 1);
    return t[k];
  };
  double v[10] = {(double)s->ticks, pct(0.50), pct(0.99), (double)s->atom_steps, s->busy_ms,
                  (double)s->max_active, (double)s->max_atoms_seen, (double)s->waits_for_memory,
                  (double)s->waits_for_slot, (double)s->n_cap};
  for (int k = 0; k < n_out && k < 10; ++k) out[k] = v[k];
  return DP_OK;
}

extern "C" void dp_server_free(dp_server* s) {
  if (!s) return;
  if (s->ctx) cudaStreamSynchronize(s->ctx->st);
  if (s->stage_x) cudaFree(s->stage_x);
  if (s->stage_v) cudaFree(s->stage_v);
  if (s->stage_f) cudaFree(s->stage_f);
  dp_free(s->ctx);
  delete s;
}

extern "C" const char* dp_server_last_error(const dp_server* s) {
  return s ? s->err.c_str() : g_server_error.c_str();
}
