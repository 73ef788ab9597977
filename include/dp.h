/*
 * dp.h -- C ABI of libdp.so: deep-potential energy, force and virial inference
 * and velocity-Verlet molecular dynamics on one NVIDIA B300 (sm_103a).
 *
 * The method is the one the paper (arXiv 2602.02234, Sec. II-III) runs inside
 * GROMACS through DeePMD-kit: a deep potential maps each atom's local
 * environment (neighbours within a cutoff, Sec. II; 0.6 nm, Sec. IV) to an
 * atomic energy, E is their sum and the forces are -dE/dx (Sec. II).  The MD
 * engine passes coordinates, species and the box and receives forces (Sec.
 * III); these calls are that interface.  Two model families are provided:
 *
 *   DP_FAMILY_ATTENTION -- DPA2-like (Sec. II: "repinit" embedding MLP,
 *     "repformer" residual self-attention layers, "fitting-net"): smooth switch
 *     and environment matrix, per-neighbour embedding MLP, gated neighbour
 *     attention, descriptor T^T T, per-atom fitting MLP.
 *   DP_FAMILY_GRAPH -- DPA3-like (Sec. II: GNN with line-graph bond and angle
 *     representations): node, edge and angle updates over the neighbour graph,
 *     then the per-atom fitting MLP.
 *
 * Units: Angstrom, femtosecond, amu, eV.  Boxes are orthorhombic and periodic;
 * coordinates may lie outside the box (they are wrapped internally only for
 * neighbour search).
 *
 * Conventions for every call:
 *   - The caller owns every array it passes; the library copies inputs and
 *     writes outputs before returning (dp_compute, dp_step synchronise the
 *     library's stream before returning).
 *   - Array arguments are host pointers unless the call's ptr_kind argument is
 *     DP_PTR_DEVICE, in which case they are device pointers on the context's
 *     device.
 *   - Return value 0 (DP_OK) on success, a negative DP_ERR_* code otherwise;
 *     dp_last_error() gives a message.  No C++ exception crosses the ABI.
 *   - A context is not thread-safe: one host thread at a time per context.
 *   - Weight blob: FP64, layout fixed by the model description (see
 *     dp_weight_count); the library keeps its own converted copies.
 */
#ifndef DP_H
#define DP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  DP_OK = 0,
  DP_ERR_ARG = -1,             /* invalid argument (message says which)      */
  DP_ERR_OOM = -2,             /* device memory (or the set budget) exceeded */
  DP_ERR_NLIST_OVERFLOW = -3,  /* more candidates than the list capacity     */
  DP_ERR_TIMEOUT = -4,         /* a device-side wait gave up                 */
  DP_ERR_NONFINITE = -5,       /* energy, forces or virial not finite, or    */
                               /* beyond the exact sums' range (a term of    */
                               /* 2^46 or a sum of 2^47 in magnitude)        */
  DP_ERR_CUDA = -6,            /* a CUDA runtime call failed                 */
  DP_ERR_UNSUPPORTED = -7      /* valid request the library does not support */
};

enum { DP_FAMILY_ATTENTION = 0, DP_FAMILY_GRAPH = 1 };

/* Arithmetic of the network:
 *   PLAIN_F64 -- unfused kernels, everything in FP64 (small systems, parity);
 *   PLAIN_F32 -- unfused kernels, one simple kernel per operation, FP32;
 *   FUSED     -- attention family: three persistent kernels per evaluation:
 *                every matrix product on the tensor cores (tcgen05) with 16-bit
 *                operands (FP16; BF16 when the library is built with
 *                DP_FUSED_BF16) and FP32 accumulation, FP32 switch/softmax/
 *                LayerNorm, FP64 energy, virial and integration.  Needs m1 =
 *                hidden = 128 with 4 heads, nmax <= 128.
 *                Graph family ("mixed"): the unfused FP32 kernels with every
 *                matrix product on the tensor cores (16-bit operands: FP16, or
 *                BF16 when built with DP_GF_BF16; FP32 accumulation).  Needs
 *                node, edge, node + edge and fitting widths that are multiples
 *                of 16, at most 256.
 *                DP_ERR_UNSUPPORTED for other sizes. */
enum { DP_PREC_PLAIN_F64 = 0, DP_PREC_PLAIN_F32 = 1, DP_PREC_FUSED = 2 };

enum { DP_PTR_HOST = 0, DP_PTR_DEVICE = 1 };

typedef struct dp_model_desc {
  int family;      /* DP_FAMILY_*                                              */
  int precision;   /* DP_PREC_*                                                */
  int n_species;   /* species indices are 0 .. n_species-1                     */
  int nmax;        /* neighbours kept per atom (nearest first)                 */
  double rcut;     /* cutoff rc (A)                                            */
  double rcut_smth;/* switch start rs (A), rs < rc                             */
  /* attention family */
  int e1, e2, m1;  /* embedding 1 -> e1 -> e2 -> m1                            */
  int m2;          /* descriptor axis width (m2 <= m1)                         */
  int n_layers;    /* attention layers                                         */
  int hidden;      /* attention width H = heads * d                            */
  int heads;
  /* graph family */
  int node_dim, edge_dim, n_gnn_layers;
  int angle_nmax;  /* angle neighbours per atom                                */
  double angle_rcut, angle_rcut_smth;
  /* fitting MLP widths (both families): in -> f1 -> f2 -> f3 -> 1            */
  int f1, f2, f3;
  /* neighbour-list maintenance (dp_step): skin (A) and rebuild period (steps).
   * The result never depends on them: lists are rebuilt early whenever an atom
   * moved more than skin/2 since the last build. 0 selects 1 A / 10 steps.   */
  double skin;
  int rebuild_every;
  /* attention family: fitting heads sharing one descriptor (the paper's
   * multi-task large atomic models, Sec. II: one branch per training set).
   * 0 or 1 = one head.  Head 0 gives dp_compute's energy, the forces, the
   * virial and the MD; every head's energy comes from dp_get_head_energies.
   * The weight blob holds the fitting nets of head 0, 1, ... in order.     */
  int fit_heads;
  /* attention family: 1 = cross-atom message passing (DPA2's repformer layers
   * exchange information between neighbouring atoms, Sec. II; DPA2 needs the
   * atoms within n_layers x rc, Sec. III).  An atom channel h (width m1)
   * starts at Wt[t_i]; before attention layer l every kept pair feature G_ip
   * gains tanh(h_j Wm_l + bm_l) of its neighbour j, and after the layer
   * h_i += (1/nmax) sum_p sw_ip G_ip.  Atom i's energy then depends on the
   * atoms up to n_layers neighbour hops away.  Plain precisions only, one
   * fitting head; every atom's activations stay resident (one chunk).     */
  int message_passing;
  int reserved[5];
} dp_model_desc;

typedef struct dp_ctx dp_ctx;

/* Number of FP64 values in the weight blob for `desc` (written to *n).
 * Attention family, in order (row-major W[in][out], W before b):
 *   per species t:  W1[1][e1] b1[e1] W2[e1][e2] b2[e2] W3[e2][m1] b3[m1]
 *   (message passing) Wt[n_species][m1]
 *   per layer l:    Wq[m1][H] Wk[m1][H] Wv[m1][H] Wo[H][m1] bo[m1]
 *                   (message passing) Wm[m1][m1] bm[m1]
 *   per species t:  F1[m1*m2][f1] c1[f1] F2[f1][f2] c2[f2] F3[f2][f3] c3[f3] F4[f3][1] c4[1]
 * Graph family (Nd = node_dim, Ed = edge_dim), in order:
 *   W_type[S][Nd] w_e[1][Ed] b_e[Ed]
 *   per layer l:    Wm[Nd][Ed] Wn[Nd+Ed][Nd] bn[Nd] Wa[Nd][Ed] Wb[Nd][Ed] Wc[Ed][Ed]
 *                   be[Ed] Wp[Ed][Ed] Wphi[4][Ed] Wq[Ed][Ed] bq[Ed]
 *   per species t:  F1[Nd][f1] c1 F2[f1][f2] c2 F3[f2][f3] c3 F4[f3][1] c4[1]
 * Errors: DP_ERR_ARG for an invalid description. */
int dp_weight_count(const dp_model_desc* desc, size_t* n);

/* Create a context for one system of n_atoms atoms.
 *   types   [n_atoms]     species index of each atom (host)
 *   masses  [n_species]   amu, only needed by dp_step (host, nullable)
 *   box     [3]           orthorhombic box lengths, A (host)
 *   weights [n_weights]   FP64 blob (host)
 *   cuda_stream           cudaStream_t to run on (NULL: the library creates one)
 * The library allocates all device buffers here and fails early with
 * DP_ERR_OOM when they do not fit.  *out is NULL on failure. */
int dp_init(dp_ctx** out, const dp_model_desc* desc, int n_atoms, const int32_t* types,
            const double* masses, const double* box, const double* weights, size_t n_weights,
            void* cuda_stream);

/* Energy (eV), forces (n_atoms x 3, eV/A, nullable) and virial (3 x 3 row-major,
 * eV, nullable) at coordinates (n_atoms x 3, A).  Virial X_ab = -sum over
 * neighbour pairs of r_a g_b with g = dE/dr.  Neighbour lists are rebuilt as
 * needed.  The coordinates become the context's resident positions. */
int dp_compute(dp_ctx* ctx, const double* coords, double* energy, double* forces, double* virial,
               int ptr_kind);

/* n_steps of velocity-Verlet NVE with time step dt_fs:
 *   v += dt/2 F/m; x += dt v; F = F(x); v += dt/2 F/m.
 * coords_io / vel_io (n_atoms x 3): when non-NULL they are uploaded before the
 * first step and overwritten with the final state; when NULL the resident
 * state is used and kept on the device.  energies_out (nullable): per step
 * {potential, kinetic} in eV, 2*n_steps values.  The whole step is one CUDA
 * graph launch.  Needs masses at dp_init. */
int dp_step(dp_ctx* ctx, int n_steps, double dt_fs, double* coords_io, double* vel_io,
            double* energies_out, int ptr_kind);

/* Copy the resident state out / in (n_atoms x 3 each, nullable), plus the step
 * counter.  Resuming from a saved state reproduces the run bit for bit. */
int dp_get_state(dp_ctx* ctx, double* coords, double* vel, long long* step, int ptr_kind);
int dp_set_state(dp_ctx* ctx, const double* coords, const double* vel, long long step,
                 int ptr_kind);

/* Inspection after dp_compute / dp_step (host pointers):
 *   nbr_j   [n_atoms x nmax]     neighbour atom, nearest first, -1 = empty slot
 *   nbr_img [n_atoms x nmax x 3] periodic image n of each neighbour
 *                                (r = (w_j - w_i) + n L, w = wrapped position)
 *   n_in_rc [n_atoms]            neighbours within rc before truncation
 * Any pointer may be NULL. */
int dp_get_neighbours(dp_ctx* ctx, int32_t* nbr_j, int32_t* nbr_img, int32_t* n_in_rc);

/* Atomic energies e_i (n_atoms, host) of the last evaluation. */
int dp_get_atom_energies(dp_ctx* ctx, double* atom_e);

/* Energies of every fitting head at the last evaluation: out[s * k + h] for
 * system s and head h (k = fit_heads; s = 0 for a single-system context), in
 * host memory, FP64.  Head 0 equals dp_compute's energy.  DP_ERR_ARG for NULL
 * pointers or before the first evaluation. */
int dp_get_head_energies(dp_ctx* ctx, double* out);

/* DP group (paper Sec. III: the deep potential covers a selected group of
 * atoms, the protein, and the rest is left to a classical force field).
 * mask: n_atoms bytes in host memory, nonzero = member; NULL = every atom
 * (the default).  With a group, only pairs of members are neighbours and only
 * members carry energy: the result equals evaluating the members alone in the
 * same box, and non-members get zero energy and zero force.  The next
 * evaluation rebuilds the neighbour lists.  DP_ERR_ARG for a NULL ctx,
 * DP_ERR_UNSUPPORTED for a multi-system (serving) context. */
int dp_set_group(dp_ctx* ctx, const unsigned char* mask);

/* Centres of one subdomain of a domain decomposition (the paper names
 * domain-decomposed inference future work, Sec. V-B, Sec. VII): the context
 * holds the owned atoms and their ghosts (every atom within rc of the
 * subdomain); mask (n_atoms bytes, host memory, nonzero = owned) selects the
 * centres.  Only centres carry energy and have neighbour lists, every atom may
 * be a neighbour, so the forces of dp_compute are the owned centres' partial
 * forces on every local atom: the ghosts' parts belong to their owners.  NULL
 * restores every atom.  Atom-local models only (the attention family without
 * message passing): DP_ERR_UNSUPPORTED otherwise, and for a multi-system
 * context; DP_ERR_ARG for a NULL ctx. */
int dp_set_centres(dp_ctx* ctx, const unsigned char* mask);

/* Energy seed of one subdomain, for every model and needed by the
 * layer-coupled ones (attention family with message passing, graph family),
 * whose energy reaches n_layers neighbour hops: the context holds the owned
 * atoms and every atom within n_layers x rc of the subdomain (Sec. III: the
 * broadened ghost area); mask (n_atoms bytes, host memory, nonzero = owned)
 * marks the atoms whose energy counts.  Every atom evaluates as a centre (the
 * ghosts' features feed the owned atoms'), only marked atoms carry energy, and
 * the adjoint is seeded with the mask, so dp_compute's forces are
 * -d(sum of owned energies)/dx on every local atom.  NULL restores every atom.
 * DP_ERR_ARG for a NULL ctx, DP_ERR_UNSUPPORTED for a multi-system context. */
int dp_set_energy_seed(dp_ctx* ctx, const unsigned char* mask);

/* Enqueue `reps` evaluations of the network alone (no neighbour update, no
 * force assembly) on the context's stream, at the resident neighbour lists,
 * without synchronising; for timing the network kernels with events on that
 * stream.  parts: bit mask of the network's kernels to run (0 = all; for the
 * fused path bit 0 = per-atom forward, bit 1 = fitting, bit 2 = per-atom
 * backward; a part reuses the intermediate results of the last evaluation).
 * Needs a prior dp_compute or dp_step. */
int dp_enqueue_network(dp_ctx* ctx, int reps, int parts);

/* Number of kernels one dp_compute / one dp_step launches (for reporting). */
int dp_kernels_per_step(dp_ctx* ctx, int* n_compute, int* n_step);

/* Device bytes held by the context. */
int dp_device_bytes(dp_ctx* ctx, size_t* bytes);

void dp_free(dp_ctx* ctx);

/* ---------------------------------------------------------------- serving
 * Continuous batching of many independent systems on one GPU (the memory
 * limits the paper reports for DPA models, Sec. V-C, become the admission
 * rule).  Requests (a system and a number of MD steps) are queued; every tick
 * admits queued requests first-in first-out while a slot is free and their
 * atoms fit the memory-sized capacity, then advances every resident system by
 * one velocity-Verlet step in one CUDA-graph launch over the packed batch.
 * A request leaves at the end of its last step.  Per-atom work does not depend
 * on the batch, so a system's trajectory is the same alone and in any mix.
 * Fused attention-family model only (DP_ERR_UNSUPPORTED otherwise). */
typedef struct dp_server dp_server;

/* max_slots: resident systems at most; max_atoms (0: no limit) and
 * mem_budget_bytes (0: 80 % of free device memory) bound the packed atoms;
 * masses [n_species] amu; dt_fs for every request. */
int dp_server_create(dp_server** out, const dp_model_desc* desc, const double* masses,
                     const double* weights, size_t n_weights, int max_slots, long long max_atoms,
                     size_t mem_budget_bytes, double dt_fs, void* cuda_stream);
/* Atoms and slots the server can hold at once. */
int dp_server_capacity(dp_server* srv, int* max_atoms, int* max_slots);
/* Queue a request (host arrays, copied): species [n], box [3], coords and
 * velocities [n x 3].  DP_ERR_OOM if the system alone exceeds the capacity. */
int dp_server_submit(dp_server* srv, int n_atoms, const int32_t* types, const double* box,
                     const double* coords, const double* vel, int n_steps, uint64_t* req_id);
/* Admit, repack if needed, advance every resident system one step. */
int dp_server_tick(dp_server* srv, int* n_active, int* n_queued);
/* state: 0 queued, 1 running, 2 done.  When done: final coords/velocities
 * [n x 3], per-step {E_pot, E_kin} [2 x n_steps] (each nullable) and
 * latency_ms[4] = {submit->done ms, submit->admit ms, tick admitted, tick done}. */
int dp_server_poll(dp_server* srv, uint64_t req_id, int* state, double* coords, double* vel,
                   double* energies, double* latency_ms);
/* out[0..9] = ticks, p50 tick ms, p99 tick ms, atom-steps, busy ms, max resident
 * systems, max resident atoms, ticks the queue head waited for memory, ticks it
 * waited for a slot, atom capacity. */
int dp_server_stats(dp_server* srv, double* out, int n_out);
void dp_server_free(dp_server* srv);
const char* dp_server_last_error(const dp_server* srv);

/* Diagnostics (no paper counterpart): one 128 x n x k BF16 tensor-core product
 * D = A B^T on the device (tcgen05.mma, FP32 accumulation in tensor memory),
 * with A (128 x k) and B (n x k) staged in shared memory in K-major (a_mn /
 * b_mn = 0) or MN-major (1) core-matrix layout; swap = 0 uses the descriptor
 * stride convention of the library's fused kernels, 1 the other assignment.
 * Host pointers, row-major FP32 (rounded to BF16 on the device).  16 <= n <=
 * 256 and 16 <= k <= 128, multiples of 16.  Allocates its own buffers.
 * Returns DP_ERR_ARG for sizes it cannot stage safely, DP_ERR_TIMEOUT if the
 * product never completed (bounded wait). */
int dp_selftest_mma(int n, int k, int a_mn, int b_mn, int swap, const float* A, const float* B,
                    float* D);

/* Diagnostics (no paper counterpart): SM cycles per tensor-core product of
 * 128 x n x 16 (16-bit operands from shared memory, FP32 accumulation in
 * tensor memory), measured on one CTA over `reps` groups of 64 products issued
 * by `issuers` threads (1..8) and waited for after each group.  16 <= n <=
 * 128, a multiple of 16; 1 <= reps <= 100000.  Allocates its own buffers.
 * Returns DP_ERR_ARG for other sizes, DP_ERR_TIMEOUT if a group never
 * completed (bounded wait). */
int dp_selftest_mma_rate(int n, int issuers, int reps, double* cycles_per_mma);

/* Diagnostics (no paper counterpart): the bounded device-side wait of the
 * fused kernels, on an mbarrier that is never completed, polled at most
 * max_polls (1..2^20) times.  Returns DP_ERR_TIMEOUT when the wait ran out and
 * the kernel returned normally (the expected outcome). */
int dp_selftest_timeout(long long max_polls);

/* Neighbour lists of one small periodic system without any device allocation.
 * The paper has no counterpart: it is for callers that cannot allocate device
 * memory (an MD engine that owns the allocator or has spent its memory budget,
 * or a plugin that only receives pointers to the engine's buffers).  The
 * lists are the ones dp_get_neighbours reports after dp_compute: every image
 * (j, n) with 0 < |r| < rcut, nearest first by (|r|^2, j, n), the first nmax.
 *   coords  [n_atoms x 3]        device pointer, A
 *   box     [3]                  host pointer, A (orthorhombic)
 *   nbr_j   [n_atoms x nmax]     device pointer, -1 = empty slot
 *   nbr_img [n_atoms x nmax x 3] device pointer
 *   n_in_rc [n_atoms]            device pointer, neighbours within rcut
 *   cuda_stream                  stream to run on (NULL: legacy default stream)
 * Limits: n_atoms <= 1024 and at most 384 neighbours within rcut per atom
 * (DP_ERR_ARG / DP_ERR_NLIST_OVERFLOW beyond).  A box whose own periodic
 * images of one atom already exceed 384 within rcut is refused before any
 * launch.  After DP_ERR_NLIST_OVERFLOW from the kernel, n_in_rc of every atom
 * that overflowed is 385 (more than the limit) and its rows of nbr_j /
 * nbr_img are empty (-1 / 0); the other atoms' rows are complete.  Its scratch memory is a static
 * array of the library (about 6.3 MB on every GPU that loads it, held until
 * the process exits), shared by all calls: calls that overlap on the GPU race
 * and must be serialised by the caller.  The first call on a device looks up
 * the array's device address; make that first call before any stream capture.
 * The call synchronises the stream to read its status.  Errors: message from
 * dp_noalloc_last_error(). */
int dp_neighbour_list_noalloc(const double* coords, int n_atoms, const double* box, double rcut,
                              int nmax, int32_t* nbr_j, int32_t* nbr_img, int32_t* n_in_rc,
                              void* cuda_stream);
const char* dp_noalloc_last_error(void);

/* Message of the last error on ctx (or of the last failed dp_init when ctx is
 * NULL).  Valid until the next call on the same context. */
const char* dp_last_error(const dp_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* DP_H */
