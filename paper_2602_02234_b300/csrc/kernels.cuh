// Launch interfaces between the runtime (ctx.cu) and the kernel files.
#pragma once

#include "common.cuh"

namespace dp {

// ----------------------------------------------------------------- neighbours
struct NlistArgs {
  int n;                 // atoms in the batch
  int ncell;             // cells in the batch
  int cap;               // skin-list capacity per atom
  int nmax;
  double rc, rskin;      // cutoff and cutoff + skin
  const double* x;       // unwrapped positions (n x 3)
  double* xref;          // positions at the last rebuild
  double* w;             // wrapped positions
  int* fl;               // floor(x / L) per component
  const int* sys_of;
  const SysInfo* sys;
  int *cell_of, *cell_cnt, *cell_fill, *cell_start, *cell_idx;
  SkinEntry* skin;
  int* skin_cnt;
  int* mirror;           // n x cap
  const unsigned char* grp;  // optional DP group: pairs only between members
  int grp_centres;           // 1: grp marks centres only (any atom is a neighbour)
  int* sel_j;            // n x nmax
  int* sel_img;          // n x nmax x 3
  double* sel_r;         // n x nmax x 3
  short* selpos;         // n x cap
  int* n_in_rc;          // n
  int* flags;
};

void launch_wrap(const NlistArgs& a, cudaStream_t st);
void launch_nlist_rebuild(const NlistArgs& a, cudaStream_t st);
void launch_select(const NlistArgs& a, cudaStream_t st);
void launch_flag_set(int* flags, int bits, cudaStream_t st);
int nlist_rebuild_kernels();
int select_max_cap();   // largest skin capacity the selection kernel supports
cudaError_t nlist_configure();

// ----------------------------------------------------------------- forces, MD
struct ForceArgs {
  int n, nmax, cap;
  int atom0;             // forces of atoms [atom0, n) only
  const int* sel_j;
  const double* sel_r;
  const SkinEntry* skin;
  const int* skin_cnt;
  const int* mirror;
  const short* selpos;
  const float* g32;      // pair gradients dE/dr (n x nmax x 3), FP32 paths
  const double* g64;     // or FP64
  double* F;             // n x 3
  double* atom_vir;      // n x 9
};
void launch_force_gather(const ForceArgs& a, cudaStream_t st);

// The per-system sums run in chunks of kReduceChunk atoms spread over the GPU,
// then one small block per system adds its chunks' exact partial sums.
constexpr int kReduceChunk = 512;
struct ReduceArgs {
  int n_sys;
  int n;                 // atoms of all systems (chunks = ceil(n / kReduceChunk) at most)
  unsigned long long* part;   // [sys][part_chunks][10] 128-bit partial sums (2 words each)
  int part_chunks;       // chunk capacity of `part` per system
  const int* sys_atom0;  // n_sys + 1 offsets
  const double* atom_e;  // n (unused by the kernel: atom_e_out is read and written)
  const double* atom_vir;// n x 9
  const double* F;       // n x 3 (finiteness check)
  double* sys_e;         // n_sys
  double* sys_vir;       // n_sys x 9
  int* flags;
  double* atom_e_out;    // with grp: energies of non-members set to 0 here
  const unsigned char* grp;
};
void launch_reduce(const ReduceArgs& a, cudaStream_t st);

struct MdArgs {
  int n;
  double dt;
  double* x;
  double* v;
  const double* F;
  const double* minv;    // kappa / m per atom
  const double* mass;    // m per atom
  const double* xref;
  double half_skin2;     // (skin / 2)^2
  int rebuild_every;
  long long* step;       // device step counter
  int* flags;
  double* atom_ke;       // n: kinetic energy per atom, written by the final kick
  int n_sys;
  const int* sys_atom0;
  const int* sys_of;
};
void launch_kick_drift(const MdArgs& a, cudaStream_t st);
void launch_kick_final(const MdArgs& a, cudaStream_t st);
// *differs |= 1 when the two arrays of `count` doubles differ in any bit
void launch_compare(long long count, const double* a, const double* b, int* differs,
                    cudaStream_t st);
void launch_record(const MdArgs& a, const double* sys_e, double* trace, int trace_len, cudaStream_t st);

// ----------------------------------------------------------------- plain model
struct AfDims {
  int n_species, e1, e2, m1, m2, n_layers, hidden, heads, f1, f2, f3, nmax;
  double rc, rs;
  int fit_heads;         // fitting heads sharing the descriptor (>= 1)
  int mp;                // 1: atom channel passed between neighbours every layer
};
// per (system, extra head) sums of atomic energies: head_e is [heads][n],
// out[s * heads + h]; members of a DP group only (grp optional)
void launch_head_reduce(int n_sys, int heads, int n, const int* sys_atom0, const double* head_e,
                        const unsigned char* grp, double* out, cudaStream_t st);

}  // namespace dp
