// The interface every network implementation exposes to the runtime: given the
// kept neighbours of every atom it writes atomic energies and the pair
// gradients g_ij = dE/dr_ij (one per neighbour slot).
#pragma once

#include <string>

#include "kernels.cuh"

namespace dp {

// The kept neighbours of every atom (slot p of atom i: atom sel_j[i*nmax+p],
// separation sel_r) and the skin-list structure that lets a kernel visit, for
// atom j, every slot (i, p) whose neighbour is j in a fixed order: skin entry
// c of j names i = skin[j*cap+c].j, mirror[j*cap+c] is the index c' of the
// reverse entry in i's skin list, and p = selpos[i*cap+c'] (-1: not kept).
struct NbrView {
  const int* sel_j;
  const double* sel_r;
  const SkinEntry* skin;
  const int* skin_cnt;
  const int* mirror;
  const short* selpos;
  int cap;
};

class Model {
 public:
  virtual ~Model() {}
  // Enqueue one evaluation on `st`; returns the number of kernels launched.
  virtual int run(const NbrView& nv, const int* types, double* atom_e, cudaStream_t st) = 0;
  // Only the kernels selected by the bit mask (implementations without
  // separable kernels run everything).
  virtual int run_parts(const NbrView& nv, const int* types, double* atom_e, cudaStream_t st,
                        int parts) {
    (void)parts;
    return run(nv, types, atom_e, st);
  }
  // Only atoms [atom0, n): their atomic energies and pair gradients (the
  // rest of both arrays is left as it was; implementations that cannot
  // restrict the range evaluate everything).
  virtual int run_range(const NbrView& nv, const int* types, double* atom_e, cudaStream_t st,
                        int atom0) {
    (void)atom0;
    return run(nv, types, atom_e, st);
  }
  // Atomic energies of fitting heads 1.. (FP64, [head - 1][capacity]; null
  // for a single head).
  virtual const double* head_energies() const { return nullptr; }
  // Pair gradients (n_atoms x nmax x 3): exactly one of the two is non-null.
  virtual const float* grad32() const { return nullptr; }
  virtual const double* grad64() const { return nullptr; }
  virtual size_t bytes() const = 0;
  // Evaluate n <= capacity atoms with these species from now on (a batch of
  // systems packed contiguously); false when the implementation cannot.
  virtual bool set_atoms(int n, const int* types_host) {
    (void)n;
    (void)types_host;
    return false;
  }
  // Device status word that kernels set bits of (kFlag*) instead of trapping.
  virtual void bind_flags(int* flags) { (void)flags; }
  // Per-atom energy seed (device bytes, 1 = the atom's energy counts; null:
  // every atom): the fitting adjoint starts from seed_i instead of 1, so the
  // pair gradients are those of sum_i seed_i e_i.  False when unsupported.
  virtual bool set_energy_seed(const unsigned char* seed) {
    (void)seed;
    return false;
  }
};

// Plain attention family (FP32 or FP64), unfused.  nmax <= 256.
Model* make_plain_af(const AfDims& m, bool f64, const double* weights, int n_atoms,
                     const int* types_host, size_t mem_budget, std::string* err);
// Fused attention family (BF16 tensor cores).  Returns nullptr and a reason when
// the sizes are outside what the fused kernels support.
bool fused_af_supported(const AfDims& m, std::string* why);
Model* make_fused_af(const AfDims& m, const double* weights, int n_atoms, const int* types_host,
                     std::string* err);

// Graph family sizes.
struct GfDims {
  int n_species, nd, ed, n_layers, f1, f2, f3, nmax, na;
  double rc, rs, rca, rsa;
};
size_t gf_weight_count(const GfDims& m);
// Whether the mixed graph form can tile these widths (reason when not).
bool gf_mixed_supported(const GfDims& m, std::string* why);
// Graph family, unfused: FP32 or FP64, or (tensor_cores) FP32 storage with
// every matrix product on the tensor cores with BF16 operands.
Model* make_plain_gf(const GfDims& m, bool f64, bool tensor_cores, const double* weights,
                     int n_atoms, const int* types_host, std::string* err);

}  // namespace dp
