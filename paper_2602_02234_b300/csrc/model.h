// The interface every network implementation exposes to the runtime: given the
// kept neighbours of every atom it writes atomic energies and the pair
// gradients g_ij = dE/dr_ij (one per neighbour slot).
#pragma once

#include <string>

#include "kernels.cuh"

namespace dp {

class Model {
 public:
  virtual ~Model() {}
  // Enqueue one evaluation on `st`; returns the number of kernels launched.
  virtual int run(const int* sel_j, const double* sel_r, const int* types, double* atom_e,
                  cudaStream_t st) = 0;
  // Pair gradients (n_atoms x nmax x 3): exactly one of the two is non-null.
  virtual const float* grad32() const { return nullptr; }
  virtual const double* grad64() const { return nullptr; }
  virtual size_t bytes() const = 0;
};

// Plain attention family (FP32 or FP64), unfused.  nmax <= 256.
Model* make_plain_af(const AfDims& m, bool f64, const double* weights, int n_atoms,
                     const int* types_host, size_t mem_budget, std::string* err);
// Fused attention family (BF16 tensor cores).  Returns nullptr and a reason when
// the sizes are outside what the fused kernels support.
bool fused_af_supported(const AfDims& m, std::string* why);
Model* make_fused_af(const AfDims& m, const double* weights, int n_atoms, const int* types_host,
                     std::string* err);

}  // namespace dp
