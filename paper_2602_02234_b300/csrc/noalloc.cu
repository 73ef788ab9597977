// Allocation-free neighbour lists: dp_neighbour_list_noalloc.
//
// Some callers cannot allocate device memory: an MD engine that owns the
// device allocator (or runs under a fixed memory budget it has already spent),
// or a plugin that only receives pointers to buffers the engine owns.  They
// still need the model's neighbour lists.  This entry point computes them for
// one small system in a single kernel whose scratch memory -- the candidate
// records of every atom -- lives in a file-scope static device array that is
// part of the loaded library, so the call allocates nothing.
//
// Limits: at most kNoallocMaxAtoms atoms and kNoallocMaxCand candidates
// within rc per atom (images included); larger requests are rejected with
// DP_ERR_ARG / DP_ERR_NLIST_OVERFLOW.  A box so small that an atom's own
// periodic images alone exceed the candidate limit is refused on the host
// before any launch, and the kernel stops scanning an atom's candidates as
// soon as they exceed the limit, so an overflowing call returns quickly.
// Every GPU that loads the library holds the array (about 6.3 MB) until the
// process exits.
//
// The array is shared by every call in the process: calls whose kernels
// overlap on the GPU (different streams, or different host threads) race on
// it and must be serialised by the caller.  Each call clears the parts that
// must start at zero (the status word) before its kernel runs.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>
#include <string>

#include "common.cuh"

namespace dp {

static constexpr int kNoallocMaxAtoms = 1024;
static constexpr int kNoallocMaxCand = 384;

struct NoallocCand {
  double d2;
  int j;
  int img;  // image components packed as 3 x 10 bits, each offset by 512
};

struct NoallocScratch {
  int status;  // bit 0: a candidate list overflowed
  int pad[63];
  NoallocCand cand[kNoallocMaxAtoms][kNoallocMaxCand];
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

__device__ __forceinline__ int pack_img(int x, int y, int z) {
  return ((x + 512) << 20) | ((y + 512) << 10) | (z + 512);
}
__device__ __forceinline__ void unpack_img(int p, int* n) {
  n[0] = ((p >> 20) & 1023) - 512;
  n[1] = ((p >> 10) & 1023) - 512;
  n[2] = (p & 1023) - 512;
}

// One warp per centre atom: every (j, image) within rc is recorded in the
// scratch array, then ranked by (r^2, j, image); the first nmax are written.
__global__ void k_neighbours_noalloc(int n, const double* __restrict__ x, double L0, double L1,
                                     double L2, double rc, int nmax, int nx, int ny, int nz,
                                     NoallocScratch* __restrict__ scr, int* __restrict__ nbr_j,
                                     int* __restrict__ nbr_img, int* __restrict__ n_in_rc) {
  int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (i >= n) return;
  const double L[3] = {L0, L1, L2};
  double wi[3];
  for (int a = 0; a < 3; ++a) {
    double f;
    wi[a] = wrap_coord(x[3 * i + a], L[a], &f);
  }
  NoallocCand* mine = scr->cand[i];
  const double rc2 = rc * rc;
  const int per_atom = (2 * nx + 1) * (2 * ny + 1) * (2 * nz + 1);
  const long long total = (long long)n * per_atom;
  int cnt = 0;
  for (long long base = 0; base < total; base += 32) {
    long long s = base + lane;
    bool take = false;
    double d2 = 0.0;
    int j = 0, nn[3] = {0, 0, 0};
    if (s < total) {
      j = (int)(s / per_atom);
      int im = (int)(s % per_atom);
      nn[0] = im / ((2 * ny + 1) * (2 * nz + 1)) - nx;
      nn[1] = (im / (2 * nz + 1)) % (2 * ny + 1) - ny;
      nn[2] = im % (2 * nz + 1) - nz;
      if (!(j == i && nn[0] == 0 && nn[1] == 0 && nn[2] == 0)) {
        double wj[3], r[3];
        for (int a = 0; a < 3; ++a) {
          double f;
          wj[a] = wrap_coord(x[3 * j + a], L[a], &f);
        }
        d2 = sep_exact(wi, wj, nn, L, r);
        take = d2 < rc2 && d2 > 0.0;
      }
    }
    unsigned b = __ballot_sync(0xffffffffu, take);
    int pos = cnt + __popc(b & ((1u << lane) - 1u));
    if (take && pos < kNoallocMaxCand) {
      mine[pos].d2 = d2;
      mine[pos].j = j;
      mine[pos].img = pack_img(nn[0], nn[1], nn[2]);
    }
    cnt += __popc(b);
    if (cnt > kNoallocMaxCand) break;   // cnt is the same in every lane
  }
  if (cnt > kNoallocMaxCand) {
    // overflow: flag it, report "more than the limit" and leave empty rows
    if (lane == 0) {
      atomicOr(&scr->status, 1);
      n_in_rc[i] = kNoallocMaxCand + 1;
    }
    for (int p = lane; p < nmax; p += 32) {
      size_t o = (size_t)i * nmax + p;
      nbr_j[o] = -1;
      for (int a = 0; a < 3; ++a) nbr_img[3 * o + a] = 0;
    }
    return;
  }
  __syncwarp();
  if (lane == 0) n_in_rc[i] = cnt;
  for (int q = lane; q < cnt; q += 32) {
    NoallocCand cq = mine[q];
    int nq[3];
    unpack_img(cq.img, nq);
    int rank = 0;
    for (int p = 0; p < cnt; ++p) {
      NoallocCand cp = mine[p];
      int np[3];
      unpack_img(cp.img, np);
      rank += key_less(cp.d2, cp.j, np, cq.d2, cq.j, nq) ? 1 : 0;
    }
    if (rank < nmax) {
      size_t o = (size_t)i * nmax + rank;
      nbr_j[o] = cq.j;
      for (int a = 0; a < 3; ++a) nbr_img[3 * o + a] = nq[a];
    }
  }
  for (int p = cnt + lane; p < nmax; p += 32) {
    size_t o = (size_t)i * nmax + p;
    nbr_j[o] = -1;
    for (int a = 0; a < 3; ++a) nbr_img[3 * o + a] = 0;
  }
}

// Device address of the scratch array, looked up once per device with that
// device current (the host-side name of a __device__ variable is not a
// device address).  The lookup is serialised by a mutex, so host threads
// that make their first calls at the same time do not race on the table.
static NoallocScratch* g_scratch_ptr[64] = {nullptr};
static std::mutex g_scratch_mutex;

// Periodic images n != 0 of one atom with |n L| < rc, counted from the
// centre outwards (0, 1, -1, 2, -2, ...) and given up once above `limit`:
// the loop stays short whether the count is small or large.
static int own_images_within(const double* L, double rc, const int* nimg, int limit) {
  auto at = [](int k) { return (k & 1) ? (k + 1) / 2 : -(k / 2); };
  int count = 0;
  const double rc2 = rc * rc;
  for (int ka = 0; ka < 2 * nimg[0] + 1; ++ka) {
    const double xa = at(ka) * L[0];
    if (xa * xa >= rc2) break;
    for (int kb = 0; kb < 2 * nimg[1] + 1; ++kb) {
      const double yb = at(kb) * L[1];
      if (xa * xa + yb * yb >= rc2) break;
      for (int kc = 0; kc < 2 * nimg[2] + 1; ++kc) {
        const double zc = at(kc) * L[2];
        const double d2 = xa * xa + yb * yb + zc * zc;
        if (d2 >= rc2) break;
        if (d2 > 0.0 && ++count > limit) return count;
      }
    }
  }
  return count;
}

static thread_local std::string g_noalloc_error;

}  // namespace dp

using namespace dp;

extern "C" const char* dp_noalloc_last_error(void) { return g_noalloc_error.c_str(); }

extern "C" int dp_neighbour_list_noalloc(const double* coords, int n_atoms, const double* box,
                                         double rcut, int nmax, int32_t* nbr_j, int32_t* nbr_img,
                                         int32_t* n_in_rc, void* cuda_stream) {
  if (!coords || !box || !nbr_j || !nbr_img || !n_in_rc) {
    g_noalloc_error = "NULL argument";
    return DP_ERR_ARG;
  }
  if (n_atoms < 1 || n_atoms > kNoallocMaxAtoms) {
    g_noalloc_error = "n_atoms must be 1.." + std::to_string(kNoallocMaxAtoms) +
                      " (the static scratch array holds that many atoms)";
    return DP_ERR_ARG;
  }
  if (nmax < 1 || nmax > kNoallocMaxCand) {
    g_noalloc_error = "nmax must be 1.." + std::to_string(kNoallocMaxCand);
    return DP_ERR_ARG;
  }
  if (!(rcut > 0)) {
    g_noalloc_error = "rcut must be positive";
    return DP_ERR_ARG;
  }
  for (int a = 0; a < 3; ++a)
    if (!(box[a] > 0)) {
      g_noalloc_error = "box lengths must be positive";
      return DP_ERR_ARG;
    }
  int img[3];
  for (int a = 0; a < 3; ++a) img[a] = (int)ceil(rcut / box[a]) + 1;
  if (img[0] > 500 || img[1] > 500 || img[2] > 500) {
    g_noalloc_error = "box too small for the cutoff";
    return DP_ERR_ARG;
  }
  if (own_images_within(box, rcut, img, kNoallocMaxCand) > kNoallocMaxCand) {
    g_noalloc_error = "more than " + std::to_string(kNoallocMaxCand) +
                      " periodic images of one atom lie within rcut";
    return DP_ERR_NLIST_OVERFLOW;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    g_noalloc_error = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return DP_ERR_CUDA;
  }
  NoallocScratch* scr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        g_noalloc_error = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return DP_ERR_CUDA;
      }
      g_scratch_ptr[dev] = (NoallocScratch*)p;
    }
    scr = g_scratch_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  e = cudaMemsetAsync(&scr->status, 0, sizeof(int), st);
  if (e != cudaSuccess) {
    g_noalloc_error = std::string("clearing the status word: ") + cudaGetErrorString(e);
    return DP_ERR_CUDA;
  }
  const int warps = 4;
  k_neighbours_noalloc<<<(n_atoms + warps - 1) / warps, 32 * warps, 0, st>>>(
      n_atoms, coords, box[0], box[1], box[2], rcut, nmax, img[0], img[1], img[2], scr, nbr_j,
      nbr_img, n_in_rc);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_noalloc_error = std::string("launch: ") + cudaGetErrorString(e);
    return DP_ERR_CUDA;
  }
  int status = 0;
  e = cudaMemcpyAsync(&status, &scr->status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    g_noalloc_error = std::string("status read: ") + cudaGetErrorString(e);
    return DP_ERR_CUDA;
  }
  if (status & 1) {
    g_noalloc_error = "more than " + std::to_string(kNoallocMaxCand) +
                      " neighbours within rcut of one atom";
    return DP_ERR_NLIST_OVERFLOW;
  }
  return DP_OK;
}
