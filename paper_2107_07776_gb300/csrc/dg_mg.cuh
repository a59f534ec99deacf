// h/p multigrid for the pressure Helmholtz systems (see dg_mg.cu).
#pragma once

#include <vector>

#include "dg_common.cuh"

namespace dg {

// Transfer between a fine level (nf nodes per direction) and the next
// coarser one (nc).  Axis a is h-coarsened when hco[a] (fine cells 2c, 2c+1
// -> coarse cell c, child bit = fine index parity) and otherwise maps cells
// one to one.  M[b][i][j] = coarse basis j at fine node i of child b on an
// h-coarsened axis; M[2][i][j] = coarse basis j at fine node i on the same
// interval (the identity when nf == nc, the p-embedding otherwise).
struct Transfer {
  int dim, nf, nc;
  int hco[3];
  int nfine[3], ncoarse[3];
  double M[3][kMaxN][kMaxN];
  float Mf[3][kMaxN][kMaxN];  // FP32 copy for the FP32 hierarchy
};

template <typename T>
__device__ __forceinline__ T transfer_w(const Transfer& tr, int s, int i, int j);
template <>
__device__ __forceinline__ double transfer_w<double>(const Transfer& tr, int s, int i, int j) {
  return tr.M[s][i][j];
}
template <>
__device__ __forceinline__ float transfer_w<float>(const Transfer& tr, int s, int i, int j) {
  return tr.Mf[s][i][j];
}

template <typename T>
struct MGLevel {
  dg_mesh* mesh = nullptr;
  bool owned = false;
  int np = 0;           // pressure nodes per direction on this level
  int kind = 0;         // relation to the finer level: 0 finest, 1 p-coarsened, 2 h-coarsened
  int hco[3] = {0, 0, 0};
  int64_t n = 0;        // DoFs
  T* x = nullptr;
  T* b = nullptr;
  T* r = nullptr;
  T* d = nullptr;
  T* t = nullptr;
  T* d2 = nullptr;                  // second Chebyshev direction (ping-pong)
  T* dinv[2] = {nullptr, nullptr};  // per cached alpha
  T* ainv[2] = {nullptr, nullptr};  // dense inverse of the coarsest level, per cached alpha
  double lmin[2] = {0, 0}, lmax[2] = {0, 0};
};

template <typename T>
struct MultiGrid {
  std::vector<MGLevel<T>> lv;
  std::vector<Transfer> tr;
  cudaStream_t stream = nullptr;
  double alpha = 0.0;
  double cache_alpha[2] = {0, 0};
  int cur = 0, next_slot = 0;
  int smooth_degree = 5;
  double* part = nullptr;
  double* host_part = nullptr;
  double* diag = nullptr;

  // V-cycles captured as CUDA graphs, per (r, z, alpha slot): the cycle is a
  // fixed launch sequence on fixed buffers, so replaying it removes the
  // per-kernel launch cost of the small coarse levels
  struct Captured {
    const double* r;
    double* z;
    int slot;
    cudaGraphExec_t exec;
    int64_t launches;
  };
  std::vector<Captured> graphs;
  bool use_graphs = true;
  cudaStream_t cap_stream = nullptr;  // private stream the cycles are recorded on

  ~MultiGrid();
  dg_status build(dg_mesh* fine, cudaStream_t s);
  dg_status set_alpha(double alpha);
  // Chebyshev degree of the smoother (drops the recorded cycles on a change)
  void set_degree(int degree);
  // z = V-cycle(r) for an FP64 residual r of the finest level
  dg_status apply(const double* r, double* z);

 private:
  dg_status apply_direct(const double* r, double* z);
  void drop_graphs(int slot);
  dg_status vcycle(int l);
  dg_status chebyshev(int l, int degree, bool x_zero);
  dg_status estimate(int l, int slot, int steps, double* lo, double* hi);
  dg_status coarse_inverse(int slot);
  dg_status dot(int64_t n, const T* a, const T* b, double* out);
  void lanczos_update(int64_t n, T a, const T* q, const T* dinv, T* r, T* z);
  void lanczos_dir(int64_t n, T b, const T* z, T* p);
};

}  // namespace dg
