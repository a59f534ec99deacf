// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/dg.h"
#include "dg_df64.cuh"

namespace dg {

// Programmatic dependent launch.  Every kernel of the library begins with
// pdl_entry(): griddepcontrol.wait returns once the kernels before it on the
// stream have completed and their writes are visible (at once when the launch
// carried no PDL attribute); launch_dependents then lets the next kernel's
// blocks be placed on free SM slots while this one still runs, so that the
// launch latency of back-to-back small kernels overlaps the tail of the one
// before.  Nothing reads or writes global memory before the wait.
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;\n\tgriddepcontrol.launch_dependents;" ::: "memory");
}

// (i, j, k) of a lexicographic cell index on an n0 x n1 x n2 box, in 32-bit
// integer division while the index fits (several times cheaper than 64-bit)
__device__ __forceinline__ void lex_coords(int64_t cell, int n0, int n1, int ci[3]) {
  if (cell <= 0x7fffffffLL) {
    const unsigned c = (unsigned)cell, q = c / (unsigned)n0;
    ci[0] = (int)(c - q * (unsigned)n0);
    ci[1] = (int)(q % (unsigned)n1);
    ci[2] = (int)(q / (unsigned)n1);
  } else {
    const int64_t q = cell / n0;
    ci[0] = (int)(cell - q * n0);
    ci[1] = (int)(q % n1);
    ci[2] = (int)(q / n1);
  }
}

// asynchronous global-to-shared copy of BYTES (4, 8 or 16; both addresses
// aligned to it), its commit and the wait for all of the thread's copies
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// The PDL attribute is set unless DG_PDL=0 in the environment, and never on
// the legacy default stream.
bool pdl_enabled();

template <typename... KArgs, typename... Args>
inline cudaError_t launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                          Args&&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed =
      (pdl_enabled() && s != nullptr && s != cudaStreamLegacy) ? 1 : 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Operator-kernel variants chosen by the autotuner: 0-4 cell-centric tile
// shapes, 5-6 face-once, 7 thread-per-cell Q1.
constexpr int kTuneVariants = 8;
constexpr int kGeneralVariants = 3;  // trilinear cells: half, default, double cells per CTA
__host__ __device__ constexpr bool variant_split(int v) { return v == 5 || v == 6; }
__host__ __device__ constexpr bool variant_q1(int v) { return v == 7; }

constexpr int kMaxN = 8;  // nodes per direction supported by the 1D tables

// 1D tables of the nodal Lagrange basis on the n Gauss-Legendre points of
// [0,1], passed to kernels by value (constant bank).
template <typename T>
struct Tab1D {
  T D[kMaxN][kMaxN];  // D[q][i] = L_i'(x_q)
  T L[2][kMaxN];      // L[s][i] = L_i(s), s = 0, 1 (cell faces)
  T dL[2][kMaxN];     // dL[s][i] = L_i'(s)
  T w[kMaxN];         // quadrature weights on [0,1]
  T x[kMaxN];         // points
};

// Pressure basis (k points) evaluated at the velocity points (k+1): the 1D
// factors of the mixed velocity-pressure forms.
template <typename T>
struct MixTab {
  T I[kMaxN][kMaxN];  // I[q][j] = psi_j(x^u_q)
  T D[kMaxN][kMaxN];  // D[q][j] = psi_j'(x^u_q)
};

// Host-side construction (FP64) of the tables for n points.
void make_tables(int n, Tab1D<double>* t);
void make_mix(const Tab1D<double>& tu, int nu, const Tab1D<double>& tp, int np, MixTab<double>* m);
template <typename T>
Tab1D<T> cast_tables(const Tab1D<double>& t);
Tab1D<df64> split_tables(const Tab1D<double>& t);
MixTab<df64> split_mix(const MixTab<double>& t);

// Cell geometry of the affine paths: per-axis cell extents (the Jacobian is
// diagonal, diag(h0, h1, h2), on Cartesian and tensor-graded meshes).
template <typename T>
struct AxisGeom {
  const T* h[3];
};

}  // namespace dg

struct dg_mesh {
  dg_mesh_desc desc;
  int dim = 0, k = 0;
  int nu = 0, np = 0;      // nodes per direction: velocity k+1, pressure k
  int nbu = 0, nbp = 0;    // nodes per cell
  int64_t ncell = 0;
  int n[3] = {1, 1, 1};
  int periodic[3] = {1, 1, 1};
  bool affine = true;
  int device = 0;
  std::vector<double> vx[3];        // vertex lattice coordinates per axis (affine)
  double* d_h64[3] = {nullptr, nullptr, nullptr};   // cell extents per axis
  float* d_h32[3] = {nullptr, nullptr, nullptr};
  double* d_hi64[3] = {nullptr, nullptr, nullptr};  // their inverses
  float* d_hi32[3] = {nullptr, nullptr, nullptr};
  dg::Tab1D<double> tu64, tp64;      // velocity / pressure tables
  dg::Tab1D<float> tu32, tp32;
  dg::MixTab<double> mix64;
  dg::Tab1D<dg::df64> tudf, tpdf;    // float-float copies of the FP64 tables
  dg::MixTab<dg::df64> mixdf;
  int fp64_arith = 0;                // FP64 operator arithmetic: 0 float-float, 1 native FP64
  int* d_status = nullptr;           // device error word
  // metric terms of trilinear cells (dg_geom.cuh); null on affine meshes
  double* gvu64 = nullptr;  // velocity-node volume terms
  float* gvu32 = nullptr;
  double* gfu64 = nullptr;  // velocity face terms
  float* gfu32 = nullptr;
  double* gvp64 = nullptr;  // pressure-node volume terms
  float* gvp32 = nullptr;
  double* gfp64 = nullptr;  // pressure face terms
  float* gfp32 = nullptr;
  double* gpen64 = nullptr; // penalty geometry per cell face
  float* gpen32 = nullptr;
  dg::df64* gvu_df = nullptr;  // the FP64 terms split into float pairs
  dg::df64* gfu_df = nullptr;
  dg::df64* gvp_df = nullptr;
  dg::df64* gfp_df = nullptr;
  dg::df64* gpen_df = nullptr;
  bool geom_u = false;      // velocity terms present (not on multigrid levels)
  // face-flux scratch of the face-once operator variant (allocated by the
  // autotuner, which is the only way that variant gets chosen)
  void* split_flux = nullptr;
  int64_t split_flux_bytes = 0;
  // float-float applies (affine meshes): the source vector and advecting
  // field split into float pairs once per apply (double-sized slots), and
  // float-float copies of the cell extents, allocated with the mesh
  double* ps_src = nullptr;         // max(dim * nbu, nbp) * ncell slots
  double* ps_ub = nullptr;          // dim * nbu * ncell slots (not on multigrid levels)
  double* d_hdf[3] = {nullptr, nullptr, nullptr};
  double* d_hidf[3] = {nullptr, nullptr, nullptr};
  // 1D tables of the Q1 pressure operator's tensor-product form (affine 3D
  // meshes with two pressure points per direction): per axis cell 4 float4,
  // the tangential weights w_i h, then the own, lower- and upper-neighbour
  // 2x2 blocks of the 1D SIP matrix; axis a starts at row q1tab_off[a]
  float4* q1tab = nullptr;
  int q1tab_off[3] = {0, 0, 0};
  // the same rows as float pairs packed in doubles (16 per row), for the
  // float-float form of the kernel
  double* q1tab_df = nullptr;
  // advecting field whose split copy may be reused while the caller keeps
  // it unchanged (the solver around its Krylov iterations), and the field
  // the copy in ps_ub was made from
  const double* ub_keep = nullptr;
  const double* ub_split_of = nullptr;
  // split copies of the explicit terms' fields (float-float right-hand
  // sides), velocity-sized, allocated on first use
  double* ps_pool[4] = {nullptr, nullptr, nullptr, nullptr};
  bool level = false;       // a multigrid level (pressure space only)
  // autotuned tile shape of the operator kernels: variant index per
  // [precision: 0 FP64, 1 FP32][operator: 0 pressure, 1 momentum, 2 momentum
  // with advection]; 1 = default cells per CTA, 0 = half, 2 = double
  int tune[2][3] = {{1, 1, 1}, {1, 1, 1}};
  bool tuned = false;
  std::string tune_report;
};

namespace dg {

// kernels launched by the library in this process (diagnostics)
void count_launch();
void count_launches(int64_t n);  // kernels of a replayed CUDA graph
int64_t launches_so_far();

// thread-local error message, set by the entry points
void set_error(const std::string& msg);
dg_status cuda_fail(cudaError_t e, const char* where);

#define DG_CUDA(call)                                     \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return dg::cuda_fail(e_, #call); \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

dg_status finish_mesh(dg_mesh* m, cudaStream_t s);
// mapped lattice vertex L of a mesh description; Gauss-Legendre rule on [0,1]
void lattice_vertex(const dg_mesh_desc& d, const int L[3], double X[3]);
void gauss_legendre_01(int n, double* x, double* w);
dg_status make_level_mesh(const dg_mesh* fine, const int coarsen[3], int degree_u, cudaStream_t s,
                          dg_mesh** out);

dg_status autotune_mesh(dg_mesh* m, cudaStream_t s);

// The advecting field `ubar` stays unchanged until the next call (nullptr:
// no such promise): float-float momentum applies with it split it once.
void keep_presplit_ubar(dg_mesh* m, const double* ubar);
// split the kept field now (no-op without one, on FP64-arithmetic meshes, or
// when already split)
dg_status presplit_kept_ubar(dg_mesh* m, cudaStream_t s);

// host-side split of a double into a float pair, packed in a double's bits
// (the layout df_bits reads)
double pack_pair(double x);

// out[i] = x[i] as float pairs in double-sized slots (one kernel on s)
dg_status presplit(int64_t n, const double* x, double* out, cudaStream_t s);

// launchers (dg_apply.cu)
template <typename T>
dg_status launch_scalar_op(const dg_mesh* m, bool pressure, T mass, T visc, T adv,
                           const T* ubar, const T* src, T* dst, int ncomp, cudaStream_t s);
// the pressure operator with a fused output stage on a multigrid level
// (modes 1-4 of op_epilogue; see dg_apply.cu and dg_mg.cu)
template <typename T>
dg_status launch_poisson_epi(int mode, const dg_mesh* m, double alpha, const T* src, T* dst, T* x, T* r,
                             const T* dinv, double c1, double c2, cudaStream_t s);

}  // namespace dg
