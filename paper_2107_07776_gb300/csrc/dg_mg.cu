// h/p multigrid preconditioner for the pressure Helmholtz systems (Section 4
// names a geometric multigrid preconditioner for them; its components are
// the project's own):
//   levels   the fine pressure space Q_{k-1}, then p-coarsening to Q_1 on the
//            same cells, then h-coarsening by 2 along every axis with an even
//            number of cells, down to at most 512 DoFs;
//   operator alpha M^p + K rediscretised on every level (same alpha, that
//            level's cell sizes and penalty, the same apply kernels);
//   transfer cell-local DG embedding: prolongation evaluates the coarse
//            polynomial at the fine nodes (exact: the coarse space is a
//            subspace), restriction is its transpose;
//   smoother Chebyshev iteration of degree 5 (an option) on D^-1 A over
//            [lambda_max/20, 1.1 lambda_max], lambda_max from 15 Lanczos
//            (Jacobi-CG) steps, each step after the first one fused launch;
//   coarse   the coarsest level (at most 2048 DoFs) is solved exactly by a
//            dense inverse built once per alpha from applies to unit vectors
//            (else a degree-30 Chebyshev over its Lanczos spectrum estimate);
//   cycle    one V-cycle (pre- and post-smoothing) per outer CG iteration.
// T = float gives the mixed-precision preconditioner (all level vectors and
// applies in FP32 inside the FP64 flexible CG), T = double the FP64 one.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dg_krylov.cuh"
#include "dg_mg.cuh"

namespace dg {

// coarsest levels up to this many DoFs are solved exactly by a dense inverse
constexpr int64_t kCoarseDenseMax = 2048;

namespace {

unsigned grid1(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// 1D Lagrange basis on nodes xs (n) at x, product form
void lagrange_at(const double* xs, int n, double x, double* out) {
  for (int j = 0; j < n; ++j) {
    double v = 1.0;
    for (int l = 0; l < n; ++l)
      if (l != j) v *= (x - xs[l]) / (xs[j] - xs[l]);
    out[j] = v;
  }
}

template <typename T>
__global__ void cvt_kernel(int64_t n, const double* __restrict__ a, T* __restrict__ b) {
  pdl_entry();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    b[k] = (T)a[k];
}
template <typename T>
__global__ void cvt_back_kernel(int64_t n, const T* __restrict__ a, double* __restrict__ b) {
  pdl_entry();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    b[k] = (double)a[k];
}
template <typename T>
__global__ void inv_diag_kernel(int64_t n, const double* __restrict__ d, T* __restrict__ dinv) {
  pdl_entry();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    dinv[k] = (T)(1.0 / d[k]);
}
// r = dinv .* (b - t) (t may be null: r = dinv .* b); d = r * inv_theta
template <typename T>
__global__ void cheb_init_kernel(int64_t n, const T* __restrict__ b, const T* __restrict__ t,
                                 const T* __restrict__ dinv, T inv_theta, T* __restrict__ r,
                                 T* __restrict__ d) {
  pdl_entry();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const T rk = dinv[k] * (t ? b[k] - t[k] : b[k]);
    r[k] = rk;
    d[k] = rk * inv_theta;
  }
}
template <typename T>
__global__ void add_kernel(int64_t n, const T* __restrict__ d, T* __restrict__ x) {
  pdl_entry();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    x[k] += d[k];
}
// I = identity (n x n)
template <typename T>
__global__ void identity_kernel(int64_t n, T* __restrict__ I) {
  pdl_entry();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n * n;
       k += (int64_t)gridDim.x * blockDim.x)
    I[k] = (k / n == k % n) ? T(1) : T(0);
}
// x = Ainv b, one warp per row: the inverse of the symmetric coarse operator
// is symmetric, so row i is read contiguously (stored column j at j*n)
template <typename T>
__global__ void __launch_bounds__(256) dense_matvec_kernel(int n, const T* __restrict__ Ainv,
                                                           const T* __restrict__ b, T* __restrict__ x) {
  pdl_entry();
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= n) return;
  const T* a = Ainv + (int64_t)row * n;
  T acc = T(0);
  for (int j = lane; j < n; j += 32) acc += a[j] * b[j];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) x[row] = acc;
}

// deterministic pseudo-random start vector in [-1, 1] (splitmix64 hash)
template <typename T>
__global__ void hash_fill_kernel(int64_t n, T* __restrict__ x) {
  pdl_entry();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = (uint64_t)k + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[k] = (T)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
  }
}
// partial dot products accumulated in double, fixed order
template <typename T>
__global__ void __launch_bounds__(256) dot_kernel(int64_t n, const T* __restrict__ a,
                                                  const T* __restrict__ b, double* __restrict__ part) {
  pdl_entry();
  __shared__ double s[256];
  double acc = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    acc += (double)a[k] * (double)b[k];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

template <typename T>
__global__ void prolong_add_kernel(const __grid_constant__ Transfer tr, int64_t nfine_dofs,
                                   const T* __restrict__ xc, T* __restrict__ xf) {
  pdl_entry();
  const int nbf = tr.dim == 3 ? tr.nf * tr.nf * tr.nf : tr.nf * tr.nf;
  const int nbc = tr.dim == 3 ? tr.nc * tr.nc * tr.nc : tr.nc * tr.nc;
  // grid-stride: the launch grid is capped (grid1), levels can be larger
  for (int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gid < nfine_dofs;
       gid += (int64_t)gridDim.x * blockDim.x) {
    const int64_t fc = gid / nbf;
    const int node = (int)(gid % nbf);
    int fi[3] = {(int)(fc % tr.nfine[0]), (int)((fc / tr.nfine[0]) % tr.nfine[1]),
                 (int)(fc / ((int64_t)tr.nfine[0] * tr.nfine[1]))};
    int ci[3], bit[3];
    for (int a = 0; a < 3; ++a) {
      ci[a] = tr.hco[a] ? fi[a] >> 1 : fi[a];
      bit[a] = tr.hco[a] ? (fi[a] & 1) : 0;
    }
    const int64_t cc = ci[0] + (int64_t)tr.ncoarse[0] * (ci[1] + (int64_t)tr.ncoarse[1] * ci[2]);
    const int ii[3] = {node % tr.nf, (node / tr.nf) % tr.nf, tr.dim == 3 ? node / (tr.nf * tr.nf) : 0};
    T acc = T(0);
    for (int j = 0; j < nbc; ++j) {
      const int jj[3] = {j % tr.nc, (j / tr.nc) % tr.nc, tr.dim == 3 ? j / (tr.nc * tr.nc) : 0};
      T w = T(1);
      for (int a = 0; a < tr.dim; ++a) w *= transfer_w<T>(tr, tr.hco[a] ? bit[a] : 2, ii[a], jj[a]);
      acc += w * xc[cc * nbc + j];
    }
    xf[gid] += acc;
  }
}

// Restriction, pass 1: part[(cc * nchild + ch) * nbc + j] = sum_i M r_f[i]
// over the fine nodes i of child ch of coarse cell cc (one thread per term
// set; the child's nodes are contiguous)
template <typename T>
__global__ void restrict_part_kernel(const __grid_constant__ Transfer tr, int64_t ncc, int nchild,
                                     const T* __restrict__ rf, T* __restrict__ part) {
  pdl_entry();
  const int nbf = tr.dim == 3 ? tr.nf * tr.nf * tr.nf : tr.nf * tr.nf;
  const int nbc = tr.dim == 3 ? tr.nc * tr.nc * tr.nc : tr.nc * tr.nc;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= ncc * nchild * nbc) return;
  const int j = (int)(gid % nbc);
  const int ch = (int)((gid / nbc) % nchild);
  const int64_t cc = gid / ((int64_t)nbc * nchild);
  const int ci[3] = {(int)(cc % tr.ncoarse[0]), (int)((cc / tr.ncoarse[0]) % tr.ncoarse[1]),
                     (int)(cc / ((int64_t)tr.ncoarse[0] * tr.ncoarse[1]))};
  const int jj[3] = {j % tr.nc, (j / tr.nc) % tr.nc, tr.dim == 3 ? j / (tr.nc * tr.nc) : 0};
  int bit[3] = {0, 0, 0}, fi[3] = {ci[0], ci[1], ci[2]}, t = ch;
  for (int a = 0; a < tr.dim; ++a)
    if (tr.hco[a]) {
      bit[a] = t & 1;
      t >>= 1;
      fi[a] = 2 * ci[a] + bit[a];
    }
  const int64_t fc = fi[0] + (int64_t)tr.nfine[0] * (fi[1] + (int64_t)tr.nfine[1] * fi[2]);
  T acc = T(0);
  for (int i = 0; i < nbf; ++i) {
    const int ii[3] = {i % tr.nf, (i / tr.nf) % tr.nf, tr.dim == 3 ? i / (tr.nf * tr.nf) : 0};
    T w = T(1);
    for (int a = 0; a < tr.dim; ++a) w *= transfer_w<T>(tr, tr.hco[a] ? bit[a] : 2, ii[a], jj[a]);
    acc += w * rf[fc * nbf + i];
  }
  part[gid] = acc;
}

// Restriction, pass 2: b_c = sum over the children, fixed order
template <typename T>
__global__ void restrict_sum_kernel(int64_t ncoarse_dofs, int nbc, int nchild,
                                    const T* __restrict__ part, T* __restrict__ bc) {
  pdl_entry();
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= ncoarse_dofs) return;
  const int64_t cc = gid / nbc;
  const int j = (int)(gid % nbc);
  T acc = T(0);
  for (int ch = 0; ch < nchild; ++ch) acc += part[(cc * nchild + ch) * nbc + j];
  bc[gid] = acc;
}

// 3D transfers between Q1 levels (two points per direction on both sides,
// the h-coarsening levels), by sum factorisation: one thread per fine cell
// (prolongation) or coarse cell (restriction) with the cell's 8 values in
// registers; along axis a the 1D map is the 2x2 matrix M[s][i][j] of the
// child's position s (0 or 1 on a coarsened axis, 2 otherwise).  Same
// weights as prolong_add_kernel / restrict_*_kernel, 3 sweeps of 2 terms
// instead of 8 terms of 3 factors per value.
template <typename T>
__device__ __forceinline__ void q1_tensor_map(const Transfer& tr, const int sel[3], bool transpose,
                                              const T in[8], T out[8]) {
  T t1[8], t2[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {  // axis 0 (x fastest)
    const int i0 = i & 1, rest = i & 6;
    const T w0 = transpose ? transfer_w<T>(tr, sel[0], 0, i0) : transfer_w<T>(tr, sel[0], i0, 0);
    const T w1 = transpose ? transfer_w<T>(tr, sel[0], 1, i0) : transfer_w<T>(tr, sel[0], i0, 1);
    t1[i] = w0 * in[rest] + w1 * in[rest | 1];
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {  // axis 1
    const int i1 = (i >> 1) & 1, rest = i & 5;
    const T w0 = transpose ? transfer_w<T>(tr, sel[1], 0, i1) : transfer_w<T>(tr, sel[1], i1, 0);
    const T w1 = transpose ? transfer_w<T>(tr, sel[1], 1, i1) : transfer_w<T>(tr, sel[1], i1, 1);
    t2[i] = w0 * t1[rest] + w1 * t1[rest | 2];
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {  // axis 2
    const int i2 = i >> 2, rest = i & 3;
    const T w0 = transpose ? transfer_w<T>(tr, sel[2], 0, i2) : transfer_w<T>(tr, sel[2], i2, 0);
    const T w1 = transpose ? transfer_w<T>(tr, sel[2], 1, i2) : transfer_w<T>(tr, sel[2], i2, 1);
    out[i] = w0 * t2[rest] + w1 * t2[rest | 4];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) prolong_q1_kernel(const __grid_constant__ Transfer tr,
                                                         int64_t nfine_cells,
                                                         const T* __restrict__ xc, T* __restrict__ xf) {
  pdl_entry();
  for (int64_t fc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; fc < nfine_cells;
       fc += (int64_t)gridDim.x * blockDim.x) {
    int fi[3];
    lex_coords(fc, tr.nfine[0], tr.nfine[1], fi);
    int ci[3], sel[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      ci[a] = tr.hco[a] ? fi[a] >> 1 : fi[a];
      sel[a] = tr.hco[a] ? (fi[a] & 1) : 2;
    }
    const int64_t cc = ci[0] + (int64_t)tr.ncoarse[0] * (ci[1] + (int64_t)tr.ncoarse[1] * ci[2]);
    T in[8], out[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) in[j] = xc[cc * 8 + j];
    q1_tensor_map<T>(tr, sel, false, in, out);
#pragma unroll
    for (int i = 0; i < 8; ++i) xf[fc * 8 + i] += out[i];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) restrict_q1_kernel(const __grid_constant__ Transfer tr,
                                                          int64_t ncoarse_cells,
                                                          const T* __restrict__ rf, T* __restrict__ bc) {
  pdl_entry();
  for (int64_t cc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; cc < ncoarse_cells;
       cc += (int64_t)gridDim.x * blockDim.x) {
    int ci[3];
    lex_coords(cc, tr.ncoarse[0], tr.ncoarse[1], ci);
    T acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = T(0);
    // children in a fixed order (bit a of ch along the a-th coarsened axis)
    for (int ch = 0; ch < 8; ++ch) {
      int fi[3] = {ci[0], ci[1], ci[2]}, sel[3] = {2, 2, 2}, t = ch;
      bool skip = false;
      for (int a = 0; a < 3; ++a) {
        if (tr.hco[a]) {
          sel[a] = t & 1;
          t >>= 1;
          fi[a] = 2 * ci[a] + sel[a];
        }
      }
      skip = t != 0;  // ch enumerates only 2^(coarsened axes) children
      if (skip) continue;
      const int64_t fc = fi[0] + (int64_t)tr.nfine[0] * (fi[1] + (int64_t)tr.nfine[1] * fi[2]);
      T in[8], out[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) in[i] = rf[fc * 8 + i];
      q1_tensor_map<T>(tr, sel, true, in, out);
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] += out[j];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) bc[cc * 8 + j] = acc[j];
  }
}

// Largest/smallest eigenvalues of a symmetric tridiagonal matrix by
// bisection on Sturm sequence counts.
void tridiag_extremes(const std::vector<double>& a, const std::vector<double>& b, double* lo,
                      double* hi) {
  const int n = (int)a.size();
  double gl = a[0], gu = a[0];
  for (int i = 0; i < n; ++i) {
    double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(b[i]) : 0.0);
    gl = std::min(gl, a[i] - r);
    gu = std::max(gu, a[i] + r);
  }
  auto count_below = [&](double x) {
    int c = 0;
    double q = a[0] - x;
    if (q < 0) ++c;
    for (int i = 1; i < n; ++i) {
      double qq = q == 0.0 ? 1e-300 : q;
      q = a[i] - x - b[i - 1] * b[i - 1] / qq;
      if (q < 0) ++c;
    }
    return c;
  };
  double l = gl, u = gu;
  for (int it = 0; it < 200; ++it) {  // largest: count_below(x) == n - 1 just below it
    double mid = 0.5 * (l + u);
    if (count_below(mid) < n) l = mid;
    else u = mid;
  }
  *hi = u;
  l = gl;
  u = gu;
  for (int it = 0; it < 200; ++it) {  // smallest
    double mid = 0.5 * (l + u);
    if (count_below(mid) >= 1) u = mid;
    else l = mid;
  }
  *lo = l;
}

}  // namespace

template <typename T>
static dg_status level_apply(const MGLevel<T>& L, double alpha, const T* x, T* y, cudaStream_t s);
template <>
dg_status level_apply<float>(const MGLevel<float>& L, double alpha, const float* x, float* y,
                             cudaStream_t s) {
  return dg_apply_poisson_f32(L.mesh, alpha, x, y, s);
}
template <>
dg_status level_apply<double>(const MGLevel<double>& L, double alpha, const double* x, double* y,
                              cudaStream_t s) {
  return dg_apply_poisson(L.mesh, alpha, x, y, s);
}

template <typename T>
MultiGrid<T>::~MultiGrid() {
  drop_graphs(-1);
  if (cap_stream) cudaStreamDestroy(cap_stream);
  for (auto& L : lv) {
    if (L.owned && L.mesh) dg_mesh_destroy(L.mesh);
    T* vs[] = {L.x, L.b, L.r, L.d, L.t, L.d2, L.dinv[0], L.dinv[1], L.ainv[0], L.ainv[1]};
    for (T* p : vs)
      if (p) cudaFree(p);
  }
  if (part) cudaFree(part);
  if (host_part) cudaFreeHost(host_part);
  if (diag) cudaFree(diag);
}

template <typename T>
dg_status MultiGrid<T>::build(dg_mesh* fine, cudaStream_t s) {
  stream = s;
  lv.clear();
  MGLevel<T> L0;
  L0.mesh = fine;
  L0.owned = false;
  L0.np = fine->np;
  lv.push_back(L0);
  // p-coarsening on the same cells down to Q1, then h-coarsening
  while (lv.back().np > 2) {
    const int nocoarsen[3] = {0, 0, 0};
    dg_mesh* m = nullptr;
    dg_status st = make_level_mesh(lv.back().mesh, nocoarsen, lv.back().np - 1, s, &m);
    if (st != DG_OK) return st;
    MGLevel<T> L;
    L.mesh = m;
    L.owned = true;
    L.np = m->np;
    L.kind = 1;
    lv.push_back(L);
  }
  while (true) {
    const dg_mesh* m0 = lv.back().mesh;
    if (m0->ncell * m0->nbp <= 512) break;
    int hco[3] = {0, 0, 0}, any = 0;
    for (int a = 0; a < m0->dim; ++a)
      if (m0->n[a] % 2 == 0) hco[a] = any = 1;
    if (!any) break;
    dg_mesh* m = nullptr;
    dg_status st = make_level_mesh(m0, hco, m0->np, s, &m);
    if (st != DG_OK) return st;
    MGLevel<T> L;
    L.mesh = m;
    L.owned = true;
    L.np = m->np;
    L.kind = 2;
    for (int a = 0; a < 3; ++a) L.hco[a] = hco[a];
    lv.push_back(L);
  }
  if (fine->tuned)
    for (size_t l = 1; l < lv.size(); ++l) {
      dg_status st = autotune_mesh(lv[l].mesh, s);
      if (st != DG_OK) return st;
    }
  int64_t nmax = 0;
  for (auto& L : lv) {
    L.n = L.mesh->ncell * L.mesh->nbp;
    nmax = std::max(nmax, L.n);
    T** vs[] = {&L.x, &L.b, &L.r, &L.d, &L.t, &L.d2, &L.dinv[0], &L.dinv[1]};
    for (T** v : vs) {
      cudaError_t e = cudaMalloc(v, sizeof(T) * L.n);
      if (e != cudaSuccess) return cuda_fail(e, "multigrid level vectors");
    }
  }
  DG_CUDA(cudaMalloc(&part, sizeof(double) * 1216));
  DG_CUDA(cudaMallocHost(&host_part, sizeof(double) * 1216));
  DG_CUDA(cudaMalloc(&diag, sizeof(double) * nmax));
  cache_alpha[0] = cache_alpha[1] = std::nan("");
  return DG_OK;
}

template <typename T>
dg_status MultiGrid<T>::dot(int64_t n, const T* a, const T* b, double* out) {
  int64_t nb = (n + 1023) / 1024;
  nb = std::max<int64_t>(1, std::min<int64_t>(nb, 1216));
  launch(dot_kernel<T>, (unsigned)nb, 256, 0, stream, n, a, b, part); count_launch();
  DG_CUDA(cudaGetLastError());
  DG_CUDA(cudaMemcpyAsync(host_part, part, sizeof(double) * nb, cudaMemcpyDeviceToHost, stream));
  DG_CUDA(cudaStreamSynchronize(stream));
  double s = 0.0;
  for (int64_t i = 0; i < nb; ++i) s += host_part[i];
  *out = s;
  return DG_OK;
}

// Lanczos extremes of D^-1 A on level l from `steps` Jacobi-CG iterations.
template <typename T>
dg_status MultiGrid<T>::estimate(int l, int slot, int steps, double* lo, double* hi) {
  MGLevel<T>& L = lv[l];
  const int64_t n = L.n;
  const T* dinv = L.dinv[slot];
  steps = (int)std::min<int64_t>(steps, n);
  // Jacobi-CG from a deterministic random right-hand side; the CG
  // coefficients give the Lanczos tridiagonal matrix of D^-1 A.
  T *r = L.r, *z = L.x, *p = L.d, *q = L.t;
  double rz;
  dg_status st;
  launch(hash_fill_kernel<T>, grid1(n), 256, 0, stream, n, r); count_launch();  // r = b
  launch(cheb_init_kernel<T>, grid1(n), 256, 0, stream, n, r, nullptr, dinv, (T)1, z, p); count_launch();  // z = p = D^-1 r
  st = dot(n, r, z, &rz);
  if (st != DG_OK) return st;
  double a_prev = 0.0, b_prev = 0.0;
  std::vector<double> diagT, offT;
  for (int k = 0; k < steps; ++k) {
    st = level_apply<T>(L, alpha, p, q, stream);
    if (st != DG_OK) return st;
    double pq;
    st = dot(n, p, q, &pq);
    if (st != DG_OK) return st;
    if (!(pq > 0.0) || !(rz > 0.0)) break;
    const double a = rz / pq;
    // r -= a q ; z = D^-1 r  (axpy in place, then scale)
    lanczos_update(n, (T)a, q, dinv, r, z);
    double rz_new;
    st = dot(n, r, z, &rz_new);
    if (st != DG_OK) return st;
    const double b = rz_new / rz;
    diagT.push_back(1.0 / a + (k > 0 ? b_prev / a_prev : 0.0));
    if (k > 0) offT.push_back(std::sqrt(b_prev) / a_prev);
    a_prev = a;
    b_prev = b;
    rz = rz_new;
    // p = z + b p
    lanczos_dir(n, (T)b, z, p);
    if (!(rz_new > 0.0)) break;
  }
  if (diagT.empty()) {
    *lo = *hi = 1.0;
    return DG_OK;
  }
  offT.resize(diagT.size() - 1);
  tridiag_extremes(diagT, offT, lo, hi);
  return DG_OK;
}

template <typename T>
__global__ void lanczos_update_kernel(int64_t n, T a, const T* __restrict__ q,
                                      const T* __restrict__ dinv, T* __restrict__ r,
                                      T* __restrict__ z) {
  pdl_entry();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const T rk = r[k] - a * q[k];
    r[k] = rk;
    z[k] = dinv[k] * rk;
  }
}
template <typename T>
__global__ void lanczos_dir_kernel(int64_t n, T b, const T* __restrict__ z, T* __restrict__ p) {
  pdl_entry();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    p[k] = z[k] + b * p[k];
}

template <typename T>
void MultiGrid<T>::lanczos_update(int64_t n, T a, const T* q, const T* dinv, T* r, T* z) {
  launch(lanczos_update_kernel<T>, grid1(n), 256, 0, stream, n, a, q, dinv, r, z); count_launch();
}
template <typename T>
void MultiGrid<T>::lanczos_dir(int64_t n, T b, const T* z, T* p) {
  launch(lanczos_dir_kernel<T>, grid1(n), 256, 0, stream, n, b, z, p); count_launch();
}

template <typename T>
dg_status MultiGrid<T>::set_alpha(double a) {
  int slot = -1;
  for (int sl = 0; sl < 2; ++sl)
    if (cache_alpha[sl] == a) slot = sl;
  if (slot >= 0) {
    cur = slot;
    alpha = a;
    return DG_OK;
  }
  slot = next_slot;
  next_slot ^= 1;
  drop_graphs(slot);  // its diagonal, bounds and coarse inverse change
  cache_alpha[slot] = a;
  alpha = a;
  cur = slot;
  for (size_t l = 0; l < lv.size(); ++l) {
    MGLevel<T>& L = lv[l];
    dg_status st = poisson_diagonal(L.mesh, a, diag, stream);
    if (st != DG_OK) return st;
    launch(inv_diag_kernel<T>, grid1(L.n), 256, 0, stream, L.n, diag, L.dinv[slot]); count_launch();
    DG_CUDA(cudaGetLastError());
    const bool coarsest = l + 1 == lv.size();
    double lo, hi;
    st = estimate((int)l, slot, coarsest ? 60 : 15, &lo, &hi);
    if (st != DG_OK) return st;
    L.lmax[slot] = 1.1 * hi;
    L.lmin[slot] = coarsest ? std::max(0.9 * lo, 1e-3 * hi) : L.lmax[slot] / 20.0;
  }
  if (lv.back().n <= kCoarseDenseMax) {
    dg_status st = coarse_inverse(slot);
    if (st != DG_OK) return st;
  }
  // transfer tables
  tr.clear();
  for (size_t l = 1; l < lv.size(); ++l) {
    const dg_mesh* f = lv[l - 1].mesh;
    const dg_mesh* c = lv[l].mesh;
    Transfer t;
    std::memset(&t, 0, sizeof(t));
    t.dim = f->dim;
    t.nf = f->np;
    t.nc = c->np;
    for (int ax = 0; ax < 3; ++ax) {
      t.hco[ax] = lv[l].hco[ax];
      t.nfine[ax] = f->n[ax];
      t.ncoarse[ax] = c->n[ax];
    }
    for (int i = 0; i < t.nf; ++i) {
      const double x = f->tp64.x[i];
      double v[kMaxN];
      for (int b = 0; b < 2; ++b) {
        lagrange_at(c->tp64.x, t.nc, 0.5 * (b + x), v);  // child b of the coarse interval
        for (int j = 0; j < t.nc; ++j) t.M[b][i][j] = v[j];
      }
      lagrange_at(c->tp64.x, t.nc, x, v);                 // same interval
      for (int j = 0; j < t.nc; ++j) t.M[2][i][j] = v[j];
    }
    for (int b = 0; b < 3; ++b)
      for (int i = 0; i < kMaxN; ++i)
        for (int j = 0; j < kMaxN; ++j) t.Mf[b][i][j] = (float)t.M[b][i][j];
    tr.push_back(t);
  }
  return DG_OK;
}

// Chebyshev smoothing on level l: x <- x + poly(D^-1 A) D^-1 (b - A x).
// From a nonzero x the start (r = D^-1 (b - A x), d = r / theta) is the
// operator apply with that output stage.  Every step after the first is one
// fused launch: the operator apply whose epilogue does x += d,
// r -= D^-1 A d, d' = c1 d + c2 r (into the second direction buffer, since
// neighbouring cells still read d); the last one adds d + d' to x instead
// and stores neither r nor d'.
template <typename T>
dg_status MultiGrid<T>::chebyshev(int l, int degree, bool x_zero) {
  MGLevel<T>& L = lv[l];
  const int64_t n = L.n;
  const T* dinv = L.dinv[cur];
  const double lmax = L.lmax[cur], lmin = L.lmin[cur];
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  dg_status st;
  if (x_zero) {
    launch(cheb_init_kernel<T>, grid1(n), 256, 0, stream, n, L.b, nullptr, dinv, (T)(1.0 / theta), L.r, L.d); count_launch();
    DG_CUDA(cudaMemsetAsync(L.x, 0, sizeof(T) * n, stream));
  } else {
    st = launch_poisson_epi<T>(3, L.mesh, alpha, L.x, L.d, L.b, L.r, dinv, 1.0 / theta, 0.0, stream);
    if (st != DG_OK) return st;
  }
  int swaps = 0;
  for (int k = 0; k + 1 < degree; ++k) {
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    const bool last = k + 2 == degree;
    st = launch_poisson_epi<T>(last ? 4 : 1, L.mesh, alpha, L.d, L.d2, L.x, L.r, dinv, rho_new * rho,
                               2.0 * rho_new / delta, stream);
    if (st != DG_OK) return st;
    if (!last) {
      T* tmp = L.d;
      L.d = L.d2;
      L.d2 = tmp;
      ++swaps;
    }
    rho = rho_new;
  }
  if (degree <= 1) {
    launch(add_kernel<T>, grid1(n), 256, 0, stream, n, L.d, L.x);
    count_launch();
  }
  DG_CUDA(cudaGetLastError());
  if (swaps & 1) {  // the direction is consumed: give every call the same buffers
    T* tmp = L.d;
    L.d = L.d2;
    L.d2 = tmp;
  }
  return DG_OK;
}

// Dense inverse of the coarsest level operator for one cached alpha: its
// columns are applies to the unit vectors, inverted on the host by
// Gauss-Jordan elimination with partial pivoting in FP64.
template <typename T>
dg_status MultiGrid<T>::coarse_inverse(int slot) {
  MGLevel<T>& L = lv.back();
  const int64_t n = L.n;
  T *I = nullptr, *Acol = nullptr;
  DG_CUDA(cudaMalloc(&I, sizeof(T) * n * n));
  DG_CUDA(cudaMalloc(&Acol, sizeof(T) * n * n));
  launch(identity_kernel<T>, grid1(n * n), 256, 0, stream, n, I); count_launch();
  dg_status st = DG_OK;
  for (int64_t j = 0; j < n && st == DG_OK; ++j)
    st = level_apply<T>(L, alpha, I + j * n, Acol + j * n, stream);
  std::vector<T> ht(n * n);
  if (st == DG_OK) {
    cudaError_t e = cudaMemcpyAsync(ht.data(), Acol, sizeof(T) * n * n, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) st = cuda_fail(e, "coarse inverse");
  }
  cudaFree(I);
  if (st != DG_OK) {
    cudaFree(Acol);
    return st;
  }
  // column j of ht is A e_j: a[i][j] = ht[j*n + i]
  std::vector<double> a(n * n), inv(n * n, 0.0);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) a[i * n + j] = (double)ht[j * n + i];
  for (int64_t i = 0; i < n; ++i) inv[i * n + i] = 1.0;
  for (int64_t c = 0; c < n; ++c) {
    int64_t piv = c;
    for (int64_t r = c + 1; r < n; ++r)
      if (std::fabs(a[r * n + c]) > std::fabs(a[piv * n + c])) piv = r;
    if (a[piv * n + c] == 0.0) {
      cudaFree(Acol);
      set_error("multigrid: singular coarse operator");
      return DG_EBREAKDOWN;
    }
    if (piv != c)
      for (int64_t k = 0; k < n; ++k) {
        std::swap(a[c * n + k], a[piv * n + k]);
        std::swap(inv[c * n + k], inv[piv * n + k]);
      }
    const double p = 1.0 / a[c * n + c];
    for (int64_t k = 0; k < n; ++k) {
      a[c * n + k] *= p;
      inv[c * n + k] *= p;
    }
    for (int64_t r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = a[r * n + c];
      if (f == 0.0) continue;
      for (int64_t k = 0; k < n; ++k) {
        a[r * n + k] -= f * a[c * n + k];
        inv[r * n + k] -= f * inv[c * n + k];
      }
    }
  }
  // store column by column: Ainv[j*n + i] = inv[i][j]
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) ht[j * n + i] = (T)inv[i * n + j];
  if (!L.ainv[slot]) {
    cudaError_t e = cudaMalloc(&L.ainv[slot], sizeof(T) * n * n);
    if (e != cudaSuccess) {
      cudaFree(Acol);
      return cuda_fail(e, "coarse inverse");
    }
  }
  cudaError_t e = cudaMemcpyAsync(L.ainv[slot], ht.data(), sizeof(T) * n * n, cudaMemcpyHostToDevice, stream);
  // ht is a host buffer that goes out of scope on return: the copy must finish
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  cudaFree(Acol);
  if (e != cudaSuccess) return cuda_fail(e, "coarse inverse");
  return DG_OK;
}

template <typename T>
dg_status MultiGrid<T>::vcycle(int l) {
  dg_status st;
  if (l + 1 == (int)lv.size()) {
    MGLevel<T>& Lc = lv[l];
    if (Lc.ainv[cur]) {
      launch(dense_matvec_kernel<T>, (unsigned)((Lc.n + 7) / 8), 256, 0, stream, (int)Lc.n, Lc.ainv[cur],
                                                                              Lc.b, Lc.x);
      count_launch();
      DG_CUDA(cudaGetLastError());
      return DG_OK;
    }
    return chebyshev(l, 30, true);
  }
  MGLevel<T>& L = lv[l];
  MGLevel<T>& C = lv[l + 1];
  st = chebyshev(l, smooth_degree, true);
  if (st != DG_OK) return st;
  // r = b - A x in one launch (the operator's residual output stage)
  st = launch_poisson_epi<T>(2, L.mesh, alpha, L.x, L.r, nullptr, L.b, nullptr, 0.0, 0.0, stream);
  if (st != DG_OK) return st;
  {
    const Transfer& t = tr[l];
    int nchild = 1;
    for (int a = 0; a < t.dim; ++a)
      if (t.hco[a]) nchild *= 2;
    const int nbc = t.dim == 3 ? t.nc * t.nc * t.nc : t.nc * t.nc;
    const int64_t ncc = C.n / nbc, nterm = C.n * nchild;
    if (t.dim == 3 && t.nf == 2 && t.nc == 2) {  // Q1 -> Q1: sum-factorised, one pass
      launch(restrict_q1_kernel<T>, grid1(ncc), 256, 0, stream, t, ncc, L.r, C.b);
      count_launch();
    } else {
      // the fine level's spare direction buffer holds the partial sums
      // (nchild * coarse DoFs = fine cells * coarse nodes <= fine DoFs)
      launch(restrict_part_kernel<T>, (unsigned)((nterm + 255) / 256), 256, 0, stream, t, ncc, nchild, L.r, L.d2);
      count_launch();
      launch(restrict_sum_kernel<T>, (unsigned)((C.n + 255) / 256), 256, 0, stream, C.n, nbc, nchild, L.d2, C.b);
      count_launch();
    }
  }
  DG_CUDA(cudaGetLastError());
  st = vcycle(l + 1);
  if (st != DG_OK) return st;
  if (tr[l].dim == 3 && tr[l].nf == 2 && tr[l].nc == 2)
    launch(prolong_q1_kernel<T>, grid1(L.n / 8), 256, 0, stream, tr[l], L.n / 8, C.x, L.x);
  else
    launch(prolong_add_kernel<T>, grid1(L.n), 256, 0, stream, tr[l], L.n, C.x, L.x);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return chebyshev(l, smooth_degree, false);
}

template <typename T>
dg_status MultiGrid<T>::apply_direct(const double* r, double* z) {
  MGLevel<T>& L = lv[0];
  launch(cvt_kernel<T>, grid1(L.n), 256, 0, stream, L.n, r, L.b); count_launch();
  dg_status st = vcycle(0);
  if (st != DG_OK) return st;
  launch(cvt_back_kernel<T>, grid1(L.n), 256, 0, stream, L.n, L.x, z); count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

template <typename T>
void MultiGrid<T>::set_degree(int degree) {
  if (degree < 1) degree = 5;
  if (degree == smooth_degree) return;
  drop_graphs(-1);
  smooth_degree = degree;
}

// slot < 0: all
template <typename T>
void MultiGrid<T>::drop_graphs(int slot) {
  std::vector<Captured> keep;
  for (auto& g : graphs) {
    if (slot < 0 || g.slot == slot) cudaGraphExecDestroy(g.exec);
    else keep.push_back(g);
  }
  graphs.swap(keep);
}

// Replays the captured V-cycle for (r, z, current alpha slot); captures it
// on first use.  Capturing runs no kernel, so the new graph is launched once
// after instantiation; its kernels were counted while they were recorded.
template <typename T>
dg_status MultiGrid<T>::apply(const double* r, double* z) {
  for (auto& g : graphs)
    if (g.r == r && g.z == z && g.slot == cur) {
      DG_CUDA(cudaGraphLaunch(g.exec, stream));
      count_launches(g.launches);
      return DG_OK;
    }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  DG_CUDA(cudaStreamIsCapturing(stream, &cs));
  if (!use_graphs || cs != cudaStreamCaptureStatusNone) return apply_direct(r, z);
  // record on a private stream (the solver's stream may be the legacy
  // default stream, which cannot be captured); nothing runs while recording
  if (!cap_stream && cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    cap_stream = nullptr;
    use_graphs = false;
    return apply_direct(r, z);
  }
  const int64_t before = launches_so_far();
  const cudaStream_t run_stream = stream;
  if (cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    use_graphs = false;
    return apply_direct(r, z);
  }
  stream = cap_stream;
  const dg_status st = apply_direct(r, z);
  stream = run_stream;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cap_stream, &graph);
  if (st != DG_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {  // fall back to direct launches for good
    cudaGetLastError();
    use_graphs = false;
    return apply_direct(r, z);
  }
  if (graphs.size() >= 8) {
    cudaGraphExecDestroy(graphs.front().exec);
    graphs.erase(graphs.begin());
  }
  graphs.push_back(Captured{r, z, cur, exec, launches_so_far() - before});
  DG_CUDA(cudaGraphLaunch(exec, stream));
  return DG_OK;
}

template struct MultiGrid<float>;
template struct MultiGrid<double>;

}  // namespace dg
