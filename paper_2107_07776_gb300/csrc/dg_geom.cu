// Precomputed metric terms of trilinear cells (layout and definitions in
// dg_geom.cuh).  Native FP64 setup kernels, run once per mesh; FP32 copies
// serve the single-precision applies.
#include <cmath>
#include <vector>

#include "dg_df64.cuh"
#include "dg_geom.cuh"

namespace dg {

namespace {

struct Lattice {
  const double* V;   // vertices [(L2 * nv1 + L1) * nv0 + L0][3]
  int nv0, nv1;
  int n[3];          // cells per axis
  int per[3];
  int dim;
  int64_t ncell;
};

__device__ void cell_of(const Lattice& g, int64_t c, int C[3]) {
  C[0] = (int)(c % g.n[0]);
  C[1] = (int)((c / g.n[0]) % g.n[1]);
  C[2] = g.dim == 3 ? (int)(c / ((int64_t)g.n[0] * g.n[1])) : 0;
}

// neighbour across face (a, s); -1 at a wall
__device__ int64_t neighbour_of(const Lattice& g, const int C[3], int a, int s, int Cn[3]) {
  for (int b = 0; b < 3; ++b) Cn[b] = C[b];
  Cn[a] += s ? 1 : -1;
  if (Cn[a] < 0 || Cn[a] >= g.n[a]) {
    if (!g.per[a]) return -1;
    Cn[a] = (Cn[a] + g.n[a]) % g.n[a];
  }
  return Cn[0] + (int64_t)g.n[0] * (Cn[1] + (int64_t)g.n[1] * Cn[2]);
}

// J[r][c] = dx_r/dxi_c of the multilinear map of cell C at xi
__device__ void jacobian(const Lattice& g, const int C[3], const double xi[3], double J[3][3]) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) J[r][c] = 0.0;
  const int d = g.dim;
  for (int corner = 0; corner < (1 << d); ++corner) {
    int L[3] = {0, 0, 0};
    double f[3], df[3];
    for (int a = 0; a < d; ++a) {
      const int bit = (corner >> a) & 1;
      L[a] = C[a] + bit;
      f[a] = bit ? xi[a] : 1.0 - xi[a];
      df[a] = bit ? 1.0 : -1.0;
    }
    const double* X = g.V + 3 * ((int64_t)(L[2] * g.nv1 + L[1]) * g.nv0 + L[0]);
    for (int c = 0; c < d; ++c) {
      double sh = df[c];
      for (int e = 0; e < d; ++e)
        if (e != c) sh *= f[e];
      for (int r = 0; r < d; ++r) J[r][c] += X[r] * sh;
    }
  }
}

// det J and Ji = J^-1 (Ji[a][r] = dxi_a/dx_r) by cofactors
__device__ double inverse(int d, const double J[3][3], double Ji[3][3]) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) Ji[r][c] = 0.0;
  if (d == 2) {
    const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    Ji[0][0] = J[1][1] / det;
    Ji[0][1] = -J[0][1] / det;
    Ji[1][0] = -J[1][0] / det;
    Ji[1][1] = J[0][0] / det;
    return det;
  }
  const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  Ji[0][0] = c00 / det;
  Ji[1][0] = c01 / det;
  Ji[2][0] = c02 / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  return det;
}

struct Rule {
  double x[kMaxN + 2], w[kMaxN + 2];
  int n;
};

// volume terms at the nodes of a space with n points per direction
__global__ void volume_kernel(const __grid_constant__ Lattice g, const __grid_constant__ Rule q,
                              bool with_b, int nfield, double* __restrict__ out) {
  pdl_entry();
  const int d = g.dim, n = q.n;
  const int nb = d == 3 ? n * n * n : n * n;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= g.ncell * nb) return;
  const int64_t c = gid / nb;
  const int node = (int)(gid % nb);
  int C[3];
  cell_of(g, c, C);
  const int ii[3] = {node % n, (node / n) % n, d == 3 ? node / (n * n) : 0};
  double xi[3] = {0, 0, 0}, w = 1.0;
  for (int a = 0; a < d; ++a) {
    xi[a] = q.x[ii[a]];
    w *= q.w[ii[a]];
  }
  double J[3][3], Ji[3][3];
  jacobian(g, C, xi, J);
  const double W = w * inverse(d, J, Ji);
  double* o = out + c * (int64_t)nfield * nb + node;
  int f = 0;
  for (int a = 0; a < d; ++a)
    for (int b = a; b < d; ++b) {
      double s = 0.0;
      for (int r = 0; r < d; ++r) s += Ji[a][r] * Ji[b][r];
      o[(int64_t)(f++) * nb] = W * s;
    }
  o[(int64_t)(f++) * nb] = W;
  if (with_b)
    for (int a = 0; a < d; ++a)
      for (int r = 0; r < d; ++r) o[(int64_t)(f++) * nb] = W * Ji[a][r];
}

// face terms at the face points of a space with n points per direction
__global__ void face_kernel(const __grid_constant__ Lattice g, const __grid_constant__ Rule q,
                            bool with_n, int nfield, double* __restrict__ out) {
  pdl_entry();
  const int d = g.dim, n = q.n;
  const int nf = d == 3 ? n * n : n;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= g.ncell * 2 * d * nf) return;
  const int64_t c = gid / (2 * d * nf);
  const int face = (int)((gid / nf) % (2 * d));
  const int t = (int)(gid % nf);
  const int a = face >> 1, s = face & 1;
  int C[3];
  cell_of(g, c, C);
  double xi[3] = {0, 0, 0}, w = 1.0;
  {
    int tt = t;
    for (int b = 0; b < d; ++b) {
      if (b == a) continue;
      xi[b] = q.x[tt % n];
      w *= q.w[tt % n];
      tt /= n;
    }
  }
  xi[a] = s;
  double J[3][3], Ji[3][3];
  jacobian(g, C, xi, J);
  const double det = inverse(d, J, Ji);
  double nv[3] = {0, 0, 0}, nn = 0.0;
  for (int r = 0; r < d; ++r) {
    nv[r] = (s ? det : -det) * Ji[a][r];
    nn += nv[r] * nv[r];
  }
  nn = sqrt(nn);
  for (int r = 0; r < d; ++r) nv[r] /= nn;
  double cown[3] = {0, 0, 0}, cnb[3] = {0, 0, 0};
  for (int b = 0; b < d; ++b)
    for (int r = 0; r < d; ++r) cown[b] += Ji[b][r] * nv[r];
  int Cn[3];
  if (neighbour_of(g, C, a, s, Cn) >= 0) {
    double xin[3] = {xi[0], xi[1], xi[2]};
    xin[a] = 1 - s;
    double Jn[3][3], Jin[3][3];
    jacobian(g, Cn, xin, Jn);
    inverse(d, Jn, Jin);
    for (int b = 0; b < d; ++b)
      for (int r = 0; r < d; ++r) cnb[b] += Jin[b][r] * nv[r];
  }
  double* o = out + ((c * 2 * d + face) * (int64_t)nfield) * nf + t;
  int f = 0;
  o[(int64_t)(f++) * nf] = w * nn;
  if (with_n)
    for (int r = 0; r < d; ++r) o[(int64_t)(f++) * nf] = nv[r];
  for (int b = 0; b < d; ++b) o[(int64_t)(f++) * nf] = cown[b];
  for (int b = 0; b < d; ++b) o[(int64_t)(f++) * nf] = cnb[b];
}

// |Gamma_f| / |K| per cell face by the rule q
__global__ void ratio_kernel(const __grid_constant__ Lattice g, const __grid_constant__ Rule q,
                             double* __restrict__ ratio) {
  pdl_entry();
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const int d = g.dim, n = q.n;
  int C[3];
  cell_of(g, c, C);
  double vol = 0.0;
  const int nqd = d == 3 ? n * n * n : n * n;
  for (int p = 0; p < nqd; ++p) {
    const int ii[3] = {p % n, (p / n) % n, d == 3 ? p / (n * n) : 0};
    double xi[3] = {0, 0, 0}, w = 1.0;
    for (int a = 0; a < d; ++a) {
      xi[a] = q.x[ii[a]];
      w *= q.w[ii[a]];
    }
    double J[3][3], Ji[3][3];
    jacobian(g, C, xi, J);
    vol += w * inverse(d, J, Ji);
  }
  const int nqf = d == 3 ? n * n : n;
  for (int face = 0; face < 2 * d; ++face) {
    const int a = face >> 1, s = face & 1;
    double area = 0.0;
    for (int p = 0; p < nqf; ++p) {
      double xi[3] = {0, 0, 0}, w = 1.0;
      int tt = p;
      for (int b = 0; b < d; ++b) {
        if (b == a) continue;
        xi[b] = q.x[tt % n];
        w *= q.w[tt % n];
        tt /= n;
      }
      xi[a] = s;
      double J[3][3], Ji[3][3];
      jacobian(g, C, xi, J);
      const double det = inverse(d, J, Ji);
      double nn = 0.0;
      for (int r = 0; r < d; ++r) nn += (det * Ji[a][r]) * (det * Ji[a][r]);
      area += w * sqrt(nn);
    }
    ratio[c * 2 * d + face] = area / vol;
  }
}

__global__ void penalty_kernel(const __grid_constant__ Lattice g, const double* __restrict__ ratio,
                               double* __restrict__ gpen) {
  pdl_entry();
  const int d = g.dim;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= g.ncell * 2 * d) return;
  const int64_t c = gid / (2 * d);
  const int face = (int)(gid % (2 * d)), a = face >> 1, s = face & 1;
  int C[3], Cn[3];
  cell_of(g, c, C);
  const int64_t nb = neighbour_of(g, C, a, s, Cn);
  gpen[gid] = nb < 0 ? ratio[gid] : 0.5 * (ratio[gid] + ratio[nb * 2 * d + 2 * a + (1 - s)]);
}

__global__ void to_pairs_kernel(int64_t n, const double* __restrict__ a, df64* __restrict__ b) {
  pdl_entry();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    b[k] = df_split(a[k]);
}

__global__ void to_f32_kernel(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  pdl_entry();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    b[k] = (float)a[k];
}

unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

dg_status alloc_pair(int64_t n, double** d64, float** d32, df64** ddf) {
  DG_CUDA(cudaMalloc(d64, sizeof(double) * n));
  DG_CUDA(cudaMalloc(d32, sizeof(float) * n));
  DG_CUDA(cudaMalloc(ddf, sizeof(df64) * n));
  return DG_OK;
}

}  // namespace

void free_geometry(dg_mesh* m) {
  double** p64[] = {&m->gvu64, &m->gfu64, &m->gvp64, &m->gfp64, &m->gpen64};
  float** p32[] = {&m->gvu32, &m->gfu32, &m->gvp32, &m->gfp32, &m->gpen32};
  df64** pdf[] = {&m->gvu_df, &m->gfu_df, &m->gvp_df, &m->gfp_df, &m->gpen_df};
  for (double** p : p64) {
    cudaFree(*p);
    *p = nullptr;
  }
  for (float** p : p32) {
    cudaFree(*p);
    *p = nullptr;
  }
  for (df64** p : pdf) {
    cudaFree(*p);
    *p = nullptr;
  }
}

dg_status build_geometry(dg_mesh* m, bool velocity, cudaStream_t s) {
  const int d = m->dim;
  // vertex lattice on the device
  const int nv0 = m->n[0] + 1, nv1 = m->n[1] + 1, nv2 = d == 3 ? m->n[2] + 1 : 1;
  std::vector<double> V((size_t)3 * nv0 * nv1 * nv2, 0.0);
  for (int L2 = 0; L2 < nv2; ++L2)
    for (int L1 = 0; L1 < nv1; ++L1)
      for (int L0 = 0; L0 < nv0; ++L0) {
        const int L[3] = {L0, L1, L2};
        lattice_vertex(m->desc, L, &V[3 * ((size_t)(L2 * nv1 + L1) * nv0 + L0)]);
      }
  double* dV = nullptr;
  double* ratio = nullptr;
  DG_CUDA(cudaMalloc(&dV, sizeof(double) * V.size()));
  cudaError_t e = cudaMemcpyAsync(dV, V.data(), sizeof(double) * V.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMalloc(&ratio, sizeof(double) * m->ncell * 2 * d);
  if (e != cudaSuccess) {
    cudaFree(dV);
    return cuda_fail(e, "geometry setup");
  }
  Lattice g;
  g.V = dV;
  g.nv0 = nv0;
  g.nv1 = nv1;
  g.dim = d;
  g.ncell = m->ncell;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = m->n[a];
    g.per[a] = m->periodic[a];
  }
  auto rule_of = [](const Tab1D<double>& t, int n) {
    Rule r;
    r.n = n;
    for (int i = 0; i < kMaxN + 2; ++i) r.x[i] = r.w[i] = 0.0;
    for (int i = 0; i < n; ++i) {
      r.x[i] = t.x[i];
      r.w[i] = t.w[i];
    }
    return r;
  };
  const Rule ru = rule_of(m->tu64, m->nu), rp = rule_of(m->tp64, m->np);
  Rule rm;  // (k+2)-point rule of the penalty measures
  rm.n = m->k + 2;
  gauss_legendre_01(rm.n, rm.x, rm.w);
  const int nfu = d == 3 ? m->nu * m->nu : m->nu, nfp = d == 3 ? m->np * m->np : m->np;
  const int NG = d * (d + 1) / 2;
  const int nvu_f = NG + 1 + d * d, nvp_f = NG + 1, nfu_f = 1 + 3 * d, nfp_f = 1 + 2 * d;
  const int64_t n_vu = m->ncell * nvu_f * m->nbu, n_fu = m->ncell * 2 * d * nfu_f * nfu;
  const int64_t n_vp = m->ncell * nvp_f * m->nbp, n_fp = m->ncell * 2 * d * nfp_f * nfp;
  const int64_t n_pen = m->ncell * 2 * d;
  dg_status st = DG_OK;
  if (velocity) {
    st = alloc_pair(n_vu, &m->gvu64, &m->gvu32, &m->gvu_df);
    if (st == DG_OK) st = alloc_pair(n_fu, &m->gfu64, &m->gfu32, &m->gfu_df);
  }
  if (st == DG_OK) st = alloc_pair(n_vp, &m->gvp64, &m->gvp32, &m->gvp_df);
  if (st == DG_OK) st = alloc_pair(n_fp, &m->gfp64, &m->gfp32, &m->gfp_df);
  if (st == DG_OK) st = alloc_pair(n_pen, &m->gpen64, &m->gpen32, &m->gpen_df);
  if (st != DG_OK) {
    cudaFree(dV);
    cudaFree(ratio);
    free_geometry(m);
    return st;
  }
  const int T = 128;
  if (velocity) {
    launch(volume_kernel, blocks_for(m->ncell * m->nbu, T), T, 0, s, g, ru, true, nvu_f, m->gvu64);
    launch(face_kernel, blocks_for(m->ncell * 2 * d * nfu, T), T, 0, s, g, ru, true, nfu_f, m->gfu64);
  }
  launch(volume_kernel, blocks_for(m->ncell * m->nbp, T), T, 0, s, g, rp, false, nvp_f, m->gvp64);
  launch(face_kernel, blocks_for(m->ncell * 2 * d * nfp, T), T, 0, s, g, rp, false, nfp_f, m->gfp64);
  launch(ratio_kernel, blocks_for(m->ncell, T), T, 0, s, g, rm, ratio);
  launch(penalty_kernel, blocks_for(n_pen, T), T, 0, s, g, ratio, m->gpen64);
  const int conv_blocks = 1216;
  if (velocity) {
    launch(to_f32_kernel, conv_blocks, 256, 0, s, n_vu, m->gvu64, m->gvu32);
    launch(to_f32_kernel, conv_blocks, 256, 0, s, n_fu, m->gfu64, m->gfu32);
  }
  launch(to_f32_kernel, conv_blocks, 256, 0, s, n_vp, m->gvp64, m->gvp32);
  launch(to_f32_kernel, conv_blocks, 256, 0, s, n_fp, m->gfp64, m->gfp32);
  launch(to_f32_kernel, conv_blocks, 256, 0, s, n_pen, m->gpen64, m->gpen32);
  if (velocity) {
    launch(to_pairs_kernel, conv_blocks, 256, 0, s, n_vu, m->gvu64, m->gvu_df);
    launch(to_pairs_kernel, conv_blocks, 256, 0, s, n_fu, m->gfu64, m->gfu_df);
  }
  launch(to_pairs_kernel, conv_blocks, 256, 0, s, n_vp, m->gvp64, m->gvp_df);
  launch(to_pairs_kernel, conv_blocks, 256, 0, s, n_fp, m->gfp64, m->gfp_df);
  launch(to_pairs_kernel, conv_blocks, 256, 0, s, n_pen, m->gpen64, m->gpen_df);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dV);
  cudaFree(ratio);
  if (e != cudaSuccess) {
    free_geometry(m);
    return cuda_fail(e, "geometry setup");
  }
  m->geom_u = velocity;
  return DG_OK;
}

}  // namespace dg
