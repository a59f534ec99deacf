// Mesh construction, 1D tables, node coordinates and error plumbing.
//
// The 1D tables hold the nodal Lagrange basis at the Gauss-Legendre points
// (the collocated basis of Section 3: quadrature points are the nodes, so
// values at quadrature points are the DoFs and the mass matrix is diagonal on
// affine cells).  Points come from Newton's method on the Legendre
// polynomial; basis values and derivatives from barycentric Lagrange
// interpolation (Berrut & Trefethen, SIAM Review 46, 2004).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "dg_common.cuh"
#include "dg_geom.cuh"

namespace dg {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_kernel_launches{0};

void count_launch() { g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }

bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("DG_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}
void count_launches(int64_t n) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_kernel_launches.load(std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }

dg_status cuda_fail(cudaError_t e, const char* where) {
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  return DG_ECUDA;
}

// Gauss-Legendre on [-1,1] by Newton iteration; Legendre values by the
// Bonnet recurrence.
static void gauss_legendre_pm1(int n, double* z, double* w) {
  for (int r = 0; r < n; ++r) {
    double t = std::cos(M_PI * (4.0 * r + 3.0) / (4.0 * n + 2.0));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * t * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      double pn = n == 0 ? 1.0 : (n == 1 ? t : p1);
      double pnm1 = n == 1 ? 1.0 : p0;
      dp = n * (pnm1 - t * pn) / (1.0 - t * t);
      double step = pn / dp;
      t -= step;
      if (std::fabs(step) <= 1e-16 * std::fmax(1.0, std::fabs(t))) break;
    }
    // refresh the derivative at the converged root
    double p0 = 1.0, p1 = t;
    for (int j = 2; j <= n; ++j) {
      double p2 = ((2.0 * j - 1.0) * t * p1 - (j - 1.0) * p0) / j;
      p0 = p1;
      p1 = p2;
    }
    double pn = n == 1 ? t : p1, pnm1 = n == 1 ? 1.0 : p0;
    dp = n * (pnm1 - t * pn) / (1.0 - t * t);
    z[r] = t;
    w[r] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

void gauss_legendre_01(int n, double* x, double* w) {
  double z[16], wz[16];
  gauss_legendre_pm1(n, z, wz);
  for (int i = 0; i < n; ++i) {
    x[i] = 0.5 * (1.0 - z[i]);
    w[i] = 0.5 * wz[i];
  }
}

void make_tables(int n, Tab1D<double>* t) {
  std::memset(t, 0, sizeof(*t));
  double z[kMaxN], wz[kMaxN];
  gauss_legendre_pm1(n, z, wz);
  for (int i = 0; i < n; ++i) {  // ascending points on [0,1]
    t->x[i] = 0.5 * (1.0 - z[i]);
    t->w[i] = 0.5 * wz[i];
  }
  // symmetrise exactly: x[n-1-i] = 1 - x[i], w[n-1-i] = w[i]
  for (int i = 0; i < n / 2; ++i) {
    double xs = 0.5 * (t->x[i] + (1.0 - t->x[n - 1 - i]));
    double ws = 0.5 * (t->w[i] + t->w[n - 1 - i]);
    t->x[i] = xs;
    t->x[n - 1 - i] = 1.0 - xs;
    t->w[i] = t->w[n - 1 - i] = ws;
  }
  if (n % 2) t->x[n / 2] = 0.5;
  // barycentric weights
  double lam[kMaxN];
  for (int j = 0; j < n; ++j) {
    double p = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != j) p *= (t->x[j] - t->x[m]);
    lam[j] = 1.0 / p;
  }
  // differentiation matrix at the nodes: D[q][i] = L_i'(x_q)
  for (int q = 0; q < n; ++q) {
    double diag = 0.0;
    for (int i = 0; i < n; ++i) {
      if (i == q) continue;
      double v = (lam[i] / lam[q]) / (t->x[q] - t->x[i]);
      t->D[q][i] = v;
      diag -= v;
    }
    t->D[q][q] = diag;
  }
  // values and derivatives at the end points s = 0, 1 (never nodes)
  for (int s = 0; s < 2; ++s) {
    double ell = 1.0;
    for (int m = 0; m < n; ++m) ell *= (s - t->x[m]);
    for (int i = 0; i < n; ++i) {
      double li = ell * lam[i] / (s - t->x[i]);
      double sum = 0.0;
      for (int m = 0; m < n; ++m)
        if (m != i) sum += 1.0 / (s - t->x[m]);
      t->L[s][i] = li;
      t->dL[s][i] = li * sum;
    }
  }
}

void make_mix(const Tab1D<double>& tu, int nu, const Tab1D<double>& tp, int np,
              MixTab<double>* m) {
  std::memset(m, 0, sizeof(*m));
  double lam[kMaxN];
  for (int j = 0; j < np; ++j) {
    double p = 1.0;
    for (int l = 0; l < np; ++l)
      if (l != j) p *= (tp.x[j] - tp.x[l]);
    lam[j] = 1.0 / p;
  }
  // Gauss points of consecutive orders interlace strictly, so a velocity
  // point is never a pressure node and the barycentric form applies.
  for (int q = 0; q < nu; ++q) {
    double x = tu.x[q], ell = 1.0;
    for (int l = 0; l < np; ++l) ell *= (x - tp.x[l]);
    for (int j = 0; j < np; ++j) {
      double v = ell * lam[j] / (x - tp.x[j]);
      double s = 0.0;
      for (int l = 0; l < np; ++l)
        if (l != j) s += 1.0 / (x - tp.x[l]);
      m->I[q][j] = v;
      m->D[q][j] = v * s;
    }
  }
}

template <typename T>
Tab1D<T> cast_tables(const Tab1D<double>& t) {
  Tab1D<T> o;
  for (int a = 0; a < kMaxN; ++a) {
    for (int b = 0; b < kMaxN; ++b) o.D[a][b] = (T)t.D[a][b];
    o.w[a] = (T)t.w[a];
    o.x[a] = (T)t.x[a];
    for (int s = 0; s < 2; ++s) {
      o.L[s][a] = (T)t.L[s][a];
      o.dL[s][a] = (T)t.dL[s][a];
    }
  }
  return o;
}
template Tab1D<float> cast_tables<float>(const Tab1D<double>&);

MixTab<df64> split_mix(const MixTab<double>& t) {
  MixTab<df64> o;
  for (int a = 0; a < kMaxN; ++a)
    for (int b = 0; b < kMaxN; ++b) {
      const float hI = (float)t.I[a][b], hD = (float)t.D[a][b];
      o.I[a][b] = df64{hI, (float)(t.I[a][b] - (double)hI)};
      o.D[a][b] = df64{hD, (float)(t.D[a][b] - (double)hD)};
    }
  return o;
}

// float-float split of every table entry: hi = fl32(x), lo = fl32(x - hi)
Tab1D<df64> split_tables(const Tab1D<double>& t) {
  Tab1D<df64> o;
  auto sp = [](double x) {
    const float h = (float)x;
    return df64{h, (float)(x - (double)h)};
  };
  for (int a = 0; a < kMaxN; ++a) {
    for (int b = 0; b < kMaxN; ++b) o.D[a][b] = sp(t.D[a][b]);
    o.w[a] = sp(t.w[a]);
    o.x[a] = sp(t.x[a]);
    for (int s = 0; s < 2; ++s) {
      o.L[s][a] = sp(t.L[s][a]);
      o.dL[s][a] = sp(t.dL[s][a]);
    }
  }
  return o;
}
template Tab1D<double> cast_tables<double>(const Tab1D<double>&);

// Vertex of the structured lattice (lattice index L) under the mesh map.
void lattice_vertex(const dg_mesh_desc& d, const int L[3], double X[3]) {
  double eta[3] = {0, 0, 0};
  for (int a = 0; a < d.dim; ++a) eta[a] = (double)L[a] / d.n_cells[a];
  for (int a = 0; a < 3; ++a) X[a] = 0.0;
  for (int a = 0; a < d.dim; ++a) {
    double s = eta[a];
    if (d.map == DG_MAP_GRADED_TANH && d.map_param[a] > 0.0) {
      double b = d.map_param[a];
      s = 0.5 * (1.0 - std::tanh(b * (1.0 - 2.0 * eta[a])) / std::tanh(b));
    }
    X[a] = d.lo[a] + (d.hi[a] - d.lo[a]) * s;
  }
  if (d.map == DG_MAP_PERTURBED_SIN) {
    double amp = d.map_param[0];
    for (int a = 0; a < d.dim; ++a) amp *= std::sin(2.0 * M_PI * eta[a]);
    for (int a = 0; a < d.dim; ++a) X[a] += amp * (d.hi[a] - d.lo[a]);
  }
}

}  // namespace dg


namespace dg {

// Tables, per-axis extents and the status word of a mesh whose sizes and
// vertex lattice are set.
// 1D tables of the pressure operator alpha M^p + K on Q1 cells in
// tensor-product form (q1_tensor_kernel).  With the collocated two-point
// Gauss rule the mass is diagonal and the SIP operator (Eqs. weakform_p_1,
// penconst1) is the sum over the axes a of the 1D DG SIP matrix along a times
// the diagonal tangential masses.  Per axis cell c (extent h, neighbours
// across the lower and upper face, wrapped on a periodic axis, none on a wall
// where the pressure operator has no face terms), with the trace L_s, its
// derivative L'_s, sgn = -1 / +1 on the lower / upper face and
// C = pen (1/h + 1/h_N) / 2:
//   own block    K_ij = (1/h) sum_q w_q D_qi D_qj
//                     + sum_s [(C L_s(j) - sgn L'_s(j)/(2h)) L_s(i) - L_s(j) sgn L'_s(i)/(2h)]
//   neighbour s  N_ij = (-C L_{1-s}(j) - sgn L'_{1-s}(j)/(2 h_N)) L_s(i) + L_{1-s}(j) sgn L'_s(i)/(2h)
// (own node i, the neighbour's node j on the same line), the terms of the
// per-face-point flux of the Q1 kernel expanded in the nodal values.
double pack_pair(double x);

static dg_status build_q1_tables(dg_mesh* m, cudaStream_t s) {
  const Tab1D<double>& t = m->tp64;
  const double pen = (double)(m->np * m->np);
  std::vector<float> tab;
  std::vector<double> tabd;
  for (int a = 0; a < 3; ++a) {
    const int na = m->n[a];
    m->q1tab_off[a] = (int)(tab.size() / 16);  // in rows (axis cells)
    for (int c = 0; c < na; ++c) {
      const double h = m->vx[a][c + 1] - m->vx[a][c], hiK = 1.0 / h;
      double K[2][2], Nb[2][2][2];
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          double v = 0.0;
          for (int q = 0; q < 2; ++q) v += t.w[q] * t.D[q][i] * t.D[q][j];
          K[i][j] = hiK * v;
          Nb[0][i][j] = Nb[1][i][j] = 0.0;
        }
      for (int sd = 0; sd < 2; ++sd) {
        int cn = c + (sd ? 1 : -1);
        if (cn < 0 || cn >= na) {
          if (!m->periodic[a]) continue;
          cn = cn < 0 ? na - 1 : 0;
        }
        const double hiN = 1.0 / (m->vx[a][cn + 1] - m->vx[a][cn]);
        const double sgn = sd ? 1.0 : -1.0, C = 0.5 * pen * (hiK + hiN);
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 2; ++j) {
            K[i][j] += (C * t.L[sd][j] - 0.5 * sgn * hiK * t.dL[sd][j]) * t.L[sd][i] -
                       0.5 * t.L[sd][j] * sgn * hiK * t.dL[sd][i];
            Nb[sd][i][j] = (-C * t.L[1 - sd][j] - 0.5 * sgn * hiN * t.dL[1 - sd][j]) * t.L[sd][i] +
                           0.5 * t.L[1 - sd][j] * sgn * hiK * t.dL[sd][i];
          }
      }
      const float row[16] = {(float)(t.w[0] * h), (float)(t.w[1] * h), 0.0f, 0.0f,
                             (float)K[0][0], (float)K[0][1], (float)K[1][0], (float)K[1][1],
                             (float)Nb[0][0][0], (float)Nb[0][0][1], (float)Nb[0][1][0], (float)Nb[0][1][1],
                             (float)Nb[1][0][0], (float)Nb[1][0][1], (float)Nb[1][1][0], (float)Nb[1][1][1]};
      tab.insert(tab.end(), row, row + 16);
      const double rowd[16] = {t.w[0] * h, t.w[1] * h, 0.0, 0.0, K[0][0], K[0][1], K[1][0], K[1][1],
                               Nb[0][0][0], Nb[0][0][1], Nb[0][1][0], Nb[0][1][1],
                               Nb[1][0][0], Nb[1][0][1], Nb[1][1][0], Nb[1][1][1]};
      for (double v : rowd) tabd.push_back(pack_pair(v));
    }
  }
  cudaError_t e = cudaMalloc(&m->q1tab, sizeof(float) * tab.size());
  if (e == cudaSuccess) e = cudaMalloc(&m->q1tab_df, sizeof(double) * tabd.size());
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m->q1tab, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m->q1tab_df, tabd.data(), sizeof(double) * tabd.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host tables die here
  if (e != cudaSuccess) return cuda_fail(e, "mesh upload (Q1 tables)");
  return DG_OK;
}

dg_status finish_mesh(dg_mesh* m, cudaStream_t s) {
  cudaGetDevice(&m->device);
  m->nu = m->k + 1;
  m->np = m->k;
  m->nbu = m->dim == 3 ? m->nu * m->nu * m->nu : m->nu * m->nu;
  m->nbp = m->dim == 3 ? m->np * m->np * m->np : m->np * m->np;
  make_tables(m->nu, &m->tu64);
  make_tables(m->np, &m->tp64);
  make_mix(m->tu64, m->nu, m->tp64, m->np, &m->mix64);
  m->tu32 = cast_tables<float>(m->tu64);
  m->tp32 = cast_tables<float>(m->tp64);
  m->tudf = split_tables(m->tu64);
  m->tpdf = split_tables(m->tp64);
  m->mixdf = split_mix(m->mix64);
  {
    const char* env = std::getenv("DG_FP64_NATIVE");
    m->fp64_arith = env && env[0] == '1' ? 1 : 0;
  }
  for (int a = 0; a < 3; ++a) {
    int na = m->n[a];
    std::vector<double> h(na), hi(na);
    std::vector<float> hf(na), hif(na);
    for (int i = 0; i < na; ++i) {
      h[i] = m->vx[a][i + 1] - m->vx[a][i];
      hi[i] = 1.0 / h[i];
      hf[i] = (float)h[i];
      hif[i] = (float)hi[i];
    }
    cudaError_t e = cudaMalloc(&m->d_h64[a], sizeof(double) * na);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_h32[a], sizeof(float) * na);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_hi64[a], sizeof(double) * na);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_hi32[a], sizeof(float) * na);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(m->d_h64[a], h.data(), sizeof(double) * na, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(m->d_h32[a], hf.data(), sizeof(float) * na, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(m->d_hi64[a], hi.data(), sizeof(double) * na, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(m->d_hi32[a], hif.data(), sizeof(float) * na, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host vectors die here
    if (e != cudaSuccess) return cuda_fail(e, "mesh upload");
  }
  cudaError_t e = cudaMalloc(&m->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(m->d_status, 0, sizeof(int), s);
  if (e != cudaSuccess) return cuda_fail(e, "mesh status word");
  // float-float applies: the per-apply split buffers of the source vector
  // and advecting field (and, on affine meshes, split copies of the extents)
  {
    const int64_t nps =
        (m->level ? (int64_t)m->nbp : std::max<int64_t>((int64_t)m->dim * m->nbu, m->nbp)) * m->ncell;
    e = cudaMalloc(&m->ps_src, sizeof(double) * nps);
    if (e == cudaSuccess && !m->level)
      e = cudaMalloc(&m->ps_ub, sizeof(double) * (int64_t)m->dim * m->nbu * m->ncell);
    if (e != cudaSuccess) return cuda_fail(e, "mesh float-float split buffers");
  }
  if (!m->affine) return build_geometry(m, !m->level, s);
  for (int a = 0; a < 3; ++a) {
    const int na = m->n[a];
    std::vector<double> hp(na), hip(na);
    for (int i = 0; i < na; ++i) {
      const double h = m->vx[a][i + 1] - m->vx[a][i];
      hp[i] = pack_pair(h);
      hip[i] = pack_pair(1.0 / h);
    }
    e = cudaMalloc(&m->d_hdf[a], sizeof(double) * na);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_hidf[a], sizeof(double) * na);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(m->d_hdf[a], hp.data(), sizeof(double) * na, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(m->d_hidf[a], hip.data(), sizeof(double) * na, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "mesh upload (float-float extents)");
  }
  if (m->dim == 3 && m->np == 2) return build_q1_tables(m, s);
  return DG_OK;
}

double pack_pair(double x) {
  const float hi = (float)x;
  const float lo = (float)(x - (double)hi);
  uint32_t a, b;
  std::memcpy(&a, &hi, 4);
  std::memcpy(&b, &lo, 4);
  const uint64_t bits = (uint64_t)a | ((uint64_t)b << 32);
  double d;
  std::memcpy(&d, &bits, 8);
  return d;
}

// Mesh of a coarser multigrid level: axes with coarsen[a] set keep every
// other vertex of `fine`; `degree_u` sets the level's pressure nodes per
// direction (np = degree_u).  Affine meshes only.
dg_status make_level_mesh(const dg_mesh* fine, const int coarsen[3], int degree_u,
                          cudaStream_t s, dg_mesh** out) {
  *out = nullptr;
  dg_mesh* m = new (std::nothrow) dg_mesh();
  if (!m) return DG_ENOMEM;
  m->desc = fine->desc;
  m->dim = fine->dim;
  m->k = degree_u;
  m->desc.degree_u = degree_u;
  m->affine = fine->affine;
  m->level = true;
  m->ncell = 1;
  for (int a = 0; a < 3; ++a) {
    m->periodic[a] = fine->periodic[a];
    const bool c = a < fine->dim && coarsen[a];
    m->n[a] = c ? fine->n[a] / 2 : fine->n[a];
    if (a < fine->dim) m->desc.n_cells[a] = m->n[a];
    m->ncell *= m->n[a];
    m->vx[a].resize(m->n[a] + 1);
    for (int i = 0; i <= m->n[a]; ++i) m->vx[a][i] = fine->vx[a][c ? 2 * i : i];
  }
  dg_status st = finish_mesh(m, s);
  if (st != DG_OK) {
    dg_mesh_destroy(m);
    return st;
  }
  *out = m;
  return DG_OK;
}

}  // namespace dg

using namespace dg;

extern "C" {

const char* dg_status_string(dg_status s) {
  switch (s) {
    case DG_OK: return "ok";
    case DG_EINVAL: return "invalid argument";
    case DG_ECUDA: return "CUDA error";
    case DG_ENOMEM: return "out of memory";
    case DG_ENOCONV: return "solver did not converge";
    case DG_EBREAKDOWN: return "solver breakdown (non-finite residual)";
    case DG_ETIMEOUT: return "solver timeout";
    case DG_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* dg_last_error(void) { return g_last_error.c_str(); }

int64_t dg_kernel_launches(void) { return g_kernel_launches.load(std::memory_order_relaxed); }

dg_status dg_mesh_set_fp64_arith(dg_mesh* m, int32_t mode) {
  if (!m || (mode != 0 && mode != 1)) {
    set_error("dg_mesh_set_fp64_arith: mode must be 0 (float-float) or 1 (native FP64)");
    return DG_EINVAL;
  }
  m->fp64_arith = mode;
  return DG_OK;
}

dg_status dg_mesh_create(const dg_mesh_desc* desc, void* stream, dg_mesh** out) {
  if (!desc || !out) {
    set_error("dg_mesh_create: null argument");
    return DG_EINVAL;
  }
  *out = nullptr;
  const dg_mesh_desc& d = *desc;
  if (d.dim != 2 && d.dim != 3) {
    set_error("dg_mesh_create: dim must be 2 or 3");
    return DG_EINVAL;
  }
  if (d.degree_u < 2 || d.degree_u > 4) {
    set_error("dg_mesh_create: degree_u must be 2..4");
    return DG_EUNSUPPORTED;
  }
  for (int a = 0; a < d.dim; ++a) {
    if (d.n_cells[a] < 1 || !(d.hi[a] > d.lo[a])) {
      set_error("dg_mesh_create: need n_cells >= 1 and hi > lo on every axis");
      return DG_EINVAL;
    }
  }
  if (d.map < 0 || d.map > 2) {
    set_error("dg_mesh_create: unknown map");
    return DG_EINVAL;
  }
  int64_t nc = 1;
  for (int a = 0; a < d.dim; ++a) nc *= d.n_cells[a];
  if (nc > (int64_t)1 << 31) {
    set_error("dg_mesh_create: more than 2^31 cells");
    return DG_EINVAL;
  }
  dg_mesh* m = new (std::nothrow) dg_mesh();
  if (!m) return DG_ENOMEM;
  m->desc = d;
  m->dim = d.dim;
  m->k = d.degree_u;
  m->ncell = nc;
  for (int a = 0; a < 3; ++a) {
    m->n[a] = a < d.dim ? d.n_cells[a] : 1;
    m->periodic[a] = a < d.dim ? (d.periodic[a] ? 1 : 0) : 1;
  }
  m->affine = d.map != DG_MAP_PERTURBED_SIN;
  // per-axis vertex lattice (affine maps; the trilinear map perturbs it)
  for (int a = 0; a < 3; ++a) {
    int na = m->n[a];
    m->vx[a].resize(na + 1);
    for (int i = 0; i <= na; ++i) {
      int L[3] = {0, 0, 0};
      L[a] = i;
      double X[3];
      if (a < d.dim) {
        dg_mesh_desc dd = d;
        dd.map = d.map == DG_MAP_PERTURBED_SIN ? DG_MAP_CARTESIAN : d.map;
        lattice_vertex(dd, L, X);
        m->vx[a][i] = X[a];
      } else {
        m->vx[a][i] = (double)i;  // unit extent in the absent axis of 2D meshes
      }
    }
  }
  dg_status st = finish_mesh(m, as_stream(stream));
  if (st != DG_OK) {
    dg_mesh_destroy(m);
    return st;
  }
  *out = m;
  return DG_OK;
}

void dg_mesh_destroy(dg_mesh* m) {
  if (!m) return;
  for (int a = 0; a < 3; ++a) {
    if (m->d_h64[a]) cudaFree(m->d_h64[a]);
    if (m->d_h32[a]) cudaFree(m->d_h32[a]);
    if (m->d_hi64[a]) cudaFree(m->d_hi64[a]);
    if (m->d_hi32[a]) cudaFree(m->d_hi32[a]);
  }
  if (m->d_status) cudaFree(m->d_status);
  if (m->split_flux) cudaFree(m->split_flux);
  for (int a = 0; a < 3; ++a) {
    if (m->d_hdf[a]) cudaFree(m->d_hdf[a]);
    if (m->d_hidf[a]) cudaFree(m->d_hidf[a]);
    if (a == 0 && m->q1tab) cudaFree(m->q1tab);
    if (a == 0 && m->q1tab_df) cudaFree(m->q1tab_df);
  }
  if (m->ps_src) cudaFree(m->ps_src);
  if (m->ps_ub) cudaFree(m->ps_ub);
  for (double* q : m->ps_pool)
    if (q) cudaFree(q);
  free_geometry(m);
  delete m;
}

dg_status dg_mesh_info(const dg_mesh* m, int64_t* n_cells, int64_t* n_dofs_u, int64_t* n_dofs_p) {
  if (!m) {
    set_error("dg_mesh_info: null mesh");
    return DG_EINVAL;
  }
  if (n_cells) *n_cells = m->ncell;
  if (n_dofs_u) *n_dofs_u = m->ncell * m->nbu * m->dim;
  if (n_dofs_p) *n_dofs_p = m->ncell * m->nbp;
  return DG_OK;
}

dg_status dg_mesh_node_coords(const dg_mesh* m, int32_t field, double* xyz, void* stream) {
  if (!m || !xyz || (field != 0 && field != 1)) {
    set_error("dg_mesh_node_coords: bad argument");
    return DG_EINVAL;
  }
  const Tab1D<double>& t = field == 0 ? m->tu64 : m->tp64;
  int n1 = field == 0 ? m->nu : m->np;
  int nb = field == 0 ? m->nbu : m->nbp;
  int d = m->dim;
  std::vector<double> host((size_t)d * m->ncell * nb);
  for (int64_t c = 0; c < m->ncell; ++c) {
    int ci[3] = {(int)(c % m->n[0]), (int)((c / m->n[0]) % m->n[1]),
                 (int)(c / ((int64_t)m->n[0] * m->n[1]))};
    // cell vertices
    double V[8][3];
    for (int b = 0; b < (1 << d); ++b) {
      int L[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) L[a] = ci[a] + ((b >> a) & 1);
      lattice_vertex(m->desc, L, V[b]);
    }
    for (int i = 0; i < nb; ++i) {
      double xi[3] = {t.x[i % n1], t.x[(i / n1) % n1], d == 3 ? t.x[i / (n1 * n1)] : 0.0};
      double X[3] = {0, 0, 0};
      for (int b = 0; b < (1 << d); ++b) {
        double sh = 1.0;
        for (int a = 0; a < d; ++a) sh *= ((b >> a) & 1) ? xi[a] : 1.0 - xi[a];
        for (int a = 0; a < d; ++a) X[a] += sh * V[b][a];
      }
      for (int a = 0; a < d; ++a) host[((size_t)a * m->ncell + c) * nb + i] = X[a];
    }
  }
  cudaStream_t s = as_stream(stream);
  DG_CUDA(cudaMemcpyAsync(xyz, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice, s));
  DG_CUDA(cudaStreamSynchronize(s));
  return DG_OK;
}

}  // extern "C"
