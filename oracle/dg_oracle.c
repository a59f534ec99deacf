/*
 * dg_oracle.c -- plain FP64 CPU oracle for the DG discretisation of
 * Orlando, Della Rocca, Barbante, Bonaventura, Parolini, "An efficient and
 * accurate implicit DG solver for the incompressible Navier-Stokes
 * equations" (arXiv 2107.07776), Section 3.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU
 * baseline of bench.py may load this code.  It shares nothing with the CUDA
 * library: every integral is evaluated by naive quadrature loops over pairs
 * of basis functions on the (tri/bi)linearly mapped cell, with no sum
 * factorisation, no collocation shortcut and no reuse of precomputed 1D
 * operators.  Operators are stored as one dense block per (row cell,
 * neighbour slot) pair and applied by a plain block sparse product.
 *
 * Notation follows the paper: velocity space Q_k (k+1 nodes per direction),
 * pressure space Q_{k-1} (k nodes per direction), nodal Lagrange bases at
 * Gauss-Legendre points, SIP penalty (Eq. penconst1 and the pressure
 * analogue), local Lax-Friedrichs flux (Eq. trilinear).
 *
 * Readings of the paper taken here (the library takes the same ones):
 *  - penalty sigma_{Gamma,K} = (k+1)^2 |Gamma|/|K| (velocity) and
 *    k^2 |Gamma|/|K| (pressure): face measure over cell volume, the 1/h
 *    scaling of the cited Fehn et al. reference; the printed
 *    diam(Gamma)/diam(K) is dimensionless and loses coercivity under
 *    refinement.
 *  - quadrature: Gauss-Legendre with k+1 points per direction for velocity
 *    and mixed forms, k points for pressure-only forms; faces likewise.
 *  - boundary LF speed lambda = |ubar+ . n|, which equals the mirror-state
 *    speed max(|ubar+ . n|, |(2 u_D - ubar+) . n|) whenever u_D . n = 0;
 *    walls are impermeable (the step refuses data with a normal
 *    component), so this is the paper's boundary flux wherever it is used.
 *  - boundary averages are interior traces (Section 3, definition of the
 *    average on boundary faces).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_MAXN 10 /* nodes or quadrature points per direction */
#define ORA_MAXB (ORA_MAXN * ORA_MAXN * ORA_MAXN)

typedef struct {
  int32_t dim;        /* 2 or 3 */
  int32_t n[3];       /* cells per axis (n[2] = 1 in 2D) */
  double lo[3], hi[3];
  int32_t periodic[3];
  int32_t degree;     /* velocity degree k >= 2; pressure degree k-1 */
  int32_t map;        /* 0 Cartesian, 1 tanh-graded, 2 sine-perturbed */
  double map_param[3];/* map 1: beta per axis (0 = uniform); map 2: amplitude in [0] */
  int32_t nq_u;       /* quadrature points per direction, velocity/mixed forms (0: k+1) */
  int32_t nq_p;       /* quadrature points per direction, pressure forms (0: k) */
} ora_mesh;

enum {
  ORA_MASS_U = 0,   /* int phi_j phi_i                                    */
  ORA_SIPG_U = 1,   /* a_u with unit viscosity, Eq. bilin_diff             */
  ORA_ADV_U = 2,    /* c with unit factor, Eq. trilinear                   */
  ORA_MASS_P = 3,   /* int psi_j psi_i                                    */
  ORA_SIPG_P = 4,   /* a_p, Eq. weakform_p_1                               */
  ORA_EXPLVISC_U = 5, /* explicit viscous part of F_u, Eq. rhs1            */
  ORA_EXPLADV_U = 6,  /* explicit advective part of F_u, Eq. rhs1          */
  ORA_GRADDG = 7,   /* int p div v - sum_E {{p}} [[v]], component c, Eq. rhs1 */
  ORA_PROJ = 8,     /* P_ij = int grad psi_j . phi_i, component c          */
  ORA_DIV = 9,      /* int u.grad q - sum_E {{u}}.[[q]], component c, Eq. weakform_p_1 */
  ORA_DIRVISC_U = 10, /* Dirichlet-data viscous terms of F_u (boundary)    */
  ORA_DIRADV_U = 11   /* Dirichlet-data advective terms of F_u (boundary)  */
};

/* ------------------------------------------------------------------ */
/* 1D Gauss-Legendre rule on [0,1]: Newton iteration on P_n(z), with P_n and
 * P_{n-1} from the three-term recurrence (m+1)P_{m+1} = (2m+1) z P_m - m P_{m-1}
 * and P_n'(z) = n (z P_n - P_{n-1}) / (z^2 - 1).  Weights 2/((1-z^2) P_n'^2)
 * on [-1,1], halved on [0,1].  Points ascending. */
int ora_gauss_legendre(int n, double* x, double* w) {
  if (n < 1 || n > ORA_MAXN) return -1;
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    double pn = 0, pn1 = 0, dp = 1;
    for (int it = 0; it < 200; ++it) {
      double pm1 = 1.0, pm = z;
      for (int m = 1; m < n; ++m) {
        double pnext = ((2.0 * m + 1.0) * z * pm - m * pm1) / (m + 1.0);
        pm1 = pm;
        pm = pnext;
      }
      pn = pm;
      pn1 = pm1;
      dp = n * (z * pn - pn1) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    {
      double pm1 = 1.0, pm = z;
      for (int m = 1; m < n; ++m) {
        double pnext = ((2.0 * m + 1.0) * z * pm - m * pm1) / (m + 1.0);
        pm1 = pm;
        pm = pnext;
      }
      dp = n * (z * pm - pm1) / (z * z - 1.0);
    }
    x[n - 1 - i] = 0.5 * (z + 1.0);
    w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
  return 0;
}

/* Lagrange basis on nodes xi[0..n-1], value and derivative at x, written out
 * from the product definition. */
void ora_lagrange(int n, const double* xi, double x, double* val, double* der) {
  for (int j = 0; j < n; ++j) {
    double v = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != j) v *= (x - xi[m]) / (xi[j] - xi[m]);
    val[j] = v;
    double d = 0.0;
    for (int m = 0; m < n; ++m) {
      if (m == j) continue;
      double t = 1.0 / (xi[j] - xi[m]);
      for (int l = 0; l < n; ++l)
        if (l != j && l != m) t *= (x - xi[l]) / (xi[j] - xi[l]);
      d += t;
    }
    der[j] = d;
  }
}

/* ------------------------------------------------------------------ */
/* Mesh geometry.  Vertices of the structured lattice, mapped. */
static void vertex(const ora_mesh* m, const int L[3], double X[3]) {
  double eta[3] = {0, 0, 0};
  for (int a = 0; a < m->dim; ++a) eta[a] = (double)L[a] / (double)m->n[a];
  X[0] = X[1] = X[2] = 0.0;
  for (int a = 0; a < m->dim; ++a) {
    double s = eta[a];
    if (m->map == 1 && m->map_param[a] > 0.0) {
      double b = m->map_param[a];
      s = 0.5 * (1.0 - tanh(b * (1.0 - 2.0 * eta[a])) / tanh(b));
    }
    X[a] = m->lo[a] + (m->hi[a] - m->lo[a]) * s;
  }
  if (m->map == 2) {
    double p = m->map_param[0];
    for (int a = 0; a < m->dim; ++a) p *= sin(2.0 * M_PI * eta[a]);
    for (int a = 0; a < m->dim; ++a) X[a] += p * (m->hi[a] - m->lo[a]);
  }
}

/* Multilinear map of cell C at reference point xi: position x and Jacobian
 * J[r][c] = d x_r / d xi_c. */
static void cell_map(const ora_mesh* m, const int C[3], const double xi[3], double x[3],
                     double J[3][3]) {
  int d = m->dim;
  for (int r = 0; r < 3; ++r) {
    x[r] = 0.0;
    for (int c = 0; c < 3; ++c) J[r][c] = 0.0;
  }
  for (int b = 0; b < (1 << d); ++b) {
    int L[3] = {0, 0, 0};
    double f[3] = {1, 1, 1}, df[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
      int bit = (b >> a) & 1;
      L[a] = C[a] + bit;
      f[a] = bit ? xi[a] : 1.0 - xi[a];
      df[a] = bit ? 1.0 : -1.0;
    }
    double X[3];
    vertex(m, L, X);
    double shape = 1.0;
    for (int a = 0; a < d; ++a) shape *= f[a];
    for (int r = 0; r < d; ++r) x[r] += X[r] * shape;
    for (int c = 0; c < d; ++c) {
      double ds = df[c];
      for (int e = 0; e < d; ++e)
        if (e != c) ds *= f[e];
      for (int r = 0; r < d; ++r) J[r][c] += X[r] * ds;
    }
  }
}

/* determinant and inverse (Jinv[c][r] = d xi_c / d x_r) */
static double invert(int d, double J[3][3], double Jinv[3][3]) {
  double det;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) Jinv[r][c] = 0.0;
  if (d == 2) {
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    Jinv[0][0] = J[1][1] / det;
    Jinv[0][1] = -J[0][1] / det;
    Jinv[1][0] = -J[1][0] / det;
    Jinv[1][1] = J[0][0] / det;
  } else {
    det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
          J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
          J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    Jinv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    Jinv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Jinv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Jinv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    Jinv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Jinv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Jinv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    Jinv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Jinv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  }
  return det;
}

static int64_t ncells(const ora_mesh* m) {
  int64_t N = 1;
  for (int a = 0; a < m->dim; ++a) N *= m->n[a];
  return N;
}

static void cell_coords(const ora_mesh* m, int64_t c, int C[3]) {
  C[0] = C[1] = C[2] = 0;
  for (int a = 0; a < m->dim; ++a) {
    C[a] = (int)(c % m->n[a]);
    c /= m->n[a];
  }
}

static int64_t cell_index(const ora_mesh* m, const int C[3]) {
  int64_t c = 0;
  for (int a = m->dim - 1; a >= 0; --a) c = c * m->n[a] + C[a];
  return c;
}

/* Neighbour across face (a, s) (s = 0: low side, 1: high side); -1 at a wall. */
static int64_t neighbour(const ora_mesh* m, const int C[3], int a, int s) {
  int N[3] = {C[0], C[1], C[2]};
  N[a] += s ? 1 : -1;
  if (N[a] < 0 || N[a] >= m->n[a]) {
    if (!m->periodic[a]) return -1;
    N[a] = (N[a] + m->n[a]) % m->n[a];
  }
  return cell_index(m, N);
}

/* Tensor-product nodal basis with n1 nodes per direction: values and
 * physical gradients (J^{-T} times the reference gradient) at xi. */
typedef struct {
  int n1, nb;
  double nodes[ORA_MAXN];
  double val[ORA_MAXB];
  double grad[ORA_MAXB][3];
} basis_eval;

static void eval_basis(basis_eval* B, int d, const double xi[3], double Jinv[3][3]) {
  double v1[3][ORA_MAXN], d1[3][ORA_MAXN];
  for (int a = 0; a < 3; ++a)
    for (int j = 0; j < ORA_MAXN; ++j) {
      v1[a][j] = 1.0;
      d1[a][j] = 0.0;
    }
  for (int a = 0; a < d; ++a) ora_lagrange(B->n1, B->nodes, xi[a], v1[a], d1[a]);
  int n1 = B->n1;
  int nz = d == 3 ? n1 : 1;
  for (int i2 = 0; i2 < nz; ++i2)
    for (int i1 = 0; i1 < n1; ++i1)
      for (int i0 = 0; i0 < n1; ++i0) {
        int i = i0 + n1 * (i1 + n1 * i2);
        double gr[3];
        B->val[i] = v1[0][i0] * v1[1][i1] * (d == 3 ? v1[2][i2] : 1.0);
        gr[0] = d1[0][i0] * v1[1][i1] * (d == 3 ? v1[2][i2] : 1.0);
        gr[1] = v1[0][i0] * d1[1][i1] * (d == 3 ? v1[2][i2] : 1.0);
        gr[2] = d == 3 ? v1[0][i0] * v1[1][i1] * d1[2][i2] : 0.0;
        for (int r = 0; r < 3; ++r) {
          double g = 0.0;
          for (int c = 0; c < d; ++c) g += Jinv[c][r] * gr[c];
          B->grad[i][r] = r < d ? g : 0.0;
        }
      }
}

static int ipow(int b, int e) {
  int r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

/* Cell volume |K| and face measures |Gamma_f| (f = 2a + s) by quadrature. */
static void cell_measures(const ora_mesh* m, const int C[3], double* volK, double area[6]) {
  int d = m->dim;
  int nq = m->degree + 2;
  double gx[ORA_MAXN], gw[ORA_MAXN];
  ora_gauss_legendre(nq, gx, gw);
  double vol = 0.0;
  int nqd = ipow(nq, d);
  for (int q = 0; q < nqd; ++q) {
    double xi[3] = {0, 0, 0}, w = 1.0;
    int t = q;
    for (int a = 0; a < d; ++a) {
      xi[a] = gx[t % nq];
      w *= gw[t % nq];
      t /= nq;
    }
    double x[3], J[3][3], Ji[3][3];
    cell_map(m, C, xi, x, J);
    vol += w * invert(d, J, Ji);
  }
  *volK = vol;
  for (int f = 0; f < 2 * d; ++f) {
    int a = f / 2, s = f % 2;
    double A = 0.0;
    int nqf = ipow(nq, d - 1);
    for (int q = 0; q < nqf; ++q) {
      double xi[3] = {0, 0, 0}, w = 1.0;
      int t = q;
      for (int b = 0; b < d; ++b) {
        if (b == a) continue;
        xi[b] = gx[t % nq];
        w *= gw[t % nq];
        t /= nq;
      }
      xi[a] = s;
      double x[3], J[3][3], Ji[3][3];
      cell_map(m, C, xi, x, J);
      double det = invert(d, J, Ji);
      double nn = 0.0;
      for (int r = 0; r < d; ++r) nn += (det * Ji[a][r]) * (det * Ji[a][r]);
      A += w * sqrt(nn);
    }
    area[f] = A;
  }
}

/* Field value of a d-component nodal velocity field F ([comp][cell][node]) in
 * cell c at a point, from the basis values held in B. */
static void field_at(const ora_mesh* m, const basis_eval* B, const double* F, int64_t c,
                     double out[3]) {
  int64_t N = ncells(m);
  for (int r = 0; r < 3; ++r) out[r] = 0.0;
  for (int r = 0; r < m->dim; ++r) {
    const double* Fr = F + (int64_t)r * N * B->nb + c * B->nb;
    double s = 0.0;
    for (int j = 0; j < B->nb; ++j) s += Fr[j] * B->val[j];
    out[r] = s;
  }
}

int ora_sizes(const ora_mesh* m, int64_t* n_cells, int32_t* nb_u, int32_t* nb_p) {
  *n_cells = ncells(m);
  *nb_u = ipow(m->degree + 1, m->dim);
  *nb_p = ipow(m->degree, m->dim);
  return 0;
}

/*
 * Assemble the rows of one operator for the selected cells (cells == NULL:
 * all cells in order).  Output blocks[sel][slot][i][j] with slot 0 = the row
 * cell, slot 1 + 2a + s = the neighbour across face (a, s); cols[sel][slot] =
 * column cell or -1.  `field` is the advecting velocity for ADV_U, DIRADV_U
 * (ubar) and EXPLADV_U (wbar), layout [comp][cell][node]; `comp` selects the
 * velocity component for GRADDG, PROJ, DIV.
 *
 * Face terms are assembled cell by cell with n the outward normal of the
 * row cell K: [u] = u_K - u_nb, {{g}} = (g_K + g_nb)/2, and the test
 * function lives on K only, which restricts the symmetric definitions of the
 * jump and average of Section 3 to the rows of K.
 */
int ora_assemble(const ora_mesh* m, int kind, const double* field, int comp, int64_t nsel,
                 const int64_t* cells, double* blocks, int64_t* cols) {
  const int d = m->dim, k = m->degree;
  const int nslot = 2 * d + 1;
  const int nq_u = m->nq_u > 0 ? m->nq_u : k + 1;
  const int nq_p = m->nq_p > 0 ? m->nq_p : k;
  int test_p = 0, trial_p = 0, nq = nq_u;
  switch (kind) {
    case ORA_MASS_P:
    case ORA_SIPG_P:
      test_p = trial_p = 1;
      nq = nq_p;
      break;
    case ORA_GRADDG:
    case ORA_PROJ:
      trial_p = 1;
      break;
    case ORA_DIV:
      test_p = 1;
      break;
    default:
      break;
  }
  if (kind < 0 || kind > 11) return -1;
  if (k + 1 > ORA_MAXN || nq > ORA_MAXN) return -2;
  const int nt = ipow(test_p ? k : k + 1, d);
  const int ns = ipow(trial_p ? k : k + 1, d);
  const double pen = test_p && trial_p ? (double)k * k : (double)(k + 1) * (k + 1);
  double qx[ORA_MAXN], qw[ORA_MAXN], nu_x[ORA_MAXN], nu_w[ORA_MAXN], np_x[ORA_MAXN],
      np_w[ORA_MAXN];
  ora_gauss_legendre(nq, qx, qw);
  ora_gauss_legendre(k + 1, nu_x, nu_w);
  ora_gauss_legendre(k, np_x, np_w);
  const int64_t N = ncells(m);
  const int64_t ncount = cells ? nsel : N;
  int err = 0;

#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t sidx = 0; sidx < ncount; ++sidx) {
    int64_t c = cells ? cells[sidx] : sidx;
    if (c < 0 || c >= N) {
      err = -3;
      continue;
    }
    int C[3];
    cell_coords(m, c, C);
    double* blk = blocks + sidx * nslot * (int64_t)nt * ns;
    int64_t* col = cols + sidx * nslot;
    memset(blk, 0, sizeof(double) * nslot * (size_t)nt * ns);
    col[0] = c;
    for (int f = 0; f < 2 * d; ++f) col[1 + f] = neighbour(m, C, f / 2, f % 2);

    /* basis evaluators: test, trial and velocity (for advecting fields) on the
     * row cell; trial and velocity on the neighbour */
    basis_eval *Bt = malloc(sizeof(basis_eval)), *Bs = malloc(sizeof(basis_eval)),
               *Bu = malloc(sizeof(basis_eval)), *Bs2 = malloc(sizeof(basis_eval)),
               *Bu2 = malloc(sizeof(basis_eval));
    Bt->n1 = test_p ? k : k + 1;
    Bs->n1 = Bs2->n1 = trial_p ? k : k + 1;
    Bu->n1 = Bu2->n1 = k + 1;
    for (int j = 0; j < ORA_MAXN; ++j) {
      Bt->nodes[j] = test_p ? np_x[j] : nu_x[j];
      Bs->nodes[j] = Bs2->nodes[j] = trial_p ? np_x[j] : nu_x[j];
      Bu->nodes[j] = Bu2->nodes[j] = nu_x[j];
    }
    Bt->nb = nt;
    Bs->nb = Bs2->nb = ns;
    Bu->nb = Bu2->nb = ipow(k + 1, d);

    double volK, areaK[6];
    cell_measures(m, C, &volK, areaK);

    /* ---- cell integrals ---- */
    int nqd = ipow(nq, d);
    for (int q = 0; q < nqd; ++q) {
      double xi[3] = {0, 0, 0}, w = 1.0;
      int t = q;
      for (int a = 0; a < d; ++a) {
        xi[a] = qx[t % nq];
        w *= qw[t % nq];
        t /= nq;
      }
      double x[3], J[3][3], Ji[3][3];
      cell_map(m, C, xi, x, J);
      double det = invert(d, J, Ji);
      double dw = w * det;
      eval_basis(Bt, d, xi, Ji);
      eval_basis(Bs, d, xi, Ji);
      double fb[3] = {0, 0, 0};
      if (kind == ORA_ADV_U || kind == ORA_EXPLADV_U) {
        eval_basis(Bu, d, xi, Ji);
        field_at(m, Bu, field, c, fb);
      }
      for (int i = 0; i < nt; ++i)
        for (int j = 0; j < ns; ++j) {
          double v = 0.0;
          const double *gi = Bt->grad[i], *gj = Bs->grad[j];
          double gg = gi[0] * gj[0] + gi[1] * gj[1] + gi[2] * gj[2];
          double fgi = fb[0] * gi[0] + fb[1] * gi[1] + fb[2] * gi[2];
          switch (kind) {
            case ORA_MASS_U:
            case ORA_MASS_P: v = Bt->val[i] * Bs->val[j]; break;
            case ORA_SIPG_U:
            case ORA_SIPG_P: v = gg; break;
            case ORA_ADV_U: v = -Bs->val[j] * fgi; break;
            case ORA_EXPLVISC_U: v = -gg; break;
            case ORA_EXPLADV_U: v = Bs->val[j] * fgi; break;
            case ORA_GRADDG: v = Bs->val[j] * gi[comp]; break;
            case ORA_PROJ: v = gj[comp] * Bt->val[i]; break;
            case ORA_DIV: v = Bs->val[j] * gi[comp]; break;
            default: v = 0.0;
          }
          blk[(int64_t)i * ns + j] += dw * v;
        }
    }

    /* ---- face integrals ---- */
    if (kind != ORA_MASS_U && kind != ORA_MASS_P && kind != ORA_PROJ) {
      for (int f = 0; f < 2 * d; ++f) {
        int a = f / 2, s = f % 2;
        int64_t nb = col[1 + f];
        int interior = nb >= 0;
        if (!interior && kind == ORA_SIPG_P) continue; /* Neumann: no boundary terms */
        if (interior && (kind == ORA_DIRVISC_U || kind == ORA_DIRADV_U)) continue;
        int Cn[3];
        if (interior) cell_coords(m, nb, Cn);
        double sig_in = pen * areaK[f] / volK, sig_nb = 0.0;
        if (interior) {
          double volN, areaN[6];
          cell_measures(m, Cn, &volN, areaN);
          sig_nb = pen * areaN[2 * a + (1 - s)] / volN;
        }
        double Cpen = interior ? 0.5 * (sig_in + sig_nb) : sig_in;
        double* bself = blk;
        double* bnb = blk + (int64_t)(1 + f) * nt * ns;
        int nqf = ipow(nq, d - 1);
        for (int q = 0; q < nqf; ++q) {
          double xi[3] = {0, 0, 0}, w = 1.0;
          int t = q;
          for (int b = 0; b < d; ++b) {
            if (b == a) continue;
            xi[b] = qx[t % nq];
            w *= qw[t % nq];
            t /= nq;
          }
          xi[a] = s;
          double x[3], J[3][3], Ji[3][3];
          cell_map(m, C, xi, x, J);
          double det = invert(d, J, Ji);
          double nv[3] = {0, 0, 0}, nn = 0.0;
          for (int r = 0; r < d; ++r) {
            nv[r] = det * (s ? 1.0 : -1.0) * Ji[a][r];
            nn += nv[r] * nv[r];
          }
          nn = sqrt(nn);
          for (int r = 0; r < d; ++r) nv[r] /= nn;
          double dS = w * nn;
          eval_basis(Bt, d, xi, Ji);
          eval_basis(Bs, d, xi, Ji);
          double ub_in[3] = {0, 0, 0}, ub_nb[3] = {0, 0, 0};
          int need_field = kind == ORA_ADV_U || kind == ORA_EXPLADV_U || kind == ORA_DIRADV_U;
          if (need_field) {
            eval_basis(Bu, d, xi, Ji);
            field_at(m, Bu, field, c, ub_in);
          }
          if (interior) {
            double xin[3] = {xi[0], xi[1], xi[2]};
            xin[a] = 1 - s;
            double xn[3], Jn[3][3], Jin[3][3];
            cell_map(m, Cn, xin, xn, Jn);
            invert(d, Jn, Jin);
            eval_basis(Bs2, d, xin, Jin);
            if (need_field) {
              eval_basis(Bu2, d, xin, Jin);
              field_at(m, Bu2, field, nb, ub_nb);
            }
          }
          double un_in = ub_in[0] * nv[0] + ub_in[1] * nv[1] + ub_in[2] * nv[2];
          double un_nb = ub_nb[0] * nv[0] + ub_nb[1] * nv[1] + ub_nb[2] * nv[2];
          double lam = interior ? fmax(fabs(un_in), fabs(un_nb)) : fabs(un_in);
          for (int i = 0; i < nt; ++i) {
            double vi = Bt->val[i];
            double dni = Bt->grad[i][0] * nv[0] + Bt->grad[i][1] * nv[1] + Bt->grad[i][2] * nv[2];
            double ni_c = vi * nv[comp];
            for (int j = 0; j < ns; ++j) {
              /* trial on the row cell */
              double uj = Bs->val[j];
              double dnj = Bs->grad[j][0] * nv[0] + Bs->grad[j][1] * nv[1] + Bs->grad[j][2] * nv[2];
              double v = 0.0;
              if (interior) {
                switch (kind) {
                  case ORA_SIPG_U:
                  case ORA_SIPG_P:
                    v = -0.5 * dnj * vi - uj * 0.5 * dni + Cpen * uj * vi;
                    break;
                  case ORA_ADV_U: v = 0.5 * uj * un_in * vi + 0.5 * lam * uj * vi; break;
                  case ORA_EXPLVISC_U: v = 0.5 * dnj * vi; break;
                  case ORA_EXPLADV_U: v = -0.5 * uj * un_in * vi; break;
                  case ORA_GRADDG: v = -0.5 * uj * ni_c; break;
                  case ORA_DIV: v = -0.5 * uj * ni_c; break;
                  default: v = 0.0;
                }
              } else {
                switch (kind) {
                  case ORA_SIPG_U: v = -dnj * vi - uj * dni + 2.0 * Cpen * uj * vi; break;
                  case ORA_ADV_U: v = lam * uj * vi; break;
                  case ORA_EXPLVISC_U: v = dnj * vi; break;
                  case ORA_EXPLADV_U: v = -uj * un_in * vi; break;
                  case ORA_GRADDG: v = -uj * ni_c; break;
                  case ORA_DIV: v = -uj * ni_c; break;
                  case ORA_DIRVISC_U: v = -uj * dni + 2.0 * Cpen * uj * vi; break;
                  case ORA_DIRADV_U: v = -uj * un_in * vi + lam * uj * vi; break;
                  default: v = 0.0;
                }
              }
              bself[(int64_t)i * ns + j] += dS * v;
              if (!interior) continue;
              /* trial on the neighbour: jump [u] = -u_nb, average halves */
              double uo = Bs2->val[j];
              double dno =
                  Bs2->grad[j][0] * nv[0] + Bs2->grad[j][1] * nv[1] + Bs2->grad[j][2] * nv[2];
              double vo = 0.0;
              switch (kind) {
                case ORA_SIPG_U:
                case ORA_SIPG_P:
                  vo = -0.5 * dno * vi + uo * 0.5 * dni - Cpen * uo * vi;
                  break;
                case ORA_ADV_U: vo = 0.5 * uo * un_nb * vi - 0.5 * lam * uo * vi; break;
                case ORA_EXPLVISC_U: vo = 0.5 * dno * vi; break;
                case ORA_EXPLADV_U: vo = -0.5 * uo * un_nb * vi; break;
                case ORA_GRADDG: vo = -0.5 * uo * ni_c; break;
                case ORA_DIV: vo = -0.5 * uo * ni_c; break;
                default: vo = 0.0;
              }
              bnb[(int64_t)i * ns + j] += dS * vo;
            }
          }
        }
      }
    }
    free(Bt);
    free(Bs);
    free(Bu);
    free(Bs2);
    free(Bu2);
  }
  return err;
}

/* y[row cell][i] = sum_slot sum_j blocks[sel][slot][i][j] x[cols[sel][slot]][j] */
int ora_block_apply(int64_t nsel, int nslot, int nt, int ns, const double* blocks,
                    const int64_t* cols, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < nsel; ++r) {
    double acc[ORA_MAXB];
    for (int i = 0; i < nt; ++i) acc[i] = 0.0;
    for (int sl = 0; sl < nslot; ++sl) {
      int64_t cc = cols[r * nslot + sl];
      if (cc < 0) continue;
      const double* B = blocks + (r * nslot + sl) * (int64_t)nt * ns;
      const double* xc = x + cc * ns;
      for (int i = 0; i < nt; ++i) {
        double s = 0.0;
        for (int j = 0; j < ns; ++j) s += B[(int64_t)i * ns + j] * xc[j];
        acc[i] += s;
      }
    }
    for (int i = 0; i < nt; ++i) y[r * nt + i] = acc[i];
  }
  return 0;
}

/* Physical coordinates of the nodes of a space (p_space: 0 velocity, 1
 * pressure), layout [dim][cell][node]. */
int ora_node_coords(const ora_mesh* m, int p_space, double* xyz) {
  int d = m->dim, k = m->degree;
  int n1 = p_space ? k : k + 1;
  double gx[ORA_MAXN], gw[ORA_MAXN];
  ora_gauss_legendre(n1, gx, gw);
  int nb = ipow(n1, d);
  int64_t N = ncells(m);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < N; ++c) {
    int C[3];
    cell_coords(m, c, C);
    for (int i = 0; i < nb; ++i) {
      double xi[3] = {0, 0, 0};
      int t = i;
      for (int a = 0; a < d; ++a) {
        xi[a] = gx[t % n1];
        t /= n1;
      }
      double x[3], J[3][3];
      cell_map(m, C, xi, x, J);
      for (int a = 0; a < d; ++a) xyz[((int64_t)a * N + c) * nb + i] = x[a];
    }
  }
  return 0;
}

/* Values and physical gradients of a scalar nodal field ([cell][node] of
 * space p_space) at an nq-point Gauss-Legendre rule per cell, with the
 * points' coordinates and weights times det J: used for error norms. */
int ora_eval_qp(const ora_mesh* m, int p_space, int nq, const double* vec, double* xyz,
                double* wdet, double* val, double* grad) {
  int d = m->dim, k = m->degree;
  int n1 = p_space ? k : k + 1;
  if (nq > ORA_MAXN) return -2;
  double gx[ORA_MAXN], gw[ORA_MAXN], nx[ORA_MAXN], nw[ORA_MAXN];
  ora_gauss_legendre(nq, gx, gw);
  ora_gauss_legendre(n1, nx, nw);
  int nb = ipow(n1, d), nqd = ipow(nq, d);
  int64_t N = ncells(m);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < N; ++c) {
    int C[3];
    cell_coords(m, c, C);
    basis_eval* B = malloc(sizeof(basis_eval));
    B->n1 = n1;
    B->nb = nb;
    for (int j = 0; j < ORA_MAXN; ++j) B->nodes[j] = nx[j];
    for (int q = 0; q < nqd; ++q) {
      double xi[3] = {0, 0, 0}, w = 1.0;
      int t = q;
      for (int a = 0; a < d; ++a) {
        xi[a] = gx[t % nq];
        w *= gw[t % nq];
        t /= nq;
      }
      double x[3], J[3][3], Ji[3][3];
      cell_map(m, C, xi, x, J);
      double det = invert(d, J, Ji);
      eval_basis(B, d, xi, Ji);
      int64_t o = c * nqd + q;
      double v = 0.0, g[3] = {0, 0, 0};
      for (int j = 0; j < nb; ++j) {
        double u = vec[c * nb + j];
        v += u * B->val[j];
        for (int r = 0; r < 3; ++r) g[r] += u * B->grad[j][r];
      }
      wdet[o] = w * det;
      val[o] = v;
      for (int a = 0; a < d; ++a) {
        xyz[(int64_t)a * N * nqd + o] = x[a];
        grad[(int64_t)a * N * nqd + o] = g[a];
      }
    }
    free(B);
  }
  return 0;
}

int ora_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
