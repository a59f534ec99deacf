// Stage right-hand sides, gradient projection and Jacobi diagonals on
// trilinear cells: the general-geometry counterparts of dg_rhs.cu, with the
// per-point metric terms of dg_geom.cuh.  Same forms (Sections 2-3): explicit
// unpenalised viscous and central advective terms of F_u, Dirichlet data
// terms, the DG pressure gradient (with mass and forcing), the divergence
// functional F_p, u~ = M^-1 P p (M diagonal: collocated nodal basis), and the
// diagonals of mass M + visc A + adv C(ubar) and alpha M^p + K.
//
// One thread per node, CPB cells per CTA, neighbour traces from global
// memory, every output written once (deterministic).  Storage FP64,
// arithmetic A = df64 (float-float) or double (dg_mesh_set_fp64_arith).
#include "dg_apply_kernel.cuh"
#include "dg_geom.cuh"

namespace dg {

namespace {

struct GG {
  int64_t ncell;
  int n[3];
  int per[3];
  const double* gvu;   // velocity volume terms
  const double* gfu;   // velocity face terms
  const double* gvp;   // pressure volume terms
  const double* gfp;   // pressure face terms
  const double* gpen;  // penalty geometry per cell face
};

GG make_gg(const dg_mesh* m) {
  GG g;
  g.ncell = m->ncell;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = m->n[a];
    g.per[a] = m->periodic[a];
  }
  g.gvu = m->gvu64;
  g.gfu = m->gfu64;
  g.gvp = m->gvp64;
  g.gfp = m->gfp64;
  g.gpen = m->gpen64;
  return g;
}

__device__ __forceinline__ void coords(const GG& g, int64_t cell, int ci[3]) {
  lex_coords(cell, g.n[0], g.n[1], ci);
}

__device__ __forceinline__ int64_t nbr(const GG& g, const int ci[3], int a, int s) {
  int nc[3] = {ci[0], ci[1], ci[2]};
  nc[a] += s ? 1 : -1;
  if (nc[a] < 0 || nc[a] >= g.n[a]) {
    if (!g.per[a]) return -1;
    nc[a] = (nc[a] + g.n[a]) % g.n[a];
  }
  return (int64_t)nc[0] + (int64_t)g.n[0] * (nc[1] + (int64_t)g.n[1] * nc[2]);
}

template <int N, int DIM>
constexpr int rhs_cpb() {
  return Shape<N, DIM>::NB <= 8 ? 16 : (Shape<N, DIM>::NB <= 27 ? 4 : (Shape<N, DIM>::NB <= 64 ? 2 : 1));
}

template <typename A>
const Tab1D<A>& tabu(const dg_mesh* m);
template <>
const Tab1D<double>& tabu<double>(const dg_mesh* m) { return m->tu64; }
template <>
const Tab1D<df64>& tabu<df64>(const dg_mesh* m) { return m->tudf; }
template <typename A>
const Tab1D<A>& tabp(const dg_mesh* m);
template <>
const Tab1D<double>& tabp<double>(const dg_mesh* m) { return m->tp64; }
template <>
const Tab1D<df64>& tabp<df64>(const dg_mesh* m) { return m->tpdf; }
template <typename A>
const MixTab<A>& tabmix(const dg_mesh* m);
template <>
const MixTab<double>& tabmix<double>(const dg_mesh* m) { return m->mix64; }
template <>
const MixTab<df64>& tabmix<df64>(const dg_mesh* m) { return m->mixdf; }

// ------------------------------------------------------------------
// Explicit terms: MODE 0 adds visc E_v w + adv E_a(wb) w (all faces, central,
// unpenalised); MODE 1 adds the Dirichlet data terms on wall faces
// (w = u_D, wb = the advecting field).
template <typename A, int DIM, int N, int MODE, int CPB>
__global__ void __launch_bounds__(((CPB * Shape<N, DIM>::NB + 31) / 32) * 32)
    gen_explicit_kernel(const __grid_constant__ GG g, const __grid_constant__ Tab1D<A> tb,
                        double visc_d, double adv_d, double pen_d, const double* __restrict__ w,
                        const double* __restrict__ wb, double* __restrict__ rhs) {
  pdl_entry();
  using Ar = Arith<A>;
  using GC = GeomCount<DIM>;
  constexpr int NB = Shape<N, DIM>::NB, NF = Shape<N, DIM>::NF, NFP = Shape<N, DIM>::NFP;
  constexpr int NG = GC::NG, NV = GC::NVU, NFF = GC::NFU;
  __shared__ A s_u[CPB][NB];
  __shared__ A s_wb[DIM][CPB][NB];
  __shared__ A s_q[DIM][CPB][NB];
  __shared__ A s_t[CPB][NFP][2];
  __shared__ A s_dn[CPB][NFP][2];
  __shared__ A s_wn[CPB][NFP][2];
  __shared__ A s_f[CPB][NFP][2];
  __shared__ A s_Q[CPB][NFP][DIM - 1];
  const int tid = threadIdx.x, cl = tid / NB, node = tid % NB;
  const int64_t cell = (int64_t)blockIdx.x * CPB + cl;
  const bool active = cl < CPB && cell < g.ncell;
  const A zero = Ar::c(0.0), half = Ar::c(0.5), two = Ar::c(2.0);
  const A visc = Ar::from(visc_d), adv = Ar::from(adv_d), pen = Ar::from(pen_d);
  int ci[3] = {0, 0, 0};
  const int ii[3] = {node % N, (node / N) % N, DIM == 3 ? node / (N * N) : 0};
  A Gm[NG], wt[DIM];
  for (int f = 0; f < NG; ++f) Gm[f] = zero;
  for (int b = 0; b < DIM; ++b) wt[b] = zero;
  if (active) {
    coords(g, cell, ci);
    const double* gv = g.gvu + cell * (int64_t)NV * NB + node;
    for (int f = 0; f < NG; ++f) Gm[f] = Ar::from(gv[f * NB]);
    A wbn[DIM];
    for (int r = 0; r < DIM; ++r) {
      wbn[r] = Ar::from(wb[((int64_t)r * g.ncell + cell) * NB + node]);
      s_wb[r][cl][node] = wbn[r];
    }
    for (int b = 0; b < DIM; ++b) {
      A acc = zero;
      for (int r = 0; r < DIM; ++r) acc += Ar::from(gv[(NG + 1 + b * DIM + r) * NB]) * wbn[r];
      wt[b] = acc;
    }
  }
  __syncthreads();
  if (active) {  // wb.n at the face points (both sides), shared by the components
    for (int fp = node; fp < NFP; fp += NB) {
      const int f = fp / NF, t = fp % NF, ax = f >> 1, s = f & 1;
      const int64_t nb = nbr(g, ci, ax, s);
      const double* gfp = g.gfu + ((cell * 2 * DIM + f) * (int64_t)NFF) * NF + t;
      A wi = zero, wo = zero;
      for (int r = 0; r < DIM; ++r) {
        const A nr = Ar::from(gfp[(1 + r) * NF]);
        A a_in = zero, a_out = zero;
        for (int i = 0; i < N; ++i) {
          const int nd = node_of(N, ax, i, t, DIM);
          a_in = Ar::fma(tb.L[s][i], s_wb[r][cl][nd], a_in);
          if (MODE == 0 && nb >= 0)
            a_out = Ar::fma(tb.L[1 - s][i], Ar::from(__ldg(&wb[((int64_t)r * g.ncell + nb) * NB + nd])), a_out);
        }
        wi += nr * a_in;
        wo += nr * a_out;
      }
      s_wn[cl][fp][0] = wi;
      s_wn[cl][fp][1] = wo;
    }
  }
  for (int c = 0; c < DIM; ++c) {
    const double* wc = w + (int64_t)c * g.ncell * NB;
    if (active) s_u[cl][node] = Ar::from(wc[cell * NB + node]);
    __syncthreads();
    if (active) {
      if (MODE == 0) {
        A gr[DIM];
        for (int b = 0; b < DIM; ++b) {
          A du = zero;
          for (int m = 0; m < N; ++m) {
            int j[3] = {ii[0], ii[1], ii[2]};
            j[b] = m;
            du += tb.D[ii[b]][m] * s_u[cl][j[0] + N * (j[1] + N * j[2])];
          }
          gr[b] = du;
        }
        for (int b = 0; b < DIM; ++b) {
          A q = zero;
          for (int e = 0; e < DIM; ++e) q += Gm[sym_index(DIM, b, e)] * gr[e];
          s_q[b][cl][node] = adv * s_u[cl][node] * wt[b] - visc * q;
        }
      }
      for (int fp = node; fp < NFP; fp += NB) {
        const int f = fp / NF, t = fp % NF, ax = f >> 1, s = f & 1;
        const int64_t nb = nbr(g, ci, ax, s);
        A uin = zero, dnin = zero, uout = zero, dnout = zero;
        for (int i = 0; i < N; ++i) {
          const A v = s_u[cl][node_of(N, ax, i, t, DIM)];
          uin = Ar::fma(tb.L[s][i], v, uin);
          dnin = Ar::fma(tb.dL[s][i], v, dnin);
        }
        if (MODE == 0 && nb >= 0) {
          for (int i = 0; i < N; ++i) {
            const A v = Ar::from(__ldg(&wc[nb * NB + node_of(N, ax, i, t, DIM)]));
            uout = Ar::fma(tb.L[1 - s][i], v, uout);
            dnout = Ar::fma(tb.dL[1 - s][i], v, dnout);
          }
        }
        s_t[cl][fp][0] = uin;
        s_t[cl][fp][1] = uout;
        s_dn[cl][fp][0] = dnin;
        s_dn[cl][fp][1] = dnout;
      }
    }
    __syncthreads();
    if (active) {
      for (int fp = node; fp < NFP; fp += NB) {
        const int f = fp / NF, t = fp % NF, ax = f >> 1, s = f & 1;
        const int64_t nb = nbr(g, ci, ax, s);
        const double* gfp = g.gfu + ((cell * 2 * DIM + f) * (int64_t)NFF) * NF + t;
        const A dS = Ar::from(gfp[0]);
        A cown[DIM], cnb[DIM];
        for (int b = 0; b < DIM; ++b) {
          cown[b] = Ar::from(gfp[(1 + DIM + b) * NF]);
          cnb[b] = Ar::from(gfp[(1 + 2 * DIM + b) * NF]);
        }
        const A uin = s_t[cl][fp][0], uout = s_t[cl][fp][1];
        const A wnin = s_wn[cl][fp][0], wnout = s_wn[cl][fp][1];
        A fv = zero, fg = zero;
        if (MODE == 0) {
          A dn_in = cown[ax] * s_dn[cl][fp][0], dn_out = cnb[ax] * s_dn[cl][fp][1];
          int stride = 1;
          for (int b = 0; b < DIM; ++b) {
            if (b == ax) continue;
            const int tb_ = (t / stride) % N;
            A gi = zero, go = zero;
            for (int m = 0; m < N; ++m) {
              const int q = f * NF + t + (m - tb_) * stride;
              gi = Ar::fma(tb.D[tb_][m], s_t[cl][q][0], gi);
              go = Ar::fma(tb.D[tb_][m], s_t[cl][q][1], go);
            }
            dn_in += cown[b] * gi;
            dn_out += cnb[b] * go;
            stride *= N;
          }
          if (nb >= 0) fv = half * (visc * (dn_in + dn_out) - adv * (uin * wnin + uout * wnout));
          else fv = visc * dn_in - adv * uin * wnin;
        } else if (nb < 0) {
          const A sig = pen * Ar::from(g.gpen[cell * 2 * DIM + f]);
          fv = visc * two * sig * uin + adv * (Ar::abs(wnin) * uin - uin * wnin);
          fg = -(visc * uin);
        }
        const A wg = dS * fg;
        s_f[cl][fp][0] = dS * fv;
        s_f[cl][fp][1] = wg * cown[ax];
        int e = 0;
        for (int b = 0; b < DIM; ++b) {
          if (b == ax) continue;
          s_Q[cl][fp][e++] = wg * cown[b];
        }
      }
    }
    __syncthreads();
    if (active) {
      A y = zero;
      if (MODE == 0) {
        for (int b = 0; b < DIM; ++b)
          for (int m = 0; m < N; ++m) {
            int j[3] = {ii[0], ii[1], ii[2]};
            j[b] = m;
            y += tb.D[m][ii[b]] * s_q[b][cl][j[0] + N * (j[1] + N * j[2])];
          }
      }
      for (int b = 0; b < DIM; ++b) {
        const int t = tang_of<N, DIM>(b, ii);
        for (int s = 0; s < 2; ++s) {
          const int f = 2 * b + s, fp = f * NF + t;
          A R = zero;
          int stride = 1, e = 0;
          for (int g2 = 0; g2 < DIM; ++g2) {
            if (g2 == b) continue;
            const int tg = ii[g2];
            for (int m = 0; m < N; ++m) R += tb.D[m][tg] * s_Q[cl][f * NF + t + (m - tg) * stride][e];
            stride *= N;
            ++e;
          }
          y += (s_f[cl][fp][0] + R) * tb.L[s][ii[b]] + s_f[cl][fp][1] * tb.dL[s][ii[b]];
        }
      }
      rhs[(int64_t)c * g.ncell * NB + cell * NB + node] += Ar::to_d(y);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------
// rhs = mass M u_mass + M f + G p (the DG pressure gradient of Eq. rhs1);
// writes (does not accumulate).
template <typename A, int DIM, int N, int NP, int CPB>
__global__ void __launch_bounds__(((CPB * Shape<N, DIM>::NB + 31) / 32) * 32)
    gen_mass_grad_kernel(const __grid_constant__ GG g, const __grid_constant__ Tab1D<A> tb,
                         const __grid_constant__ Tab1D<A> tp, const __grid_constant__ MixTab<A> mx,
                         double mass_d, const double* __restrict__ u_mass,
                         const double* __restrict__ f, const double* __restrict__ p,
                         double* __restrict__ rhs) {
  pdl_entry();
  using Ar = Arith<A>;
  using GC = GeomCount<DIM>;
  constexpr int NB = Shape<N, DIM>::NB, NF = Shape<N, DIM>::NF, NFP = Shape<N, DIM>::NFP;
  constexpr int NBP = Shape<NP, DIM>::NB;
  constexpr int NG = GC::NG, NV = GC::NVU, NFF = GC::NFU;
  __shared__ A s_p[CPB][NBP];
  __shared__ A s_pu[CPB][NB];
  __shared__ A s_q[DIM][CPB][NB];
  __shared__ A s_f[CPB][NFP];
  const int tid = threadIdx.x, cl = tid / NB, node = tid % NB;
  const int64_t cell = (int64_t)blockIdx.x * CPB + cl;
  const bool active = cl < CPB && cell < g.ncell;
  const A zero = Ar::c(0.0), half = Ar::c(0.5), mass = Ar::from(mass_d);
  int ci[3] = {0, 0, 0};
  const int ii[3] = {node % N, (node / N) % N, DIM == 3 ? node / (N * N) : 0};
  const double* gv = g.gvu + cell * (int64_t)NV * NB + node;
  A W = zero;
  if (active) {
    coords(g, cell, ci);
    W = Ar::from(gv[NG * NB]);
    if (p && node < NBP) s_p[cl][node] = Ar::from(p[cell * NBP + node]);
  }
  __syncthreads();
  if (active && p) {  // p at the velocity nodes (exact: Q_{k-1} lies in Q_k)
    A pu = zero;
    for (int j = 0; j < NBP; ++j) {
      const int j0 = j % NP, j1 = (j / NP) % NP, j2 = DIM == 3 ? j / (NP * NP) : 0;
      A wgt = mx.I[ii[0]][j0] * mx.I[ii[1]][j1];
      if (DIM == 3) wgt = wgt * mx.I[ii[2]][j2];
      pu = Ar::fma(wgt, s_p[cl][j], pu);
    }
    s_pu[cl][node] = pu;
  }
  __syncthreads();
  if (active && p) {  // {{p}} dS at the face points
    for (int fp = node; fp < NFP; fp += NB) {
      const int fc = fp / NF, t = fp % NF, ax = fc >> 1, s = fc & 1;
      const int64_t nb = nbr(g, ci, ax, s);
      int tb3[3] = {0, 0, 0};
      {
        int tt = t;
        for (int b = 0; b < DIM; ++b) {
          if (b == ax) continue;
          tb3[b] = tt % N;
          tt /= N;
        }
      }
      A pin = zero;
      for (int i = 0; i < N; ++i) pin += tb.L[s][i] * s_pu[cl][node_of(N, ax, i, t, DIM)];
      A pav = pin;
      if (nb >= 0) {
        A pout = zero;
        for (int j = 0; j < NBP; ++j) {
          const int jj[3] = {j % NP, (j / NP) % NP, DIM == 3 ? j / (NP * NP) : 0};
          A wgt = tp.L[1 - s][jj[ax]];
          for (int b = 0; b < DIM; ++b)
            if (b != ax) wgt = wgt * mx.I[tb3[b]][jj[b]];
          pout = Ar::fma(wgt, Ar::from(__ldg(&p[nb * NBP + j])), pout);
        }
        pav = half * (pin + pout);
      }
      const double* gfp = g.gfu + ((cell * 2 * DIM + fc) * (int64_t)NFF) * NF + t;
      s_f[cl][fp] = Ar::from(gfp[0]) * pav;
    }
  }
  for (int c = 0; c < DIM; ++c) {
    if (active && p)
      for (int a = 0; a < DIM; ++a) s_q[a][cl][node] = s_pu[cl][node] * Ar::from(gv[(NG + 1 + a * DIM + c) * NB]);
    __syncthreads();
    if (active) {
      const int64_t o = (int64_t)c * g.ncell * NB + cell * NB + node;
      A y = zero;
      if (u_mass) y += mass * W * Ar::from(u_mass[o]);
      if (f) y += W * Ar::from(f[o]);
      if (p) {
        for (int a = 0; a < DIM; ++a)
          for (int m = 0; m < N; ++m) {
            int j[3] = {ii[0], ii[1], ii[2]};
            j[a] = m;
            y += tb.D[m][ii[a]] * s_q[a][cl][j[0] + N * (j[1] + N * j[2])];
          }
        for (int b = 0; b < DIM; ++b) {
          const int t = tang_of<N, DIM>(b, ii);
          for (int s = 0; s < 2; ++s) {
            const int fc = 2 * b + s, fp = fc * NF + t;
            const double* gfp = g.gfu + ((cell * 2 * DIM + fc) * (int64_t)NFF) * NF + t;
            y -= s_f[cl][fp] * Ar::from(gfp[(1 + c) * NF]) * tb.L[s][ii[b]];
          }
        }
      }
      rhs[o] = Ar::to_d(y);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------
// rhs_p = alpha M^p p_old + (1/tau) sum_c D_c uss_c (Eq. weakform_p_1), one
// thread per pressure node, integrated with the velocity rule.
template <typename A, int DIM, int N, int NP, int CPB>
__global__ void __launch_bounds__(((CPB * Shape<NP, DIM>::NB + 31) / 32) * 32)
    gen_pressure_rhs_kernel(const __grid_constant__ GG g, const __grid_constant__ Tab1D<A> tb,
                            const __grid_constant__ Tab1D<A> tp, const __grid_constant__ MixTab<A> mx,
                            double alpha_d, double inv_tau_d, const double* __restrict__ uss,
                            const double* __restrict__ p_old, double* __restrict__ rhs) {
  pdl_entry();
  using Ar = Arith<A>;
  using GC = GeomCount<DIM>;
  constexpr int NB = Shape<N, DIM>::NB, NF = Shape<N, DIM>::NF, NFP = Shape<N, DIM>::NFP;
  constexpr int NBP = Shape<NP, DIM>::NB;
  constexpr int NG = GC::NG, NV = GC::NVU, NFF = GC::NFU, NVP = GC::NVP;
  __shared__ A s_u[DIM][CPB][NB];   // uss, then B uss (contravariant)
  __shared__ A s_f[CPB][NFP];
  const int tid = threadIdx.x, cl = tid / NBP, node = tid % NBP;
  const int64_t cell = (int64_t)blockIdx.x * CPB + cl;
  const bool active = cl < CPB && cell < g.ncell;
  const A zero = Ar::c(0.0), half = Ar::c(0.5);
  int ci[3] = {0, 0, 0};
  if (active) {
    coords(g, cell, ci);
    for (int idx = node; idx < DIM * NB; idx += NBP) {
      const int c = idx / NB, nd = idx % NB;
      s_u[c][cl][nd] = Ar::from(uss[((int64_t)c * g.ncell + cell) * NB + nd]);
    }
  }
  __syncthreads();
  if (active) {  // {{uss}}.n dS at the velocity face points
    for (int fp = node; fp < NFP; fp += NBP) {
      const int fc = fp / NF, t = fp % NF, ax = fc >> 1, s = fc & 1;
      const int64_t nb = nbr(g, ci, ax, s);
      const double* gfp = g.gfu + ((cell * 2 * DIM + fc) * (int64_t)NFF) * NF + t;
      A acc = zero;
      for (int r = 0; r < DIM; ++r) {
        A uin = zero, uout = zero;
        for (int i = 0; i < N; ++i) {
          const int nd = node_of(N, ax, i, t, DIM);
          uin = Ar::fma(tb.L[s][i], s_u[r][cl][nd], uin);
          if (nb >= 0) uout += tb.L[1 - s][i] * Ar::from(__ldg(&uss[((int64_t)r * g.ncell + nb) * NB + nd]));
        }
        acc += Ar::from(gfp[(1 + r) * NF]) * (nb >= 0 ? half * (uin + uout) : uin);
      }
      s_f[cl][fp] = Ar::from(gfp[0]) * acc;
    }
  }
  __syncthreads();
  // contravariant components B uss at the velocity nodes (in place)
  A tmp[DIM * ((NB + NBP - 1) / NBP)];
  if (active) {
    int k = 0;
    for (int q = node; q < NB; q += NBP) {
      const double* gv = g.gvu + cell * (int64_t)NV * NB + q;
      for (int a = 0; a < DIM; ++a) {
        A acc = zero;
        for (int c = 0; c < DIM; ++c) acc += Ar::from(gv[(NG + 1 + a * DIM + c) * NB]) * s_u[c][cl][q];
        tmp[k++] = acc;
      }
    }
  }
  __syncthreads();
  if (active) {
    int k = 0;
    for (int q = node; q < NB; q += NBP)
      for (int a = 0; a < DIM; ++a) s_u[a][cl][q] = tmp[k++];
  }
  __syncthreads();
  if (active) {
    const int pi[3] = {node % NP, (node / NP) % NP, DIM == 3 ? node / (NP * NP) : 0};
    A acc = zero;
    for (int q = 0; q < NB; ++q) {
      const int qq[3] = {q % N, (q / N) % N, DIM == 3 ? q / (N * N) : 0};
      A v[DIM];
      for (int b = 0; b < DIM; ++b) v[b] = mx.I[qq[b]][pi[b]];
      for (int a = 0; a < DIM; ++a) {
        A dpsi = mx.D[qq[a]][pi[a]];
        for (int b = 0; b < DIM; ++b)
          if (b != a) dpsi = dpsi * v[b];
        acc += s_u[a][cl][q] * dpsi;
      }
    }
    for (int fc = 0; fc < 2 * DIM; ++fc) {
      const int ax = fc >> 1, s = fc & 1;
      for (int t = 0; t < NF; ++t) {
        A psi = tp.L[s][pi[ax]];
        int tt = t;
        for (int b = 0; b < DIM; ++b) {
          if (b == ax) continue;
          psi = psi * mx.I[tt % N][pi[b]];
          tt /= N;
        }
        acc -= s_f[cl][fc * NF + t] * psi;
      }
    }
    const A Wp = Ar::from(g.gvp[cell * (int64_t)NVP * NBP + NG * NBP + node]);
    rhs[cell * NBP + node] =
        Ar::to_d(Ar::from(alpha_d) * Wp * Ar::from(p_old[cell * NBP + node]) + Ar::from(inv_tau_d) * acc);
  }
}

// ------------------------------------------------------------------
// u~_c = M^-1 P_c p = the physical gradient of p at the velocity nodes
// (collocation makes M diagonal with entries W).
template <typename A, int DIM, int N, int NP, int CPB>
__global__ void __launch_bounds__(((CPB * Shape<N, DIM>::NB + 31) / 32) * 32)
    gen_project_kernel(const __grid_constant__ GG g, const __grid_constant__ MixTab<A> mx,
                       const double* __restrict__ p, double* __restrict__ ut) {
  pdl_entry();
  using Ar = Arith<A>;
  using GC = GeomCount<DIM>;
  constexpr int NB = Shape<N, DIM>::NB, NBP = Shape<NP, DIM>::NB;
  constexpr int NG = GC::NG, NV = GC::NVU;
  __shared__ A s_p[CPB][NBP];
  const int tid = threadIdx.x, cl = tid / NB, node = tid % NB;
  const int64_t cell = (int64_t)blockIdx.x * CPB + cl;
  const bool active = cl < CPB && cell < g.ncell;
  if (active && node < NBP) s_p[cl][node] = Ar::from(p[cell * NBP + node]);
  __syncthreads();
  if (!active) return;
  const int ii[3] = {node % N, (node / N) % N, DIM == 3 ? node / (N * N) : 0};
  A gref[DIM];
  for (int a = 0; a < DIM; ++a) {
    A acc = Ar::c(0.0);
    for (int j = 0; j < NBP; ++j) {
      const int jj[3] = {j % NP, (j / NP) % NP, DIM == 3 ? j / (NP * NP) : 0};
      A wgt = a == 0 ? mx.D[ii[0]][jj[0]] : mx.I[ii[0]][jj[0]];
      for (int b = 1; b < DIM; ++b) wgt = wgt * (b == a ? mx.D[ii[b]][jj[b]] : mx.I[ii[b]][jj[b]]);
      acc = Ar::fma(wgt, s_p[cl][j], acc);
    }
    gref[a] = acc;
  }
  const double* gv = g.gvu + cell * (int64_t)NV * NB + node;
  const double W = gv[NG * NB];
  for (int c = 0; c < DIM; ++c) {
    A acc = Ar::c(0.0);
    for (int a = 0; a < DIM; ++a) acc += Ar::from(gv[(NG + 1 + a * DIM + c) * NB]) * gref[a];
    ut[((int64_t)c * g.ncell + cell) * NB + node] = Ar::to_d(acc) / W;
  }
}

// ------------------------------------------------------------------
// Diagonal of mass M + visc A + adv C(ubar) (velocity space, walls) or of
// alpha M^p + K (pressure space, VEL = false, no wall terms), one thread per
// node, arithmetic R.
template <int DIM, int N, bool VEL, typename R>
__global__ void gen_diag_kernel(const __grid_constant__ GG g, const __grid_constant__ Tab1D<R> tb,
                                R mass, R visc, R adv, R pen, const double* __restrict__ ub,
                                double* __restrict__ diag) {
  pdl_entry();
  using Ar = Arith<R>;
  using GC = GeomCount<DIM>;
  constexpr int NB = Shape<N, DIM>::NB, NF = Shape<N, DIM>::NF;
  constexpr int NG = GC::NG;
  constexpr int NV = VEL ? GC::NVU : GC::NVP;
  constexpr int NFF = VEL ? GC::NFU : GC::NFP;
  constexpr int OFF_C = VEL ? 1 + DIM : 1;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= g.ncell * NB) return;
  const int64_t cell = gid / NB;
  const int node = (int)(gid % NB);
  int ci[3];
  coords(g, cell, ci);
  const int ii[3] = {node % N, (node / N) % N, DIM == 3 ? node / (N * N) : 0};
  const double* gvb = (VEL ? g.gvu : g.gvp) + cell * (int64_t)NV * NB;
  const double* gfb = (VEL ? g.gfu : g.gfp) + cell * 2 * DIM * (int64_t)NFF * NF;
  R d = mass * (R)gvb[NG * NB + node];
  // volume: sum_a sum_m G_aa(line) D[m][i_a]^2 + sum_{a != b} G_ab(i) D_aa D_bb
  R vol = 0;
  for (int a = 0; a < DIM; ++a) {
    for (int m = 0; m < N; ++m) {
      int j[3] = {ii[0], ii[1], ii[2]};
      j[a] = m;
      const int nd = j[0] + N * (j[1] + N * j[2]);
      const R Dm = tb.D[m][ii[a]];
      vol += (R)gvb[sym_index(DIM, a, a) * NB + nd] * Dm * Dm;
    }
    for (int b = 0; b < DIM; ++b)
      if (b != a) vol += (R)gvb[sym_index(DIM, a, b) * NB + node] * tb.D[ii[a]][ii[a]] * tb.D[ii[b]][ii[b]];
  }
  d += visc * vol;
  if (VEL && adv != R(0)) {  // - adv sum_a (B ubar)_a(i) D[i_a][i_a]
    for (int a = 0; a < DIM; ++a) {
      R uta = 0;
      for (int r = 0; r < DIM; ++r)
        uta += (R)gvb[(NG + 1 + a * DIM + r) * NB + node] * (R)ub[((int64_t)r * g.ncell + cell) * NB + node];
      d -= adv * uta * tb.D[ii[a]][ii[a]];
    }
  }
  for (int ax = 0; ax < DIM; ++ax) {
    const int t = tang_of<N, DIM>(ax, ii);
    for (int s = 0; s < 2; ++s) {
      const int f = 2 * ax + s;
      const int64_t nb = nbr(g, ci, ax, s);
      if (nb < 0 && !VEL) continue;  // pressure: Neumann walls, no terms
      const double* gfp = gfb + (int64_t)f * NFF * NF + t;
      const R dS = (R)gfp[0];
      R cown[DIM], cnb[DIM];
      for (int b = 0; b < DIM; ++b) {
        cown[b] = (R)gfp[(OFF_C + b) * NF];
        cnb[b] = (R)gfp[(OFF_C + DIM + b) * NF];
      }
      const R Lv = tb.L[s][ii[ax]];
      R dn = cown[ax] * tb.dL[s][ii[ax]];
      for (int b = 0; b < DIM; ++b)
        if (b != ax) dn += cown[b] * Lv * tb.D[ii[b]][ii[b]];
      const R sig = pen * (R)g.gpen[cell * 2 * DIM + f];
      R unin = 0, unout = 0;
      if (VEL && adv != R(0)) {
        for (int r = 0; r < DIM; ++r) {
          R wi = 0, wo = 0;
          for (int i = 0; i < N; ++i) {
            const int nd = node_of(N, ax, i, t, DIM);
            wi = Ar::fma(tb.L[s][i], (R)ub[((int64_t)r * g.ncell + cell) * NB + nd], wi);
            if (nb >= 0) wo += tb.L[1 - s][i] * (R)ub[((int64_t)r * g.ncell + nb) * NB + nd];
          }
          const R nr = (R)gfp[(1 + r) * NF];
          unin += nr * wi;
          unout += nr * wo;
        }
      }
      R term;
      if (nb >= 0) {
        // a one-cell period makes the cell its own neighbour: the outside
        // trace of the same basis function enters too
        R uo = 0, dno = 0;
        if (nb == cell) {
          uo = tb.L[1 - s][ii[ax]];
          dno = cnb[ax] * tb.dL[1 - s][ii[ax]];
          for (int b = 0; b < DIM; ++b)
            if (b != ax) dno += cnb[b] * uo * tb.D[ii[b]][ii[b]];
        }
        const R jump = Lv - uo;
        term = visc * (sig * jump * Lv - R(0.5) * (dn + dno) * Lv - R(0.5) * jump * dn);
        if (VEL && adv != R(0)) {
          const R lam = fmax(fabs(unin), fabs(unout));
          term += adv * (R(0.5) * (Lv * unin + uo * unout) + R(0.5) * lam * jump) * Lv;
        }
      } else {
        term = visc * (R(2) * sig * Lv * Lv - R(2) * dn * Lv);
        if (adv != R(0)) term += adv * fabs(unin) * Lv * Lv;
      }
      d += dS * term;
    }
  }
  diag[gid] = (double)d;
}

template <typename A, int DIM, int N>
dg_status run_explicit(const dg_mesh* m, int mode, double visc, double adv, const double* w,
                       const double* wb, double* rhs, cudaStream_t s) {
  constexpr int CPB = rhs_cpb<N, DIM>();
  constexpr int threads = ((CPB * Shape<N, DIM>::NB + 31) / 32) * 32;
  const unsigned blocks = (unsigned)((m->ncell + CPB - 1) / CPB);
  const double pen = (double)(N * N);
  if (mode == 0)
    launch(gen_explicit_kernel<A, DIM, N, 0, CPB>, blocks, threads, 0, s, make_gg(m), tabu<A>(m), visc, adv, pen, w, wb, rhs);
  else
    launch(gen_explicit_kernel<A, DIM, N, 1, CPB>, blocks, threads, 0, s, make_gg(m), tabu<A>(m), visc, adv, pen, w, wb, rhs);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

template <typename A, int DIM, int N>
dg_status run_mass_grad(const dg_mesh* m, double mass, const double* um, const double* f,
                        const double* p, double* rhs, cudaStream_t s) {
  constexpr int CPB = rhs_cpb<N, DIM>();
  constexpr int threads = ((CPB * Shape<N, DIM>::NB + 31) / 32) * 32;
  const unsigned blocks = (unsigned)((m->ncell + CPB - 1) / CPB);
  launch(gen_mass_grad_kernel<A, DIM, N, N - 1, CPB>, blocks, threads, 0, s, 
      make_gg(m), tabu<A>(m), tabp<A>(m), tabmix<A>(m), mass, um, f, p, rhs);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

template <typename A, int DIM, int N>
dg_status run_pressure_rhs(const dg_mesh* m, double alpha, double inv_tau, const double* uss,
                           const double* p_old, double* rhs, cudaStream_t s) {
  constexpr int NP = N - 1;
  constexpr int CPB = rhs_cpb<NP, DIM>();
  constexpr int threads = ((CPB * Shape<NP, DIM>::NB + 31) / 32) * 32;
  const unsigned blocks = (unsigned)((m->ncell + CPB - 1) / CPB);
  launch(gen_pressure_rhs_kernel<A, DIM, N, NP, CPB>, blocks, threads, 0, s, 
      make_gg(m), tabu<A>(m), tabp<A>(m), tabmix<A>(m), alpha, inv_tau, uss, p_old, rhs);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

template <typename A, int DIM, int N>
dg_status run_project(const dg_mesh* m, const double* p, double* ut, cudaStream_t s) {
  constexpr int CPB = rhs_cpb<N, DIM>();
  constexpr int threads = ((CPB * Shape<N, DIM>::NB + 31) / 32) * 32;
  const unsigned blocks = (unsigned)((m->ncell + CPB - 1) / CPB);
  launch(gen_project_kernel<A, DIM, N, N - 1, CPB>, blocks, threads, 0, s, make_gg(m), tabmix<A>(m), p, ut);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

template <int DIM, int N, bool VEL>
dg_status run_diag(const dg_mesh* m, double mass, double visc, double adv, const double* ub,
                   double* diag, bool fp32, cudaStream_t s) {
  const int64_t total = m->ncell * Shape<N, DIM>::NB;
  const unsigned blocks = (unsigned)((total + 255) / 256);
  const double pen = VEL ? (double)((m->k + 1) * (m->k + 1)) : (double)(m->k * m->k);
  if (fp32)
    launch(gen_diag_kernel<DIM, N, VEL, float>, blocks, 256, 0, s, 
        make_gg(m), VEL ? m->tu32 : m->tp32, (float)mass, (float)visc, (float)adv, (float)pen, ub, diag);
  else
    launch(gen_diag_kernel<DIM, N, VEL, double>, blocks, 256, 0, s, 
        make_gg(m), VEL ? m->tu64 : m->tp64, mass, visc, adv, pen, ub, diag);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

// dispatch on (dim, velocity nodes) and the arithmetic of the mesh
#define DG_GEN_DISPATCH(m, FN, ...)                                                          \
  ((m)->fp64_arith                                                                           \
       ? ((m)->dim == 2 ? ((m)->nu == 3 ? FN<double, 2, 3>(__VA_ARGS__)                      \
                           : (m)->nu == 4 ? FN<double, 2, 4>(__VA_ARGS__)                    \
                                          : FN<double, 2, 5>(__VA_ARGS__))                   \
                        : ((m)->nu == 3 ? FN<double, 3, 3>(__VA_ARGS__)                      \
                           : (m)->nu == 4 ? FN<double, 3, 4>(__VA_ARGS__)                    \
                                          : FN<double, 3, 5>(__VA_ARGS__)))                  \
       : ((m)->dim == 2 ? ((m)->nu == 3 ? FN<df64, 2, 3>(__VA_ARGS__)                        \
                           : (m)->nu == 4 ? FN<df64, 2, 4>(__VA_ARGS__)                      \
                                          : FN<df64, 2, 5>(__VA_ARGS__))                     \
                        : ((m)->nu == 3 ? FN<df64, 3, 3>(__VA_ARGS__)                        \
                           : (m)->nu == 4 ? FN<df64, 3, 4>(__VA_ARGS__)                      \
                                          : FN<df64, 3, 5>(__VA_ARGS__))))

bool check_geom(const dg_mesh* m, const char* who) {
  if (!m->geom_u) {
    set_error(std::string(who) + ": velocity metric terms missing on this mesh");
    return false;
  }
  if (m->nu < 3 || m->nu > 5) {
    set_error(std::string(who) + ": unsupported degree on trilinear cells");
    return false;
  }
  return true;
}

}  // namespace

dg_status general_explicit(const dg_mesh* m, int mode, double visc, double adv, const double* w,
                           const double* wb, double* rhs, cudaStream_t s) {
  if (!check_geom(m, "dg_rhs_momentum")) return DG_EUNSUPPORTED;
  return DG_GEN_DISPATCH(m, run_explicit, m, mode, visc, adv, w, wb, rhs, s);
}

dg_status general_mass_grad(const dg_mesh* m, double mass, const double* um, const double* f,
                            const double* p, double* rhs, cudaStream_t s) {
  if (!check_geom(m, "dg_rhs_momentum")) return DG_EUNSUPPORTED;
  return DG_GEN_DISPATCH(m, run_mass_grad, m, mass, um, f, p, rhs, s);
}

dg_status general_pressure_rhs(const dg_mesh* m, double alpha, double inv_tau, const double* uss,
                               const double* p_old, double* rhs, cudaStream_t s) {
  if (!check_geom(m, "dg_rhs_pressure")) return DG_EUNSUPPORTED;
  return DG_GEN_DISPATCH(m, run_pressure_rhs, m, alpha, inv_tau, uss, p_old, rhs, s);
}

dg_status general_project(const dg_mesh* m, const double* p, double* ut, cudaStream_t s) {
  if (!check_geom(m, "dg_project_gradient")) return DG_EUNSUPPORTED;
  return DG_GEN_DISPATCH(m, run_project, m, p, ut, s);
}

dg_status general_diag(const dg_mesh* m, bool pressure, double mass, double visc, double adv,
                       const double* ub, double* diag, bool fp32, cudaStream_t s) {
  if (pressure) {
    switch (m->dim * 10 + m->np) {
      case 22: return run_diag<2, 2, false>(m, mass, visc, 0.0, nullptr, diag, fp32, s);
      case 23: return run_diag<2, 3, false>(m, mass, visc, 0.0, nullptr, diag, fp32, s);
      case 24: return run_diag<2, 4, false>(m, mass, visc, 0.0, nullptr, diag, fp32, s);
      case 32: return run_diag<3, 2, false>(m, mass, visc, 0.0, nullptr, diag, fp32, s);
      case 33: return run_diag<3, 3, false>(m, mass, visc, 0.0, nullptr, diag, fp32, s);
      case 34: return run_diag<3, 4, false>(m, mass, visc, 0.0, nullptr, diag, fp32, s);
    }
    set_error("pressure diagonal: unsupported degree on trilinear cells");
    return DG_EUNSUPPORTED;
  }
  if (!check_geom(m, "momentum diagonal")) return DG_EUNSUPPORTED;
  switch (m->dim * 10 + m->nu) {
    case 23: return run_diag<2, 3, true>(m, mass, visc, adv, ub, diag, fp32, s);
    case 24: return run_diag<2, 4, true>(m, mass, visc, adv, ub, diag, fp32, s);
    case 25: return run_diag<2, 5, true>(m, mass, visc, adv, ub, diag, fp32, s);
    case 33: return run_diag<3, 3, true>(m, mass, visc, adv, ub, diag, fp32, s);
    case 34: return run_diag<3, 4, true>(m, mass, visc, adv, ub, diag, fp32, s);
    case 35: return run_diag<3, 5, true>(m, mass, visc, adv, ub, diag, fp32, s);
  }
  set_error("momentum diagonal: unsupported degree on trilinear cells");
  return DG_EUNSUPPORTED;
}

}  // namespace dg
