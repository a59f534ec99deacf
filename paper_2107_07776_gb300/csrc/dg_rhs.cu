// Stage right-hand sides, gradient projection and Jacobi diagonals on affine
// cells (Sections 2-3): the explicit viscous and advective terms of F_u
// (Eq. rhs1 and its stage-2 analogue), the DG pressure gradient, the
// Dirichlet data terms, the divergence functional F_p (Eq. weakform_p_1),
// u~ = M^-1 P p, and diag(mass M + visc A + adv C(ubar)) / diag(alpha M^p + K).
//
// Same collocated layout as the operator kernels: one thread per node, CPB
// cells per CTA, cell data in shared memory, neighbour traces from global
// memory, every output written once (deterministic).  These run once per
// stage, not per Krylov iteration.
#include <type_traits>

#include "dg_common.cuh"
#include "dg_df64.cuh"
#include "dg_geom.cuh"
#include "dg_faces.cuh"

namespace dg {

namespace {

template <int N, int DIM>
struct Sh {
  static constexpr int NB = DIM == 3 ? N * N * N : N * N;
  static constexpr int NF = DIM == 3 ? N * N : N;
  static constexpr int NFP = 2 * DIM * NF;
};

struct Grid {
  int64_t ncell;
  int n[3];
  int per[3];
  const double* h[3];
  const double* hi[3];  // inverse extents (no FP64 division in the kernels)
};

__device__ __forceinline__ int nodeof(int N, int dim, int a, int i, int t) {
  // node with coordinate i along axis a and tangential index t (other axes
  // in increasing order); array-free, so a run-time axis stays in registers
  if (dim == 2) return a == 0 ? i + N * t : t + N * i;
  return a == 0 ? i + N * t : (a == 1 ? t % N + N * (i + N * (t / N)) : t + N * N * i);
}

template <typename X>
__device__ __forceinline__ X sel3(int ax, X v0, X v1, X v2) {
  return ax == 0 ? v0 : (ax == 1 ? v1 : v2);
}

__device__ __forceinline__ int tangof(int N, int dim, int a, const int i[3]) {
  int t = 0, mul = 1;
  for (int b = 0; b < dim; ++b) {
    if (b == a) continue;
    t += i[b] * mul;
    mul *= N;
  }
  return t;
}

template <typename A>
__device__ __forceinline__ A b0_or(bool c, A x, A y) { return c ? x : y; }

// neighbour of cell ci across face (a, s); -1 at a wall
__device__ __forceinline__ int64_t neighbour(const Grid& g, const int ci[3], int a, int s) {
  const int ca = sel3(a, ci[0], ci[1], ci[2]), na = sel3(a, g.n[0], g.n[1], g.n[2]);
  int cn = ca + (s ? 1 : -1);
  if (cn < 0 || cn >= na) {
    if (!sel3(a, g.per[0], g.per[1], g.per[2])) return -1;
    cn = cn < 0 ? na - 1 : 0;
  }
  const int64_t stride = a == 0 ? 1 : (a == 1 ? (int64_t)g.n[0] : (int64_t)g.n[0] * g.n[1]);
  const int64_t cell = (int64_t)ci[0] + (int64_t)g.n[0] * (ci[1] + (int64_t)g.n[1] * ci[2]);
  return cell + (int64_t)(cn - ca) * stride;
}

// coordinate along axis a of the neighbour across face s (periodic wrap;
// only meaningful where neighbour() is not -1), without a division
__device__ __forceinline__ int neighbour_coord(const Grid& g, const int ci[3], int a, int s) {
  const int ca = sel3(a, ci[0], ci[1], ci[2]), na = sel3(a, g.n[0], g.n[1], g.n[2]);
  return s ? (ca + 1 == na ? 0 : ca + 1) : (ca == 0 ? na - 1 : ca - 1);
}

__device__ __forceinline__ void cell_coords(const Grid& g, int64_t cell, int ci[3]) {
  lex_coords(cell, g.n[0], g.n[1], ci);
}

// All kernels below keep FP64 storage and compute in the arithmetic type A:
// df64 (float-float on the FP32 pipes, the default) or double (native FP64;
// selected per mesh with dg_mesh_set_fp64_arith).

// ------------------------------------------------------------------
// Explicit terms: MODE 0 adds visc E_v w + adv E_a(wb) w (all faces, central,
// unpenalised); MODE 1 adds the Dirichlet data terms visc B_v w + adv B_a(wb) w
// on wall faces (w = u_D, wb = the stage's advecting field).
template <typename A, int DIM, int N, int MODE, int CPB>
__global__ void __launch_bounds__(((CPB * Sh<N, DIM>::NB + 31) / 32) * 32)
    explicit_kernel(const __grid_constant__ Grid g, const __grid_constant__ Tab1D<A> tb,
                    double visc_d, double adv_d, double pen_d, const double* __restrict__ w,
                    const double* __restrict__ wb, double* __restrict__ rhs) {
  pdl_entry();
  using Ar = Arith<A>;
  constexpr int NB = Sh<N, DIM>::NB, NF = Sh<N, DIM>::NF, NFP = Sh<N, DIM>::NFP;
  __shared__ A s_u[CPB][NB];
  __shared__ A s_wb[DIM][CPB][NB];
  __shared__ A s_q[DIM][CPB][NB];
  __shared__ A s_f[CPB][NFP][2];
  const int tid = threadIdx.x, cl = tid / NB, node = tid % NB;
  const int64_t cell = (int64_t)blockIdx.x * CPB + cl;
  const bool active = cl < CPB && cell < g.ncell;
  const A zero = Ar::c(0.0), half = Ar::c(0.5), two = Ar::c(2.0);
  const A visc = Ar::from(visc_d), adv = Ar::from(adv_d), pen = Ar::from(pen_d);
  int ci[3] = {0, 0, 0};
  const int ii[3] = {node % N, (node / N) % N, DIM == 3 ? node / (N * N) : 0};
  A h[3] = {Ar::c(1.0), Ar::c(1.0), Ar::c(1.0)}, hi[3] = {Ar::c(1.0), Ar::c(1.0), Ar::c(1.0)};
  A W = zero;
  if (active) {
    cell_coords(g, cell, ci);
    for (int b = 0; b < DIM; ++b) {
      h[b] = Ar::from(g.h[b][ci[b]]);
      hi[b] = Ar::from(g.hi[b][ci[b]]);
    }
    W = Ar::c(1.0);
    for (int b = 0; b < DIM; ++b) W = W * tb.w[ii[b]] * h[b];
    for (int b = 0; b < DIM; ++b) s_wb[b][cl][node] = Ar::from(wb[((int64_t)b * g.ncell + cell) * NB + node]);
  }
  for (int c = 0; c < DIM; ++c) {
    const double* wc = w + (int64_t)c * g.ncell * NB;
    if (active) s_u[cl][node] = Ar::from(wc[cell * NB + node]);
    __syncthreads();
    if (active) {
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        A q = zero;
        if (MODE == 0) {
          A du = zero;
#pragma unroll
          for (int m = 0; m < N; ++m) {
            int j[3] = {ii[0], ii[1], ii[2]};
            j[b] = m;
            du += tb.D[ii[b]][m] * s_u[cl][j[0] + N * (j[1] + N * j[2])];
          }
          q = W * (adv * s_u[cl][node] * s_wb[b][cl][node] - visc * du * hi[b]);
        }
        s_q[b][cl][node] = q;
      }
      for (int fp = node; fp < NFP; fp += NB) {
        const int f = fp / NF, t = fp % NF, ax = f >> 1, s = f & 1;
        const A sgn = s ? Ar::c(1.0) : Ar::c(-1.0);
        const int64_t nb = neighbour(g, ci, ax, s);
        const A hiK = sel3(ax, hi[0], hi[1], hi[2]);
        A wt = Ar::c(1.0);
        {
          int tt = t;
          for (int b = 0; b < DIM; ++b) {
            if (b == ax) continue;
            wt = wt * tb.w[tt % N] * h[b];
            tt /= N;
          }
        }
        A uin = zero, dnin = zero, wnin = zero;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const int nd = nodeof(N, DIM, ax, i, t);
          uin = Ar::fma(tb.L[s][i], s_u[cl][nd], uin);
          dnin = Ar::fma(tb.dL[s][i], s_u[cl][nd], dnin);
          wnin = Ar::fma(tb.L[s][i], s_wb[ax][cl][nd], wnin);
        }
        dnin = dnin * sgn * hiK;
        wnin = wnin * sgn;
        A fv = zero, fg = zero;
        if (MODE == 0) {
          if (nb >= 0) {
            const A hiN = Ar::from(sel3(ax, g.hi[0], g.hi[1], g.hi[2])[neighbour_coord(g, ci, ax, s)]);
            A uout = zero, dnout = zero, wnout = zero;
#pragma unroll
            for (int i = 0; i < N; ++i) {
              const int nd = nodeof(N, DIM, ax, i, t);
              const A v = Ar::from(__ldg(&wc[nb * NB + nd]));
              uout = Ar::fma(tb.L[1 - s][i], v, uout);
              dnout = Ar::fma(tb.dL[1 - s][i], v, dnout);
              wnout = Ar::fma(tb.L[1 - s][i], Ar::from(__ldg(&wb[((int64_t)ax * g.ncell + nb) * NB + nd])), wnout);
            }
            dnout = dnout * sgn * hiN;
            wnout = wnout * sgn;
            fv = half * (visc * (dnin + dnout) - adv * (uin * wnin + uout * wnout));
          } else {
            fv = visc * dnin - adv * uin * wnin;
          }
        } else if (nb < 0) {
          const A sig = pen * hiK;
          fv = visc * two * sig * uin + adv * (Ar::abs(wnin) * uin - uin * wnin);
          fg = -(visc * uin);
        }
        s_f[cl][fp][0] = wt * fv;
        s_f[cl][fp][1] = wt * fg * sgn * hiK;
      }
    }
    __syncthreads();
    if (active) {
      A y = zero;
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        A acc = zero;
#pragma unroll
        for (int m = 0; m < N; ++m) {
          int j[3] = {ii[0], ii[1], ii[2]};
          j[b] = m;
          acc += tb.D[m][ii[b]] * s_q[b][cl][j[0] + N * (j[1] + N * j[2])];
        }
        y += acc * hi[b];
        const int t = tangof(N, DIM, b, ii);
        for (int s = 0; s < 2; ++s) {
          const int fp = (2 * b + s) * NF + t;
          y += s_f[cl][fp][0] * tb.L[s][ii[b]] + s_f[cl][fp][1] * tb.dL[s][ii[b]];
        }
      }
      rhs[(int64_t)c * g.ncell * NB + cell * NB + node] += Ar::to_d(y);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------
// The explicit terms of one stage in one pass: rhs += sum_t (visc_t E_v w_t +
// adv_t E_a(wb_t) w_t) over NT = 1 or 2 terms (stage 2 has two).  E_v is
// linear, so it is evaluated once on v = sum_t visc_t w_t; the normal traces
// of the advecting fields are computed once per cell, not per component.
struct ExplTerms {
  double visc[2], adv[2];
  const double* w[2];
  const double* wb[2];
};

// The explicit-term kernels in float-float arithmetic read their fields w,
// wbar pre-split into float pairs (one split pass per field and call instead
// of one split per read; run_explicit_terms_a makes the copies); in native
// FP64 they read the fields themselves.
template <typename A>
__device__ __forceinline__ A ldw(double v) {
  if constexpr (std::is_same<A, df64>::value) return df_bits(v);
  else return Arith<A>::from(v);
}

template <int N, int DIM>
constexpr int expl_minb(int threads) {
  return 65536 / (threads * 96) < 1 ? 1 : 65536 / (threads * 96);
}

// resident CTAs per SM that keep a thread at 72 registers at most
constexpr int minb_cap72(int threads) { return 65536 / (threads * 72) < 1 ? 1 : 65536 / (threads * 72); }

template <typename A, int DIM, int N, int NT, int CPB>
__global__ void __launch_bounds__(((CPB * Sh<N, DIM>::NB + 31) / 32) * 32,
                                  expl_minb<N, DIM>(((CPB * Sh<N, DIM>::NB + 31) / 32) * 32))
    explicit_terms_kernel(const __grid_constant__ Grid g, const __grid_constant__ Tab1D<A> tb,
                          const __grid_constant__ ExplTerms et, double* __restrict__ rhs) {
  pdl_entry();
  using Ar = Arith<A>;
  constexpr int NB = Sh<N, DIM>::NB, NF = Sh<N, DIM>::NF, NFP = Sh<N, DIM>::NFP;
  __shared__ A s_u[NT][CPB][NB];
  __shared__ A s_v[CPB][NB];
  __shared__ A s_wb[NT][DIM][CPB][NB];
  __shared__ A s_q[DIM][CPB][NB];
  __shared__ A s_f[CPB][NFP];
  __shared__ A s_wn[NT][CPB][NFP][2];
  const int tid = threadIdx.x, cl = tid / NB, node = tid % NB;
  const int64_t cell = (int64_t)blockIdx.x * CPB + cl;
  const bool active = cl < CPB && cell < g.ncell;
  const A zero = Ar::c(0.0), half = Ar::c(0.5);
  A visc[NT], adv[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    visc[t] = Ar::from(et.visc[t]);
    adv[t] = Ar::from(et.adv[t]);
  }
  int ci[3] = {0, 0, 0};
  const int ii[3] = {node % N, (node / N) % N, DIM == 3 ? node / (N * N) : 0};
  A h[3] = {Ar::c(1.0), Ar::c(1.0), Ar::c(1.0)}, hi[3] = {Ar::c(1.0), Ar::c(1.0), Ar::c(1.0)};
  A W = zero;
  if (active) {
    cell_coords(g, cell, ci);
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      h[b] = Ar::from(g.h[b][ci[b]]);
      hi[b] = Ar::from(g.hi[b][ci[b]]);
    }
    W = Ar::c(1.0);
#pragma unroll
    for (int b = 0; b < DIM; ++b) W = W * tb.w[ii[b]] * h[b];
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
      for (int b = 0; b < DIM; ++b)
        s_wb[t][b][cl][node] = ldw<A>(et.wb[t][((int64_t)b * g.ncell + cell) * NB + node]);
  }
  __syncthreads();
  if (active) {  // normal traces of the advecting fields, both sides (walls: inside only)
    for (int fp = node; fp < NFP; fp += NB) {
      const int f = fp / NF, t = fp % NF, ax = f >> 1, s = f & 1;
      const A sgn = s ? Ar::c(1.0) : Ar::c(-1.0);
      const int64_t nb = neighbour(g, ci, ax, s);
#pragma unroll
      for (int tt = 0; tt < NT; ++tt) {
        A wi = zero, wo = zero;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const int nd = nodeof(N, DIM, ax, i, t);
          wi = Ar::fma(tb.L[s][i], s_wb[tt][ax][cl][nd], wi);
          if (nb >= 0) wo += tb.L[1 - s][i] * ldw<A>(__ldg(&et.wb[tt][((int64_t)ax * g.ncell + nb) * NB + nd]));
        }
        s_wn[tt][cl][fp][0] = wi * sgn;
        s_wn[tt][cl][fp][1] = wo * sgn;
      }
    }
  }
  for (int c = 0; c < DIM; ++c) {
    if (active) {
      A v = zero;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const A u = ldw<A>(et.w[t][((int64_t)c * g.ncell + cell) * NB + node]);
        s_u[t][cl][node] = u;
        v += visc[t] * u;
      }
      s_v[cl][node] = v;
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        A dv = zero;
#pragma unroll
        for (int m = 0; m < N; ++m) {
          int j[3] = {ii[0], ii[1], ii[2]};
          j[b] = m;
          dv += tb.D[ii[b]][m] * s_v[cl][j[0] + N * (j[1] + N * j[2])];
        }
        A q = -(dv * hi[b]);
#pragma unroll
        for (int t = 0; t < NT; ++t) q += adv[t] * s_u[t][cl][node] * s_wb[t][b][cl][node];
        s_q[b][cl][node] = W * q;
      }
      for (int fp = node; fp < NFP; fp += NB) {
        const int f = fp / NF, t = fp % NF, ax = f >> 1, s = f & 1;
        const A sgn = s ? Ar::c(1.0) : Ar::c(-1.0);
        const int64_t nb = neighbour(g, ci, ax, s);
        const A hiK = sel3(ax, hi[0], hi[1], hi[2]);
        A wt = Ar::c(1.0);
        {
          int tt = t;
#pragma unroll
          for (int b = 0; b < DIM; ++b) {
            if (b == ax) continue;
            wt = wt * tb.w[tt % N] * h[b];
            tt /= N;
          }
        }
        A vin = zero, dvin = zero, uin[NT];
#pragma unroll
        for (int tt = 0; tt < NT; ++tt) uin[tt] = zero;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const int nd = nodeof(N, DIM, ax, i, t);
          const A v = s_v[cl][nd];
          vin = Ar::fma(tb.L[s][i], v, vin);
          dvin = Ar::fma(tb.dL[s][i], v, dvin);
#pragma unroll
          for (int tt = 0; tt < NT; ++tt) uin[tt] += tb.L[s][i] * s_u[tt][cl][nd];
        }
        dvin = dvin * sgn * hiK;
        A fv;
        if (nb >= 0) {
          const A hiN = Ar::from(sel3(ax, g.hi[0], g.hi[1], g.hi[2])[neighbour_coord(g, ci, ax, s)]);
          A vout = zero, dvout = zero, uout[NT];
#pragma unroll
          for (int tt = 0; tt < NT; ++tt) uout[tt] = zero;
#pragma unroll
          for (int i = 0; i < N; ++i) {
            const int nd = nodeof(N, DIM, ax, i, t);
            A v = zero;
#pragma unroll
            for (int tt = 0; tt < NT; ++tt) {
              const A u = ldw<A>(__ldg(&et.w[tt][((int64_t)c * g.ncell + nb) * NB + nd]));
              uout[tt] += tb.L[1 - s][i] * u;
              v += visc[tt] * u;
            }
            vout = Ar::fma(tb.L[1 - s][i], v, vout);
            dvout = Ar::fma(tb.dL[1 - s][i], v, dvout);
          }
          dvout = dvout * sgn * hiN;
          A a = zero;
#pragma unroll
          for (int tt = 0; tt < NT; ++tt)
            a += adv[tt] * (uin[tt] * s_wn[tt][cl][fp][0] + uout[tt] * s_wn[tt][cl][fp][1]);
          fv = half * (dvin + dvout - a);
        } else {
          A a = zero;
#pragma unroll
          for (int tt = 0; tt < NT; ++tt) a += adv[tt] * uin[tt] * s_wn[tt][cl][fp][0];
          fv = dvin - a;
        }
        s_f[cl][fp] = wt * fv;
      }
    }
    __syncthreads();
    if (active) {
      A y = zero;
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        A acc = zero;
#pragma unroll
        for (int m = 0; m < N; ++m) {
          int j[3] = {ii[0], ii[1], ii[2]};
          j[b] = m;
          acc += tb.D[m][ii[b]] * s_q[b][cl][j[0] + N * (j[1] + N * j[2])];
        }
        y += acc * hi[b];
        const int t = tangof(N, DIM, b, ii);
#pragma unroll
        for (int s = 0; s < 2; ++s) y += s_f[cl][(2 * b + s) * NF + t] * tb.L[s][ii[b]];
      }
      rhs[(int64_t)c * g.ncell * NB + cell * NB + node] += Ar::to_d(y);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------
// Face-once form of the explicit terms (used when the mesh's momentum
// operator runs in the face-once form and its flux scratch exists): one
// thread per face point of every face computes the central flux once, in the
// orientation of the face's lower-side cell (the flux is antisymmetric, so
// the upper-side cell takes -F0); the cell kernel adds the volume terms and
// the stored fluxes.  Wall faces store their single cell's flux in the same
// convention.
template <typename A, int DIM, int N, int NT>
__global__ void __launch_bounds__(256)
    explicit_face_kernel(const __grid_constant__ Grid g, const __grid_constant__ Tab1D<A> tb,
                         const __grid_constant__ ExplTerms et, A* __restrict__ flux) {
  pdl_entry();
  using Ar = Arith<A>;
  constexpr int NB = Sh<N, DIM>::NB, NF = Sh<N, DIM>::NF;
  const int64_t f0 = faces_of_axis(0, g.n, g.per), f1 = faces_of_axis(1, g.n, g.per);
  const int64_t f2 = DIM == 3 ? faces_of_axis(2, g.n, g.per) : 0;
  const int64_t nface = f0 + f1 + f2;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nface * NF) return;
  const int t = (int)(gid % NF);
  const int64_t fg = gid / NF;
  const int ax = fg < f0 ? 0 : (fg < f0 + f1 ? 1 : 2);
  const int64_t fl = fg - (ax == 0 ? 0 : (ax == 1 ? f0 : f0 + f1));
  const int d0 = ax == 0 ? face_layers(g.n[0], g.per[0]) : g.n[0];
  const int d1 = ax == 1 ? face_layers(g.n[1], g.per[1]) : g.n[1];
  int fc[3];
  lex_coords(fl, d0, d1, fc);
  const int layer = sel3(ax, fc[0], fc[1], fc[2]);
  const int nax = sel3(ax, g.n[0], g.n[1], g.n[2]);
  const bool pax = sel3(ax, g.per[0], g.per[1], g.per[2]) != 0;
  const int cl_ax = pax ? (layer - 1 + nax) % nax : layer - 1;
  const int cr_ax = layer;
  const bool hasL = pax || layer >= 1, hasR = pax || layer < nax;
  const int64_t cstr = ax == 0 ? 1 : (ax == 1 ? (int64_t)g.n[0] : (int64_t)g.n[0] * g.n[1]);
  const int64_t cbase = (ax == 0 ? 0 : fc[0]) +
                        (int64_t)g.n[0] * ((ax == 1 ? 0 : fc[1]) + (int64_t)g.n[1] * (ax == 2 ? 0 : fc[2]));
  const int64_t cL = cbase + (int64_t)cl_ax * cstr, cR = cbase + (int64_t)cr_ax * cstr;
  const double* hiax = sel3(ax, g.hi[0], g.hi[1], g.hi[2]);
  const A zero = Ar::c(0.0), half = Ar::c(0.5);
  const A hiL = hasL ? Ar::from(hiax[cl_ax]) : zero, hiR = hasR ? Ar::from(hiax[cr_ax]) : zero;
  A visc[NT], adv[NT];
#pragma unroll
  for (int tt = 0; tt < NT; ++tt) {
    visc[tt] = Ar::from(et.visc[tt]);
    adv[tt] = Ar::from(et.adv[tt]);
  }
  A wt = Ar::c(1.0);
  {
    int tt = t;
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      if (b == ax) continue;
      wt = wt * tb.w[tt % N] * Ar::from(g.h[b][fc[b]]);
      tt /= N;
    }
  }
  // advecting fields' traces along +e_ax
  A wnL[NT], wnR[NT];
#pragma unroll
  for (int tt = 0; tt < NT; ++tt) {
    const double* wa = et.wb[tt] + (int64_t)ax * g.ncell * NB;
    SumOf<A> l, r;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int nd = nodeof(N, DIM, ax, i, t);
      if (hasL) {
        const A x = ldw<A>(__ldg(&wa[cL * NB + nd]));
        if (i == 0) l.start(tb.L[1][i], x);
        else l.fma(tb.L[1][i], x);
      }
      if (hasR) {
        const A x = ldw<A>(__ldg(&wa[cR * NB + nd]));
        if (i == 0) r.start(tb.L[0][i], x);
        else r.fma(tb.L[0][i], x);
      }
    }
    wnL[tt] = hasL ? l.value() : zero;
    wnR[tt] = hasR ? r.value() : zero;
  }
  // Flux coefficients of this face point, the same for every component:
  //   F0 = sum_t (cdL_t dL_t + cuL_t uL_t + cdR_t dR_t + cuR_t uR_t)
  // with u the traces and d the reference normal derivatives of term t's
  // field on each side.  Interior (central flux, normal +e_ax seen from the
  // lower cell): cd = wt visc_t / (2h), cu = -wt adv_t wn_t / 2 on both
  // sides.  Wall of one cell: the one-sided flux, coefficients wt visc_t / h
  // and -wt adv_t wn_t of its single side, in the same orientation (the
  // reader takes -F0 on a cell's lower face).
  A cdL[NT], cuL[NT], cdR[NT], cuR[NT];
  {
    const bool interior = hasL && hasR;
    const A fL = interior ? half * wt : wt, fR = interior ? half * wt : wt;
#pragma unroll
    for (int tt = 0; tt < NT; ++tt) {
      cdL[tt] = hasL ? fL * hiL * visc[tt] : zero;
      cuL[tt] = hasL ? -(fL * adv[tt] * wnL[tt]) : zero;
      cdR[tt] = hasR ? fR * hiR * visc[tt] : zero;
      cuR[tt] = hasR ? -(fR * adv[tt] * wnR[tt]) : zero;
    }
  }
  for (int c = 0; c < DIM; ++c) {
    SumOf<A> f;
    bool started = false;
#pragma unroll
    for (int tt = 0; tt < NT; ++tt) {
      const double* wc = et.w[tt] + (int64_t)c * g.ncell * NB;
      if (hasL) {
        SumOf<A> u, d;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const A x = ldw<A>(__ldg(&wc[cL * NB + nodeof(N, DIM, ax, i, t)]));
          if (i == 0) {
            u.start(tb.L[1][i], x);
            d.start(tb.dL[1][i], x);
          } else {
            u.fma(tb.L[1][i], x);
            d.fma(tb.dL[1][i], x);
          }
        }
        if (!started) f.start(cdL[tt], d.value());
        else f.fma(cdL[tt], d.value());
        started = true;
        f.fma(cuL[tt], u.value());
      }
      if (hasR) {
        SumOf<A> u, d;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const A x = ldw<A>(__ldg(&wc[cR * NB + nodeof(N, DIM, ax, i, t)]));
          if (i == 0) {
            u.start(tb.L[0][i], x);
            d.start(tb.dL[0][i], x);
          } else {
            u.fma(tb.L[0][i], x);
            d.fma(tb.dL[0][i], x);
          }
        }
        if (!started) f.start(cdR[tt], d.value());
        else f.fma(cdR[tt], d.value());
        started = true;
        f.fma(cuR[tt], u.value());
      }
    }
    const A F0 = started ? f.value() : zero;
    flux[(c * nface + fg) * NF + t] = F0;
  }
}

template <typename A, int DIM, int N, int NT, int CPB>
__global__ void __launch_bounds__(((CPB * Sh<N, DIM>::NB + 31) / 32) * 32,
                                  minb_cap72(((CPB * Sh<N, DIM>::NB + 31) / 32) * 32))
    explicit_cell_kernel(const __grid_constant__ Grid g, const __grid_constant__ Tab1D<A> tb,
                         const __grid_constant__ ExplTerms et, const A* __restrict__ flux,
                         double* __restrict__ rhs) {
  pdl_entry();
  using Ar = Arith<A>;
  constexpr int NB = Sh<N, DIM>::NB, NF = Sh<N, DIM>::NF;
  // every component's values and gradient terms: the three phases below run
  // once for all components, each between the same two barriers
  __shared__ A s_v[DIM][CPB][NB];
  __shared__ A s_q[DIM][DIM][CPB][NB];
  // the thread's own advective factors W adv_t ubar_t,b / h_b (shared memory
  // rather than registers)
  __shared__ A s_ca[CPB][NB][NT * DIM];
  const int tid = threadIdx.x, cl = tid / NB, node = tid % NB;
  const int64_t cell = (int64_t)blockIdx.x * CPB + cl;
  const bool active = cl < CPB && cell < g.ncell;
  const A zero = Ar::c(0.0);
  A visc[NT];
#pragma unroll
  for (int tt = 0; tt < NT; ++tt) visc[tt] = Ar::from(et.visc[tt]);
  const int64_t f0 = faces_of_axis(0, g.n, g.per), f1 = faces_of_axis(1, g.n, g.per);
  const int64_t nface = f0 + f1 + (DIM == 3 ? faces_of_axis(2, g.n, g.per) : 0);
  int ci[3] = {0, 0, 0};
  const int ii[3] = {node % N, (node / N) % N, DIM == 3 ? node / (N * N) : 0};
  // per-node factors, the same for every component: the viscous one
  // -W / h_b^2 (both inverse extents of the gradient and its transpose
  // folded in) and the advective ones above
  A cv[DIM];
#pragma unroll
  for (int b = 0; b < DIM; ++b) cv[b] = zero;
  if (active) {
    cell_coords(g, cell, ci);
    A h[3], hi[3];
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      h[b] = Ar::from(g.h[b][ci[b]]);
      hi[b] = Ar::from(g.hi[b][ci[b]]);
    }
    A W = Ar::c(1.0);
#pragma unroll
    for (int b = 0; b < DIM; ++b) W = W * tb.w[ii[b]] * h[b];
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      cv[b] = -(W * hi[b] * hi[b]);
#pragma unroll
      for (int tt = 0; tt < NT; ++tt)
        s_ca[cl][node][tt * DIM + b] =
            W * hi[b] * Ar::from(et.adv[tt]) * ldw<A>(et.wb[tt][((int64_t)b * g.ncell + cell) * NB + node]);
    }
  }
  int64_t fpos[2 * DIM];
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    const int t = tangof(N, DIM, b, ii);
    const int64_t foff = b == 0 ? 0 : (b == 1 ? f0 : f0 + f1);
    const int hi_l = g.per[b] ? (ci[b] + 1) % g.n[b] : ci[b] + 1;
    fpos[2 * b] = (foff + face_index(b, ci[b], ci, g.n, g.per)) * NF + t;
    fpos[2 * b + 1] = (foff + face_index(b, hi_l, ci, g.n, g.per)) * NF + t;
  }
  A u[DIM][NT];
#pragma unroll
  for (int c = 0; c < DIM; ++c)
#pragma unroll
    for (int tt = 0; tt < NT; ++tt) u[c][tt] = zero;
  if (active) {
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      SumOf<A> v;
#pragma unroll
      for (int tt = 0; tt < NT; ++tt) {
        u[c][tt] = ldw<A>(et.w[tt][((int64_t)c * g.ncell + cell) * NB + node]);
        if (tt == 0) v.start(visc[tt], u[c][tt]);
        else v.fma(visc[tt], u[c][tt]);
      }
      s_v[c][cl][node] = v.value();
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        SumOf<A> dv;
#pragma unroll
        for (int m = 0; m < N; ++m) {
          int j[3] = {ii[0], ii[1], ii[2]};
          j[b] = m;
          const A x = s_v[c][cl][j[0] + N * (j[1] + N * j[2])];
          if (m == 0) dv.start(tb.D[ii[b]][m], x);
          else dv.fma(tb.D[ii[b]][m], x);
        }
        SumOf<A> q;
        q.start(cv[b], dv.value());
#pragma unroll
        for (int tt = 0; tt < NT; ++tt) q.fma(s_ca[cl][node][tt * DIM + b], u[c][tt]);
        s_q[c][b][cl][node] = q.value();
      }
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const A* fl = flux + (int64_t)c * nface * NF;
      SumOf<A> y[DIM];  // one partial sum per direction, merged at the end
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
#pragma unroll
        for (int m = 0; m < N; ++m) {
          int j[3] = {ii[0], ii[1], ii[2]};
          j[b] = m;
          const A x = s_q[c][b][cl][j[0] + N * (j[1] + N * j[2])];
          if (m == 0) y[b].start(tb.D[m][ii[b]], x);
          else y[b].fma(tb.D[m][ii[b]], x);
        }
        const A F0lo = fl[fpos[2 * b]], F0hi = fl[fpos[2 * b + 1]];
        y[b].fma(-F0lo, tb.L[0][ii[b]]);
        y[b].fma(F0hi, tb.L[1][ii[b]]);
      }
#pragma unroll
      for (int b = 1; b < DIM; ++b) y[0].merge(y[b]);
      rhs[(int64_t)c * g.ncell * NB + cell * NB + node] += Ar::to_d(y[0].value());
    }
  }
}

// ------------------------------------------------------------------
// rhs = mass M u_mass + M f + G p (G the DG pressure gradient of Eq. rhs1);
// writes (does not accumulate).  N velocity, NP pressure nodes per direction.
// p reaches the velocity nodes by sum factorisation (the value table one
// axis at a time; exact, Q_{k-1} lies in Q_k); the face average {{p}} is
// formed in the pressure basis of the face (own and neighbour trace, NP
// values along the normal each) and then interpolated to the face points.
template <typename A, int DIM, int N, int NP, int CPB>
__global__ void __launch_bounds__(((CPB * Sh<N, DIM>::NB + 31) / 32) * 32)
    mass_grad_kernel(const __grid_constant__ Grid g, const __grid_constant__ Tab1D<A> tb,
                     const __grid_constant__ Tab1D<A> tp, const __grid_constant__ MixTab<A> mx,
                     double mass_d, const double* __restrict__ u_mass, const double* __restrict__ f,
                     const double* __restrict__ p, double* __restrict__ rhs) {
  pdl_entry();
  using Ar = Arith<A>;
  constexpr int NB = Sh<N, DIM>::NB, NF = Sh<N, DIM>::NF, NFP = Sh<N, DIM>::NFP;
  constexpr int NBP = Sh<NP, DIM>::NB, NPF = Sh<NP, DIM>::NF;
  constexpr int SA = DIM == 3 ? N * NP * NP : N * NP;  // after the axis-0 interpolation
  constexpr int SB = DIM == 3 ? N * N * NP : 1;        // after the axis-1 interpolation (3D)
  __shared__ A s_p[CPB][NBP];
  __shared__ A s_a[CPB][SA];
  __shared__ A s_b[CPB][SB];
  __shared__ A s_g[CPB][NB];
  __shared__ A s_t[CPB][2 * DIM * NPF];  // {{p}} per face, pressure tangential basis
  __shared__ A s_f[CPB][NFP];
  const int tid = threadIdx.x, cl = tid / NB, node = tid % NB;
  const int64_t cell = (int64_t)blockIdx.x * CPB + cl;
  const bool active = cl < CPB && cell < g.ncell;
  const A zero = Ar::c(0.0), half = Ar::c(0.5), mass = Ar::from(mass_d);
  int ci[3] = {0, 0, 0};
  const int ii[3] = {node % N, (node / N) % N, DIM == 3 ? node / (N * N) : 0};
  A h[3] = {Ar::c(1.0), Ar::c(1.0), Ar::c(1.0)}, W = zero;
  if (active) {
    cell_coords(g, cell, ci);
    for (int b = 0; b < DIM; ++b) h[b] = Ar::from(g.h[b][ci[b]]);
    W = Ar::c(1.0);
    for (int b = 0; b < DIM; ++b) W = W * tb.w[ii[b]] * h[b];
    if (p) {
      if (node < NBP) s_p[cl][node] = Ar::from(p[cell * NBP + node]);
      for (int idx = node; idx < 2 * DIM * NPF; idx += NB) {
        const int fc = idx / NPF, t = idx % NPF, ax = fc >> 1, s = fc & 1;
        // {{p}} = (p_in + p_out) / 2 as one compensated sum of both traces
        const int64_t nb = neighbour(g, ci, ax, s);
        const A wi = nb >= 0 ? half : Ar::c(1.0);
        SumOf<A> pav;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          const A x = Ar::from(__ldg(&p[cell * NBP + nodeof(NP, DIM, ax, j, t)]));
          if (j == 0) pav.start(wi * tp.L[s][j], x);
          else pav.fma(wi * tp.L[s][j], x);
        }
        if (nb >= 0) {
#pragma unroll
          for (int j = 0; j < NP; ++j)
            pav.fma(half * tp.L[1 - s][j], Ar::from(__ldg(&p[nb * NBP + nodeof(NP, DIM, ax, j, t)])));
        }
        s_t[cl][idx] = pav.value();
      }
    }
  }
  __syncthreads();
  if (active && p) {
    for (int idx = node; idx < SA; idx += NB) {  // axis 0
      const int i0 = idx % N, rest = idx / N;
      A av = zero;
#pragma unroll
      for (int j0 = 0; j0 < NP; ++j0) av = Ar::fma(mx.I[i0][j0], s_p[cl][j0 + NP * rest], av);
      s_a[cl][idx] = av;
    }
    for (int fp = node; fp < NFP; fp += NB) {  // - w |face| n {{p}} at the face points
      const int fc = fp / NF, t = fp % NF, ax = fc >> 1, s = fc & 1;
      const A sgn = s ? Ar::c(1.0) : Ar::c(-1.0);
      const int ta = t % N, tb2 = DIM == 3 ? t / N : 0;
      const int ba = ax == 0 ? 1 : 0, bb = ax == 2 ? 1 : 2;
      A wt = tb.w[ta] * sel3(ba, h[0], h[1], h[2]);
      if (DIM == 3) wt = wt * tb.w[tb2] * sel3(bb, h[0], h[1], h[2]);
      A pv = zero;
      if (DIM == 3) {
#pragma unroll
        for (int b2 = 0; b2 < NP; ++b2) {
          A r = zero;
#pragma unroll
          for (int a2 = 0; a2 < NP; ++a2) r = Ar::fma(mx.I[ta][a2], s_t[cl][fc * NPF + a2 + NP * b2], r);
          pv = Ar::fma(mx.I[tb2][b2], r, pv);
        }
      } else {
#pragma unroll
        for (int a2 = 0; a2 < NP; ++a2) pv = Ar::fma(mx.I[ta][a2], s_t[cl][fc * NPF + a2], pv);
      }
      s_f[cl][fp] = -(wt * sgn * pv);
    }
  }
  __syncthreads();
  if (DIM == 3) {
    if (active && p) {
      for (int idx = node; idx < SB; idx += NB) {  // axis 1
        const int i0 = idx % N, i1 = (idx / N) % N, j2 = idx / (N * N);
        A bv = zero;
#pragma unroll
        for (int j1 = 0; j1 < NP; ++j1) bv = Ar::fma(mx.I[i1][j1], s_a[cl][i0 + N * (j1 + NP * j2)], bv);
        s_b[cl][idx] = bv;
      }
    }
    __syncthreads();
  }
  if (active && p) {  // last axis: p at the velocity nodes
    A pu = zero;
    if (DIM == 3) {
#pragma unroll
      for (int j2 = 0; j2 < NP; ++j2) pu = Ar::fma(mx.I[ii[2]][j2], s_b[cl][ii[0] + N * (ii[1] + N * j2)], pu);
    } else {
#pragma unroll
      for (int j1 = 0; j1 < NP; ++j1) pu = Ar::fma(mx.I[ii[1]][j1], s_a[cl][ii[0] + N * j1], pu);
    }
    s_g[cl][node] = W * pu;
  }
  __syncthreads();
  if (active) {
    // compensated sums of the node's terms (one rounding per output)
    const A mW = mass * W;
    A hic[3] = {zero, zero, zero};
    if (p)
      for (int b = 0; b < DIM; ++b) hic[b] = Ar::from(g.hi[b][ci[b]]);
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const int64_t o = (int64_t)c * g.ncell * NB + cell * NB + node;
      SumOf<A> y;
      if (u_mass) y.start(mW, Ar::from(u_mass[o]));
      else y.start(zero, zero);
      if (f) y.fma(W, Ar::from(f[o]));
      if (p) {
        const int ic = sel3(c, ii[0], ii[1], ii[2]);
        SumOf<A> acc;
#pragma unroll
        for (int m = 0; m < N; ++m) {
          const int j0 = c == 0 ? m : ii[0], j1 = c == 1 ? m : ii[1], j2 = c == 2 ? m : ii[2];
          if (m == 0) acc.start(tb.D[m][ic], s_g[cl][j0 + N * (j1 + N * j2)]);
          else acc.fma(tb.D[m][ic], s_g[cl][j0 + N * (j1 + N * j2)]);
        }
        y.fma(acc.value(), hic[c]);
        const int t = tangof(N, DIM, c, ii);
#pragma unroll
        for (int s = 0; s < 2; ++s) y.fma(s_f[cl][(2 * c + s) * NF + t], tb.L[s][ic]);
      }
      rhs[o] = Ar::to_d(y.value());
    }
  }
}

// ------------------------------------------------------------------
// rhs_p = alpha M^p p_old + (1/tau) sum_c D_c uss_c, one thread per pressure
// node; D the DG divergence of Eq. weakform_p_1, integrated with the
// velocity rule.  Cell term by sum factorisation over the transposed
// pressure-to-velocity tables: component 0 takes D^T along axis 0 and I^T
// along the others, and so on; partial sums that meet the same remaining
// tables are added before they are contracted further.  Face term: the
// quadrature-weighted normal flux w |face| n {{u}} is tested against the
// pressure basis, tangential axes first.  In float-float arithmetic uss
// arrives pre-split (run_pressure_rhs_a).
template <typename A, int DIM, int N, int NP, int CPB>
__global__ void __launch_bounds__(((CPB * Sh<NP, DIM>::NB + 31) / 32) * 32)
    pressure_rhs_kernel(const __grid_constant__ Grid g, const __grid_constant__ Tab1D<A> tb,
                        const __grid_constant__ Tab1D<A> tp, const __grid_constant__ MixTab<A> mx,
                        double alpha_d, double inv_tau_d, const double* __restrict__ uss,
                        const double* __restrict__ p_old, double* __restrict__ rhs) {
  pdl_entry();
  using Ar = Arith<A>;
  constexpr int NB = Sh<N, DIM>::NB, NF = Sh<N, DIM>::NF, NFP = Sh<N, DIM>::NFP;
  constexpr int NBP = Sh<NP, DIM>::NB, NPF = Sh<NP, DIM>::NF;
  constexpr int SX = DIM == 3 ? NP * N * N : NP * N;  // after the axis-0 contraction
  constexpr int SY = DIM == 3 ? NP * NP * N : 1;      // after the axis-1 contraction (3D)
  __shared__ A s_u[DIM][CPB][NB];         // W hi_c u_c at the velocity nodes
  __shared__ A s_f[CPB][NFP];             // w |face| n {{u}} at the face points
  __shared__ A s_F[CPB][2 * DIM * NPF];   // the same tested in the tangential pressure basis
  __shared__ A s_x[DIM][CPB][SX];
  __shared__ A s_y[2][CPB][SY];
  const int tid = threadIdx.x, cl = tid / NBP, node = tid % NBP;
  const int64_t cell = (int64_t)blockIdx.x * CPB + cl;
  const bool active = cl < CPB && cell < g.ncell;
  const A zero = Ar::c(0.0), half = Ar::c(0.5);
  int ci[3] = {0, 0, 0};
  A h[3] = {Ar::c(1.0), Ar::c(1.0), Ar::c(1.0)}, hiv[3] = {Ar::c(1.0), Ar::c(1.0), Ar::c(1.0)};
  if (active) {
    cell_coords(g, cell, ci);
    for (int b = 0; b < DIM; ++b) {
      h[b] = Ar::from(g.h[b][ci[b]]);
      hiv[b] = Ar::from(g.hi[b][ci[b]]);
    }
    for (int idx = node; idx < DIM * NB; idx += NBP) {
      const int c = idx / NB, nd = idx % NB;
      const int q0 = nd % N, q1 = (nd / N) % N, q2 = DIM == 3 ? nd / (N * N) : 0;
      A Wq = tb.w[q0] * h[0] * tb.w[q1] * h[1];
      if (DIM == 3) Wq = Wq * tb.w[q2] * h[2];
      s_u[c][cl][nd] = Wq * sel3(c, hiv[0], hiv[1], hiv[2]) *
                       ldw<A>(uss[((int64_t)c * g.ncell + cell) * NB + nd]);
    }
    for (int fp = node; fp < NFP; fp += NBP) {
      const int fc = fp / NF, t = fp % NF, ax = fc >> 1, s = fc & 1;
      const A sgn = s ? Ar::c(1.0) : Ar::c(-1.0);
      const int64_t nb = neighbour(g, ci, ax, s);
      const int ta = t % N, tb2 = DIM == 3 ? t / N : 0;
      const int ba = ax == 0 ? 1 : 0, bb = ax == 2 ? 1 : 2;
      A wt = tb.w[ta] * sel3(ba, h[0], h[1], h[2]);
      if (DIM == 3) wt = wt * tb.w[tb2] * sel3(bb, h[0], h[1], h[2]);
      // w |face| n {{u}}: both traces in one compensated sum, the weight
      // folded into the coefficients
      const A wf = sgn * (nb >= 0 ? half * wt : wt);
      SumOf<A> uav;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const A x = ldw<A>(__ldg(&uss[((int64_t)ax * g.ncell + cell) * NB + nodeof(N, DIM, ax, i, t)]));
        if (i == 0) uav.start(wf * tb.L[s][i], x);
        else uav.fma(wf * tb.L[s][i], x);
      }
      if (nb >= 0) {
#pragma unroll
        for (int i = 0; i < N; ++i)
          uav.fma(wf * tb.L[1 - s][i], ldw<A>(__ldg(&uss[((int64_t)ax * g.ncell + nb) * NB + nodeof(N, DIM, ax, i, t)])));
      }
      s_f[cl][fp] = uav.value();
    }
  }
  __syncthreads();
  if (active) {
    for (int idx = node; idx < SX; idx += NBP) {  // axis 0
      const int p0 = idx % NP, rest = idx / NP;
      A x[DIM];
#pragma unroll
      for (int c = 0; c < DIM; ++c) x[c] = zero;
#pragma unroll
      for (int q0 = 0; q0 < N; ++q0) {
        x[0] = Ar::fma(mx.D[q0][p0], s_u[0][cl][q0 + N * rest], x[0]);
#pragma unroll
        for (int c = 1; c < DIM; ++c) x[c] = Ar::fma(mx.I[q0][p0], s_u[c][cl][q0 + N * rest], x[c]);
      }
#pragma unroll
      for (int c = 0; c < DIM; ++c) s_x[c][cl][idx] = x[c];
    }
    for (int idx = node; idx < 2 * DIM * NPF; idx += NBP) {  // face fluxes, tangential axes
      const int fc = idx / NPF, t = idx % NPF, a2 = t % NP, b2 = DIM == 3 ? t / NP : 0;
      A F = zero;
      if (DIM == 3) {
#pragma unroll
        for (int tb2 = 0; tb2 < N; ++tb2) {
          A r = zero;
#pragma unroll
          for (int ta = 0; ta < N; ++ta) r = Ar::fma(mx.I[ta][a2], s_f[cl][fc * NF + ta + N * tb2], r);
          F = Ar::fma(mx.I[tb2][b2], r, F);
        }
      } else {
#pragma unroll
        for (int ta = 0; ta < N; ++ta) F = Ar::fma(mx.I[ta][a2], s_f[cl][fc * NF + ta], F);
      }
      s_F[cl][idx] = F;
    }
  }
  __syncthreads();
  if (DIM == 3) {
    if (active) {
      for (int idx = node; idx < SY; idx += NBP) {  // axis 1: (x0, x2 with I^T; x1 with D^T)
        const int p0 = idx % NP, p1 = (idx / NP) % NP, q2 = idx / (NP * NP);
        A y0 = zero, y1 = zero;
#pragma unroll
        for (int q1 = 0; q1 < N; ++q1) {
          const int q = p0 + NP * (q1 + N * q2);
          y0 = Ar::fma(mx.I[q1][p1], s_x[0][cl][q], y0);
          y0 = Ar::fma(mx.D[q1][p1], s_x[1][cl][q], y0);
          y1 = Ar::fma(mx.I[q1][p1], s_x[DIM - 1][cl][q], y1);
        }
        s_y[0][cl][idx] = y0;
        s_y[1][cl][idx] = y1;
      }
    }
    __syncthreads();
  }
  if (!active) return;
  const int pi[3] = {node % NP, (node / NP) % NP, DIM == 3 ? node / (NP * NP) : 0};
  // the cell and face terms as one compensated sum
  SumOf<A> acc;
  if (DIM == 3) {  // axis 2: I^T on (x0 + x1 so far), D^T on x2
#pragma unroll
    for (int q2 = 0; q2 < N; ++q2) {
      const int q = pi[0] + NP * (pi[1] + NP * q2);
      if (q2 == 0) acc.start(mx.I[q2][pi[2]], s_y[0][cl][q]);
      else acc.fma(mx.I[q2][pi[2]], s_y[0][cl][q]);
      acc.fma(mx.D[q2][pi[2]], s_y[1][cl][q]);
    }
  } else {  // axis 1 in 2D: I^T on x0, D^T on x1
#pragma unroll
    for (int q1 = 0; q1 < N; ++q1) {
      const int q = pi[0] + NP * q1;
      if (q1 == 0) acc.start(mx.I[q1][pi[1]], s_x[0][cl][q]);
      else acc.fma(mx.I[q1][pi[1]], s_x[0][cl][q]);
      acc.fma(mx.D[q1][pi[1]], s_x[DIM - 1][cl][q]);
    }
  }
  // face term: - sum_faces (tested flux) L_s(normal index)
#pragma unroll
  for (int fc = 0; fc < 2 * DIM; ++fc) {
    const int ax = fc >> 1, s = fc & 1;
    acc.fma(-tp.L[s][sel3(ax, pi[0], pi[1], pi[2])], s_F[cl][fc * NPF + tangof(NP, DIM, ax, pi)]);
  }
  A Wp = Ar::c(1.0);
  for (int b = 0; b < DIM; ++b) Wp = Wp * tp.w[pi[b]] * h[b];
  SumOf<A> r;
  r.start(Ar::from(alpha_d) * Wp, Ar::from(p_old[cell * NBP + node]));
  r.fma(Ar::from(inv_tau_d), acc.value());
  rhs[cell * NBP + node] = Ar::to_d(r.value());
}

// ------------------------------------------------------------------
// u~_c = M^-1 P_c p: the broken gradient of p at the velocity nodes (exact
// on affine cells, where M is diagonal and P_c p = W d_c p at the nodes), by
// sum factorisation: the pressure-to-velocity tables applied one axis at a
// time (value table I or derivative table D per axis), sharing the partial
// contractions between the components.  Optional fused update (out != null):
// out = base + tau (u~ - sub) (sub may be null), the stage updates of
// Section 2 (u** = u* + tau u~old, u = u* - tau (u~new - u~old)).
template <typename A, int DIM, int N, int NP, int CPB>
__global__ void __launch_bounds__(((CPB * Sh<N, DIM>::NB + 31) / 32) * 32)
    project_kernel(const __grid_constant__ Grid g, const __grid_constant__ MixTab<A> mx,
                   const double* __restrict__ p, double* __restrict__ ut,
                   const double* __restrict__ base, double tau, const double* __restrict__ sub,
                   double* __restrict__ out) {
  pdl_entry();
  using Ar = Arith<A>;
  constexpr int NB = Sh<N, DIM>::NB, NBP = Sh<NP, DIM>::NB;
  constexpr int SA = DIM == 3 ? N * NP * NP : N * NP;  // after the axis-0 contraction
  constexpr int SB = DIM == 3 ? N * N * NP : 1;        // after the axis-1 contraction (3D)
  __shared__ A s_p[CPB][NBP];
  __shared__ A s_a[2][CPB][SA];   // I0 p, D0 p
  __shared__ A s_b[3][CPB][SB];   // I1 I0 p, D1 I0 p, I1 D0 p
  const int tid = threadIdx.x, cl = tid / NB, node = tid % NB;
  const int64_t cell = (int64_t)blockIdx.x * CPB + cl;
  const bool active = cl < CPB && cell < g.ncell;
  const A zero = Ar::c(0.0);
  if (active && node < NBP) s_p[cl][node] = Ar::from(p[cell * NBP + node]);
  __syncthreads();
  if (active) {  // axis 0
    for (int idx = node; idx < SA; idx += NB) {
      const int i0 = idx % N, rest = idx / N;  // rest = j1 (+ NP j2)
      A av = zero, bv = zero;
#pragma unroll
      for (int j0 = 0; j0 < NP; ++j0) {
        const A pv = s_p[cl][j0 + NP * rest];
        av = Ar::fma(mx.I[i0][j0], pv, av);
        bv = Ar::fma(mx.D[i0][j0], pv, bv);
      }
      s_a[0][cl][idx] = av;
      s_a[1][cl][idx] = bv;
    }
  }
  __syncthreads();
  if (DIM == 3) {
    if (active) {  // axis 1
      for (int idx = node; idx < SB; idx += NB) {
        const int i0 = idx % N, i1 = (idx / N) % N, j2 = idx / (N * N);
        A ai = zero, ad = zero, bi = zero;
#pragma unroll
        for (int j1 = 0; j1 < NP; ++j1) {
          const int q = i0 + N * (j1 + NP * j2);
          ai = Ar::fma(mx.I[i1][j1], s_a[0][cl][q], ai);
          ad = Ar::fma(mx.D[i1][j1], s_a[0][cl][q], ad);
          bi = Ar::fma(mx.I[i1][j1], s_a[1][cl][q], bi);
        }
        s_b[0][cl][idx] = ai;
        s_b[1][cl][idx] = ad;
        s_b[2][cl][idx] = bi;
      }
    }
    __syncthreads();
  }
  if (!active) return;
  int ci[3];
  cell_coords(g, cell, ci);
  const int ii[3] = {node % N, (node / N) % N, DIM == 3 ? node / (N * N) : 0};
  A uc[DIM];
  if (DIM == 3) {  // axis 2: x-derivative (I2 I1 D0), y (I2 D1 I0), z (D2 I1 I0)
    A u0 = zero, u1 = zero, u2 = zero;
#pragma unroll
    for (int j2 = 0; j2 < NP; ++j2) {
      const int q = ii[0] + N * (ii[1] + N * j2);
      u0 = Ar::fma(mx.I[ii[2]][j2], s_b[2][cl][q], u0);
      u1 = Ar::fma(mx.I[ii[2]][j2], s_b[1][cl][q], u1);
      u2 = Ar::fma(mx.D[ii[2]][j2], s_b[0][cl][q], u2);
    }
    uc[0] = u0;
    uc[1] = u1;
    uc[DIM - 1] = u2;
  } else {  // axis 1 in 2D: x (I1 D0), y (D1 I0)
    A u0 = zero, u1 = zero;
#pragma unroll
    for (int j1 = 0; j1 < NP; ++j1) {
      const int q = ii[0] + N * j1;
      u0 = Ar::fma(mx.I[ii[1]][j1], s_a[1][cl][q], u0);
      u1 = Ar::fma(mx.D[ii[1]][j1], s_a[0][cl][q], u1);
    }
    uc[0] = u0;
    uc[DIM - 1] = u1;
  }
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const int64_t o = ((int64_t)c * g.ncell + cell) * NB + node;
    const double v = Ar::to_d(uc[c] * Ar::from(g.hi[c][ci[c]]));
    ut[o] = v;
    if (out) out[o] = base[o] + tau * (sub ? v - sub[o] : v);
  }
}

// ------------------------------------------------------------------
// FP64 data in the diagonal's arithmetic type: float by integer narrowing
// (no FP64-pipe conversion), double as is; and 1/d stored as double (FP32
// reciprocal widened exactly for float, an FP64 division for double).
template <typename R>
__device__ __forceinline__ R to_r(double v) {
  if constexpr (sizeof(R) == 4) return df_narrow(v);
  else return v;
}
// an advecting-field value for the diagonal: from the float-pair copy (its
// leading float) when the field arrives pre-split, else narrowed
template <typename R>
__device__ __forceinline__ R ld_ub(double v, int pairs) {
  if constexpr (sizeof(R) == 4) {
    if (pairs) return df_bits(v).hi;
  }
  return to_r<R>(v);
}
template <typename R>
__device__ __forceinline__ R abs_r(R x) { return x < R(0.0) ? -x : x; }
template <typename R>
__device__ __forceinline__ R max_r(R x, R y) { return x < y ? y : x; }
template <typename R>
__device__ __forceinline__ double inv_r(R d) {
  if constexpr (sizeof(R) == 4) return df_widen(__frcp_rn(d));
  else return 1.0 / d;
}

// Diagonal of mass M + visc A + adv C(ubar) (walls = 1) or of
// alpha M^p + K (walls = 0, adv = 0), one thread per node.  A face point's
// contribution to the node i on its normal line (i the node's index along
// the normal, t its tangential index) factors into per-face-point
// coefficients and per-node table values: with u_in = L_s(i) and
// dn_in = sgn h^-1 L'_s(i),
//   interior face:  w_t (K u_in^2 - visc u_in dn_in),
//                   K = visc C + adv (un_in + lambda) / 2, C = pen (h_K^-1 + h_N^-1) / 2
//   wall face:      w_t (K u_in^2 - 2 visc u_in dn_in),  K = 2 visc pen h_K^-1 + adv |un_in|
// (the SIP and Lax-Friedrichs terms of the operator, Section 3, with the
// outer trace of a basis function zero).  The coefficients are formed once
// per face point (P = w_t K, Q = kappa w_t visc sgn h_K^-1) and each node
// adds P L_s(i)^2 - Q L_s(i) L'_s(i).  On a one-cell periodic axis the
// outer trace is the cell's own: those faces take the full flux per node.
template <int DIM, int N, typename R, int CPB>
__global__ void __launch_bounds__(((CPB * Sh<N, DIM>::NB + 31) / 32) * 32)
    diag_kernel(const __grid_constant__ Grid g, const __grid_constant__ Tab1D<R> tb, R mass, R visc, R adv,
                R pen, int walls, const double* __restrict__ ub, int ub_pairs, double* __restrict__ diag,
                int inv_copies) {
  pdl_entry();
  using Ar = Arith<R>;
  constexpr int NB = Sh<N, DIM>::NB, NF = Sh<N, DIM>::NF, NFP = Sh<N, DIM>::NFP;
  // per face point: the normal advecting velocity (own and neighbour trace)
  // and the two coefficients P and Q above
  __shared__ R s_in[CPB][NFP];
  __shared__ R s_out[CPB][NFP];
  __shared__ R s_P[CPB][NFP];
  __shared__ R s_Q[CPB][NFP];
  const int tid = threadIdx.x, cl = tid / NB, node = tid % NB;
  const int64_t cell = (int64_t)blockIdx.x * CPB + cl;
  const bool active = cl < CPB && cell < g.ncell;
  int ci[3] = {0, 0, 0};
  R h[3] = {1, 1, 1}, hi[3] = {1, 1, 1};
  if (active) {
    cell_coords(g, cell, ci);
    for (int b = 0; b < DIM; ++b) {
      h[b] = to_r<R>(g.h[b][ci[b]]);
      hi[b] = to_r<R>(g.hi[b][ci[b]]);
    }
    for (int fp = node; fp < NFP; fp += NB) {
      const int fc = fp / NF, t = fp % NF, ax = fc >> 1, s = fc & 1;
      const R sgn = s ? R(1.0) : R(-1.0);
      const int64_t nb = neighbour(g, ci, ax, s);
      R unin = 0.0, unout = 0.0;
      if (adv != R(0.0)) {
        const double* ua = ub + (int64_t)ax * g.ncell * NB;
#pragma unroll
        for (int i = 0; i < N; ++i)
          unin = Ar::fma(tb.L[s][i], ld_ub<R>(__ldg(&ua[cell * NB + nodeof(N, DIM, ax, i, t)]), ub_pairs), unin);
        if (nb >= 0) {
#pragma unroll
          for (int i = 0; i < N; ++i)
            unout = Ar::fma(tb.L[1 - s][i], ld_ub<R>(__ldg(&ua[nb * NB + nodeof(N, DIM, ax, i, t)]), ub_pairs), unout);
        }
        unin = sgn * unin;
        unout = sgn * unout;
      }
      s_in[cl][fp] = unin;
      s_out[cl][fp] = unout;
      // tangential weight of the face point
      const int b0 = ax == 0 ? 1 : 0, b1 = ax == 2 ? 1 : 2;
      R wt = tb.w[t % N] * sel3(b0, h[0], h[1], h[2]);
      if (DIM == 3) wt *= tb.w[t / N] * sel3(b1, h[0], h[1], h[2]);
      const R hiK = sel3(ax, hi[0], hi[1], hi[2]);
      R P = 0.0, Q = 0.0;
      if (nb >= 0) {
        const R hiN = to_r<R>(g.hi[ax][neighbour_coord(g, ci, ax, s)]);
        const R C = R(0.5) * pen * (hiK + hiN);
        const R lam = max_r(abs_r(unin), abs_r(unout));
        P = wt * (visc * C + R(0.5) * adv * (unin + lam));
        Q = wt * visc;
      } else if (walls) {
        P = wt * (R(2.0) * visc * pen * hiK + adv * abs_r(unin));
        Q = R(2.0) * wt * visc;
      }
      s_P[cl][fp] = P;
      s_Q[cl][fp] = Q * sgn * hiK;
    }
  }
  __syncthreads();
  if (!active) return;
  const int ii[3] = {node % N, (node / N) % N, DIM == 3 ? node / (N * N) : 0};
  // W = prod_b w(i_b) h_b.  The stiffness diagonal along axis b is
  // sum_m W(j: j_b = m) (D[m][i_b] / h_b)^2 = (W / w(i_b)) h_b^-2 sum_m w(m) D[m][i_b]^2:
  // the tangential weights factor out of the 1D sum.
  R wl[3] = {1, 1, 1};
  for (int b = 0; b < DIM; ++b) wl[b] = tb.w[ii[b]] * h[b];
  const R W = DIM == 3 ? wl[0] * wl[1] * wl[2] : wl[0] * wl[1];
  R d = mass * W;
  for (int b = 0; b < DIM; ++b) {
    R sb = 0.0;
#pragma unroll
    for (int m = 0; m < N; ++m) sb += tb.w[m] * tb.D[m][ii[b]] * tb.D[m][ii[b]];
    R wt = h[b];  // W / w(i_b), times h_b h_b^-2 below
    for (int c = 0; c < DIM; ++c)
      if (c != b) wt *= wl[c];
    const R acc = wt * sb * hi[b] * hi[b];
    d += visc * acc;
    if (adv != R(0.0)) d -= adv * W * ld_ub<R>(ub[((int64_t)b * g.ncell + cell) * NB + node], ub_pairs) * tb.D[ii[b]][ii[b]] * hi[b];
  }
  for (int ax = 0; ax < DIM; ++ax) {
    const int t = tangof(N, DIM, ax, ii), i = ii[ax];
    const bool self = g.per[ax] && g.n[ax] == 1;  // the cell is its own neighbour
    for (int s = 0; s < 2; ++s) {
      const int fp = (2 * ax + s) * NF + t;
      const R Ls = tb.L[s][i], dLs = tb.dL[s][i];
      if (!self) {
        d += s_P[cl][fp] * Ls * Ls - s_Q[cl][fp] * Ls * dLs;
        continue;
      }
      const R sgn = s ? R(1.0) : R(-1.0);
      R wt = 1.0;
      for (int b = 0; b < DIM; ++b)
        if (b != ax) wt *= wl[b];
      const R hiK = hi[ax];
      const R uin = Ls, dnin = sgn * dLs * hiK;
      const R uout = tb.L[1 - s][i], dnout = sgn * tb.dL[1 - s][i] * hiK;
      const R unin = s_in[cl][fp], unout = s_out[cl][fp];
      const R C = pen * hiK;
      const R jump = uin - uout;
      R fv = visc * (R(-0.5) * (dnin + dnout) + C * jump);
      const R fg = R(-0.5) * visc * jump;
      if (adv != R(0.0)) {
        const R lam = max_r(abs_r(unin), abs_r(unout));
        fv += adv * (R(0.5) * (uin * unin + uout * unout) + R(0.5) * lam * jump);
      }
      d += wt * (fv * uin + fg * dnin);
    }
  }
  if (inv_copies > 0) {  // the Jacobi scaling itself, 1/d, for each of inv_copies components
    const double id = inv_r<R>(d);
    for (int c = 0; c < inv_copies; ++c) diag[((int64_t)c * g.ncell + cell) * NB + node] = id;
  } else {
    diag[cell * NB + node] = sizeof(R) == 4 ? df_widen((float)d) : (double)d;
  }
}

template <int DIM>
Grid make_grid(const dg_mesh* m) {
  Grid g;
  g.ncell = m->ncell;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = m->n[a];
    g.per[a] = m->periodic[a];
    g.h[a] = m->d_h64[a];
    g.hi[a] = m->d_hi64[a];
  }
  return g;
}

template <int N, int DIM>
constexpr int cpb_for() {
  return Sh<N, DIM>::NB <= 8 ? 16 : (Sh<N, DIM>::NB <= 27 ? 8 : (Sh<N, DIM>::NB <= 64 ? 4 : 2));
}

template <typename A>
const Tab1D<A>& tab_u(const dg_mesh* m);
template <>
const Tab1D<double>& tab_u<double>(const dg_mesh* m) { return m->tu64; }
template <>
const Tab1D<df64>& tab_u<df64>(const dg_mesh* m) { return m->tudf; }
template <typename A>
const Tab1D<A>& tab_p(const dg_mesh* m);
template <>
const Tab1D<double>& tab_p<double>(const dg_mesh* m) { return m->tp64; }
template <>
const Tab1D<df64>& tab_p<df64>(const dg_mesh* m) { return m->tpdf; }
template <typename A>
const MixTab<A>& tab_mix(const dg_mesh* m);
template <>
const MixTab<double>& tab_mix<double>(const dg_mesh* m) { return m->mix64; }
template <>
const MixTab<df64>& tab_mix<df64>(const dg_mesh* m) { return m->mixdf; }

template <typename A, int DIM, int N>
dg_status run_explicit_a(const dg_mesh* m, int mode, double visc, double adv, const double* w,
                         const double* wb, double* rhs, cudaStream_t s) {
  constexpr int CPB = cpb_for<N, DIM>();
  constexpr int threads = ((CPB * Sh<N, DIM>::NB + 31) / 32) * 32;
  const unsigned blocks = (unsigned)((m->ncell + CPB - 1) / CPB);
  const Grid g = make_grid<DIM>(m);
  const double pen = (double)(N * N);
  if (mode == 0)
    launch(explicit_kernel<A, DIM, N, 0, CPB>, blocks, threads, 0, s, g, tab_u<A>(m), visc, adv, pen, w, wb, rhs);
  else
    launch(explicit_kernel<A, DIM, N, 1, CPB>, blocks, threads, 0, s, g, tab_u<A>(m), visc, adv, pen, w, wb, rhs);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

// Float-float explicit terms: each distinct field of et split once into the
// mesh's pool (slots allocated on first use), the kernels then read pairs.
dg_status split_fields(const dg_mesh* mc, ExplTerms& et, cudaStream_t s) {
  dg_mesh* m = const_cast<dg_mesh*>(mc);
  const int64_t n = (int64_t)m->dim * m->ncell * m->nbu;
  const double* src[4];
  int nsrc = 0;
  const double** fields[4] = {&et.w[0], &et.w[1], &et.wb[0], &et.wb[1]};
  for (const double** f : fields) {
    int k = 0;
    while (k < nsrc && src[k] != *f) ++k;
    if (k == nsrc) {
      src[nsrc++] = *f;
      if (!m->ps_pool[k]) DG_CUDA(cudaMalloc(&m->ps_pool[k], sizeof(double) * n));
      const dg_status st = presplit(n, *f, m->ps_pool[k], s);
      if (st != DG_OK) return st;
    }
    *f = m->ps_pool[k];
  }
  return DG_OK;
}

template <typename A, int DIM, int N>
dg_status run_explicit_terms_a(const dg_mesh* m, const ExplTerms& et_in, int nt, double* rhs,
                               cudaStream_t s) {
  ExplTerms et = et_in;
  if constexpr (std::is_same<A, df64>::value) {
    const dg_status st = split_fields(m, et, s);
    if (st != DG_OK) return st;
  }
  constexpr int CPB = cpb_for<N, DIM>();
  constexpr int threads = ((CPB * Sh<N, DIM>::NB + 31) / 32) * 32;
  const unsigned blocks = (unsigned)((m->ncell + CPB - 1) / CPB);
  int64_t nface = 0;
  for (int ax = 0; ax < DIM; ++ax) nface += faces_of_axis(ax, m->n, m->periodic);
  const int64_t need = nface * Sh<N, DIM>::NF * DIM * (int64_t)sizeof(A);
  const bool face_once = (variant_split(m->tune[0][2]) || variant_split(m->tune[0][1])) && m->split_flux &&
                         need <= m->split_flux_bytes;
  if (face_once) {
    A* flux = static_cast<A*>(m->split_flux);
    const Grid g = make_grid<DIM>(m);
    const unsigned fb = (unsigned)((nface * Sh<N, DIM>::NF + 255) / 256);
    if (nt == 2) {
      launch(explicit_face_kernel<A, DIM, N, 2>, fb, 256, 0, s, g, tab_u<A>(m), et, flux);
      launch(explicit_cell_kernel<A, DIM, N, 2, CPB>, blocks, threads, 0, s, g, tab_u<A>(m), et, flux, rhs);
    } else {
      launch(explicit_face_kernel<A, DIM, N, 1>, fb, 256, 0, s, g, tab_u<A>(m), et, flux);
      launch(explicit_cell_kernel<A, DIM, N, 1, CPB>, blocks, threads, 0, s, g, tab_u<A>(m), et, flux, rhs);
    }
    count_launch();
    count_launch();
    DG_CUDA(cudaGetLastError());
    return DG_OK;
  }
  if (nt == 2)
    launch(explicit_terms_kernel<A, DIM, N, 2, CPB>, blocks, threads, 0, s, make_grid<DIM>(m), tab_u<A>(m), et, rhs);
  else
    launch(explicit_terms_kernel<A, DIM, N, 1, CPB>, blocks, threads, 0, s, make_grid<DIM>(m), tab_u<A>(m), et, rhs);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

template <int DIM, int N>
dg_status run_explicit_terms(const dg_mesh* m, const ExplTerms& et, int nt, double* rhs,
                             cudaStream_t s) {
  return m->fp64_arith ? run_explicit_terms_a<double, DIM, N>(m, et, nt, rhs, s)
                       : run_explicit_terms_a<df64, DIM, N>(m, et, nt, rhs, s);
}

template <int DIM, int N>
dg_status run_explicit(const dg_mesh* m, int mode, double visc, double adv, const double* w,
                       const double* wb, double* rhs, cudaStream_t s) {
  return m->fp64_arith ? run_explicit_a<double, DIM, N>(m, mode, visc, adv, w, wb, rhs, s)
                       : run_explicit_a<df64, DIM, N>(m, mode, visc, adv, w, wb, rhs, s);
}

template <typename A, int DIM, int N>
dg_status run_mass_grad_a(const dg_mesh* m, double mass, const double* um, const double* f,
                          const double* p, double* rhs, cudaStream_t s) {
  constexpr int CPB = cpb_for<N, DIM>();
  constexpr int threads = ((CPB * Sh<N, DIM>::NB + 31) / 32) * 32;
  const unsigned blocks = (unsigned)((m->ncell + CPB - 1) / CPB);
  launch(mass_grad_kernel<A, DIM, N, N - 1, CPB>, blocks, threads, 0, s, 
      make_grid<DIM>(m), tab_u<A>(m), tab_p<A>(m), tab_mix<A>(m), mass, um, f, p, rhs);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

template <int DIM, int N>
dg_status run_mass_grad(const dg_mesh* m, double mass, const double* um, const double* f,
                        const double* p, double* rhs, cudaStream_t s) {
  return m->fp64_arith ? run_mass_grad_a<double, DIM, N>(m, mass, um, f, p, rhs, s)
                       : run_mass_grad_a<df64, DIM, N>(m, mass, um, f, p, rhs, s);
}

template <typename A, int DIM, int N>
dg_status run_pressure_rhs_a(const dg_mesh* m, double alpha, double inv_tau, const double* uss,
                             const double* p_old, double* rhs, cudaStream_t s) {
  if constexpr (std::is_same<A, df64>::value) {  // the kernel reads uss pre-split
    dg_mesh* mm = const_cast<dg_mesh*>(m);
    const int64_t n = (int64_t)m->dim * m->ncell * m->nbu;
    if (!mm->ps_pool[0]) DG_CUDA(cudaMalloc(&mm->ps_pool[0], sizeof(double) * n));
    const dg_status st = presplit(n, uss, mm->ps_pool[0], s);
    if (st != DG_OK) return st;
    uss = mm->ps_pool[0];
  }
  constexpr int NP = N - 1;
  constexpr int CPB = cpb_for<NP, DIM>();
  constexpr int threads = ((CPB * Sh<NP, DIM>::NB + 31) / 32) * 32;
  const unsigned blocks = (unsigned)((m->ncell + CPB - 1) / CPB);
  launch(pressure_rhs_kernel<A, DIM, N, NP, CPB>, blocks, threads, 0, s, 
      make_grid<DIM>(m), tab_u<A>(m), tab_p<A>(m), tab_mix<A>(m), alpha, inv_tau, uss, p_old, rhs);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

template <int DIM, int N>
dg_status run_pressure_rhs(const dg_mesh* m, double alpha, double inv_tau, const double* uss,
                           const double* p_old, double* rhs, cudaStream_t s) {
  return m->fp64_arith ? run_pressure_rhs_a<double, DIM, N>(m, alpha, inv_tau, uss, p_old, rhs, s)
                       : run_pressure_rhs_a<df64, DIM, N>(m, alpha, inv_tau, uss, p_old, rhs, s);
}

template <typename A, int DIM, int N>
dg_status run_project_a(const dg_mesh* m, const double* p, double* ut, const double* base,
                        double tau, const double* sub, double* out, cudaStream_t s) {
  constexpr int CPB = cpb_for<N, DIM>();
  constexpr int threads = ((CPB * Sh<N, DIM>::NB + 31) / 32) * 32;
  const unsigned blocks = (unsigned)((m->ncell + CPB - 1) / CPB);
  launch(project_kernel<A, DIM, N, N - 1, CPB>, blocks, threads, 0, s, make_grid<DIM>(m), tab_mix<A>(m), p,
                                                                   ut, base, tau, sub, out);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

template <int DIM, int N>
dg_status run_project(const dg_mesh* m, const double* p, double* ut, const double* base,
                      double tau, const double* sub, double* out, cudaStream_t s) {
  return m->fp64_arith ? run_project_a<double, DIM, N>(m, p, ut, base, tau, sub, out, s)
                       : run_project_a<df64, DIM, N>(m, p, ut, base, tau, sub, out, s);
}

template <int DIM, int N>
dg_status run_diag(const dg_mesh* m, bool pressure, double mass, double visc, double adv,
                   const double* ub, double* diag, cudaStream_t s, bool fp32 = false, int inv_copies = 0) {
  constexpr int CPB = cpb_for<N, DIM>();
  constexpr int threads = ((CPB * Sh<N, DIM>::NB + 31) / 32) * 32;
  const unsigned blocks = (unsigned)((m->ncell + CPB - 1) / CPB);
  // the FP32 diagonal reads the float-pair copy of ubar when the mesh holds
  // one for this field (kept for a solve: keep_presplit_ubar)
  const bool pairs = fp32 && ub && m->ps_ub && m->ub_keep == ub && m->ub_split_of == ub;
  if (fp32)
    launch(diag_kernel<DIM, N, float, CPB>, blocks, threads, 0, s, 
        make_grid<DIM>(m), pressure ? m->tp32 : m->tu32, (float)mass, (float)visc, (float)adv,
        (float)(N * N), pressure ? 0 : 1, pairs ? (const double*)m->ps_ub : ub, pairs ? 1 : 0, diag,
        inv_copies);
  else
    launch(diag_kernel<DIM, N, double, CPB>, blocks, threads, 0, s, 
        make_grid<DIM>(m), pressure ? m->tp64 : m->tu64, mass, visc, adv, (double)(N * N),
        pressure ? 0 : 1, ub, 0, diag, inv_copies);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

// dispatch on (dim, velocity nodes) for velocity-space kernels
#define DG_DISPATCH_U(m, FN, ...)                                        \
  ((m)->dim == 2 ? ((m)->nu == 3 ? FN<2, 3>(__VA_ARGS__)                 \
                    : (m)->nu == 4 ? FN<2, 4>(__VA_ARGS__)               \
                                   : FN<2, 5>(__VA_ARGS__))              \
                 : ((m)->nu == 3 ? FN<3, 3>(__VA_ARGS__)                 \
                    : (m)->nu == 4 ? FN<3, 4>(__VA_ARGS__)               \
                                   : FN<3, 5>(__VA_ARGS__)))


}  // namespace

// internal entry used by the solver: the momentum diagonal in FP32
// arithmetic (it only scales the Jacobi preconditioner)
dg_status momentum_diagonal_fp32(const dg_mesh* m, const dg_momentum_coeffs* co, const double* ub,
                                 double* diag, cudaStream_t s) {
  if (!m->affine) return general_diag(m, false, co->mass, co->visc, co->adv, ub, diag, true, s);
  return DG_DISPATCH_U(m, run_diag, m, false, co->mass, co->visc, co->adv, ub, diag, s, true);
}

// internal entry used by the solver on affine meshes: the momentum Jacobi
// scaling 1/diag for all components in one pass (FP32 diagonal arithmetic,
// as above)
dg_status momentum_inv_diagonal_fp32(const dg_mesh* m, const dg_momentum_coeffs* co, const double* ub,
                                     double* dinv, cudaStream_t s) {
  if (!m->affine) {
    set_error("momentum_inv_diagonal_fp32: affine meshes only");
    return DG_EINVAL;
  }
  return DG_DISPATCH_U(m, run_diag, m, false, co->mass, co->visc, co->adv, ub, dinv, s, true, m->dim);
}

// out = base + tau (ut - sub) elementwise (sub may be null)
__global__ void __launch_bounds__(256)
    update_kernel(int64_t n, const double* __restrict__ base, double tau, const double* __restrict__ ut,
                  const double* __restrict__ sub, double* __restrict__ out) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = base[i] + tau * (sub ? ut[i] - sub[i] : ut[i]);
}

dg_status axpby_update(int64_t n, const double* base, double tau, const double* ut, const double* sub,
                       double* out, cudaStream_t s) {
  const int64_t want = (n + 255) / 256;
  const unsigned blocks = (unsigned)(want < 152 * 16 ? (want > 0 ? want : 1) : 152 * 16);
  launch(update_kernel, blocks, 256, 0, s, n, base, tau, ut, sub, out);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

// internal entry used by the solver: u~ = M^-1 P p into ut, and optionally
// out = base + tau (u~ - sub) in the same pass
dg_status project_fused(const dg_mesh* m, const double* p, double* ut, const double* base,
                        double tau, const double* sub, double* out, cudaStream_t s) {
  if (!m->affine) {
    dg_status st = general_project(m, p, ut, s);
    if (st != DG_OK || !out) return st;
    // trilinear cells: the update as a separate pass
    return axpby_update(m->ncell * m->nbu * m->dim, base, tau, ut, sub, out, s);
  }
  return DG_DISPATCH_U(m, run_project, m, p, ut, base, tau, sub, out, s);
}

// internal entry used by the solver: diagonal of a pressure-space operator
dg_status poisson_diagonal(const dg_mesh* m, double alpha, double* diag, cudaStream_t s) {
  if (!m->affine) return general_diag(m, true, alpha, 1.0, 0.0, nullptr, diag, false, s);
  switch (m->dim * 10 + m->np) {
    case 22: return run_diag<2, 2>(m, true, alpha, 1.0, 0.0, nullptr, diag, s);
    case 23: return run_diag<2, 3>(m, true, alpha, 1.0, 0.0, nullptr, diag, s);
    case 24: return run_diag<2, 4>(m, true, alpha, 1.0, 0.0, nullptr, diag, s);
    case 32: return run_diag<3, 2>(m, true, alpha, 1.0, 0.0, nullptr, diag, s);
    case 33: return run_diag<3, 3>(m, true, alpha, 1.0, 0.0, nullptr, diag, s);
    case 34: return run_diag<3, 4>(m, true, alpha, 1.0, 0.0, nullptr, diag, s);
  }
  set_error("poisson_diagonal: unsupported degree");
  return DG_EUNSUPPORTED;
}

}  // namespace dg

using namespace dg;

extern "C" {

dg_status dg_rhs_momentum(dg_mesh* m, const dg_momentum_rhs* d, double* rhs, void* stream) {
  if (!m || !d || !rhs || d->n_terms < 0 || d->n_terms > 2) {
    set_error("dg_rhs_momentum: bad argument");
    return DG_EINVAL;
  }
  for (int t = 0; t < d->n_terms; ++t) {
    if (!d->w[t] || (d->adv[t] != 0.0 && !d->wbar[t]) || d->w[t] == rhs || d->wbar[t] == rhs) {
      set_error("dg_rhs_momentum: bad explicit term");
      return DG_EINVAL;
    }
  }
  if (d->uD && !d->ubar) {
    set_error("dg_rhs_momentum: Dirichlet data need the stage's advecting field");
    return DG_EINVAL;
  }
  if (d->u_mass == rhs || d->p == rhs || d->uD == rhs || d->f == rhs || d->ubar == rhs) {
    set_error("dg_rhs_momentum: rhs aliases an input");
    return DG_EINVAL;
  }
  cudaStream_t s = as_stream(stream);
  dg_status st = m->affine ? DG_DISPATCH_U(m, run_mass_grad, m, d->mass, d->u_mass, d->f, d->p, rhs, s)
                           : general_mass_grad(m, d->mass, d->u_mass, d->f, d->p, rhs, s);
  if (st != DG_OK) return st;
  if (m->affine && d->n_terms > 0) {
    // all explicit terms in one pass; a term without advection still needs
    // a field for the shared-memory staging: its own w stands in (times 0)
    ExplTerms et;
    for (int t = 0; t < 2; ++t) {
      const int u = t < d->n_terms ? t : 0;
      et.visc[t] = t < d->n_terms ? d->visc[t] : 0.0;
      et.adv[t] = t < d->n_terms ? d->adv[t] : 0.0;
      et.w[t] = d->w[u];
      et.wb[t] = d->wbar[u] ? d->wbar[u] : d->w[u];
    }
    st = DG_DISPATCH_U(m, run_explicit_terms, m, et, d->n_terms, rhs, s);
    if (st != DG_OK) return st;
  }
  for (int t = 0; t < d->n_terms && !m->affine; ++t) {
    const double* wb = d->wbar[t] ? d->wbar[t] : d->w[t];
    st = general_explicit(m, 0, d->visc[t], d->adv[t], d->w[t], wb, rhs, s);
    if (st != DG_OK) return st;
  }
  bool walls = false;
  for (int a = 0; a < m->dim; ++a) walls |= !m->periodic[a];
  if (d->uD && walls) {
    st = m->affine
             ? DG_DISPATCH_U(m, run_explicit, m, 1, d->dir_visc, d->dir_adv, d->uD, d->ubar, rhs, s)
             : general_explicit(m, 1, d->dir_visc, d->dir_adv, d->uD, d->ubar, rhs, s);
    if (st != DG_OK) return st;
  }
  return DG_OK;
}

dg_status dg_project_gradient(dg_mesh* m, const double* p, double* ut, void* stream) {
  if (!m || !p || !ut) {
    set_error("dg_project_gradient: bad argument");
    return DG_EINVAL;
  }
  return project_fused(m, p, ut, nullptr, 0.0, nullptr, nullptr, as_stream(stream));
}

dg_status dg_rhs_pressure(dg_mesh* m, double alpha, double tau, const double* uss,
                          const double* p_old, double* rhs, void* stream) {
  if (!m || !uss || !p_old || !rhs || !(tau != 0.0) || rhs == p_old) {
    set_error("dg_rhs_pressure: bad argument");
    return DG_EINVAL;
  }
  if (!m->affine) return general_pressure_rhs(m, alpha, 1.0 / tau, uss, p_old, rhs, as_stream(stream));
  return DG_DISPATCH_U(m, run_pressure_rhs, m, alpha, 1.0 / tau, uss, p_old, rhs, as_stream(stream));
}

dg_status dg_momentum_diagonal(dg_mesh* m, const dg_momentum_coeffs* co, const double* ubar,
                               double* diag, void* stream) {
  if (!m || !co || !diag || (co->adv != 0.0 && !ubar)) {
    set_error("dg_momentum_diagonal: bad argument");
    return DG_EINVAL;
  }
  if (!m->affine)
    return general_diag(m, false, co->mass, co->visc, co->adv, ubar, diag, false, as_stream(stream));
  return DG_DISPATCH_U(m, run_diag, m, false, co->mass, co->visc, co->adv, ubar, diag,
                       as_stream(stream));
}

dg_status dg_poisson_diagonal(dg_mesh* m, double alpha, double* diag, void* stream) {
  if (!m || !diag) {
    set_error("dg_poisson_diagonal: bad argument");
    return DG_EINVAL;
  }
  return poisson_diagonal(m, alpha, diag, as_stream(stream));
}

}  // extern "C"
