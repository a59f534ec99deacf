// Face-once variant of the affine operator kernel: the same operator as
// scalar_op_kernel, in two launches.
//
//  1. face_flux_kernel: one thread per face point of every face, each face
//     once.  It takes both sides' traces and normal derivatives (and the
//     advecting field's normal traces), forms the SIP + LF flux of Section 3
//     and stores the pair (F0, G) = (w_t fv, w_t fg) per face point and
//     component, in the orientation of the face's lower-side cell.  The
//     upper-side cell sees the antisymmetric pair: its value flux is -F0, and
//     its normal-derivative coefficient is G times its own inverse extent
//     (for both sides).  Wall faces store the one-sided flux of their single
//     cell in the same convention.
//  2. cell_split_kernel: the volume terms (as in scalar_op_kernel) plus the
//     stored fluxes of the cell's 2d faces.
//
// Every face is evaluated once instead of once per side, which removes
// about half of the face arithmetic.  The flux pairs make a round trip
// through L2/HBM: 2 values per face point and component.  Results equal
// those of the single-kernel variant up to rounding order; each output is
// still written once, without atomics.
#pragma once

#include "dg_common.cuh"
#include "dg_df64.cuh"
#include "dg_faces.cuh"

namespace dg {

template <typename T, typename A, int DIM, int N, bool ADV>
__global__ void __launch_bounds__(256)
    face_flux_kernel(const __grid_constant__ OpArgs<T> a, const __grid_constant__ Tab1D<A> tb,
                     const T* __restrict__ src, const T* __restrict__ ub, A* __restrict__ flux) {
  pdl_entry();
  using Ar = Arith<A>;
  constexpr int NB = Shape<N, DIM>::NB, NF = Shape<N, DIM>::NF;
  const int n[3] = {a.n0, a.n1, a.n2};
  const int per[3] = {a.per0, a.per1, a.per2};
  const int64_t f0 = faces_of_axis(0, n, per), f1 = faces_of_axis(1, n, per);
  const int64_t f2 = DIM == 3 ? faces_of_axis(2, n, per) : 0;
  const int64_t nface = f0 + f1 + f2;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nface * NF) return;
  const int t = (int)(gid % NF);
  int64_t fg = gid / NF;  // global face index (axis 0 faces, then 1, then 2)
  int ax;
  int64_t fl;
  if (fg < f0) {
    ax = 0;
    fl = fg;
  } else if (fg < f0 + f1) {
    ax = 1;
    fl = fg - f0;
  } else {
    ax = 2;
    fl = fg - f0 - f1;
  }
  // face coordinates
  const int d0 = ax == 0 ? face_layers(n[0], per[0]) : n[0];
  const int d1 = ax == 1 ? face_layers(n[1], per[1]) : n[1];
  int fc[3];
  lex_coords(fl, d0, d1, fc);
  const int layer = pick3(ax, fc[0], fc[1], fc[2]);
  const int nax = pick3(ax, n[0], n[1], n[2]);
  const bool pax = pick3(ax, per[0], per[1], per[2]) != 0;
  // cells on both sides (lower side L: the face is its upper face)
  const int cl_ax = pax ? (layer - 1 + nax) % nax : layer - 1;
  const int cr_ax = layer;
  const bool hasL = pax || layer >= 1, hasR = pax || layer < nax;
  const int64_t cstr = ax == 0 ? 1 : (ax == 1 ? (int64_t)n[0] : (int64_t)n[0] * n[1]);
  const int64_t cbase = (ax == 0 ? 0 : fc[0]) + (int64_t)n[0] * ((ax == 1 ? 0 : fc[1]) +
                                                             (int64_t)n[1] * (ax == 2 ? 0 : fc[2]));
  const int64_t cL = cbase + (int64_t)cl_ax * cstr, cR = cbase + (int64_t)cr_ax * cstr;
  const T* hiax = ax == 0 ? a.hi0 : (ax == 1 ? a.hi1 : a.hi2);
  const A zero = Ar::c(0.0), half = Ar::c(0.5), two = Ar::c(2.0);
  const A visc = ld_val<T, A>(a.visc), advc = ld_val<T, A>(a.adv), pen = ld_val<T, A>(a.pen);
  const A hiL = hasL ? ld_val<T, A>(hiax[cl_ax]) : zero, hiR = hasR ? ld_val<T, A>(hiax[cr_ax]) : zero;
  // tangential weight: face quadrature weight times the face measure
  A wt = Ar::c(1.0);
  {
    int tt = t;
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      if (b == ax) continue;
      const T* hb = b == 0 ? a.h0 : (b == 1 ? a.h1 : a.h2);
      wt = wt * tb.w[tt % N] * ld_val<T, A>(hb[pick3(b, fc[0], fc[1], fc[2])]);
      tt /= N;
    }
  }
  // normal traces of the advecting field along +e_ax
  A unL = zero, unR = zero;
  if (ADV) {
    const T* uba = ub + (int64_t)ax * a.ncell * NB;
    SumOf<A> sL, sR;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int nd = node_of(N, ax, i, t, DIM);
      if (hasL) {
        const A v = ld_val<T, A>(__ldg(&uba[cL * NB + nd]));
        if (i == 0) sL.start(tb.L[1][i], v);
        else sL.fma(tb.L[1][i], v);
      }
      if (hasR) {
        const A v = ld_val<T, A>(__ldg(&uba[cR * NB + nd]));
        if (i == 0) sR.start(tb.L[0][i], v);
        else sR.fma(tb.L[0][i], v);
      }
    }
    if (hasL) unL = sL.value();
    if (hasR) unR = sR.value();
  }
  // Flux coefficients of this face point, the same for every component.
  // Interior face (normal +e_ax, seen from the lower cell L), with C the
  // penalty average and lambda = max(|unL|, |unR|):
  //   F0 = aL uL + aR uR + cDL dL + cDR dR,   G = cG (uL - uR)
  //   aL = wt (visc C + adv (unL + lambda)/2), aR = wt (adv (unR - lambda)/2 - visc C)
  //   cDL = -wt visc hiL / 2, cDR = -wt visc hiR / 2, cG = -wt visc / 2
  // (the SIP terms and the LF flux of Section 3 with the traces u and the
  // reference normal derivatives d of both sides).  Wall face of one cell
  // (sg = -1 when the wall is the cell's lower face): with its trace u_in,
  // derivative d_in and sigma = pen / h,
  //   F0 = aL u_in + cDL d_in,  G = cG u_in
  //   aL = sg wt (2 visc sigma + adv |un|), cDL = -wt visc / h, cG = -sg wt visc
  // so that the reader's rule (value flux -F0 below, +F0 above; derivative
  // coefficient G over its own extent) reproduces the one-sided flux.
  const bool interior = hasL && hasR;
  const bool low = hasR;  // on a wall: the wall is the lower face of cell R
  A aL = zero, aR = zero, cDL = zero, cDR = zero, cG = zero;
  if (interior) {
    const A Cv = visc * (half * pen * (hiL + hiR));
    const A hw = half * (wt * visc);
    if (ADV) {
      const A lam = Ar::max(Ar::abs(unL), Ar::abs(unR));
      const A ha = half * advc;
      aL = wt * (Cv + ha * (unL + lam));
      aR = wt * (ha * (unR - lam) - Cv);
    } else {
      aL = wt * Cv;
      aR = -aL;
    }
    cDL = -(hw * hiL);
    cDR = -(hw * hiR);
    cG = -hw;
  } else if (a.walls) {
    const A hin = low ? hiR : hiL;
    const A wv = wt * visc;
    A base = two * (wv * (pen * hin));
    if (ADV) base = base + wt * (advc * Ar::abs(low ? unR : unL));
    aL = low ? -base : base;
    cDL = -(wv * hin);
    cG = low ? wv : -wv;
  }
  for (int c = 0; c < a.ncomp; ++c) {
    const T* srcc = src + (int64_t)c * a.ncell * NB;
    A F0 = zero, G = zero;
    if (interior) {
      SumOf<A> uL, dL, uR, dR;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int nd = node_of(N, ax, i, t, DIM);
        const A vl = ld_val<T, A>(__ldg(&srcc[cL * NB + nd]));
        const A vr = ld_val<T, A>(__ldg(&srcc[cR * NB + nd]));
        if (i == 0) {
          uL.start(tb.L[1][i], vl);
          dL.start(tb.dL[1][i], vl);
          uR.start(tb.L[0][i], vr);
          dR.start(tb.dL[0][i], vr);
        } else {
          uL.fma(tb.L[1][i], vl);
          dL.fma(tb.dL[1][i], vl);
          uR.fma(tb.L[0][i], vr);
          dR.fma(tb.dL[0][i], vr);
        }
      }
      const A ul = uL.value(), ur = uR.value();
      SumOf<A> f;
      f.start(aL, ul);
      f.fma(aR, ur);
      f.fma(cDL, dL.value());
      f.fma(cDR, dR.value());
      F0 = f.value();
      G = cG * (ul - ur);
    } else if (a.walls) {
      const int64_t cin = low ? cR : cL;
      const int sd = low ? 0 : 1;
      SumOf<A> ui, di;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const A v = ld_val<T, A>(__ldg(&srcc[cin * NB + node_of(N, ax, i, t, DIM)]));
        if (i == 0) {
          ui.start(tb.L[sd][i], v);
          di.start(tb.dL[sd][i], v);
        } else {
          ui.fma(tb.L[sd][i], v);
          di.fma(tb.dL[sd][i], v);
        }
      }
      const A u_in = ui.value();
      SumOf<A> f;
      f.start(aL, u_in);
      f.fma(cDL, di.value());
      F0 = f.value();
      G = cG * u_in;
    }
    A* fo = flux + ((c * nface + fg) * NF + t) * 2;
    fo[0] = F0;
    fo[1] = G;
  }
}

template <typename T, typename A, int DIM, int N, bool ADV, int CPB, int MINB>
__global__ void __launch_bounds__(((CPB * Shape<N, DIM>::NB + 31) / 32) * 32, MINB)
    cell_split_kernel(const __grid_constant__ OpArgs<T> a, const __grid_constant__ Tab1D<A> tb,
                      const T* __restrict__ src, const T* __restrict__ ub,
                      const A* __restrict__ flux, T* __restrict__ dst) {
  pdl_entry();
  using Ar = Arith<A>;
  constexpr int NB = Shape<N, DIM>::NB, NF = Shape<N, DIM>::NF;
  __shared__ A s_u[CPB][NB];
  __shared__ A s_q[DIM][CPB][NB];
  __shared__ __align__(16) A s_fl[CPB][NB][2 * DIM][2];
  // the thread's own gradient-term factors (cv, ca), kept in shared memory
  // rather than registers: more resident CTAs per SM
  __shared__ A s_cva[CPB][NB][2 * DIM];
  const int tid = threadIdx.x;
  const int cl = tid / NB, node = tid - (tid / NB) * NB;
  const int64_t cell = (int64_t)blockIdx.x * CPB + cl;
  const bool active = cl < CPB && cell < a.ncell;
  const A zero = Ar::c(0.0);
  const int n[3] = {a.n0, a.n1, a.n2};
  const int per[3] = {a.per0, a.per1, a.per2};
  const int64_t f0 = faces_of_axis(0, n, per), f1 = faces_of_axis(1, n, per);
  const int64_t f2 = DIM == 3 ? faces_of_axis(2, n, per) : 0;
  const int64_t nface = f0 + f1 + f2;
  int ci[3] = {0, 0, 0};
  const int ii[3] = {node % N, (node / N) % N, DIM == 3 ? node / (N * N) : 0};
  // per-node coefficients, the same for every component: the mass weight
  // mass W, the gradient-term factors visc W / h_b^2 and -adv W ubar_b / h_b
  // (both inverse extents of the gradient and its transpose folded in), and
  // the normal-derivative weights L_i'(s) / h_b of the face terms
  A cm = zero, gdl[DIM][2];
#pragma unroll
  for (int b = 0; b < DIM; ++b) gdl[b][0] = gdl[b][1] = zero;
  if (active) {
    lex_coords(cell, a.n0, a.n1, ci);
    A h[3], hi[3];
    h[0] = ld_val<T, A>(a.h0[ci[0]]);
    h[1] = ld_val<T, A>(a.h1[ci[1]]);
    hi[0] = ld_val<T, A>(a.hi0[ci[0]]);
    hi[1] = ld_val<T, A>(a.hi1[ci[1]]);
    h[2] = hi[2] = Ar::c(1.0);
    if (DIM == 3) {
      h[2] = ld_val<T, A>(a.h2[ci[2]]);
      hi[2] = ld_val<T, A>(a.hi2[ci[2]]);
    }
    A W = tb.w[ii[0]] * tb.w[ii[1]] * h[0] * h[1];
    if (DIM == 3) W = W * tb.w[ii[2]] * h[2];
    cm = ld_val<T, A>(a.mass) * W;
    const A vW = ld_val<T, A>(a.visc) * W, aW = -(ld_val<T, A>(a.adv) * W);
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      s_cva[cl][node][b] = vW * hi[b] * hi[b];
      s_cva[cl][node][DIM + b] =
          ADV ? aW * hi[b] * ld_val<T, A>(ub[((int64_t)b * a.ncell + cell) * NB + node]) : zero;
      gdl[b][0] = tb.dL[0][ii[b]] * hi[b];
      gdl[b][1] = tb.dL[1][ii[b]] * hi[b];
    }
  }
  // face indices of this node's 2d face points (the same for every component)
  int64_t fpos[2 * DIM];
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    const int t = tang_of<N, DIM>(b, ii);
    const int64_t foff = b == 0 ? 0 : (b == 1 ? f0 : f0 + f1);
    const int cb = ci[b], nb_ = n[b];
    const int lo = cb, hi_l = per[b] ? (cb + 1) % nb_ : cb + 1;
    fpos[2 * b] = (foff + face_index(b, lo, ci, n, per)) * NF + t;
    fpos[2 * b + 1] = (foff + face_index(b, hi_l, ci, n, per)) * NF + t;
  }
  for (int c = 0; c < a.ncomp; ++c) {
    const T* srcc = src + (int64_t)c * a.ncell * NB;
    // this component's flux pairs (F0, G) at the node's 2d face points,
    // copied asynchronously into the thread's own shared-memory slots first,
    // so that their latency overlaps the cell-term phase
    if (active) {
      const A* fl = flux + (int64_t)c * nface * NF * 2;
#pragma unroll
      for (int q = 0; q < 2 * DIM; ++q) cp_async<2 * sizeof(A)>(&s_fl[cl][node][q][0], fl + fpos[q] * 2);
    }
    cp_async_commit();
    if (active) s_u[cl][node] = ld_val<T, A>(srcc[cell * NB + node]);
    __syncthreads();
    if (active) {
      const A u = s_u[cl][node];
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        SumOf<A> du;
#pragma unroll
        for (int m = 0; m < N; ++m) {
          int j[3] = {ii[0], ii[1], ii[2]};
          j[b] = m;
          const A v = s_u[cl][j[0] + N * (j[1] + N * j[2])];
          if (m == 0) du.start(tb.D[ii[b]][m], v);
          else du.fma(tb.D[ii[b]][m], v);
        }
        SumOf<A> q;
        q.start(s_cva[cl][node][b], du.value());
        if (ADV) q.fma(s_cva[cl][node][DIM + b], u);
        s_q[b][cl][node] = q.value();
      }
    }
    __syncthreads();
    if (active) {
      // one partial sum per direction (the mass term joins the first), so
      // that the three dependency chains interleave; merged at the end
      SumOf<A> y[DIM];
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
#pragma unroll
        for (int m = 0; m < N; ++m) {
          int j[3] = {ii[0], ii[1], ii[2]};
          j[b] = m;
          const A q = s_q[b][cl][j[0] + N * (j[1] + N * j[2])];
          if (m == 0) y[b].start(tb.D[m][ii[b]], q);
          else y[b].fma(tb.D[m][ii[b]], q);
        }
      }
      y[0].fma(cm, s_u[cl][node]);
      cp_async_wait_all();  // the thread's own copies (no barrier needed)
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const A F0 = s_fl[cl][node][2 * b + s][0], G = s_fl[cl][node][2 * b + s][1];
          y[b].fma(s ? F0 : -F0, tb.L[s][ii[b]]);
          y[b].fma(G, gdl[b][s]);
        }
      }
#pragma unroll
      for (int b = 1; b < DIM; ++b) y[0].merge(y[b]);
      const A yv = y[0].value();
      const int64_t o = (int64_t)c * a.ncell * NB + cell * NB + node;
      const T yt = sizeof(T) == 8 ? (T)Ar::to_d(yv) : (T)Ar::to_f(yv);
      op_epilogue(a, o, yt, dst);
    }
    __syncthreads();
  }
}

// Components-interleaved cell pass of the face-once form (NC components,
// 1 or DIM): the volume sums of all components run between the same two
// barriers -- NC x DIM independent dependency chains per phase instead of
// NC sequential phase pairs with a barrier each -- and the flux pairs of all
// components are staged per face into shared memory by asynchronous copies
// issued at entry, each face point once per cell rather than once per node
// (a third of the shared memory of the per-node staging).  Dynamic shared
// memory: NcSplitSmem::bytes.
template <typename A, int DIM, int N, int NC, int CPB>
struct NcSplitSmem {
  static constexpr int NB = Shape<N, DIM>::NB, NF = Shape<N, DIM>::NF;
  static constexpr int kAlign = 16 / (int)sizeof(A);  // elements per 16 bytes
  static constexpr int u = 0;
  static constexpr int q = u + NC * CPB * NB;
  static constexpr int fl = (q + NC * DIM * CPB * NB + kAlign - 1) / kAlign * kAlign;
  static constexpr int cva = fl + CPB * NC * 2 * DIM * NF * 2;
  static constexpr int bytes = (int)sizeof(A) * (cva + CPB * NB * 2 * DIM);
};

template <typename T, typename A, int DIM, int N, int NC, bool ADV, int CPB, int MINB>
__global__ void __launch_bounds__(((CPB * Shape<N, DIM>::NB + 31) / 32) * 32, MINB)
    cell_split_nc_kernel(const __grid_constant__ OpArgs<T> a, const __grid_constant__ Tab1D<A> tb,
                         const T* __restrict__ src, const T* __restrict__ ub,
                         const A* __restrict__ flux, T* __restrict__ dst) {
  pdl_entry();
  using Ar = Arith<A>;
  constexpr int NB = Shape<N, DIM>::NB, NF = Shape<N, DIM>::NF;
  constexpr int NFC = 2 * DIM * NF;  // face points of a cell
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // [NC][CPB][NB] values, [NC][DIM][CPB][NB] gradient terms, then the flux
  // pairs [CPB][NC][2 DIM][NF][2] and the per-node factors [CPB][NB][2 DIM]
  using L = NcSplitSmem<A, DIM, N, NC, CPB>;
  A* s_u = reinterpret_cast<A*>(smem_raw) + L::u;
  A* s_q = reinterpret_cast<A*>(smem_raw) + L::q;
  A* s_fl = reinterpret_cast<A*>(smem_raw) + L::fl;
  A* s_cva = reinterpret_cast<A*>(smem_raw) + L::cva;
  const int tid = threadIdx.x;
  const int cl = tid / NB, node = tid - (tid / NB) * NB;
  const int64_t cell = (int64_t)blockIdx.x * CPB + cl;
  const bool active = cl < CPB && cell < a.ncell;
  const A zero = Ar::c(0.0);
  const int n[3] = {a.n0, a.n1, a.n2};
  const int per[3] = {a.per0, a.per1, a.per2};
  const int64_t f0 = faces_of_axis(0, n, per), f1 = faces_of_axis(1, n, per);
  const int64_t f2 = DIM == 3 ? faces_of_axis(2, n, per) : 0;
  const int64_t nface = f0 + f1 + f2;
  int ci[3] = {0, 0, 0};
  const int ii[3] = {node % N, (node / N) % N, DIM == 3 ? node / (N * N) : 0};
  if (active) lex_coords(cell, a.n0, a.n1, ci);
  // the cell's faces (2b: lower, 2b+1: upper face of axis b), global indices
  int64_t fidx[2 * DIM];
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    const int64_t foff = b == 0 ? 0 : (b == 1 ? f0 : f0 + f1);
    const int cb = ci[b], hi_l = per[b] ? (cb + 1) % n[b] : cb + 1;
    fidx[2 * b] = foff + face_index(b, cb, ci, n, per);
    fidx[2 * b + 1] = foff + face_index(b, hi_l, ci, n, per);
  }
  if (active) {
    A* fcell = s_fl + (int64_t)cl * NC * NFC * 2;
    for (int q = node; q < NC * NFC; q += NB) {
      const int c = q / NFC, r = q - c * NFC, f = r / NF, t = r - f * NF;
      int64_t F = fidx[0];
#pragma unroll
      for (int j = 1; j < 2 * DIM; ++j)
        if (f == j) F = fidx[j];
      cp_async<2 * sizeof(A)>(fcell + (int64_t)q * 2, flux + (((int64_t)c * nface + F) * NF + t) * 2);
    }
  }
  cp_async_commit();
  // per-node coefficients, the same for every component (as in
  // cell_split_kernel): mass weight, gradient-term factors, normal-derivative
  // weights of the face terms
  A cm = zero, gdl[DIM][2];
  A uo[NC];
#pragma unroll
  for (int b = 0; b < DIM; ++b) gdl[b][0] = gdl[b][1] = zero;
#pragma unroll
  for (int c = 0; c < NC; ++c) uo[c] = zero;
  if (active) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      uo[c] = ld_val<T, A>(src[((int64_t)c * a.ncell + cell) * NB + node]);
      s_u[(c * CPB + cl) * NB + node] = uo[c];
    }
    A h[3], hi[3];
    h[0] = ld_val<T, A>(a.h0[ci[0]]);
    h[1] = ld_val<T, A>(a.h1[ci[1]]);
    hi[0] = ld_val<T, A>(a.hi0[ci[0]]);
    hi[1] = ld_val<T, A>(a.hi1[ci[1]]);
    h[2] = hi[2] = Ar::c(1.0);
    if (DIM == 3) {
      h[2] = ld_val<T, A>(a.h2[ci[2]]);
      hi[2] = ld_val<T, A>(a.hi2[ci[2]]);
    }
    A W = tb.w[ii[0]] * tb.w[ii[1]] * h[0] * h[1];
    if (DIM == 3) W = W * tb.w[ii[2]] * h[2];
    cm = ld_val<T, A>(a.mass) * W;
    const A vW = ld_val<T, A>(a.visc) * W, aW = -(ld_val<T, A>(a.adv) * W);
    A* cva = s_cva + ((int64_t)cl * NB + node) * 2 * DIM;
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      cva[b] = vW * hi[b] * hi[b];
      cva[DIM + b] = ADV ? aW * hi[b] * ld_val<T, A>(ub[((int64_t)b * a.ncell + cell) * NB + node]) : zero;
      gdl[b][0] = tb.dL[0][ii[b]] * hi[b];
      gdl[b][1] = tb.dL[1][ii[b]] * hi[b];
    }
  }
  __syncthreads();
  if (active) {
    const A* cva = s_cva + ((int64_t)cl * NB + node) * 2 * DIM;
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      const A cv = cva[b], ca = ADV ? cva[DIM + b] : zero;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const A* uc = s_u + (c * CPB + cl) * NB;
        SumOf<A> du;
#pragma unroll
        for (int m = 0; m < N; ++m) {
          int j[3] = {ii[0], ii[1], ii[2]};
          j[b] = m;
          const A v = uc[j[0] + N * (j[1] + N * j[2])];
          if (m == 0) du.start(tb.D[ii[b]][m], v);
          else du.fma(tb.D[ii[b]][m], v);
        }
        SumOf<A> q;
        q.start(cv, du.value());
        if (ADV) q.fma(ca, uo[c]);
        s_q[((c * DIM + b) * CPB + cl) * NB + node] = q.value();
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
  if (active) {
    const A* fcell = s_fl + (int64_t)cl * NC * NFC * 2;
    int tq[DIM];
#pragma unroll
    for (int b = 0; b < DIM; ++b) tq[b] = tang_of<N, DIM>(b, ii);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      SumOf<A> y[DIM];  // one partial sum per direction, merged at the end
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        const A* qb = s_q + ((c * DIM + b) * CPB + cl) * NB;
#pragma unroll
        for (int m = 0; m < N; ++m) {
          int j[3] = {ii[0], ii[1], ii[2]};
          j[b] = m;
          const A q = qb[j[0] + N * (j[1] + N * j[2])];
          if (m == 0) y[b].start(tb.D[m][ii[b]], q);
          else y[b].fma(tb.D[m][ii[b]], q);
        }
      }
      y[0].fma(cm, uo[c]);
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const A* pr = fcell + ((c * 2 * DIM + 2 * b + s) * NF + tq[b]) * 2;
          const A F0 = pr[0], G = pr[1];
          y[b].fma(s ? F0 : -F0, tb.L[s][ii[b]]);
          y[b].fma(G, gdl[b][s]);
        }
      }
#pragma unroll
      for (int b = 1; b < DIM; ++b) y[0].merge(y[b]);
      const A yv = y[0].value();
      const int64_t o = (int64_t)c * a.ncell * NB + cell * NB + node;
      const T yt = sizeof(T) == 8 ? (T)Ar::to_d(yv) : (T)Ar::to_f(yv);
      op_epilogue(a, o, yt, dst);
    }
  }
}

}  // namespace dg
