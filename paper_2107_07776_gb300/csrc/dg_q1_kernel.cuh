// Scalar operator alpha M + visc K_SIP on Q1 elements (two Gauss points per
// direction, 3D, no advection: the pressure space of Q2/Q1 and every
// multigrid level after p-coarsening), one thread per cell.  With N = 2 a
// cell's 8 values, each face's 4 points and the 2 nodes on each normal line
// are compile-time indices, so the whole cell lives in registers: the cell
// term (sum factorisation, axis by axis), then the 6 faces one after
// another (the neighbour's 8 values, the SIP flux of Eqs. weakform_p_1 and
// the penalty of Eq. penconst1 at the 4 face points, lifted back onto the 2
// nodes of each normal line), then the plain or Chebyshev epilogue.  The
// arithmetic is term by term that of scalar_op_kernel, in the same order.
#pragma once

#include "dg_common.cuh"
#include "dg_df64.cuh"

namespace dg {

template <typename T, typename A>
__device__ __forceinline__ void q1_load(const T* __restrict__ p, bool vec, T out[8]) {
  if (vec) {
    if constexpr (sizeof(T) == 4) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(p));
      const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
      out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
      out[4] = b.x; out[5] = b.y; out[6] = b.z; out[7] = b.w;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(p) + q);
        out[2 * q] = a.x;
        out[2 * q + 1] = a.y;
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) out[i] = __ldg(p + i);
  }
}

// node of a Q1 cell with coordinate i along axis ax and tangential index t
// (the other two axes in increasing order, t = t0 + 2 t1)
__host__ __device__ constexpr int q1_node(int ax, int i, int t) {
  return ax == 0 ? i + 2 * t : (ax == 1 ? (t & 1) + 2 * i + 4 * (t >> 1) : t + 4 * i);
}

template <typename T, typename A>
__global__ void __launch_bounds__(128)
    q1_cell_kernel(const __grid_constant__ OpArgs<T> a, const __grid_constant__ Tab1D<A> tb,
                   const T* __restrict__ src, T* __restrict__ dst) {
  pdl_entry();
  using Ar = Arith<A>;
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= a.ncell) return;
  const A zero = Ar::c(0.0), half = Ar::c(0.5), two = Ar::c(2.0);
  const A mass = Ar::from(a.mass), visc = Ar::from(a.visc), pen = Ar::from(a.pen);
  int ci[3];
  lex_coords(cell, a.n0, a.n1, ci);
  const A h[3] = {Ar::from(a.h0[ci[0]]), Ar::from(a.h1[ci[1]]), Ar::from(a.h2[ci[2]])};
  const A hi[3] = {Ar::from(a.hi0[ci[0]]), Ar::from(a.hi1[ci[1]]), Ar::from(a.hi2[ci[2]])};
  // 16-byte vector access when every base pointer allows it (a cell's 8
  // values then start on a 32- or 64-byte boundary)
  uintptr_t align = reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst);
  if (a.cheb)
    align |= reinterpret_cast<uintptr_t>(a.cx) | reinterpret_cast<uintptr_t>(a.cr) |
             reinterpret_cast<uintptr_t>(a.cdinv);
  const bool vec = (align & 15u) == 0;
  T ut[8];
  q1_load<T, A>(src + cell * 8, vec, ut);
  A u[8], W[8], y[8];
#pragma unroll
  for (int nd = 0; nd < 8; ++nd) {
    u[nd] = Ar::from(ut[nd]);
    W[nd] = tb.w[nd & 1] * tb.w[(nd >> 1) & 1] * h[0] * h[1] * tb.w[nd >> 2] * h[2];
    y[nd] = mass * W[nd] * u[nd];
  }
  // cell term: y += hi_b D_b^T (W visc hi_b D_b u), axis by axis
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    A q[8];
#pragma unroll
    for (int nd = 0; nd < 8; ++nd) {
      const int ib = (nd >> b) & 1, lo = nd & ~(1 << b), up = lo | (1 << b);
      A du = zero;
      du += tb.D[ib][0] * u[lo];
      du += tb.D[ib][1] * u[up];
      q[nd] = W[nd] * (visc * du * hi[b]);
    }
#pragma unroll
    for (int nd = 0; nd < 8; ++nd) {
      const int ib = (nd >> b) & 1, lo = nd & ~(1 << b), up = lo | (1 << b);
      A acc = zero;
      acc += tb.D[0][ib] * q[lo];
      acc += tb.D[1][ib] * q[up];
      y[nd] += acc * hi[b];
    }
  }
  // faces, in the order of the cell-centric kernel's lifting (axis, side)
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const int cax = ci[ax];
    const int nax = ax == 0 ? a.n0 : (ax == 1 ? a.n1 : a.n2);
    const int per = ax == 0 ? a.per0 : (ax == 1 ? a.per1 : a.per2);
    const int64_t cstr = ax == 0 ? 1 : (ax == 1 ? (int64_t)a.n0 : (int64_t)a.n0 * a.n1);
    const T* hiax = ax == 0 ? a.hi0 : (ax == 1 ? a.hi1 : a.hi2);
    const int b0 = ax == 0 ? 1 : 0, b1 = ax == 2 ? 1 : 2;  // tangential axes
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const A sgn = s ? Ar::c(1.0) : Ar::c(-1.0);
      int cn = cax + (s ? 1 : -1);
      bool interior = true;
      if (cn < 0 || cn >= nax) {
        if (per) cn = cn < 0 ? nax - 1 : 0;
        else interior = false;
      }
      if (!interior && !a.walls) continue;  // Neumann: no face terms
      const A hiK = hi[ax];
      A hiN = zero;
      T vt[8];
      if (interior) {
        hiN = Ar::from(hiax[cn]);
        q1_load<T, A>(src + (cell + (int64_t)(cn - cax) * cstr) * 8, vec, vt);
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int n0 = q1_node(ax, 0, t), n1 = q1_node(ax, 1, t);
        A wt = Ar::c(1.0);
        wt = wt * tb.w[t & 1] * h[b0];
        wt = wt * tb.w[t >> 1] * h[b1];
        A uin = zero, dnin = zero;
        uin = Ar::fma(tb.L[s][0], u[n0], uin);
        dnin = Ar::fma(tb.dL[s][0], u[n0], dnin);
        uin = Ar::fma(tb.L[s][1], u[n1], uin);
        dnin = Ar::fma(tb.dL[s][1], u[n1], dnin);
        dnin = dnin * sgn * hiK;
        A fv, fg;
        if (interior) {
          const A v0 = Ar::from(vt[n0]), v1 = Ar::from(vt[n1]);
          A uout = zero, dnout = zero;
          uout = Ar::fma(tb.L[1 - s][0], v0, uout);
          dnout = Ar::fma(tb.dL[1 - s][0], v0, dnout);
          uout = Ar::fma(tb.L[1 - s][1], v1, uout);
          dnout = Ar::fma(tb.dL[1 - s][1], v1, dnout);
          dnout = dnout * sgn * hiN;
          const A Cpen = half * pen * (hiK + hiN);
          const A jump = uin - uout;
          fv = visc * (Cpen * jump - half * (dnin + dnout));
          fg = -(half * visc * jump);
        } else {
          const A sig = pen * hiK;
          fv = visc * (two * sig * uin - dnin);
          fg = -(visc * uin);
        }
        const A f0 = wt * fv, f1 = wt * fg * sgn * hiK;
        y[n0] += f0 * tb.L[s][0] + f1 * tb.dL[s][0];
        y[n1] += f0 * tb.L[s][1] + f1 * tb.dL[s][1];
      }
    }
  }
  const int64_t o = cell * 8;
  T yt[8];
#pragma unroll
  for (int nd = 0; nd < 8; ++nd) yt[nd] = sizeof(T) == 8 ? (T)Ar::to_d(y[nd]) : (T)Ar::to_f(y[nd]);
  if (a.cheb) {
    // x += d; r -= dinv y; dst = c1 d + c2 r
#pragma unroll
    for (int nd = 0; nd < 8; ++nd) {
      const T dk = ut[nd];
      a.cx[o + nd] += dk;
      const T rk = a.cr[o + nd] - a.cdinv[o + nd] * yt[nd];
      a.cr[o + nd] = rk;
      dst[o + nd] = a.cc1 * dk + a.cc2 * rk;
    }
  } else if (vec) {
    if constexpr (sizeof(T) == 4) {
      reinterpret_cast<float4*>(dst + o)[0] = make_float4(yt[0], yt[1], yt[2], yt[3]);
      reinterpret_cast<float4*>(dst + o)[1] = make_float4(yt[4], yt[5], yt[6], yt[7]);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) reinterpret_cast<double2*>(dst + o)[q] = make_double2(yt[2 * q], yt[2 * q + 1]);
    }
  } else {
#pragma unroll
    for (int nd = 0; nd < 8; ++nd) dst[o + nd] = yt[nd];
  }
}

}  // namespace dg
