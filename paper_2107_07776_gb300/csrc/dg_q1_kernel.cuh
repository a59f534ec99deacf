// Scalar operator alpha M + visc K_SIP on Q1 elements (two Gauss points per
// direction, 3D, no advection: the pressure space of Q2/Q1 and every
// multigrid level after p-coarsening), two threads per cell.  With N = 2 a
// cell's 8 values, each face's 4 points and the 2 nodes on each normal line
// are compile-time indices, so the cell lives in registers.  Thread h of a
// lane pair owns the 4 nodes of the z-layer i2 = h: it evaluates the x and y
// derivative terms and the x and y faces of its layer alone, the z
// derivative and the z face on its side (s = h) for the whole cell, and
// trades the halves that belong to its partner by warp shuffles.  Terms
// follow scalar_op_kernel (the SIP flux of Eqs. weakform_p_1, the penalty
// of Eq. penconst1) and are added to each node in the same order.
#pragma once

#include "dg_common.cuh"
#include "dg_df64.cuh"

#include <type_traits>

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

template <typename A>
__device__ __forceinline__ A shfl_pair(A v) {
  if constexpr (sizeof(A) == 8 && !std::is_same<A, double>::value) {  // float-float
    v.hi = __shfl_xor_sync(0xffffffffu, v.hi, 1);
    v.lo = __shfl_xor_sync(0xffffffffu, v.lo, 1);
    return v;
  } else {
    return __shfl_xor_sync(0xffffffffu, v, 1);
  }
}

template <typename T>
__device__ __forceinline__ void q1_load4(const T* __restrict__ p, bool vec, T out[4]) {
  if (vec) {
    if constexpr (sizeof(T) == 4) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(p));
      out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
    } else {
      const double2 a = __ldg(reinterpret_cast<const double2*>(p));
      const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
      out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) out[i] = __ldg(p + i);
  }
}

template <typename T, typename A>
__global__ void __launch_bounds__(128)
    q1_cell_kernel(const __grid_constant__ OpArgs<T> a, const __grid_constant__ Tab1D<A> tb,
                   const T* __restrict__ src, T* __restrict__ dst) {
  pdl_entry();
  using Ar = Arith<A>;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int h = (int)(gt & 1);  // the thread's z-layer
  // pairs are whole (2 ncell threads); threads past the end compute the last
  // cell again so that every lane takes part in the shuffles, and store nothing
  const bool active = (gt >> 1) < a.ncell;
  const int64_t cell = active ? (gt >> 1) : a.ncell - 1;
  const A zero = Ar::c(0.0), half = Ar::c(0.5), two = Ar::c(2.0);
  const A mass = ld_val<T, A>(a.mass), visc = ld_val<T, A>(a.visc), pen = ld_val<T, A>(a.pen);
  int ci[3];
  lex_coords(cell, a.n0, a.n1, ci);
  const A h3[3] = {ld_val<T, A>(a.h0[ci[0]]), ld_val<T, A>(a.h1[ci[1]]), ld_val<T, A>(a.h2[ci[2]])};
  const A hi[3] = {ld_val<T, A>(a.hi0[ci[0]]), ld_val<T, A>(a.hi1[ci[1]]), ld_val<T, A>(a.hi2[ci[2]])};
  uintptr_t align = reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst);
  if (a.cheb)
    align |= reinterpret_cast<uintptr_t>(a.cx) | reinterpret_cast<uintptr_t>(a.cr) |
             reinterpret_cast<uintptr_t>(a.cdinv);
  const bool vec = (align & 15u) == 0;
  T ut[8];
  q1_load<T, A>(src + cell * 8, vec, ut);
  A u[8];
#pragma unroll
  for (int nd = 0; nd < 8; ++nd) u[nd] = ld_val<T, A>(ut[nd]);
  // own nodes nd = 4 h + k (k = i0 + 2 i1), picked by selects (a run-time
  // index into u would put it in local memory)
  A uo[4], W[4], y[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    uo[k] = h ? u[4 + k] : u[k];
    W[k] = tb.w[k & 1] * tb.w[k >> 1] * h3[0] * h3[1] * tb.w[h] * h3[2];
    y[k] = mass * W[k] * uo[k];
  }
  // x and y derivative terms within the layer
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    A q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int ib = (k >> b) & 1, lo = k & ~(1 << b), up = lo | (1 << b);
      A du = zero;
      du += tb.D[ib][0] * uo[lo];
      du += tb.D[ib][1] * uo[up];
      q[k] = W[k] * (visc * du * hi[b]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int ib = (k >> b) & 1, lo = k & ~(1 << b), up = lo | (1 << b);
      A acc = zero;
      acc += tb.D[0][ib] * q[lo];
      acc += tb.D[1][ib] * q[up];
      y[k] += acc * hi[b];
    }
  }
  // z derivative: q on the own layer, the partner's layer by shuffle
  {
    A qo[4], qp[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      A du = zero;
      du += tb.D[h][0] * u[k];
      du += tb.D[h][1] * u[4 + k];
      qo[k] = W[k] * (visc * du * hi[2]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) qp[k] = shfl_pair(qo[k]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const A q0 = h == 0 ? qo[k] : qp[k], q1 = h == 0 ? qp[k] : qo[k];
      A acc = zero;
      acc += tb.D[0][h] * q0;
      acc += tb.D[1][h] * q1;
      y[k] += acc * hi[2];
    }
  }
  // x and y faces: the layer's 2 points on each
#pragma unroll
  for (int ax = 0; ax < 2; ++ax) {
    const int cax = ci[ax];
    const int nax = ax == 0 ? a.n0 : a.n1;
    const int per = ax == 0 ? a.per0 : a.per1;
    const int64_t cstr = ax == 0 ? 1 : (int64_t)a.n0;
    const T* hiax = ax == 0 ? a.hi0 : a.hi1;
    const int b0 = ax == 0 ? 1 : 0;  // tangential axes b0 and z
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
      T vt[4];  // the neighbour's layer h
      if (interior) {
        hiN = ld_val<T, A>(hiax[cn]);
        q1_load4<T>(src + (cell + (int64_t)(cn - cax) * cstr) * 8 + 4 * h, vec, vt);
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        // layer-local nodes on the normal line through tangential index j
        const int k0 = ax == 0 ? 2 * j : j, k1 = ax == 0 ? 2 * j + 1 : j + 2;
        A wt = Ar::c(1.0);
        wt = wt * tb.w[j] * h3[b0];
        wt = wt * tb.w[h] * h3[2];
        A uin = zero, dnin = zero;
        uin = Ar::fma(tb.L[s][0], uo[k0], uin);
        dnin = Ar::fma(tb.dL[s][0], uo[k0], dnin);
        uin = Ar::fma(tb.L[s][1], uo[k1], uin);
        dnin = Ar::fma(tb.dL[s][1], uo[k1], dnin);
        dnin = dnin * sgn * hiK;
        A fv, fg;
        if (interior) {
          const A v0 = ld_val<T, A>(vt[k0]), v1 = ld_val<T, A>(vt[k1]);
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
        y[k0] += f0 * tb.L[s][0] + f1 * tb.dL[s][0];
        y[k1] += f0 * tb.L[s][1] + f1 * tb.dL[s][1];
      }
    }
  }
  // z faces: this thread evaluates side s = h at all 4 points; the lift onto
  // the partner's layer is traded by shuffle, and each node adds side 0 first
  {
    const int s = h;
    const A sgn = s ? Ar::c(1.0) : Ar::c(-1.0);
    int cn = ci[2] + (s ? 1 : -1);
    bool interior = true;
    if (cn < 0 || cn >= a.n2) {
      if (a.per2) cn = cn < 0 ? a.n2 - 1 : 0;
      else interior = false;
    }
    const bool any = interior || a.walls;
    const A hiK = hi[2];
    A hiN = zero;
    T vt[8];
    if (interior) {
      hiN = ld_val<T, A>(a.hi2[cn]);
      q1_load<T, A>(src + (cell + (int64_t)(cn - ci[2]) * a.n0 * (int64_t)a.n1) * 8, vec, vt);
    }
    A c_own[4], c_par[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      c_own[t] = zero;
      c_par[t] = zero;
      if (any) {
        A wt = Ar::c(1.0);
        wt = wt * tb.w[t & 1] * h3[0];
        wt = wt * tb.w[t >> 1] * h3[1];
        A uin = zero, dnin = zero;
        uin = Ar::fma(tb.L[s][0], u[t], uin);
        dnin = Ar::fma(tb.dL[s][0], u[t], dnin);
        uin = Ar::fma(tb.L[s][1], u[4 + t], uin);
        dnin = Ar::fma(tb.dL[s][1], u[4 + t], dnin);
        dnin = dnin * sgn * hiK;
        A fv, fg;
        if (interior) {
          const A v0 = ld_val<T, A>(vt[t]), v1 = ld_val<T, A>(vt[4 + t]);
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
        // node t (layer 0) takes index 0 of the normal line, node 4 + t index 1
        const A c0 = f0 * tb.L[s][0] + f1 * tb.dL[s][0];
        const A c1 = f0 * tb.L[s][1] + f1 * tb.dL[s][1];
        c_own[t] = h == 0 ? c0 : c1;
        c_par[t] = h == 0 ? c1 : c0;
      }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const A from_partner = shfl_pair(c_par[t]);  // the partner's side, lifted onto this layer
      if (h == 0) {
        y[t] += c_own[t];
        y[t] += from_partner;
      } else {
        y[t] += from_partner;
        y[t] += c_own[t];
      }
    }
  }
  if (!active) return;
  const int64_t o = cell * 8 + 4 * h;
  T yt[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) yt[k] = sizeof(T) == 8 ? (T)Ar::to_d(y[k]) : (T)Ar::to_f(y[k]);
  if (a.cheb) {
#pragma unroll
    for (int k = 0; k < 4; ++k) op_epilogue(a, o + k, yt[k], dst);
  } else if (vec) {
    if constexpr (sizeof(T) == 4) {
      reinterpret_cast<float4*>(dst + o)[0] = make_float4(yt[0], yt[1], yt[2], yt[3]);
    } else {
      reinterpret_cast<double2*>(dst + o)[0] = make_double2(yt[0], yt[1]);
      reinterpret_cast<double2*>(dst + o)[1] = make_double2(yt[2], yt[3]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) dst[o + k] = yt[k];
  }
}

// The FP32 pressure operator alpha M^p + visc K on Q1 cells of a Cartesian
// mesh in tensor-product form, one thread per cell.  The mass is diagonal
// (alpha w_i0 h_0 w_i1 h_1 w_i2 h_2 per node) and K is the sum over the axes
// of the 1D SIP matrix along the axis times the tangential masses: along axis
// a, each of the cell's 4 lines takes its own 2x2 block and the blocks of its
// lower and upper neighbours' lines, all tabulated per axis cell at mesh
// setup (build_q1_tables).  The same operator as q1_cell_kernel, with the
// face terms folded into the tables instead of formed per face point.
template <int AX>
__device__ __forceinline__ void q1_line_block(const float4 K, const float v[8], const float mt[4], float s[8]) {
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int n0 = q1_node(AX, 0, t), n1 = q1_node(AX, 1, t);
    const float a0 = fmaf(K.y, v[n1], K.x * v[n0]);
    const float a1 = fmaf(K.w, v[n1], K.z * v[n0]);
    s[n0] = fmaf(mt[t], a0, s[n0]);
    s[n1] = fmaf(mt[t], a1, s[n1]);
  }
}

template <int AX>
__device__ __forceinline__ void q1_axis_terms(const OpArgs<float>& a, const float4* row, const int ci[3],
                                              int64_t cell, const float* __restrict__ src, bool vec,
                                              const float u[8], const float mt[4], float s[8]) {
  const int c = ci[AX], n = AX == 0 ? a.n0 : (AX == 1 ? a.n1 : a.n2);
  const int per = AX == 0 ? a.per0 : (AX == 1 ? a.per1 : a.per2);
  const int64_t stride = AX == 0 ? 1 : (AX == 1 ? (int64_t)a.n0 : (int64_t)a.n0 * a.n1);
  q1_line_block<AX>(__ldg(row + 1), u, mt, s);
#pragma unroll
  for (int sd = 0; sd < 2; ++sd) {
    int cn = c + (sd ? 1 : -1);
    if (cn < 0 || cn >= n) {
      if (!per) continue;  // wall: the pressure operator has no face terms there
      cn = cn < 0 ? n - 1 : 0;
    }
    float v[8];
    q1_load<float, float>(src + (cell + (int64_t)(cn - c) * stride) * 8, vec, v);
    q1_line_block<AX>(__ldg(row + 2 + sd), v, mt, s);
  }
}

template <typename T>
__global__ void __launch_bounds__(128)
    q1_tensor_kernel(const __grid_constant__ OpArgs<T> a, const T* __restrict__ src, T* __restrict__ dst) {
  pdl_entry();
  static_assert(std::is_same<T, float>::value, "q1_tensor_kernel: FP32 only");
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= a.ncell) return;
  int ci[3];
  lex_coords(cell, a.n0, a.n1, ci);
  const float4* r0 = a.q1tab + 4 * (int64_t)ci[0];
  const float4* r1 = a.q1tab + 4 * ((int64_t)a.q1tab_off1 + ci[1]);
  const float4* r2 = a.q1tab + 4 * ((int64_t)a.q1tab_off2 + ci[2]);
  const float4 w0 = __ldg(r0), w1 = __ldg(r1), w2 = __ldg(r2);  // (w_0 h, w_1 h, -, -) per axis
  uintptr_t align = reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst);
  const bool vec = (align & 15u) == 0;
  // the epilogue's vectors too (a null pointer is aligned)
  const bool vec_all = vec && ((reinterpret_cast<uintptr_t>(a.cx) | reinterpret_cast<uintptr_t>(a.cr) |
                                reinterpret_cast<uintptr_t>(a.cdinv) | reinterpret_cast<uintptr_t>(a.csrc)) &
                               15u) == 0;
  float u[8], s[8];
  q1_load<float, float>(src + cell * 8, vec, u);
#pragma unroll
  for (int k = 0; k < 8; ++k) s[k] = 0.0f;
  {  // axis 0: lines t = i1 + 2 i2
    const float mt[4] = {w1.x * w2.x, w1.y * w2.x, w1.x * w2.y, w1.y * w2.y};
    q1_axis_terms<0>(a, r0, ci, cell, src, vec, u, mt, s);
  }
  {  // axis 1: lines t = i0 + 2 i2
    const float mt[4] = {w0.x * w2.x, w0.y * w2.x, w0.x * w2.y, w0.y * w2.y};
    q1_axis_terms<1>(a, r1, ci, cell, src, vec, u, mt, s);
  }
  {  // axis 2: lines t = i0 + 2 i1
    const float mt[4] = {w0.x * w1.x, w0.y * w1.x, w0.x * w1.y, w0.y * w1.y};
    q1_axis_terms<2>(a, r2, ci, cell, src, vec, u, mt, s);
  }
  float y[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float m = ((k & 1) ? w0.y : w0.x) * ((k & 2) ? w1.y : w1.x) * ((k & 4) ? w2.y : w2.x);
    y[k] = fmaf(a.visc, s[k], a.mass * m * u[k]);
  }
  const int64_t o = cell * 8;
  if (a.cheb && vec_all) {  // op_epilogue's modes on the cell's 8 contiguous values, 16-byte accesses
    float d[8], r[8], x[8], di[8], out[8];
    if (a.cheb == 1 || a.cheb == 4) q1_load<float, float>(a.csrc + o, true, d);
    // x and r are written in this launch (each element by its own thread
    // only): plain loads, not the read-only path
    auto ld8 = [](const float* p, float v[8]) {
      const float4 lo = reinterpret_cast<const float4*>(p)[0], hi = reinterpret_cast<const float4*>(p)[1];
      v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w;
      v[4] = hi.x; v[5] = hi.y; v[6] = hi.z; v[7] = hi.w;
    };
    if (a.cheb != 3) ld8(a.cr + o, r);
    if (a.cheb != 2) q1_load<float, float>(a.cdinv + o, true, di);
    if (a.cheb != 2) ld8(a.cx + o, x);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      switch (a.cheb) {
        case 1: {
          x[k] += d[k];
          r[k] = r[k] - di[k] * y[k];
          out[k] = a.cc1 * d[k] + a.cc2 * r[k];
          break;
        }
        case 2: out[k] = r[k] - y[k]; break;
        case 3: {
          r[k] = di[k] * (x[k] - y[k]);
          out[k] = a.cc1 * r[k];
          break;
        }
        default: {
          const float rk = r[k] - di[k] * y[k];
          x[k] += d[k] + (a.cc1 * d[k] + a.cc2 * rk);
        }
      }
    }
    float4* xv = reinterpret_cast<float4*>(a.cx + o);
    float4* rv = reinterpret_cast<float4*>(a.cr + o);
    float4* ov = reinterpret_cast<float4*>(dst + o);
    if (a.cheb == 1 || a.cheb == 4) {
      xv[0] = make_float4(x[0], x[1], x[2], x[3]);
      xv[1] = make_float4(x[4], x[5], x[6], x[7]);
    }
    if (a.cheb == 1 || a.cheb == 3) {
      rv[0] = make_float4(r[0], r[1], r[2], r[3]);
      rv[1] = make_float4(r[4], r[5], r[6], r[7]);
    }
    if (a.cheb != 4) {
      ov[0] = make_float4(out[0], out[1], out[2], out[3]);
      ov[1] = make_float4(out[4], out[5], out[6], out[7]);
    }
  } else if (a.cheb) {
#pragma unroll
    for (int k = 0; k < 8; ++k) op_epilogue(a, o + k, y[k], dst);
  } else if (vec) {
    reinterpret_cast<float4*>(dst + o)[0] = make_float4(y[0], y[1], y[2], y[3]);
    reinterpret_cast<float4*>(dst + o)[1] = make_float4(y[4], y[5], y[6], y[7]);
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) dst[o + k] = y[k];
  }
}

// The same tensor-product operator in float-float FP64 arithmetic (T =
// double storage, the source pre-split into float pairs, the tables' rows as
// float pairs): one compensated sum per node for the stiffness terms, then
// y = (alpha w h w h w h) u + visc K u rounded once.
template <int AX>
__device__ __forceinline__ void q1_line_block_df(const double* __restrict__ K, const df64 v[8], const df64 mt[4],
                                                 DfAcc st[8]) {
  const df64 k00 = df_bits(__ldg(K)), k01 = df_bits(__ldg(K + 1)), k10 = df_bits(__ldg(K + 2)),
             k11 = df_bits(__ldg(K + 3));
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int n0 = q1_node(AX, 0, t), n1 = q1_node(AX, 1, t);
    SumOf<df64> a0, a1;
    a0.start(k00, v[n0]);
    a0.fma(k01, v[n1]);
    a1.start(k10, v[n0]);
    a1.fma(k11, v[n1]);
    acc_fma(st[n0], mt[t], a0.value());
    acc_fma(st[n1], mt[t], a1.value());
  }
}

template <int AX>
__device__ __forceinline__ void q1_axis_terms_df(const OpArgs<double>& a, const double* row, const int ci[3],
                                                 int64_t cell, const double* __restrict__ src, bool vec,
                                                 const df64 u[8], const df64 mt[4], DfAcc st[8]) {
  const int c = ci[AX], n = AX == 0 ? a.n0 : (AX == 1 ? a.n1 : a.n2);
  const int per = AX == 0 ? a.per0 : (AX == 1 ? a.per1 : a.per2);
  const int64_t stride = AX == 0 ? 1 : (AX == 1 ? (int64_t)a.n0 : (int64_t)a.n0 * a.n1);
  q1_line_block_df<AX>(row + 4, u, mt, st);
#pragma unroll
  for (int sd = 0; sd < 2; ++sd) {
    int cn = c + (sd ? 1 : -1);
    if (cn < 0 || cn >= n) {
      if (!per) continue;  // wall: the pressure operator has no face terms there
      cn = cn < 0 ? n - 1 : 0;
    }
    double vt[8];
    q1_load<double, df64>(src + (cell + (int64_t)(cn - c) * stride) * 8, vec, vt);
    df64 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = df_bits(vt[k]);
    q1_line_block_df<AX>(row + 8 + 4 * sd, v, mt, st);
  }
}

template <typename T>
__global__ void __launch_bounds__(128, 4)
    q1_tensor_df_kernel(const __grid_constant__ OpArgs<T> a, const T* __restrict__ src, T* __restrict__ dst) {
  pdl_entry();
  static_assert(std::is_same<T, double>::value, "q1_tensor_df_kernel: FP64 storage only");
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= a.ncell) return;
  int ci[3];
  lex_coords(cell, a.n0, a.n1, ci);
  const double* r0 = a.q1tab_df + 16 * (int64_t)ci[0];
  const double* r1 = a.q1tab_df + 16 * ((int64_t)a.q1tab_off1 + ci[1]);
  const double* r2 = a.q1tab_df + 16 * ((int64_t)a.q1tab_off2 + ci[2]);
  const df64 w0[2] = {df_bits(__ldg(r0)), df_bits(__ldg(r0 + 1))};
  const df64 w1[2] = {df_bits(__ldg(r1)), df_bits(__ldg(r1 + 1))};
  const df64 w2[2] = {df_bits(__ldg(r2)), df_bits(__ldg(r2 + 1))};
  const bool vec = (reinterpret_cast<uintptr_t>(src) & 15u) == 0;
  double ut[8];
  q1_load<double, df64>(src + cell * 8, vec, ut);
  df64 u[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) u[k] = df_bits(ut[k]);
  DfAcc st[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) st[k] = acc_prod(df_const(0.0), df_const(0.0));
  {  // axis 0: lines t = i1 + 2 i2
    const df64 mt[4] = {w1[0] * w2[0], w1[1] * w2[0], w1[0] * w2[1], w1[1] * w2[1]};
    q1_axis_terms_df<0>(a, r0, ci, cell, src, vec, u, mt, st);
  }
  {  // axis 1: lines t = i0 + 2 i2
    const df64 mt[4] = {w0[0] * w2[0], w0[1] * w2[0], w0[0] * w2[1], w0[1] * w2[1]};
    q1_axis_terms_df<1>(a, r1, ci, cell, src, vec, u, mt, st);
  }
  {  // axis 2: lines t = i0 + 2 i1
    const df64 mt[4] = {w0[0] * w1[0], w0[1] * w1[0], w0[0] * w1[1], w0[1] * w1[1]};
    q1_axis_terms_df<2>(a, r2, ci, cell, src, vec, u, mt, st);
  }
  const df64 mass = df_bits(a.mass), visc = df_bits(a.visc);
  const int64_t o = cell * 8;
  double yd[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const df64 m = w0[k & 1] * w1[(k >> 1) & 1] * w2[k >> 2];
    SumOf<df64> y;
    y.start(mass * m, u[k]);
    y.fma(visc, acc_value(st[k]));
    yd[k] = df_to(y.value());
  }
  if (a.cheb || (reinterpret_cast<uintptr_t>(dst) & 15u) != 0) {
#pragma unroll
    for (int k = 0; k < 8; ++k) op_epilogue(a, o + k, yd[k], dst);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) reinterpret_cast<double2*>(dst + o)[q] = make_double2(yd[2 * q], yd[2 * q + 1]);
  }
}

}  // namespace dg
