// Operator kernel of the matrix-free DG applies on trilinear cells (the
// general-geometry counterpart of scalar_op_kernel): the same forms of
// Section 3 -- mass, SIP diffusion (Eq. bilin_diff / weakform_p_1) and local
// Lax-Friedrichs advection (Eq. trilinear) -- with the per-point metric terms
// of dg_geom.cuh in place of the per-axis cell extents.
//
// One thread per cell node, CPB cells per CTA.  Per component:
//  1. the cell's values go to shared memory;
//  2. volume: reference gradient by d 1D sweeps, flux q_a = visc G[a][:] g -
//     adv u ubar~_a (ubar~ = B ubar, the contravariant advecting field);
//     face points: own and neighbour traces and reference normal derivatives
//     (neighbour pencils gathered from global memory / L2);
//  3. face points: tangential reference derivatives of both traces (sweeps
//     within the face), physical normal derivatives d/dn = c . grad_ref, the
//     SIP + LF fluxes, and the coefficients of the test function's value,
//     its reference normal derivative and its tangential derivatives;
//  4. node: mass + transposed volume sweeps + face contributions (the
//     tangential part by a transposed sweep within each face).
// Every output is written once, without atomics: deterministic.
#pragma once

#include "dg_apply_kernel.cuh"
#include "dg_geom.cuh"

#include <type_traits>

namespace dg {

template <typename T>
struct GenArgs {
  int64_t ncell;
  int n0, n1, n2;
  int per0, per1, per2;
  const T* gv;    // volume terms [cell][field][node]
  const T* gf;    // face terms [cell][face][field][point]
  const T* gpen;  // penalty geometry [cell][face]
  // the same terms split into float pairs once at setup, read by the
  // float-float variant instead of splitting a double at every load
  const df64* gv2;
  const df64* gf2;
  const df64* gpen2;
  T mass, visc, adv, pen;
  int walls;      // 1: SIP + LF wall terms (homogeneous Dirichlet); 0: none (Neumann)
  int ncomp;
  int cheb;       // fused epilogue, as in OpArgs (op_epilogue)
  T* cx;
  T* cr;
  const T* cdinv;
  T cc1, cc2;
  int variant;    // tile shape: 0 half, 1 default, 2 double the cells per CTA
  const T* csrc;  // the caller's source vector (the Chebyshev update reads it)
};

// metric term i: from the float-pair copy in float-float arithmetic, else
// converted from the storage type
template <typename A, typename T>
__device__ __forceinline__ A gload(const T* p, const df64* q, int64_t i) {
  if constexpr (std::is_same<A, df64>::value) return q[i];
  else return Arith<A>::from(p[i]);
}

template <int N, int DIM, bool ADV>
constexpr int gen_smem_words(int cpb) {
  // s_u, s_q, s_f, s_t, s_dn, s_Q, (s_ub, s_un)
  return cpb * (Shape<N, DIM>::NB * (1 + DIM) + Shape<N, DIM>::NFP * (6 + (DIM - 1)) +
                (ADV ? DIM * Shape<N, DIM>::NB + 3 * Shape<N, DIM>::NFP : 2));
}

template <typename T, int DIM, int N, bool ADV>
constexpr int gen_cpb(int variant = 1) {
  int c = default_cpb<N, DIM>();
  if (variant == 0) c = c > 1 ? c / 2 : 1;
  if (variant == 2) c *= 2;
  // shared-memory words are 8 bytes (double or float-float) at most
  while (c > 1 && (c * Shape<N, DIM>::NB > 1024 || 8 * gen_smem_words<N, DIM, ADV>(c) > 46 * 1024))
    c /= 2;
  return c;
}

// T: storage type (double or float); A: arithmetic type (double, float or
// df64).  VEL: velocity-space metric layout (with normals and B); pressure
// layout otherwise.  ADV requires VEL.
template <typename T, typename A, int DIM, int N, bool ADV, bool VEL, int CPB>
__global__ void __launch_bounds__(((CPB * Shape<N, DIM>::NB + 31) / 32) * 32)
    general_op_kernel(const __grid_constant__ GenArgs<T> a, const __grid_constant__ Tab1D<A> tb,
                      const T* __restrict__ src, const T* __restrict__ ub, T* __restrict__ dst) {
  pdl_entry();
  using Ar = Arith<A>;
  using GC = GeomCount<DIM>;
  constexpr int NB = Shape<N, DIM>::NB, NF = Shape<N, DIM>::NF, NFP = Shape<N, DIM>::NFP;
  constexpr int NG = GC::NG;
  constexpr int NV = VEL ? GC::NVU : GC::NVP;
  constexpr int NFF = VEL ? GC::NFU : GC::NFP;
  constexpr int OFF_C = VEL ? 1 + DIM : 1;   // first cown field of a face
  __shared__ A s_u[CPB][NB];
  __shared__ A s_q[DIM][CPB][NB];
  __shared__ A s_f[CPB][NFP][2];
  __shared__ A s_t[CPB][NFP][2];
  __shared__ A s_dn[CPB][NFP][2];
  __shared__ A s_Q[CPB][NFP][DIM - 1];
  __shared__ A s_ub[ADV ? DIM : 1][CPB][ADV ? NB : 1];
  __shared__ A s_un[ADV ? CPB : 1][ADV ? NFP : 1][3];  // ubar.n inside, outside, lambda

  const int tid = threadIdx.x;
  const int cl = tid / NB, node = tid - (tid / NB) * NB;
  const int64_t cell = (int64_t)blockIdx.x * CPB + cl;
  const bool active = cl < CPB && cell < a.ncell;
  const A zero = Ar::c(0.0), half = Ar::c(0.5), two = Ar::c(2.0);
  const A mass = ld_val<T, A>(a.mass), visc = ld_val<T, A>(a.visc), advc = ld_val<T, A>(a.adv),
          pen = ld_val<T, A>(a.pen);

  int ci[3] = {0, 0, 0};
  const int ii[3] = {node % N, (node / N) % N, DIM == 3 ? node / (N * N) : 0};
  A Gm[NG], Wm = zero, ut[DIM];
#pragma unroll
  for (int f = 0; f < NG; ++f) Gm[f] = zero;
#pragma unroll
  for (int b = 0; b < DIM; ++b) ut[b] = zero;
  if (active) {
    lex_coords(cell, a.n0, a.n1, ci);
    const int64_t gvo = cell * (int64_t)NV * NB + node;
    const T* gv = a.gv + gvo;
    const df64* gv2 = a.gv2 + gvo;
#pragma unroll
    for (int f = 0; f < NG; ++f) Gm[f] = gload<A>(gv, gv2, f * NB);
    Wm = gload<A>(gv, gv2, NG * NB);
    if (ADV) {
      A ubn[DIM];
#pragma unroll
      for (int r = 0; r < DIM; ++r) {
        ubn[r] = ld_val<T, A>(ub[((int64_t)r * a.ncell + cell) * NB + node]);
        s_ub[r][cl][node] = ubn[r];
      }
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        A acc = zero;
#pragma unroll
        for (int r = 0; r < DIM; ++r) acc = Ar::fma(gload<A>(gv, gv2, (NG + 1 + b * DIM + r) * NB), ubn[r], acc);
        ut[b] = acc;
      }
    }
  }

  for (int c = 0; c < a.ncomp; ++c) {
    const T* srcc = src + (int64_t)c * a.ncell * NB;
    if (active) s_u[cl][node] = ld_val<T, A>(srcc[cell * NB + node]);
    __syncthreads();
    if (active) {
      // ---- volume flux at this node ----
      A g[DIM];
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        A du = zero;
#pragma unroll
        for (int m = 0; m < N; ++m) {
          int j[3] = {ii[0], ii[1], ii[2]};
          j[b] = m;
          du += tb.D[ii[b]][m] * s_u[cl][j[0] + N * (j[1] + N * j[2])];
        }
        g[b] = du;
      }
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        A q = zero;
#pragma unroll
        for (int e = 0; e < DIM; ++e) q += Gm[sym_index(DIM, b, e)] * g[e];
        q = visc * q;
        if (ADV) q -= advc * s_u[cl][node] * ut[b];
        s_q[b][cl][node] = q;
      }
      // ---- face points: traces and reference normal derivatives ----
      for (int fp = node; fp < NFP; fp += NB) {
        const int f = fp / NF, t = fp - (fp / NF) * NF;
        const int ax = f >> 1, s = f & 1;
        const int cax = pick3(ax, ci[0], ci[1], ci[2]);
        const int nax = pick3(ax, a.n0, a.n1, a.n2);
        const int64_t cstr = ax == 0 ? 1 : (ax == 1 ? (int64_t)a.n0 : (int64_t)a.n0 * a.n1);
        int cn = cax + (s ? 1 : -1);
        bool interior = true;
        if (cn < 0 || cn >= nax) {
          if (pick3(ax, a.per0, a.per1, a.per2)) cn = cn < 0 ? nax - 1 : 0;
          else interior = false;
        }
        const int64_t nb = cell + (int64_t)(cn - cax) * cstr;
        A uin = zero, dnin = zero, uout = zero, dnout = zero;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const A v = s_u[cl][node_of(N, ax, i, t, DIM)];
          uin = Ar::fma(tb.L[s][i], v, uin);
          dnin = Ar::fma(tb.dL[s][i], v, dnin);
        }
        if (interior) {
#pragma unroll
          for (int i = 0; i < N; ++i) {
            const A v = ld_val<T, A>(__ldg(&srcc[nb * NB + node_of(N, ax, i, t, DIM)]));
            uout = Ar::fma(tb.L[1 - s][i], v, uout);
            dnout = Ar::fma(tb.dL[1 - s][i], v, dnout);
          }
        }
        s_t[cl][fp][0] = uin;
        s_t[cl][fp][1] = uout;
        s_dn[cl][fp][0] = dnin;
        s_dn[cl][fp][1] = dnout;
        if (ADV && c == 0) {
          const int64_t gfo = ((cell * 2 * DIM + f) * (int64_t)NFF) * NF + t;
          const T* gfp = a.gf + gfo;
          const df64* gfp2 = a.gf2 + gfo;
          A unin = zero, unout = zero;
#pragma unroll
          for (int r = 0; r < DIM; ++r) {
            const A nr = gload<A>(gfp, gfp2, (1 + r) * NF);
            A wi = zero, wo = zero;
#pragma unroll
            for (int i = 0; i < N; ++i) {
              const int nd = node_of(N, ax, i, t, DIM);
              wi = Ar::fma(tb.L[s][i], s_ub[r][cl][nd], wi);
              if (interior)
                wo = Ar::fma(tb.L[1 - s][i], ld_val<T, A>(__ldg(&ub[((int64_t)r * a.ncell + nb) * NB + nd])), wo);
            }
            unin += nr * wi;
            unout += nr * wo;
          }
          s_un[cl][fp][0] = unin;
          s_un[cl][fp][1] = unout;
          s_un[cl][fp][2] = interior ? Ar::max(Ar::abs(unin), Ar::abs(unout)) : Ar::abs(unin);
        }
      }
    }
    __syncthreads();
    if (active) {
      // ---- face points: fluxes ----
      for (int fp = node; fp < NFP; fp += NB) {
        const int f = fp / NF, t = fp - (fp / NF) * NF;
        const int ax = f >> 1, s = f & 1;
        const int cax = pick3(ax, ci[0], ci[1], ci[2]);
        const bool interior =
            pick3(ax, a.per0, a.per1, a.per2) || (s ? cax + 1 < pick3(ax, a.n0, a.n1, a.n2) : cax > 0);
        const int64_t gfo = ((cell * 2 * DIM + f) * (int64_t)NFF) * NF + t;
        const T* gfp = a.gf + gfo;
        const df64* gfp2 = a.gf2 + gfo;
        const A dS = gload<A>(gfp, gfp2, 0);
        A cown[DIM], cnb[DIM];
#pragma unroll
        for (int b = 0; b < DIM; ++b) {
          cown[b] = gload<A>(gfp, gfp2, (OFF_C + b) * NF);
          cnb[b] = gload<A>(gfp, gfp2, (OFF_C + DIM + b) * NF);
        }
        const A uin = s_t[cl][fp][0], uout = s_t[cl][fp][1];
        const A cown_ax = pick<DIM>(ax, cown[0], cown[1], cown[DIM - 1]);
        const A cnb_ax = pick<DIM>(ax, cnb[0], cnb[1], cnb[DIM - 1]);
        A dn_in = cown_ax * s_dn[cl][fp][0], dn_out = cnb_ax * s_dn[cl][fp][1];
        {
          int stride = 1;
#pragma unroll
          for (int b = 0; b < DIM; ++b) {
            if (b == ax) continue;
            const int tb_ = (t / stride) % N;
            A gi = zero, go = zero;
#pragma unroll
            for (int m = 0; m < N; ++m) {
              const int q = f * NF + t + (m - tb_) * stride;
              gi = Ar::fma(tb.D[tb_][m], s_t[cl][q][0], gi);
              go = Ar::fma(tb.D[tb_][m], s_t[cl][q][1], go);
            }
            dn_in += cown[b] * gi;
            dn_out += cnb[b] * go;
            stride *= N;
          }
        }
        A fv = zero, fg = zero;
        const A sig = pen * gload<A>(a.gpen, a.gpen2, cell * 2 * DIM + f);
        if (interior) {
          const A jump = uin - uout;
          fv = visc * (sig * jump - half * (dn_in + dn_out));
          fg = -(half * visc * jump);
          if (ADV)
            fv += advc * (half * (uin * s_un[cl][fp][0] + uout * s_un[cl][fp][1]) +
                          half * s_un[cl][fp][2] * jump);
        } else if (a.walls) {
          fv = visc * (two * sig * uin - dn_in);
          fg = -(visc * uin);
          if (ADV) fv += advc * s_un[cl][fp][2] * uin;
        }
        const A wg = dS * fg;
        s_f[cl][fp][0] = dS * fv;
        s_f[cl][fp][1] = wg * cown_ax;
        int e = 0;
#pragma unroll
        for (int b = 0; b < DIM; ++b) {
          if (b == ax) continue;
          s_Q[cl][fp][e++] = wg * cown[b];
        }
      }
    }
    __syncthreads();
    if (active) {
      A y = mass * Wm * s_u[cl][node];
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
#pragma unroll
        for (int m = 0; m < N; ++m) {
          int j[3] = {ii[0], ii[1], ii[2]};
          j[b] = m;
          y += tb.D[m][ii[b]] * s_q[b][cl][j[0] + N * (j[1] + N * j[2])];
        }
      }
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        const int t = tang_of<N, DIM>(b, ii);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int f = 2 * b + s, fp = f * NF + t;
          A R = zero;
          int stride = 1, e = 0;
#pragma unroll
          for (int g2 = 0; g2 < DIM; ++g2) {
            if (g2 == b) continue;
            const int tg = ii[g2];
#pragma unroll
            for (int m = 0; m < N; ++m)
              R = Ar::fma(tb.D[m][tg], s_Q[cl][f * NF + t + (m - tg) * stride][e], R);
            stride *= N;
            ++e;
          }
          y += (s_f[cl][fp][0] + R) * tb.L[s][ii[b]] + s_f[cl][fp][1] * tb.dL[s][ii[b]];
        }
      }
      const int64_t o = (int64_t)c * a.ncell * NB + cell * NB + node;
      const T yt = sizeof(T) == 8 ? (T)Ar::to_d(y) : (T)Ar::to_f(y);
      op_epilogue(a, o, yt, dst);
    }
    __syncthreads();
  }
}

template <typename T, typename A, int DIM, int N, bool ADV, bool VEL, int CPB>
dg_status launch_general_cpb(const GenArgs<T>& args, const Tab1D<A>& tb, const T* ub,
                             const T* src, T* dst, cudaStream_t s) {
  constexpr int threads = ((CPB * Shape<N, DIM>::NB + 31) / 32) * 32;
  const int64_t blocks = (args.ncell + CPB - 1) / CPB;
  if (blocks > 0x7fffffff) {
    set_error("operator apply: grid too large");
    return DG_EINVAL;
  }
  launch(general_op_kernel<T, A, DIM, N, ADV, VEL, CPB>, (unsigned)blocks, threads, 0, s, args, tb, src, ub, dst);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

// the autotuner's tile shape (GenArgs::variant); the clamped cell counts of
// neighbouring variants can coincide
template <typename T, typename A, int DIM, int N, bool ADV, bool VEL>
dg_status launch_general_fixed(const GenArgs<T>& args, const Tab1D<A>& tb, const T* ub,
                               const T* src, T* dst, cudaStream_t s) {
  switch (args.variant) {
    case 0: return launch_general_cpb<T, A, DIM, N, ADV, VEL, gen_cpb<T, DIM, N, ADV>(0)>(args, tb, ub, src, dst, s);
    case 2: return launch_general_cpb<T, A, DIM, N, ADV, VEL, gen_cpb<T, DIM, N, ADV>(2)>(args, tb, ub, src, dst, s);
    default: return launch_general_cpb<T, A, DIM, N, ADV, VEL, gen_cpb<T, DIM, N, ADV>(1)>(args, tb, ub, src, dst, s);
  }
}

// kind: 0 pressure (pressure layout, no advection), 1 velocity without
// advection, 2 velocity with advection
template <typename T, typename A, int DIM>
dg_status launch_general_dim(int kind, int N, const GenArgs<T>& args, const Tab1D<A>& tb,
                             const T* ub, const T* src, T* dst, cudaStream_t s) {
  if (kind == 0) {
    switch (N) {
      case 2: return launch_general_fixed<T, A, DIM, 2, false, false>(args, tb, ub, src, dst, s);
      case 3: return launch_general_fixed<T, A, DIM, 3, false, false>(args, tb, ub, src, dst, s);
      case 4: return launch_general_fixed<T, A, DIM, 4, false, false>(args, tb, ub, src, dst, s);
      default: break;
    }
  } else if (kind == 1) {
    switch (N) {
      case 3: return launch_general_fixed<T, A, DIM, 3, false, true>(args, tb, ub, src, dst, s);
      case 4: return launch_general_fixed<T, A, DIM, 4, false, true>(args, tb, ub, src, dst, s);
      case 5: return launch_general_fixed<T, A, DIM, 5, false, true>(args, tb, ub, src, dst, s);
      default: break;
    }
  } else {
    switch (N) {
      case 3: return launch_general_fixed<T, A, DIM, 3, true, true>(args, tb, ub, src, dst, s);
      case 4: return launch_general_fixed<T, A, DIM, 4, true, true>(args, tb, ub, src, dst, s);
      case 5: return launch_general_fixed<T, A, DIM, 5, true, true>(args, tb, ub, src, dst, s);
      default: break;
    }
  }
  set_error("operator apply (trilinear cells): unsupported number of nodes");
  return DG_EUNSUPPORTED;
}

}  // namespace dg
