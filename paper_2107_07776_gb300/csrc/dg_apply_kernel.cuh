// Operator kernel of the matrix-free DG applies (templates); instantiated in
// dg_apply_inst_*.cu, dispatched from dg_apply.cu.
#pragma once

#include <cstdio>
#include <type_traits>

#include "dg_common.cuh"
#include "dg_df64.cuh"

namespace dg {

template <int N, int DIM>
struct Shape {
  static constexpr int NB = DIM == 3 ? N * N * N : N * N;   // nodes per cell
  static constexpr int NF = DIM == 3 ? N * N : N;           // nodes per face
  static constexpr int NFP = 2 * DIM * NF;                  // face points per cell
};

template <typename T>
struct OpArgs {
  int64_t ncell;
  int n0, n1, n2;
  int per0, per1, per2;
  const T* h0;
  const T* h1;
  const T* h2;
  const T* hi0;  // inverse extents
  const T* hi1;
  const T* hi2;
  T mass, visc, adv, pen;
  int walls;   // 1: SIP + LF Dirichlet terms on wall faces; 0: none (Neumann)
  int ncomp;
  // fused epilogue (multigrid smoothing, one component; op_epilogue): 0 none,
  // 1 a Chebyshev step, 2 the residual, 3 the smoother's start from a
  // nonzero iterate, 4 the last Chebyshev step with the final update
  int cheb;
  T* cx;
  T* cr;
  const T* cdinv;
  T cc1, cc2;
  // face-flux scratch of the face-once variant (null: not available)
  void* flux;
  int64_t flux_bytes;
  // the caller's source vector in its storage type (the Chebyshev update
  // reads it; the kernels' src may be a pre-split copy)
  const T* csrc;
  // the mesh's Q1 tensor-product tables (null: none) and the first rows of
  // axes 1 and 2 (a row: one axis cell, 4 float4)
  const float4* q1tab;
  const double* q1tab_df;  // the same rows as float pairs
  int q1tab_off1, q1tab_off2;
};

// The operator kernels' output stage at output index o, y = (A src)_o
// (fields as in OpArgs / GenArgs):
//   0  dst = y
//   1  Chebyshev step, d = the caller's src:  x += d; r -= dinv y; dst = c1 d + c2 r
//   2  residual, r holding b:                  dst = r - y
//   3  smoother start from the iterate src, x holding b:
//                                              r = dinv (b - y); dst = c1 r
//   4  last Chebyshev step and final update:   x += d + c1 d + c2 (r - dinv y)
//      (r and the next direction are not stored)
template <typename Args, typename T>
__device__ __forceinline__ void op_epilogue(const Args& a, int64_t o, T y, T* __restrict__ dst) {
  switch (a.cheb) {
    case 1: {
      const T dk = a.csrc[o];
      a.cx[o] += dk;
      const T rk = a.cr[o] - a.cdinv[o] * y;
      a.cr[o] = rk;
      dst[o] = a.cc1 * dk + a.cc2 * rk;
      break;
    }
    case 2: dst[o] = a.cr[o] - y; break;
    case 3: {
      const T rk = a.cdinv[o] * (a.cx[o] - y);
      a.cr[o] = rk;
      dst[o] = a.cc1 * rk;
      break;
    }
    case 4: {
      const T dk = a.csrc[o];
      const T rk = a.cr[o] - a.cdinv[o] * y;
      a.cx[o] += dk + (a.cc1 * dk + a.cc2 * rk);
      break;
    }
    default: dst[o] = y;
  }
}

// Float-float kernels on FP64 storage (T = double, A = df64) receive every
// FP64 input pre-split: the source vector and advecting field as float
// pairs in double-sized slots (one split pass per apply instead of one split
// per read), the cell extents from the mesh's float-float copies and the
// scalar coefficients split on the host.  ld_val reads a storage value in
// the arithmetic type either way.
template <typename T, typename A>
constexpr bool kPreSplit = std::is_same<T, double>::value && std::is_same<A, df64>::value;

template <typename T, typename A>
__device__ __forceinline__ A ld_val(T v) {
  if constexpr (kPreSplit<T, A>) return df_bits(v);
  else return Arith<A>::from(v);
}

__device__ __forceinline__ int node_of(int N, int a, int i, int t, int dim) {
  // node index with coordinate i along axis a and tangential index t (the
  // other axes in increasing order, t = t0 + N t1); no local arrays, so a
  // run-time axis costs no local-memory traffic
  if (dim == 2) return a == 0 ? i + N * t : t + N * i;
  return a == 0 ? i + N * t : (a == 1 ? t % N + N * (i + N * (t / N)) : t + N * N * i);
}

// v[ax] for a run-time axis without a local-memory array access (the
// elements are passed by value, so the array itself stays in registers)
template <int DIM, typename X>
__device__ __forceinline__ X pick(int ax, X v0, X v1, X v2) {
  return ax == 0 ? v0 : (ax == 1 || DIM == 2 ? v1 : v2);
}
__device__ __forceinline__ int pick3(int ax, int v0, int v1, int v2) {
  return ax == 0 ? v0 : (ax == 1 ? v1 : v2);
}

template <int N, int DIM>
__device__ __forceinline__ int tang_of(int a, const int i[3]) {
  // tangential index of node i on the faces normal to axis a
  int t = 0, mul = 1;
  for (int b = 0; b < DIM; ++b) {
    if (b == a) continue;
    t += i[b] * mul;
    mul *= N;
  }
  return t;
}

}  // namespace dg

#include "dg_split_kernel.cuh"
#include "dg_q1_kernel.cuh"

namespace dg {

// T: storage type of the vectors (double or float); A: arithmetic type
// (double, float, or df64 = float-float on the FP32 pipes).
template <typename T, typename A, int DIM, int N, bool ADV, int CPB, int MINB = 1>
__global__ void __launch_bounds__(((CPB * Shape<N, DIM>::NB + 31) / 32) * 32, MINB)
    scalar_op_kernel(const __grid_constant__ OpArgs<T> a, const __grid_constant__ Tab1D<A> tb,
                     const T* __restrict__ src, const T* __restrict__ ub, T* __restrict__ dst) {
  pdl_entry();
  using Ar = Arith<A>;
  constexpr int NB = Shape<N, DIM>::NB, NF = Shape<N, DIM>::NF, NFP = Shape<N, DIM>::NFP;
  __shared__ A s_u[CPB][NB];
  __shared__ A s_q[DIM][CPB][NB];
  __shared__ A s_f[CPB][NFP][2];
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
  A h[3] = {Ar::c(1.0), Ar::c(1.0), Ar::c(1.0)}, hi[3] = {Ar::c(1.0), Ar::c(1.0), Ar::c(1.0)};
  int ii[3] = {node % N, (node / N) % N, DIM == 3 ? node / (N * N) : 0};
  A W = zero;
  if (active) {
    lex_coords(cell, a.n0, a.n1, ci);
    h[0] = ld_val<T, A>(a.h0[ci[0]]);
    h[1] = ld_val<T, A>(a.h1[ci[1]]);
    hi[0] = ld_val<T, A>(a.hi0[ci[0]]);
    hi[1] = ld_val<T, A>(a.hi1[ci[1]]);
    if (DIM == 3) {
      h[2] = ld_val<T, A>(a.h2[ci[2]]);
      hi[2] = ld_val<T, A>(a.hi2[ci[2]]);
    }
    W = tb.w[ii[0]] * tb.w[ii[1]] * h[0] * h[1];
    if (DIM == 3) W = W * tb.w[ii[2]] * h[2];
    if (ADV) {
#pragma unroll
      for (int b = 0; b < DIM; ++b) s_ub[b][cl][node] = ld_val<T, A>(ub[((int64_t)b * a.ncell + cell) * NB + node]);
    }
  }
  for (int c = 0; c < a.ncomp; ++c) {
    const T* srcc = src + (int64_t)c * a.ncell * NB;
    if (active) s_u[cl][node] = ld_val<T, A>(srcc[cell * NB + node]);
    __syncthreads();
    if (active) {
      // ---- cell integrand at this node: W * (visc grad u - adv u ubar) ----
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        A du = zero;
#pragma unroll
        for (int m = 0; m < N; ++m) {
          int j[3] = {ii[0], ii[1], ii[2]};
          j[b] = m;
          du += tb.D[ii[b]][m] * s_u[cl][j[0] + N * (j[1] + N * j[2])];
        }
        A q = visc * du * hi[b];
        if (ADV) q -= advc * s_u[cl][node] * s_ub[b][cl][node];
        s_q[b][cl][node] = W * q;
      }
      // ---- face fluxes at the face points handled by this thread ----
      for (int fp = node; fp < NFP; fp += NB) {
        const int f = fp / NF, t = fp - (fp / NF) * NF;
        const int ax = f >> 1, s = f & 1;
        const A sgn = s ? Ar::c(1.0) : Ar::c(-1.0);
        // neighbour across this face (selects instead of run-time indexed
        // arrays: no local memory)
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
        const T* hiax = ax == 0 ? a.hi0 : (ax == 1 ? a.hi1 : a.hi2);
        const A hiK = ax == 0 ? hi[0] : (ax == 1 ? hi[1] : hi[2]);
        // tangential weight: face quadrature weight times the face measure
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
        A uin = zero, dnin = zero;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const A v = s_u[cl][node_of(N, ax, i, t, DIM)];
          uin = Ar::fma(tb.L[s][i], v, uin);
          dnin = Ar::fma(tb.dL[s][i], v, dnin);
        }
        dnin = dnin * sgn * hiK;
        A fv = zero, fg = zero;
        if (interior) {
          const A hiN = ld_val<T, A>(hiax[cn]);
          A uout = zero, dnout = zero;
#pragma unroll
          for (int i = 0; i < N; ++i) {
            const A v = ld_val<T, A>(__ldg(&srcc[nb * NB + node_of(N, ax, i, t, DIM)]));
            uout = Ar::fma(tb.L[1 - s][i], v, uout);
            dnout = Ar::fma(tb.dL[1 - s][i], v, dnout);
          }
          dnout = dnout * sgn * hiN;
          const A Cpen = half * pen * (hiK + hiN);
          const A jump = uin - uout;
          fv = visc * (Cpen * jump - half * (dnin + dnout));
          fg = -(half * visc * jump);
          if (ADV) {
            A unin, unout, lam;
            if (c == 0) {
              unin = zero;
              unout = zero;
#pragma unroll
              for (int i = 0; i < N; ++i) {
                unin = Ar::fma(tb.L[s][i], s_ub[ax][cl][node_of(N, ax, i, t, DIM)], unin);
                unout += tb.L[1 - s][i] *
                         ld_val<T, A>(__ldg(&ub[((int64_t)ax * a.ncell + nb) * NB + node_of(N, ax, i, t, DIM)]));
              }
              unin = unin * sgn;
              unout = unout * sgn;
              lam = Ar::max(Ar::abs(unin), Ar::abs(unout));
              s_un[cl][fp][0] = unin;
              s_un[cl][fp][1] = unout;
              s_un[cl][fp][2] = lam;
            } else {
              unin = s_un[cl][fp][0];
              unout = s_un[cl][fp][1];
              lam = s_un[cl][fp][2];
            }
            fv += advc * (half * (uin * unin + uout * unout) + half * lam * jump);
          }
        } else if (a.walls) {
          const A sig = pen * hiK;
          fv = visc * (two * sig * uin - dnin);
          fg = -(visc * uin);
          if (ADV) {
            A unin, lam;
            if (c == 0) {
              unin = zero;
#pragma unroll
              for (int i = 0; i < N; ++i)
                unin = Ar::fma(tb.L[s][i], s_ub[ax][cl][node_of(N, ax, i, t, DIM)], unin);
              unin = unin * sgn;
              lam = Ar::abs(unin);
              s_un[cl][fp][0] = unin;
              s_un[cl][fp][2] = lam;
            } else {
              lam = s_un[cl][fp][2];
            }
            fv += advc * lam * uin;
          }
        }
        s_f[cl][fp][0] = wt * fv;
        s_f[cl][fp][1] = wt * fg * sgn * hiK;
      }
    }
    __syncthreads();
    if (active) {
      A y = mass * W * s_u[cl][node];
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
      }
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        const int t = tang_of<N, DIM>(b, ii);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int fp = (2 * b + s) * NF + t;
          y += s_f[cl][fp][0] * tb.L[s][ii[b]] + s_f[cl][fp][1] * tb.dL[s][ii[b]];
        }
      }
      const int64_t o = (int64_t)c * a.ncell * NB + cell * NB + node;
      const T yt = sizeof(T) == 8 ? (T)Ar::to_d(y) : (T)Ar::to_f(y);
      op_epilogue(a, o, yt, dst);
    }
    __syncthreads();
  }
}

template <int N, int DIM>
constexpr int default_cpb() {
  return Shape<N, DIM>::NB <= 8 ? 16 : (Shape<N, DIM>::NB <= 27 ? 8 : (Shape<N, DIM>::NB <= 64 ? 4 : 2));
}

// shared memory of one CTA (arithmetic type of size sizeof(T); float-float
// has the size of double)
template <int N, int DIM, bool ADV>
constexpr int smem_words(int cpb) {
  return cpb * (Shape<N, DIM>::NB * (1 + DIM) + 2 * Shape<N, DIM>::NFP +
                (ADV ? DIM * Shape<N, DIM>::NB + 3 * Shape<N, DIM>::NFP : 4));
}

// Tile-shape candidates of the autotuner: variants 0-2 take half, the
// default and double the default cells per CTA, each clamped to the 48 KB
// static shared-memory and 1024-thread limits; variants 3 and 4 take the
// default cells per CTA with the registers per thread capped at 96 and 80
// (more resident CTAs per SM, possibly at the price of spills); variants 5
// and 6 are the face-once form (face fluxes, then cells) with the default
// cells per CTA and 72 registers (variant 6 with the components-interleaved
// cell pass, cell_split_nc_kernel); variant 7 is the
// thread-per-cell Q1 kernel (3D scalar operators without advection on two
// points per direction; elsewhere it runs as variant 1).
// (kTuneVariants, variant_split and variant_q1 are in dg_common.cuh.)

template <typename T, int DIM, int N, bool ADV>
constexpr int cpb_variant(int v) {
  int c = v == 0 ? default_cpb<N, DIM>() / 2 : (v == 2 ? default_cpb<N, DIM>() * 2 : default_cpb<N, DIM>());
  if (c < 1) c = 1;
  while (c > 1 && (c * Shape<N, DIM>::NB > 1024 || (int)sizeof(T) * smem_words<N, DIM, ADV>(c) > 46 * 1024))
    c /= 2;
  return c;
}

// minimum resident CTAs per SM requested from the compiler for variant v
template <typename T, int DIM, int N, bool ADV>
constexpr int minb_variant(int v) {
  const int threads = ((cpb_variant<T, DIM, N, ADV>(v) * Shape<N, DIM>::NB + 31) / 32) * 32;
  const int cap = v == 3 ? 96 : (v == 4 ? 80 : (v == 5 || v == 6 ? 72 : 0));
  if (cap == 0) return 1;
  const int b = 65536 / (threads * cap);
  return b < 1 ? 1 : b;
}

template <typename T, typename A, int DIM, int N, bool ADV, int CPB, int MINB>
static dg_status launch_cpb(const OpArgs<T>& args, const Tab1D<A>& tb, const T* ub, const T* src,
                            T* dst, cudaStream_t s) {
  constexpr int threads = ((CPB * Shape<N, DIM>::NB + 31) / 32) * 32;
  const int64_t blocks = (args.ncell + CPB - 1) / CPB;
  if (blocks > 0x7fffffff) {
    set_error("operator apply: grid too large");
    return DG_EINVAL;
  }
  launch(scalar_op_kernel<T, A, DIM, N, ADV, CPB, MINB>, (unsigned)blocks, threads, 0, s, args, tb, src, ub, dst);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

// the components-interleaved cell pass (dynamic shared memory, above the
// 48 KB static limit for some shapes: the opt-in is set once per device)
template <typename T, typename A, int DIM, int N, int NC, bool ADV, int CPB, int MINB>
static dg_status launch_cell_nc(const OpArgs<T>& args, const Tab1D<A>& tb, const T* ub, const T* src,
                                const A* flux, T* dst, cudaStream_t s) {
  constexpr int smem = NcSplitSmem<A, DIM, N, NC, CPB>::bytes;
  static_assert(smem <= 227 * 1024, "cell_split_nc_kernel: shared memory");
  auto kern = cell_split_nc_kernel<T, A, DIM, N, NC, ADV, CPB, MINB>;
  if (smem > 48 * 1024) {
    static unsigned long long opted = 0;  // devices (bit i: device i < 64) already opted in
    int dev = 0;
    DG_CUDA(cudaGetDevice(&dev));
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (!bit || !(__atomic_load_n(&opted, __ATOMIC_ACQUIRE) & bit)) {
      DG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      if (bit) __atomic_fetch_or(&opted, bit, __ATOMIC_ACQ_REL);
    }
  }
  constexpr int threads = ((CPB * Shape<N, DIM>::NB + 31) / 32) * 32;
  const int64_t blocks = (args.ncell + CPB - 1) / CPB;
  launch(kern, (unsigned)blocks, threads, smem, s, args, tb, src, ub, flux, dst);
  count_launch();
  return DG_OK;
}

template <typename T, typename A, int DIM, int N, bool ADV, int CPB, int MINB, bool NCK = false>
static dg_status launch_split(const OpArgs<T>& args, const Tab1D<A>& tb, const T* ub, const T* src,
                              T* dst, cudaStream_t s) {
  const int n[3] = {args.n0, args.n1, args.n2};
  const int per[3] = {args.per0, args.per1, args.per2};
  int64_t nface = faces_of_axis(0, n, per) + faces_of_axis(1, n, per);
  if (DIM == 3) nface += faces_of_axis(2, n, per);
  const int64_t need = nface * Shape<N, DIM>::NF * 2 * args.ncomp * (int64_t)sizeof(A);
  if (!args.flux || need > args.flux_bytes) {  // no scratch: the single-kernel form
    return launch_cpb<T, A, DIM, N, ADV, cpb_variant<T, DIM, N, ADV>(1), 1>(args, tb, ub, src, dst, s);
  }
  A* flux = static_cast<A*>(args.flux);
  const int64_t fthreads = nface * Shape<N, DIM>::NF;
  launch(face_flux_kernel<T, A, DIM, N, ADV>, (unsigned)((fthreads + 255) / 256), 256, 0, s, args, tb, src, ub, flux);
  count_launch();
  if constexpr (NCK) {
    if (args.ncomp == DIM || args.ncomp == 1) {
      const dg_status st =
          args.ncomp == DIM ? launch_cell_nc<T, A, DIM, N, DIM, ADV, CPB, MINB>(args, tb, ub, src, flux, dst, s)
                            : launch_cell_nc<T, A, DIM, N, 1, ADV, CPB, MINB>(args, tb, ub, src, flux, dst, s);
      if (st != DG_OK) return st;
      DG_CUDA(cudaGetLastError());
      return DG_OK;
    }
  }
  constexpr int threads = ((CPB * Shape<N, DIM>::NB + 31) / 32) * 32;
  const int64_t blocks = (args.ncell + CPB - 1) / CPB;
  launch(cell_split_kernel<T, A, DIM, N, ADV, CPB, MINB>, (unsigned)blocks, threads, 0, s, args, tb, src, ub,
         flux, dst);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

template <typename T, typename A>
static dg_status launch_q1(const OpArgs<T>& args, const Tab1D<A>& tb, const T* src, T* dst,
                           cudaStream_t s) {
  if constexpr ((std::is_same<T, float>::value && std::is_same<A, float>::value) || kPreSplit<T, A>) {
    // FP32 or float-float pressure operator (no wall terms): the
    // tensor-product form
    if ((kPreSplit<T, A> ? args.q1tab_df != nullptr : args.q1tab != nullptr) && !args.walls) {
      const int64_t tblocks = (args.ncell + 127) / 128;
      if (tblocks > 0x7fffffff) {
        set_error("operator apply: grid too large");
        return DG_EINVAL;
      }
      if constexpr (kPreSplit<T, A>)
        launch(q1_tensor_df_kernel<T>, (unsigned)tblocks, 128, 0, s, args, src, dst);
      else
        launch(q1_tensor_kernel<T>, (unsigned)tblocks, 128, 0, s, args, src, dst);
      count_launch();
      DG_CUDA(cudaGetLastError());
      return DG_OK;
    }
  }
  const int64_t blocks = (2 * args.ncell + 127) / 128;  // two threads per cell
  if (blocks > 0x7fffffff) {
    set_error("operator apply: grid too large");
    return DG_EINVAL;
  }
  launch(q1_cell_kernel<T, A>, (unsigned)blocks, 128, 0, s, args, tb, src, dst);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

template <typename T, typename A, int DIM, int N, bool ADV, int V>
static dg_status launch_v(const OpArgs<T>& args, const Tab1D<A>& tb, const T* ub, const T* src,
                          T* dst, cudaStream_t s) {
  if constexpr (variant_q1(V)) {
    if constexpr (N == 2 && DIM == 3 && !ADV) {
      if (args.ncomp == 1) return launch_q1<T, A>(args, tb, src, dst, s);
    }
    return launch_v<T, A, DIM, N, ADV, 1>(args, tb, ub, src, dst, s);
  } else if constexpr (variant_split(V))
    return launch_split<T, A, DIM, N, ADV, cpb_variant<T, DIM, N, ADV>(V), minb_variant<T, DIM, N, ADV>(V),
                        V == 6>(args, tb, ub, src, dst, s);
  else
    return launch_cpb<T, A, DIM, N, ADV, cpb_variant<T, DIM, N, ADV>(V), minb_variant<T, DIM, N, ADV>(V)>(
        args, tb, ub, src, dst, s);
}

template <typename T, typename A, int DIM, int N, bool ADV>
static dg_status launch_fixed(int variant, const OpArgs<T>& args, const Tab1D<A>& tb, const T* ub,
                              const T* src, T* dst, cudaStream_t s) {
  switch (variant) {
    case 0: return launch_v<T, A, DIM, N, ADV, 0>(args, tb, ub, src, dst, s);
    case 2: return launch_v<T, A, DIM, N, ADV, 2>(args, tb, ub, src, dst, s);
    case 3: return launch_v<T, A, DIM, N, ADV, 3>(args, tb, ub, src, dst, s);
    case 4: return launch_v<T, A, DIM, N, ADV, 4>(args, tb, ub, src, dst, s);
    case 5: return launch_v<T, A, DIM, N, ADV, 5>(args, tb, ub, src, dst, s);
    case 6: return launch_v<T, A, DIM, N, ADV, 6>(args, tb, ub, src, dst, s);
    case 7: return launch_v<T, A, DIM, N, ADV, 7>(args, tb, ub, src, dst, s);
    default: return launch_v<T, A, DIM, N, ADV, 1>(args, tb, ub, src, dst, s);
  }
}

template <typename T, int DIM, int N, bool ADV>
static int cpb_of(int variant) {
  return cpb_variant<T, DIM, N, ADV>(variant);
}

template <typename T, typename A, int DIM, bool ADV>
static dg_status launch_dim(int variant, int N, const OpArgs<T>& args, const Tab1D<A>& tb,
                            const T* ub, const T* src, T* dst, cudaStream_t s) {
  switch (N) {
    case 2: return launch_fixed<T, A, DIM, 2, ADV>(variant, args, tb, ub, src, dst, s);
    case 3: return launch_fixed<T, A, DIM, 3, ADV>(variant, args, tb, ub, src, dst, s);
    case 4: return launch_fixed<T, A, DIM, 4, ADV>(variant, args, tb, ub, src, dst, s);
    case 5: return launch_fixed<T, A, DIM, 5, ADV>(variant, args, tb, ub, src, dst, s);
    default: set_error("operator apply: unsupported number of nodes"); return DG_EUNSUPPORTED;
  }
}

template <typename T, int DIM, bool ADV>
static int cpb_dim(int variant, int N) {
  switch (N) {
    case 2: return cpb_of<T, DIM, 2, ADV>(variant);
    case 3: return cpb_of<T, DIM, 3, ADV>(variant);
    case 4: return cpb_of<T, DIM, 4, ADV>(variant);
    default: return cpb_of<T, DIM, 5, ADV>(variant);
  }
}

}  // namespace dg
