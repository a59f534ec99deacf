// Matrix-free application of the DG operators of Section 3 on affine
// (Cartesian or tensor-graded) cells:
//
//   momentum, per velocity component (the operator is the same scalar
//   operator for every component):
//     mass M + visc A + adv C(ubar)
//     A: SIP form a_u (Eq. bilin_diff), C: local Lax-Friedrichs form (Eq. trilinear)
//   pressure Helmholtz:
//     alpha M^p + K, K the SIP form a_p (Eq. weakform_p_1), interior faces only.
//
// Basis: nodal Lagrange at the Gauss-Legendre points (collocation): the
// quadrature points of cells and faces are the nodes and the traces of the
// face-normal pencils, so cell values need no interpolation and gradients
// are 1D differentiation sweeps (sum factorisation).  One thread per cell
// node; one CTA handles CPB cells; cell data are staged in shared memory and
// each cell computes the face fluxes of its 2d faces itself (neighbour traces
// from the neighbour's pencils), so every output is written once, without
// atomics, and the result is deterministic.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dg_common.cuh"

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
};

__device__ __forceinline__ int node_of(int N, int a, int i, int t, int dim) {
  // node index with coordinate i along axis a and tangential index t
  int idx[3] = {0, 0, 0};
  idx[a] = i;
  for (int b = 0; b < dim; ++b) {
    if (b == a) continue;
    idx[b] = t % N;
    t /= N;
  }
  return idx[0] + N * (idx[1] + N * idx[2]);
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

template <typename T, int DIM, int N, bool ADV, int CPB>
__global__ void __launch_bounds__(((CPB * Shape<N, DIM>::NB + 31) / 32) * 32)
    scalar_op_kernel(const __grid_constant__ OpArgs<T> a, const __grid_constant__ Tab1D<T> tb,
                     const T* __restrict__ src, const T* __restrict__ ub, T* __restrict__ dst) {
  constexpr int NB = Shape<N, DIM>::NB, NF = Shape<N, DIM>::NF, NFP = Shape<N, DIM>::NFP;
  __shared__ T s_u[CPB][NB];
  __shared__ T s_q[DIM][CPB][NB];
  __shared__ T s_f[CPB][NFP][2];
  __shared__ T s_ub[ADV ? DIM : 1][CPB][ADV ? NB : 1];
  __shared__ T s_un[ADV ? CPB : 1][ADV ? NFP : 1][3];  // ubar.n inside, outside, lambda

  const int tid = threadIdx.x;
  const int cl = tid / NB, node = tid - (tid / NB) * NB;
  const int64_t cell = (int64_t)blockIdx.x * CPB + cl;
  const bool active = cl < CPB && cell < a.ncell;

  int ci[3] = {0, 0, 0};
  T h[3] = {T(1), T(1), T(1)}, hi[3] = {T(1), T(1), T(1)};
  int ii[3] = {node % N, (node / N) % N, DIM == 3 ? node / (N * N) : 0};
  T W = T(0);
  if (active) {
    ci[0] = (int)(cell % a.n0);
    ci[1] = (int)((cell / a.n0) % a.n1);
    ci[2] = DIM == 3 ? (int)(cell / ((int64_t)a.n0 * a.n1)) : 0;
    h[0] = a.h0[ci[0]];
    h[1] = a.h1[ci[1]];
    hi[0] = a.hi0[ci[0]];
    hi[1] = a.hi1[ci[1]];
    if (DIM == 3) {
      h[2] = a.h2[ci[2]];
      hi[2] = a.hi2[ci[2]];
    }
    W = tb.w[ii[0]] * tb.w[ii[1]] * h[0] * h[1];
    if (DIM == 3) W *= tb.w[ii[2]] * h[2];
    if (ADV) {
#pragma unroll
      for (int b = 0; b < DIM; ++b) s_ub[b][cl][node] = ub[((int64_t)b * a.ncell + cell) * NB + node];
    }
  }
  const int nn[3] = {a.n0, a.n1, a.n2};
  const int per[3] = {a.per0, a.per1, a.per2};

  for (int c = 0; c < a.ncomp; ++c) {
    const T* srcc = src + (int64_t)c * a.ncell * NB;
    if (active) s_u[cl][node] = srcc[cell * NB + node];
    __syncthreads();
    if (active) {
      // ---- cell integrand at this node: W * (visc grad u - adv u ubar) ----
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        T du = T(0);
#pragma unroll
        for (int m = 0; m < N; ++m) {
          int j[3] = {ii[0], ii[1], ii[2]};
          j[b] = m;
          du += tb.D[ii[b]][m] * s_u[cl][j[0] + N * (j[1] + N * j[2])];
        }
        T q = a.visc * du * hi[b];
        if (ADV) q -= a.adv * s_u[cl][node] * s_ub[b][cl][node];
        s_q[b][cl][node] = W * q;
      }
      // ---- face fluxes at the face points handled by this thread ----
      for (int fp = node; fp < NFP; fp += NB) {
        const int f = fp / NF, t = fp - (fp / NF) * NF;
        const int ax = f >> 1, s = f & 1;
        const T sgn = s ? T(1) : T(-1);
        // neighbour across this face
        int nc[3] = {ci[0], ci[1], ci[2]};
        nc[ax] += s ? 1 : -1;
        bool interior = true;
        if (nc[ax] < 0 || nc[ax] >= nn[ax]) {
          if (per[ax]) nc[ax] = (nc[ax] + nn[ax]) % nn[ax];
          else interior = false;
        }
        const int64_t nb = (int64_t)nc[0] + (int64_t)a.n0 * (nc[1] + (int64_t)a.n1 * nc[2]);
        const T* hiax = ax == 0 ? a.hi0 : (ax == 1 ? a.hi1 : a.hi2);
        const T hiK = hi[ax];
        // tangential weight: face quadrature weight times the face measure
        T wt = T(1);
        {
          int tt = t;
#pragma unroll
          for (int b = 0; b < DIM; ++b) {
            if (b == ax) continue;
            wt *= tb.w[tt % N] * h[b];
            tt /= N;
          }
        }
        T uin = T(0), dnin = T(0);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          T v = s_u[cl][node_of(N, ax, i, t, DIM)];
          uin += tb.L[s][i] * v;
          dnin += tb.dL[s][i] * v;
        }
        dnin *= sgn * hiK;
        T fv = T(0), fg = T(0);
        if (interior) {
          const T hiN = hiax[nc[ax]];
          T uout = T(0), dnout = T(0);
#pragma unroll
          for (int i = 0; i < N; ++i) {
            T v = __ldg(&srcc[nb * NB + node_of(N, ax, i, t, DIM)]);
            uout += tb.L[1 - s][i] * v;
            dnout += tb.dL[1 - s][i] * v;
          }
          dnout *= sgn * hiN;
          const T Cpen = T(0.5) * a.pen * (hiK + hiN);
          const T jump = uin - uout;
          fv = a.visc * (T(-0.5) * (dnin + dnout) + Cpen * jump);
          fg = T(-0.5) * a.visc * jump;
          if (ADV) {
            T unin, unout, lam;
            if (c == 0) {
              unin = T(0);
              unout = T(0);
#pragma unroll
              for (int i = 0; i < N; ++i) {
                unin += tb.L[s][i] * s_ub[ax][cl][node_of(N, ax, i, t, DIM)];
                unout += tb.L[1 - s][i] *
                         __ldg(&ub[((int64_t)ax * a.ncell + nb) * NB + node_of(N, ax, i, t, DIM)]);
              }
              unin *= sgn;
              unout *= sgn;
              lam = fmax(fabs(unin), fabs(unout));
              s_un[cl][fp][0] = unin;
              s_un[cl][fp][1] = unout;
              s_un[cl][fp][2] = lam;
            } else {
              unin = s_un[cl][fp][0];
              unout = s_un[cl][fp][1];
              lam = s_un[cl][fp][2];
            }
            fv += a.adv * (T(0.5) * (uin * unin + uout * unout) + T(0.5) * lam * jump);
          }
        } else if (a.walls) {
          const T sig = a.pen * hiK;
          fv = a.visc * (-dnin + T(2) * sig * uin);
          fg = -a.visc * uin;
          if (ADV) {
            T unin, lam;
            if (c == 0) {
              unin = T(0);
#pragma unroll
              for (int i = 0; i < N; ++i)
                unin += tb.L[s][i] * s_ub[ax][cl][node_of(N, ax, i, t, DIM)];
              unin *= sgn;
              lam = fabs(unin);
              s_un[cl][fp][0] = unin;
              s_un[cl][fp][2] = lam;
            } else {
              lam = s_un[cl][fp][2];
            }
            fv += a.adv * lam * uin;
          }
        }
        s_f[cl][fp][0] = wt * fv;
        s_f[cl][fp][1] = wt * fg * sgn * hiK;
      }
    }
    __syncthreads();
    if (active) {
      T y = a.mass * W * s_u[cl][node];
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        T acc = T(0);
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
      dst[(int64_t)c * a.ncell * NB + cell * NB + node] = y;
    }
    __syncthreads();
  }
}

template <int N, int DIM>
constexpr int default_cpb() {
  return Shape<N, DIM>::NB <= 8 ? 16 : (Shape<N, DIM>::NB <= 27 ? 8 : (Shape<N, DIM>::NB <= 64 ? 4 : 2));
}

template <typename T, int DIM, int N, bool ADV, int CPB>
constexpr int smem_bytes() {
  return (int)sizeof(T) * CPB *
         (Shape<N, DIM>::NB * (1 + DIM) + 2 * Shape<N, DIM>::NFP +
          (ADV ? DIM * Shape<N, DIM>::NB + 3 * Shape<N, DIM>::NFP : 4));
}

// Tile-shape candidates of the autotuner: half, default and double the
// default cells per CTA, each clamped to the 48 KB static shared-memory and
// 1024-thread limits.
template <typename T, int DIM, int N, bool ADV>
constexpr int cpb_variant(int v) {
  int c = v == 0 ? default_cpb<N, DIM>() / 2 : (v == 2 ? default_cpb<N, DIM>() * 2 : default_cpb<N, DIM>());
  if (c < 1) c = 1;
  while (c > 1 && (c * Shape<N, DIM>::NB > 1024 ||
                   (int)sizeof(T) * c * (Shape<N, DIM>::NB * (1 + DIM) + 2 * Shape<N, DIM>::NFP +
                                          (ADV ? DIM * Shape<N, DIM>::NB + 3 * Shape<N, DIM>::NFP : 4)) >
                       48 * 1024))
    c /= 2;
  return c;
}

template <typename T, int DIM, int N, bool ADV, int CPB>
static dg_status launch_cpb(const OpArgs<T>& args, const Tab1D<T>& tb, const T* ub, const T* src,
                            T* dst, cudaStream_t s) {
  constexpr int threads = ((CPB * Shape<N, DIM>::NB + 31) / 32) * 32;
  const int64_t blocks = (args.ncell + CPB - 1) / CPB;
  if (blocks > 0x7fffffff) {
    set_error("operator apply: grid too large");
    return DG_EINVAL;
  }
  scalar_op_kernel<T, DIM, N, ADV, CPB><<<(unsigned)blocks, threads, 0, s>>>(args, tb, src, ub, dst); count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

template <typename T, int DIM, int N, bool ADV>
static dg_status launch_fixed(int variant, const OpArgs<T>& args, const Tab1D<T>& tb, const T* ub,
                              const T* src, T* dst, cudaStream_t s) {
  switch (variant) {
    case 0: return launch_cpb<T, DIM, N, ADV, cpb_variant<T, DIM, N, ADV>(0)>(args, tb, ub, src, dst, s);
    case 2: return launch_cpb<T, DIM, N, ADV, cpb_variant<T, DIM, N, ADV>(2)>(args, tb, ub, src, dst, s);
    default: return launch_cpb<T, DIM, N, ADV, cpb_variant<T, DIM, N, ADV>(1)>(args, tb, ub, src, dst, s);
  }
}

template <typename T, int DIM, int N, bool ADV>
static int cpb_of(int variant) {
  return cpb_variant<T, DIM, N, ADV>(variant);
}

template <typename T, int DIM, bool ADV>
static dg_status launch_dim(int variant, int N, const OpArgs<T>& args, const Tab1D<T>& tb,
                            const T* ub, const T* src, T* dst, cudaStream_t s) {
  switch (N) {
    case 2: return launch_fixed<T, DIM, 2, ADV>(variant, args, tb, ub, src, dst, s);
    case 3: return launch_fixed<T, DIM, 3, ADV>(variant, args, tb, ub, src, dst, s);
    case 4: return launch_fixed<T, DIM, 4, ADV>(variant, args, tb, ub, src, dst, s);
    case 5: return launch_fixed<T, DIM, 5, ADV>(variant, args, tb, ub, src, dst, s);
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

template <typename T>
const T* axis_h(const dg_mesh* m, int a, bool inv);
template <>
const double* axis_h<double>(const dg_mesh* m, int a, bool inv) { return inv ? m->d_hi64[a] : m->d_h64[a]; }
template <>
const float* axis_h<float>(const dg_mesh* m, int a, bool inv) { return inv ? m->d_hi32[a] : m->d_h32[a]; }
template <typename T>
const Tab1D<T>& tabs(const dg_mesh* m, bool pressure);
template <>
const Tab1D<double>& tabs<double>(const dg_mesh* m, bool p) { return p ? m->tp64 : m->tu64; }
template <>
const Tab1D<float>& tabs<float>(const dg_mesh* m, bool p) { return p ? m->tp32 : m->tu32; }

template <typename T>
dg_status launch_scalar_op(const dg_mesh* m, bool pressure, T mass, T visc, T adv, const T* ubar,
                           const T* src, T* dst, int ncomp, cudaStream_t s) {
  if (!m->affine) {
    set_error("operator apply: trilinear (perturbed) cells are not built in this library");
    return DG_EUNSUPPORTED;
  }
  OpArgs<T> a;
  a.ncell = m->ncell;
  a.n0 = m->n[0];
  a.n1 = m->n[1];
  a.n2 = m->n[2];
  a.per0 = m->periodic[0];
  a.per1 = m->periodic[1];
  a.per2 = m->periodic[2];
  a.h0 = axis_h<T>(m, 0, false);
  a.h1 = axis_h<T>(m, 1, false);
  a.h2 = axis_h<T>(m, 2, false);
  a.hi0 = axis_h<T>(m, 0, true);
  a.hi1 = axis_h<T>(m, 1, true);
  a.hi2 = axis_h<T>(m, 2, true);
  a.mass = mass;
  a.visc = visc;
  a.adv = adv;
  const int N = pressure ? m->np : m->nu;
  a.pen = (T)(N * N);  // (k+1)^2 for velocity, k^2 for pressure
  a.walls = pressure ? 0 : 1;
  a.ncomp = ncomp;
  const Tab1D<T>& tb = tabs<T>(m, pressure);
  const bool use_adv = !pressure && ubar != nullptr && adv != T(0);
  const int v = m->tune[sizeof(T) == 8 ? 0 : 1][pressure ? 0 : (use_adv ? 2 : 1)];
  if (m->dim == 2)
    return use_adv ? launch_dim<T, 2, true>(v, N, a, tb, ubar, src, dst, s)
                   : launch_dim<T, 2, false>(v, N, a, tb, ubar, src, dst, s);
  return use_adv ? launch_dim<T, 3, true>(v, N, a, tb, ubar, src, dst, s)
                 : launch_dim<T, 3, false>(v, N, a, tb, ubar, src, dst, s);
}

// cells per CTA of a tuning variant (reporting)
template <typename T>
static int cpb_for_mesh(const dg_mesh* m, bool pressure, bool adv, int v) {
  const int N = pressure ? m->np : m->nu;
  if (m->dim == 2) return adv ? cpb_dim<T, 2, true>(v, N) : cpb_dim<T, 2, false>(v, N);
  return adv ? cpb_dim<T, 3, true>(v, N) : cpb_dim<T, 3, false>(v, N);
}

// Time every tile-shape variant of the mesh's operator kernels (CUDA events,
// median of 7 launches after 2 warm-up launches, inputs zero: the kernels'
// work does not depend on values) and keep the fastest.  Results do not
// depend on the choice: each output is computed by one thread in a fixed
// order whatever the number of cells per CTA.
dg_status autotune_mesh(dg_mesh* m, cudaStream_t s) {
  const int64_t nu = m->ncell * m->nbu * m->dim, np = m->ncell * m->nbp;
  void* buf = nullptr;
  const size_t bytes = sizeof(double) * (size_t)(3 * nu + 2 * np);
  DG_CUDA(cudaMalloc(&buf, bytes));
  DG_CUDA(cudaMemsetAsync(buf, 0, bytes, s));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double* d = static_cast<double*>(buf);
  std::string rep = "[";
  dg_status st = DG_OK;
  const char* opname[3] = {"pressure", "momentum", "momentum+advection"};
  for (int prec = 0; prec < 2 && st == DG_OK; ++prec) {
    for (int op = 0; op < 3 && st == DG_OK; ++op) {
      float best = 1e30f, times[3] = {0, 0, 0};
      int bestv = 1;
      for (int v = 0; v < 3 && st == DG_OK; ++v) {
        m->tune[prec][op] = v;
        auto run = [&]() -> dg_status {
          const bool p = op == 0;
          if (prec == 0)
            return launch_scalar_op<double>(m, p, 1.0, 1.0, op == 2 ? 0.5 : 0.0, op == 2 ? d : nullptr,
                                            d + nu, d + 2 * nu, p ? 1 : m->dim, s);
          float* f = reinterpret_cast<float*>(buf);
          return launch_scalar_op<float>(m, p, 1.0f, 1.0f, op == 2 ? 0.5f : 0.0f, op == 2 ? f : nullptr,
                                         f + nu, f + 2 * nu, p ? 1 : m->dim, s);
        };
        for (int w = 0; w < 2 && st == DG_OK; ++w) st = run();
        std::vector<float> ms;
        for (int r = 0; r < 7 && st == DG_OK; ++r) {
          cudaEventRecord(e0, s);
          st = run();
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          float t = 0.0f;
          cudaEventElapsedTime(&t, e0, e1);
          ms.push_back(t);
        }
        if (st != DG_OK) break;
        std::sort(ms.begin(), ms.end());
        times[v] = ms[ms.size() / 2];
        if (times[v] < best) {
          best = times[v];
          bestv = v;
        }
      }
      m->tune[prec][op] = bestv;
      char line[256];
      const bool p = op == 0, adv = op == 2;
      auto cp = [&](int v) {
        return prec == 0 ? cpb_for_mesh<double>(m, p, adv, v) : cpb_for_mesh<float>(m, p, adv, v);
      };
      std::snprintf(line, sizeof(line),
                    "%s{\"op\": \"%s\", \"precision\": \"%s\", \"cells_per_cta\": [%d, %d, %d], "
                    "\"ms\": [%.5f, %.5f, %.5f], \"chosen\": %d}",
                    rep.size() > 1 ? ", " : "", opname[op], prec == 0 ? "f64" : "f32", cp(0), cp(1),
                    cp(2), times[0], times[1], times[2], cp(bestv));
      rep += line;
    }
  }
  rep += "]";
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(buf);
  if (st != DG_OK) return st;
  m->tuned = true;
  m->tune_report = rep;
  return DG_OK;
}

template dg_status launch_scalar_op<double>(const dg_mesh*, bool, double, double, double,
                                            const double*, const double*, double*, int,
                                            cudaStream_t);
template dg_status launch_scalar_op<float>(const dg_mesh*, bool, float, float, float, const float*,
                                           const float*, float*, int, cudaStream_t);

}  // namespace dg

using namespace dg;

extern "C" {

dg_status dg_apply_momentum(dg_mesh* m, const dg_momentum_coeffs* co, const double* ubar,
                            const double* src, double* dst, void* stream) {
  if (!m || !co || !src || !dst || (co->adv != 0.0 && !ubar) || src == dst || ubar == dst) {
    set_error("dg_apply_momentum: bad argument");
    return DG_EINVAL;
  }
  return launch_scalar_op<double>(m, false, co->mass, co->visc, co->adv, ubar, src, dst, m->dim,
                                  as_stream(stream));
}

dg_status dg_apply_momentum_f32(dg_mesh* m, const dg_momentum_coeffs* co, const float* ubar,
                                const float* src, float* dst, void* stream) {
  if (!m || !co || !src || !dst || (co->adv != 0.0 && !ubar) || src == dst || ubar == dst) {
    set_error("dg_apply_momentum_f32: bad argument");
    return DG_EINVAL;
  }
  return launch_scalar_op<float>(m, false, (float)co->mass, (float)co->visc, (float)co->adv, ubar,
                                 src, dst, m->dim, as_stream(stream));
}

dg_status dg_apply_poisson(dg_mesh* m, double alpha, const double* src, double* dst, void* stream) {
  if (!m || !src || !dst || src == dst) {
    set_error("dg_apply_poisson: bad argument");
    return DG_EINVAL;
  }
  return launch_scalar_op<double>(m, true, alpha, 1.0, 0.0, nullptr, src, dst, 1,
                                  as_stream(stream));
}

dg_status dg_autotune(dg_mesh* m, void* stream) {
  if (!m) {
    set_error("dg_autotune: null mesh");
    return DG_EINVAL;
  }
  return autotune_mesh(m, as_stream(stream));
}

dg_status dg_autotune_report(const dg_mesh* m, char* buf, int64_t size) {
  if (!m || !buf || size < 1) {
    set_error("dg_autotune_report: bad argument");
    return DG_EINVAL;
  }
  const std::string& r = m->tuned ? m->tune_report : std::string("[]");
  if ((int64_t)r.size() + 1 > size) {
    set_error("dg_autotune_report: buffer too small");
    return DG_EINVAL;
  }
  std::memcpy(buf, r.c_str(), r.size() + 1);
  return DG_OK;
}

dg_status dg_apply_poisson_f32(dg_mesh* m, double alpha, const float* src, float* dst,
                               void* stream) {
  if (!m || !src || !dst || src == dst) {
    set_error("dg_apply_poisson_f32: bad argument");
    return DG_EINVAL;
  }
  return launch_scalar_op<float>(m, true, (float)alpha, 1.0f, 0.0f, nullptr, src, dst, 1,
                                 as_stream(stream));
}

}  // extern "C"
