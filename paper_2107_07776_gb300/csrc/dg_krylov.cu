// Krylov solvers for the stage systems (Section 4: GMRES with Jacobi for the
// momentum predictors, preconditioned CG for the pressure Helmholtz
// equations).  All vector work runs in the fused kernels below; the host only
// keeps the (restart x restart) Hessenberg least-squares problem and the
// scalar recurrences.  Reductions are deterministic: every inner product uses
// a fixed grid, a fixed per-block tree and a fixed-order second pass, so a
// solve gives the same bits on every run.
#include <chrono>
#include <cmath>
#include <vector>

#include "dg_krylov.cuh"

namespace dg {

namespace {

constexpr int kRedThreads = 256;

int red_blocks(int64_t n) {
  int64_t b = (n + 4 * kRedThreads - 1) / (4 * kRedThreads);
  if (b < 1) b = 1;
  if (b > 1216) b = 1216;  // 8 CTAs per SM on 152 SMs
  return (int)b;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partial[blk * nv + i] = sum over this block's range of w * V_i (fixed
// per-thread order, fixed block tree)
__global__ void __launch_bounds__(kRedThreads)
    multi_dot_kernel(int64_t n, int nv, const double* __restrict__ w, const double* __restrict__ V,
                     int64_t ldv, double* __restrict__ partial) {
  pdl_entry();
  __shared__ double s[kRedThreads];
  for (int i = 0; i < nv; ++i) {
    const double* v = V + (int64_t)i * ldv;
    double acc = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
      acc += w[k] * v[k];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int st = kRedThreads / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * nv + i] = s[0];
    __syncthreads();
  }
}

// out[i] = sum_blk partial[blk * nv + i], fixed order (one block per i)
__global__ void __launch_bounds__(kRedThreads)
    reduce_kernel(int nblk, int nv, const double* __restrict__ partial, double* __restrict__ out) {
  pdl_entry();
  constexpr int kWarps = kRedThreads / 32;
  __shared__ double s[kWarps];
  const int i = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += partial[(int64_t)b * nv + i];
  acc = warp_sum(acc);
  if (lane == 0) s[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) t += s[q];
    out[i] = t;
  }
}

// block sums of a 256-thread block's values in the fixed tree of
// multi_dot_kernel (s: the block's shared scratch)
__device__ __forceinline__ double block_tree_sum(double v, double* s) {
  s[threadIdx.x] = v;
  __syncthreads();
  for (int st = kRedThreads / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
    __syncthreads();
  }
  const double t = s[0];
  __syncthreads();
  return t;
}

// r = b - q with this block's partial sums of <b, b> and <r, r> in one pass
// (partial[blk * 2 + 0, 1]); the same per-thread order and block tree as
// multi_dot_kernel, so the sums equal those of two separate inner products
__global__ void __launch_bounds__(kRedThreads)
    residual_norms_kernel(int64_t n, const double* __restrict__ b, const double* __restrict__ q,
                          double* __restrict__ r, double* __restrict__ partial) {
  pdl_entry();
  __shared__ double s[kRedThreads];
  double bb = 0.0, rr = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double bk = b[k];
    const double rk = 1.0 * bk + (-1.0) * q[k];
    r[k] = rk;
    bb += bk * bk;
    rr += rk * rk;
  }
  bb = block_tree_sum(bb, s);
  rr = block_tree_sum(rr, s);
  if (threadIdx.x == 0) {
    partial[(int64_t)blockIdx.x * 2] = bb;
    partial[(int64_t)blockIdx.x * 2 + 1] = rr;
  }
}

// w -= sum_i h[i] V_i, then this block's partial sums of <w, U_i>
// (i < nu; U = V, or U = w itself when self_dot) in multi_dot_kernel's
// per-thread order and block tree, so the sums equal those of
// multi_dot_kernel run after the update.  Each thread reads back only the w
// elements it wrote.  Grid: red_blocks(n).
__global__ void __launch_bounds__(kRedThreads)
    axpy_dots_kernel(int64_t n, int nv, const double* __restrict__ h, const double* __restrict__ V,
                     int64_t ldv, double* __restrict__ w, int nu, int self_dot,
                     double* __restrict__ partial) {
  pdl_entry();
  __shared__ double s[kRedThreads];
  const int64_t k0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, dk = (int64_t)gridDim.x * blockDim.x;
  if (nu == 1) {  // one pass: the update and the single product together
    const double* u = self_dot ? nullptr : V;
    double acc = 0.0;
    for (int64_t k = k0; k < n; k += dk) {
      double wk = w[k];
      for (int i = 0; i < nv; ++i) wk -= h[i] * V[(int64_t)i * ldv + k];
      w[k] = wk;
      acc += wk * (u ? u[k] : wk);
    }
    acc = block_tree_sum(acc, s);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
    return;
  }
  for (int64_t k = k0; k < n; k += dk) {
    double wk = w[k];
    for (int i = 0; i < nv; ++i) wk -= h[i] * V[(int64_t)i * ldv + k];
    w[k] = wk;
  }
  for (int i = 0; i < nu; ++i) {
    const double* u = self_dot ? w : V + (int64_t)i * ldv;
    double acc = 0.0;
    for (int64_t k = k0; k < n; k += dk) acc += w[k] * u[k];
    acc = block_tree_sum(acc, s);
    if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * nu + i] = acc;
  }
}

// v = a x (in place allowed), z = dinv .* v: a new Arnoldi vector and its
// Jacobi-preconditioned copy in one pass
__global__ void scale_precondition_kernel(int64_t n, double a, const double* x, double* v,
                                          const double* __restrict__ dinv, double* __restrict__ z) {
  pdl_entry();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double vk = a * x[k] + 0.0;
    v[k] = vk;
    z[k] = dinv[k] * vk;
  }
}

// x += dinv .* sum_i y[i] V_i  (dinv NULL: identity)
__global__ void gmres_update_kernel(int64_t n, int nv, const double* __restrict__ y,
                                    const double* __restrict__ V, int64_t ldv,
                                    const double* __restrict__ dinv, double* __restrict__ x) {
  pdl_entry();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < nv; ++i) acc += y[i] * V[(int64_t)i * ldv + k];
    x[k] += dinv ? dinv[k] * acc : acc;
  }
}

__global__ void axpby_kernel(int64_t n, double a, const double* __restrict__ x, double b,
                             const double* __restrict__ y, double* __restrict__ z) {
  pdl_entry();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    z[k] = a * x[k] + (b == 0.0 ? 0.0 : b * y[k]);
}

__global__ void mul_kernel(int64_t n, const double* __restrict__ d, const double* __restrict__ x,
                           double* __restrict__ z) {
  pdl_entry();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    z[k] = d[k] * x[k];
}

__global__ void inv_kernel(int64_t n, const double* __restrict__ d, int64_t period,
                           double* __restrict__ out) {
  pdl_entry();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = 1.0 / d[k % period];
}

// CG update x += a p, r_old = r, r -= a q with a = sc[irz] / sc[ipq] read on
// the device, and this block's partial sum of the new <r, r>
// (multi_dot_kernel's order and tree)
__global__ void __launch_bounds__(kRedThreads)
    cg_update_dev_kernel(int64_t n, const double* __restrict__ sc, int irz, int ipq,
                         const double* __restrict__ p, const double* __restrict__ q,
                         double* __restrict__ x, double* __restrict__ r, double* __restrict__ r_old,
                         double* __restrict__ partial) {
  pdl_entry();
  __shared__ double s[kRedThreads];
  const double a = sc[irz] / sc[ipq];
  double rr = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    x[k] += a * p[k];
    const double rk = r[k];
    r_old[k] = rk;
    const double rn = rk - a * q[k];
    r[k] = rn;
    rr += rn * rn;
  }
  rr = block_tree_sum(rr, s);
  if (threadIdx.x == 0) partial[blockIdx.x] = rr;
}

// flexible (Polak-Ribiere) direction: p = z + beta p, beta = (<z, r> -
// <z, r_old>) / rz_old with sc[izr] = <z, r>, sc[izr + 1] = <z, r_old>,
// sc[irz] = rz_old
__global__ void cg_direction_kernel(int64_t n, const double* __restrict__ sc, int izr, int irz,
                                    const double* __restrict__ z, double* __restrict__ p) {
  pdl_entry();
  const double beta = (sc[izr] - sc[izr + 1]) / sc[irz];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    p[k] = z[k] + beta * p[k];
}

unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

// --------------------------------------------------------------- VecOps
dg_status VecOps::dots(int64_t n, int nv, const double* w, const double* V, int64_t ldv,
                       double* out_dev) {
  const int nb = red_blocks(n);
  launch(multi_dot_kernel, nb, kRedThreads, 0, stream, n, nv, w, V, ldv, partial); count_launch();
  launch(reduce_kernel, nv, kRedThreads, 0, stream, nb, nv, partial, out_dev); count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status VecOps::residual_norms(int64_t n, const double* b, const double* q, double* r,
                                 double* out_dev) {
  const int nb = red_blocks(n);
  launch(residual_norms_kernel, nb, kRedThreads, 0, stream, n, b, q, r, partial); count_launch();
  launch(reduce_kernel, 2, kRedThreads, 0, stream, nb, 2, partial, out_dev); count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status VecOps::dots_host(int64_t n, int nv, const double* w, const double* V, int64_t ldv,
                            double* out_host) {
  dg_status st = dots(n, nv, w, V, ldv, scal);
  if (st != DG_OK) return st;
  DG_CUDA(cudaMemcpyAsync(host_scal, scal, sizeof(double) * nv, cudaMemcpyDeviceToHost, stream));
  DG_CUDA(cudaStreamSynchronize(stream));
  for (int i = 0; i < nv; ++i) out_host[i] = host_scal[i];
  return DG_OK;
}

dg_status VecOps::axpby(int64_t n, double a, const double* x, double b, const double* y,
                        double* z) {
  launch(axpby_kernel, grid_for(n), 256, 0, stream, n, a, x, b, y, z); count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status VecOps::mul(int64_t n, const double* d, const double* x, double* z) {
  launch(mul_kernel, grid_for(n), 256, 0, stream, n, d, x, z); count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status VecOps::invert(int64_t n, const double* d, int64_t period, double* out) {
  launch(inv_kernel, grid_for(n), 256, 0, stream, n, d, period, out); count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

// --------------------------------------------------------------- GMRES
// Restarted GMRES(m), right Jacobi preconditioning (x = x0 + D^-1 V y, so the
// Arnoldi residual is the true residual), classical Gram-Schmidt applied
// twice (CGS2) through the fused multi-dot / multi-axpy kernels.
// Restarted GMRES(m) with right Jacobi preconditioning and two classical
// Gram-Schmidt passes.  Host round trips: one per cycle start (|b| and |r0|
// together) and one per Arnoldi step (both passes' coefficients and |w| in
// one copy); the small Hessenberg problem is solved on the host.
//   hdev: >= 3 * 256 doubles: [0, 256) pass-1 coefficients and y, [256, 512)
//   pass-2 coefficients, [512] |w|^2.  vo.host_scal: >= 1024 doubles (pinned),
//   [768, 1024) stages y.
dg_status gmres_solve(VecOps& vo, int64_t n, const LinOp& A, const double* dinv, const double* b,
                      double* x, double* V /* (m+1) n */, double* w, double* hdev, int m,
                      double tol, int max_iter, double timeout_s, dg_solve_info* info) {
  using clock = std::chrono::steady_clock;
  const auto t0 = clock::now();
  info->iterations = 0;
  info->res0 = info->res_final = 0.0;
  if (m > 255) {
    set_error("gmres: restart above 255");
    return DG_EINVAL;
  }
  double* const h1 = hdev;
  double* const h2 = hdev + 256;
  double* const hw = hdev + 512;
  double* const hs = vo.host_scal;
  double* const hy = vo.host_scal + 768;
  std::vector<double> H((size_t)(m + 1) * m), g(m + 1), cs(m), sn(m), hcol(m + 2);
  int it = 0;
  bool first = true;
  double bnorm = 0.0;
  while (true) {
    // r = b - A x -> V_0, with |b|^2 (first cycle) and |r|^2 in one round trip
    dg_status st = A(x, w);
    if (st != DG_OK) return st;
    st = vo.residual_norms(n, b, w, V, vo.scal);  // V_0 = b - A x, |b|^2, |V_0|^2
    if (st != DG_OK) return st;
    DG_CUDA(cudaMemcpyAsync(hs, vo.scal, sizeof(double) * 2, cudaMemcpyDeviceToHost, vo.stream));
    DG_CUDA(cudaStreamSynchronize(vo.stream));
    if (first) {
      bnorm = std::sqrt(hs[0]);
      if (!std::isfinite(bnorm)) return DG_EBREAKDOWN;
      if (bnorm == 0.0) {
        DG_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, vo.stream));
        return DG_OK;
      }
    }
    const double beta = std::sqrt(hs[1]);
    if (!std::isfinite(beta)) return DG_EBREAKDOWN;
    if (first) {
      info->res0 = beta;
      first = false;
    }
    info->res_final = beta;
    if (beta <= tol * bnorm) return DG_OK;
    if (it >= max_iter) return DG_ENOCONV;
    // V_0 = r / beta, and its preconditioned copy z = D^-1 V_0 staged in V_1
    if (dinv) {
      launch(scale_precondition_kernel, grid_for(n), 256, 0, vo.stream, n, 1.0 / beta, V, V, dinv, V + n);
      count_launch();
      DG_CUDA(cudaGetLastError());
    } else {
      st = vo.axpby(n, 1.0 / beta, V, 0.0, nullptr, V);
      if (st != DG_OK) return st;
    }
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    bool done = false;
    for (; j < m && it < max_iter; ++j, ++it) {
      double* vj = V + (int64_t)j * n;
      double* vj1 = V + (int64_t)(j + 1) * n;
      // w = A D^-1 v_j   (z = D^-1 v_j staged in v_{j+1} by the kernel that
      // wrote v_j)
      st = A(dinv ? vj1 : vj, w);
      if (st != DG_OK) return st;
      // two classical Gram-Schmidt passes on the device, then |w|^2: each
      // pass's update fused with the next pass's products
      {
        const int nb = red_blocks(n);
        st = vo.dots(n, j + 1, w, V, n, h1);
        if (st != DG_OK) return st;
        launch(axpy_dots_kernel, nb, kRedThreads, 0, vo.stream, n, j + 1, h1, V, (int64_t)n, w, j + 1, 0,
               vo.partial);
        count_launch();
        launch(reduce_kernel, j + 1, kRedThreads, 0, vo.stream, nb, j + 1, vo.partial, h2);
        count_launch();
        launch(axpy_dots_kernel, nb, kRedThreads, 0, vo.stream, n, j + 1, h2, V, (int64_t)n, w, 1, 1,
               vo.partial);
        count_launch();
        launch(reduce_kernel, 1, kRedThreads, 0, vo.stream, nb, 1, vo.partial, hw);
        count_launch();
        DG_CUDA(cudaGetLastError());
      }
      DG_CUDA(cudaMemcpyAsync(hs, h1, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, vo.stream));
      DG_CUDA(cudaMemcpyAsync(hs + 256, h2, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, vo.stream));
      DG_CUDA(cudaMemcpyAsync(hs + 512, hw, sizeof(double), cudaMemcpyDeviceToHost, vo.stream));
      DG_CUDA(cudaStreamSynchronize(vo.stream));
      const double hn2 = hs[512];
      for (int i = 0; i <= j; ++i) hcol[i] = hs[i] + hs[256 + i];
      hcol[j + 1] = std::sqrt(hn2);
      if (!std::isfinite(hcol[j + 1])) return DG_EBREAKDOWN;
      // Givens rotations
      for (int i = 0; i < j; ++i) {
        const double a = hcol[i], bb = hcol[i + 1];
        hcol[i] = cs[i] * a + sn[i] * bb;
        hcol[i + 1] = -sn[i] * a + cs[i] * bb;
      }
      const double a = hcol[j], bb = hcol[j + 1];
      const double r = std::hypot(a, bb);
      cs[j] = r == 0.0 ? 1.0 : a / r;
      sn[j] = r == 0.0 ? 0.0 : bb / r;
      hcol[j] = r;
      hcol[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
      const double hnext = std::sqrt(hn2);
      info->iterations = it + 1;
      info->res_final = std::fabs(g[j + 1]);
      if (std::fabs(g[j + 1]) <= tol * bnorm || hnext == 0.0) {
        ++j;
        ++it;
        done = true;
        break;
      }
      // v_{j+1} = w / |w| only when the cycle goes on (a converged cycle
      // never reads it), with the next step's z = D^-1 v_{j+1} in v_{j+2}
      // when that step belongs to this cycle
      if (dinv && j + 1 < m) {
        launch(scale_precondition_kernel, grid_for(n), 256, 0, vo.stream, n, 1.0 / hnext, w, vj1, dinv,
               vj1 + n);
        count_launch();
        DG_CUDA(cudaGetLastError());
      } else {
        st = vo.axpby(n, 1.0 / hnext, w, 0.0, nullptr, vj1);
        if (st != DG_OK) return st;
      }
      if (timeout_s > 0 &&
          std::chrono::duration<double>(clock::now() - t0).count() > timeout_s) {
        ++j;
        ++it;
        break;
      }
    }
    // y = H^-1 g (upper triangular) in pinned host memory, x += D^-1 V y.  The
    // copy is asynchronous: the staging area is written again only after the
    // next cycle's round trip.
    for (int i = j - 1; i >= 0; --i) {
      double s = g[i];
      for (int l = i + 1; l < j; ++l) s -= H[(size_t)i * m + l] * hy[l];
      hy[i] = s / H[(size_t)i * m + i];
    }
    DG_CUDA(cudaMemcpyAsync(h1, hy, sizeof(double) * j, cudaMemcpyHostToDevice, vo.stream));
    launch(gmres_update_kernel, grid_for(n), 256, 0, vo.stream, n, j, h1, V, n, dinv, x); count_launch();
    DG_CUDA(cudaGetLastError());
    if (timeout_s > 0 && std::chrono::duration<double>(clock::now() - t0).count() > timeout_s)
      return DG_ETIMEOUT;
    // with two Gram-Schmidt passes the Arnoldi residual tracks the true one,
    // so a converged cycle returns without another operator application
    if (done) return DG_OK;
  }
}

// --------------------------------------------------------------- FCG
// Flexible preconditioned CG (Polak-Ribiere beta = <z, r - r_old>/<z_old, r_old>),
// robust when the preconditioner varies between iterations (multigrid in
// reduced precision).  P == nullptr: unpreconditioned.
// Flexible preconditioned CG.  Its scalars stay on the device: the step
// length and the direction update read them there, so each iteration needs
// one host round trip (the residual norm for the stopping test, with <p, A p>
// for the breakdown test) instead of three.
//   device scalars (vo.scal): [0] <b, b>  [1] <r, r>  [2] <p, A p>
//   [3], [4] <z, r>, <z, r_old>  [5], [6] <z, r> of alternate iterations (rz)
dg_status cg_solve(VecOps& vo, int64_t n, const LinOp& A, const LinOp* P, const double* b,
                   double* x, double* r, double* r_old, double* z, double* p, double* q,
                   double tol, int max_iter, double timeout_s, dg_solve_info* info) {
  using clock = std::chrono::steady_clock;
  const auto t0 = clock::now();
  info->iterations = 0;
  double* sc = vo.scal;
  dg_status st = A(x, q);
  if (st != DG_OK) return st;
  st = vo.residual_norms(n, b, q, r, sc + 0);  // r = b - A x, <b, b>, <r, r>
  if (st != DG_OK) return st;
  DG_CUDA(cudaMemcpyAsync(vo.host_scal, sc, sizeof(double) * 2, cudaMemcpyDeviceToHost, vo.stream));
  DG_CUDA(cudaStreamSynchronize(vo.stream));
  const double bnorm = std::sqrt(vo.host_scal[0]);
  double rr = vo.host_scal[1];
  if (!std::isfinite(bnorm)) return DG_EBREAKDOWN;
  if (bnorm == 0.0) {
    DG_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, vo.stream));
    info->res0 = info->res_final = 0.0;
    return DG_OK;
  }
  info->res0 = info->res_final = std::sqrt(rr);
  if (!std::isfinite(rr)) return DG_EBREAKDOWN;
  if (info->res0 <= tol * bnorm) return DG_OK;
  if (P) {
    st = (*P)(r, z);
    if (st != DG_OK) return st;
  } else {
    DG_CUDA(cudaMemcpyAsync(z, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, vo.stream));
  }
  int irz = 5;  // slot of the current <z, r>
  st = vo.dots(n, 1, z, r, n, sc + irz);
  if (st != DG_OK) return st;
  DG_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, vo.stream));
  for (int it = 0; it < max_iter; ++it) {
    st = A(p, q);
    if (st != DG_OK) return st;
    st = vo.dots(n, 1, p, q, n, sc + 2);
    if (st != DG_OK) return st;
    {  // x += a p, r_old = r, r -= a q, and <r, r>
      const int nb = red_blocks(n);
      launch(cg_update_dev_kernel, nb, kRedThreads, 0, vo.stream, n, sc, irz, 2, p, q, x, r, r_old,
             vo.partial);
      count_launch();
      launch(reduce_kernel, 1, kRedThreads, 0, vo.stream, nb, 1, vo.partial, sc + 1);
      count_launch();
      DG_CUDA(cudaGetLastError());
    }
    DG_CUDA(cudaMemcpyAsync(vo.host_scal, sc + 1, sizeof(double) * 2, cudaMemcpyDeviceToHost, vo.stream));
    DG_CUDA(cudaStreamSynchronize(vo.stream));
    rr = vo.host_scal[0];
    const double pq = vo.host_scal[1];
    info->iterations = it + 1;
    // a non-positive <p, A p> means the step just taken was not a CG step:
    // report the breakdown (x and r hold that step)
    if (!std::isfinite(pq) || pq <= 0.0) return DG_EBREAKDOWN;
    info->res_final = std::sqrt(rr);
    if (!std::isfinite(rr)) return DG_EBREAKDOWN;
    if (info->res_final <= tol * bnorm) return DG_OK;
    if (timeout_s > 0 && std::chrono::duration<double>(clock::now() - t0).count() > timeout_s)
      return DG_ETIMEOUT;
    if (P) {
      st = (*P)(r, z);
      if (st != DG_OK) return st;
    } else {
      DG_CUDA(cudaMemcpyAsync(z, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, vo.stream));
    }
    // <z, r> and <z, r_old> in one pass (r_old = r + its distance in the
    // caller's workspace), then the direction on the device
    st = vo.dots(n, 2, z, r, r_old - r, sc + 3);
    if (st != DG_OK) return st;
    launch(cg_direction_kernel, grid_for(n), 256, 0, vo.stream, n, sc, 3, irz, z, p);
    count_launch();
    DG_CUDA(cudaGetLastError());
    // the new <z, r> becomes the next iteration's rz (alternate slot)
    irz = irz == 5 ? 6 : 5;
    DG_CUDA(cudaMemcpyAsync(sc + irz, sc + 3, sizeof(double), cudaMemcpyDeviceToDevice, vo.stream));
  }
  return DG_ENOCONV;
}

}  // namespace dg
