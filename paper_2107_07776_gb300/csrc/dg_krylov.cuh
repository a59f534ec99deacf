// Krylov building blocks shared by the solver translation units.
#pragma once

#include <functional>

#include "dg_common.cuh"

namespace dg {

// y = A x on the solver's stream
using LinOp = std::function<dg_status(const double* x, double* y)>;

// Deterministic vector kernels bound to one stream and one scratch area.
struct VecOps {
  cudaStream_t stream = nullptr;
  double* partial = nullptr;    // device, >= 1216 * (max vectors) doubles
  double* scal = nullptr;       // device, >= 64 doubles
  double* host_scal = nullptr;  // pinned host, >= 64 doubles
  dg_status dots(int64_t n, int nv, const double* w, const double* V, int64_t ldv,
                 double* out_dev);
  // r = b - q with <b, b> and <r, r> into out_dev[0, 1] (one pass)
  dg_status residual_norms(int64_t n, const double* b, const double* q, double* r, double* out_dev);
  dg_status dots_host(int64_t n, int nv, const double* w, const double* V, int64_t ldv,
                      double* out_host);
  dg_status axpby(int64_t n, double a, const double* x, double b, const double* y, double* z);
  dg_status mul(int64_t n, const double* d, const double* x, double* z);
  dg_status invert(int64_t n, const double* d, int64_t period, double* out);
};

dg_status gmres_solve(VecOps& vo, int64_t n, const LinOp& A, const double* dinv, const double* b,
                      double* x, double* V, double* w, double* hdev, int m, double tol,
                      int max_iter, double timeout_s, dg_solve_info* info);

// r_old must lie in the same allocation as r (their distance is used as a
// vector stride).
dg_status cg_solve(VecOps& vo, int64_t n, const LinOp& A, const LinOp* P, const double* b,
                   double* x, double* r, double* r_old, double* z, double* p, double* q,
                   double tol, int max_iter, double timeout_s, dg_solve_info* info);

dg_status poisson_diagonal(const dg_mesh* m, double alpha, double* diag, cudaStream_t s);
// ut = M^-1 P p (the projection's broken pressure gradient); when out is not
// null also out = base + tau (ut - sub) in the same pass (sub may be null).
dg_status project_fused(const dg_mesh* m, const double* p, double* ut, const double* base,
                        double tau, const double* sub, double* out, cudaStream_t s);
dg_status momentum_diagonal_fp32(const dg_mesh* m, const dg_momentum_coeffs* co, const double* ub,
                                 double* diag, cudaStream_t s);
// affine meshes: 1/diag of the momentum operator for every component at once
dg_status momentum_inv_diagonal_fp32(const dg_mesh* m, const dg_momentum_coeffs* co, const double* ub,
                                     double* dinv, cudaStream_t s);

}  // namespace dg
