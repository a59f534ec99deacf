// Stage solves and the TR-BDF2 projection step (Section 2: Eqs. trbdf2,
// first_stage, helmholtz2a, second_stage, helmholtz3a; algebraic form at the
// end of Section 3).  Every vector operation of the step runs in the
// library's kernels on the solver's stream; the host sequences them.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "dg_krylov.cuh"
#include "dg_mg.cuh"
#include "dg_guess.cuh"

struct dg_solver {
  dg_mesh* mesh = nullptr;
  double Re = 1.0, c = 1e3;
  // the solver's own non-blocking stream: every call first waits for the work
  // the caller has enqueued on the caller's stream (join_caller; the legacy
  // default stream unless dg_solver_set_stream named another) and
  // synchronises this stream before it returns
  cudaStream_t stream = nullptr;
  cudaStream_t caller = nullptr;  // nullptr: cudaStreamLegacy
  cudaEvent_t ev_in = nullptr;
  dg::VecOps vo;
  int64_t nu = 0, np = 0, nus = 0;  // velocity (all comps), pressure, one component
  int m_alloc = 0;
  double* V = nullptr;  // GMRES basis (m_alloc + 1) * nu
  double* w = nullptr;
  double* hdev = nullptr;
  double* dinv_u = nullptr;
  double* diag_s = nullptr;
  double* dinv_p = nullptr;
  double* cgbuf = nullptr;  // r, r_old, z, p, q (np each)
  // step state
  double *ub = nullptr, *ustar = nullptr, *ut_old = nullptr, *ut_new = nullptr, *uss = nullptr,
         *rhs_u = nullptr, *u_g = nullptr, *u_hist = nullptr, *fcomb = nullptr;
  double *rhs_p = nullptr, *p_g = nullptr;
  bool has_hist = false;
  int fp_iters[2] = {1, 1};  // Picard solves of the last step's momentum stages
  double* u_pred = nullptr;  // BDF2 projection steps: the last predicted velocity
  bool has_pred = false;
  std::vector<void*> allocs;
  dg::MultiGrid<float>* mg32 = nullptr;   // built on first use
  dg::MultiGrid<double>* mg64 = nullptr;
  dg::GuessState guess;                   // stage histories and learned-guess nets
  // per-phase CUDA-event tracing of trbdf2_step (dg_solver_set_tracing)
  bool tracing = false;
  cudaEvent_t ev[24] = {};
  double phase_ms[6] = {0, 0, 0, 0, 0, 0};
  int64_t traced_steps = 0;
};

namespace dg {
namespace {

dg_status join_caller(dg_solver* s) {
  DG_CUDA(cudaEventRecord(s->ev_in, s->caller ? s->caller : cudaStreamLegacy));
  DG_CUDA(cudaStreamWaitEvent(s->stream, s->ev_in, 0));
  return DG_OK;
}

dg_status dalloc(dg_solver* s, double** p, int64_t n) {
  cudaError_t e = cudaMalloc(p, sizeof(double) * (n > 0 ? n : 1));
  if (e != cudaSuccess) {
    set_error(std::string("solver workspace: ") + cudaGetErrorString(e));
    return DG_ENOMEM;
  }
  s->allocs.push_back(*p);
  return DG_OK;
}

dg_status ensure_basis(dg_solver* s, int m) {
  if (m <= s->m_alloc) return DG_OK;
  if (s->V) {
    for (auto& a : s->allocs)
      if (a == s->V) a = nullptr;
    cudaFree(s->V);
    s->V = nullptr;
  }
  dg_status st = dalloc(s, &s->V, (int64_t)(m + 1) * s->nu);
  if (st != DG_OK) return st;
  s->m_alloc = m;
  return DG_OK;
}

bool check_opts(const dg_solve_opts* o, const char* who) {
  if (!o || !(o->tol_rel > 0.0) || o->max_iter < 1 || o->restart < 1 || o->restart > 200) {
    set_error(std::string(who) + ": bad solve options");
    return false;
  }
  return true;
}

dg_status solve_momentum(dg_solver* s, const dg_momentum_coeffs* co, const double* ubar,
                         const double* rhs, double* x, const dg_solve_opts* o,
                         dg_solve_info* info) {
  dg_mesh* m = s->mesh;
  dg_status st;
  const double* dinv = nullptr;
  // ubar stays unchanged during the solve: the float-float applies split it
  // once instead of once per iteration, and the FP32 diagonal reads the pairs
  keep_presplit_ubar(m, ubar);
  if (o->precond == DG_PC_JACOBI) {
    if (m->affine) {  // diagonal and its inverse in one pass
      st = presplit_kept_ubar(m, s->stream);
      if (st == DG_OK) st = momentum_inv_diagonal_fp32(m, co, ubar, s->dinv_u, s->stream);
    } else {
      st = momentum_diagonal_fp32(m, co, ubar, s->diag_s, s->stream);
      if (st == DG_OK) st = s->vo.invert(s->nu, s->diag_s, s->nus, s->dinv_u);
    }
    if (st != DG_OK) {
      keep_presplit_ubar(m, nullptr);
      return st;
    }
    dinv = s->dinv_u;
  } else if (o->precond != DG_PC_NONE) {
    keep_presplit_ubar(m, nullptr);
    set_error("dg_solve_stage: momentum systems take NONE or JACOBI preconditioning");
    return DG_EINVAL;
  }
  if (o->guess == DG_GUESS_ZERO) {
    const cudaError_t e = cudaMemsetAsync(x, 0, sizeof(double) * s->nu, s->stream);
    if (e != cudaSuccess) {
      keep_presplit_ubar(m, nullptr);
      return cuda_fail(e, "dg_solve_stage");
    }
  }
  st = ensure_basis(s, o->restart);
  if (st != DG_OK) {
    keep_presplit_ubar(m, nullptr);
    return st;
  }
  LinOp A = [&](const double* in, double* out) {
    return dg_apply_momentum(m, co, ubar, in, out, s->stream);
  };
  st = gmres_solve(s->vo, s->nu, A, dinv, rhs, x, s->V, s->w, s->hdev, o->restart, o->tol_rel,
                   o->max_iter, o->timeout_s, info);
  keep_presplit_ubar(m, nullptr);
  return st;
}

dg_status solve_helmholtz(dg_solver* s, double alpha, const double* rhs, double* x,
                          const dg_solve_opts* o, dg_solve_info* info) {
  dg_mesh* m = s->mesh;
  dg_status st;
  if (o->guess == DG_GUESS_ZERO) DG_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * s->np, s->stream));
  LinOp A = [&](const double* in, double* out) {
    return dg_apply_poisson(m, alpha, in, out, s->stream);
  };
  LinOp J = [&](const double* in, double* out) { return s->vo.mul(s->np, s->dinv_p, in, out); };
  const LinOp* P = nullptr;
  if (o->precond == DG_PC_JACOBI) {
    st = poisson_diagonal(m, alpha, s->dinv_p, s->stream);
    if (st != DG_OK) return st;
    st = s->vo.invert(s->np, s->dinv_p, s->np, s->dinv_p);
    if (st != DG_OK) return st;
    P = &J;
  } else if (o->precond == DG_PC_MG_FP32 || o->precond == DG_PC_MG_FP64) {
    if (o->precond == DG_PC_MG_FP32) {
      if (!s->mg32) {
        s->mg32 = new (std::nothrow) MultiGrid<float>();
        if (!s->mg32) return DG_ENOMEM;
        st = s->mg32->build(m, s->stream);
        if (st != DG_OK) {
          delete s->mg32;
          s->mg32 = nullptr;
          return st;
        }
      }
      s->mg32->set_degree(o->mg_degree);
      st = s->mg32->set_alpha(alpha);
    } else {
      if (!s->mg64) {
        s->mg64 = new (std::nothrow) MultiGrid<double>();
        if (!s->mg64) return DG_ENOMEM;
        st = s->mg64->build(m, s->stream);
        if (st != DG_OK) {
          delete s->mg64;
          s->mg64 = nullptr;
          return st;
        }
      }
      s->mg64->set_degree(o->mg_degree);
      st = s->mg64->set_alpha(alpha);
    }
    if (st != DG_OK) return st;
  } else if (o->precond != DG_PC_NONE) {
    set_error("dg_solve_stage: unknown preconditioner");
    return DG_EINVAL;
  }
  LinOp MGP = [s, o](const double* in, double* out) {
    return o->precond == DG_PC_MG_FP32 ? s->mg32->apply(in, out) : s->mg64->apply(in, out);
  };
  if (o->precond == DG_PC_MG_FP32 || o->precond == DG_PC_MG_FP64) P = &MGP;
  double* r = s->cgbuf;
  return cg_solve(s->vo, s->np, A, P, rhs, x, r, r + s->np, r + 2 * s->np, r + 3 * s->np,
                  r + 4 * s->np, o->tol_rel, o->max_iter, o->timeout_s, info);
}


// ---------------------------------------------------------------- tracing
// phases: 0 extrapolation + momentum RHS, 1 initial guesses (history,
// learned prediction and training), 2 momentum solves, 3 projections +
// pressure RHS + velocity updates, 4 Helmholtz solves
struct Tracer {
  dg_solver* s;
  int n = 0;
  int phase[24];
  void mark(int ph) {
    if (!s->tracing || n >= 24) return;
    cudaEventRecord(s->ev[n], s->stream);
    phase[n] = ph;
    ++n;
  }
  void finish() {
    if (!s->tracing || n < 2) return;
    cudaEventSynchronize(s->ev[n - 1]);
    for (int i = 0; i + 1 < n; ++i) {
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, s->ev[i], s->ev[i + 1]);
      s->phase_ms[phase[i]] += ms;
    }
    ++s->traced_steps;
  }
};

// ---------------------------------------------------------------- guesses
// slot = 2 (stage - 1) + (0 momentum, 1 Helmholtz)
struct SysShape {
  int ncomp, nbc;
  int64_t n;
};

SysShape shape_of(const dg_solver* s, int slot) {
  const dg_mesh* m = s->mesh;
  if (slot & 1) return {1, m->nbp, s->np};
  return {m->dim, m->nbu, s->nu};
}

dg_status ensure_net(dg_solver* s, int k, const SysShape& sh) {
  GuessState& G = s->guess;
  if (G.net[k]) return DG_OK;
  Mlp* net = new (std::nothrow) Mlp();
  if (!net) return DG_ENOMEM;
  const int nbs = sh.ncomp * sh.nbc;
  dg_status st = net->init(5 * nbs, G.hidden, nbs, G.seed + 7919ull * k, s->stream);
  if (st != DG_OK) {
    delete net;
    return st;
  }
  G.net[k] = net;
  return DG_OK;
}

// x = xe + theta d with theta = (<d, b> - <A d, xe>) / <d, A d> from sc =
// [<d, A d>, <d, b>, <A d, xe>] (0 when d carries no energy): the energy-
// norm-optimal multiple of the learned correction d on top of the
// extrapolated guess xe
__global__ void theta_axpy_kernel(int64_t n, const double* __restrict__ sc,
                                  const double* __restrict__ xe, const double* __restrict__ d,
                                  double* __restrict__ x) {
  pdl_entry();
  const double den = sc[0];
  const double th = den > 0.0 ? (sc[1] - sc[2]) / den : 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    x[k] = xe[k] + th * d[k];
}

// Writes the initial guess of a stage solve into x (the caller's value
// stays when there is no history).  For the pressure Helmholtz systems the
// learned correction is scaled by the multiple that minimises the energy
// norm of the initial error along it (one line search of CG, two applies of
// alpha M^p + K), so the learned guess is never worse than the
// extrapolation in that norm.
dg_status prepare_guess(dg_solver* s, int slot, int mode, const double* rhs, double* x,
                        double alpha = 0.0) {
  GuessState& G = s->guess;
  G.predicted = false;
  if (mode != DG_GUESS_EXTRAP && mode != DG_GUESS_LEARNED) return DG_OK;
  const SysShape sh = shape_of(s, slot);
  const int cnt = G.count[slot];
  double* const* h = G.hist[slot];
  const dg_mesh* m = s->mesh;
  if (cnt == 1) {
    DG_CUDA(cudaMemcpyAsync(x, h[0], sizeof(double) * sh.n, cudaMemcpyDeviceToDevice, s->stream));
    return DG_OK;
  }
  if (cnt < 2) return DG_OK;
  const int k = (slot & 1) ? 0 : 1;
  const bool use_net = mode == DG_GUESS_LEARNED && G.enable && ((G.systems >> k) & 1) && cnt >= 4;
  if (!use_net) return guess_apply(m->ncell, sh.ncomp, sh.nbc, h[0], h[1], nullptr, nullptr, x, s->stream);
  dg_status st = ensure_net(s, k, sh);
  if (st != DG_OK) return st;
  if (!G.part) {
    DG_CUDA(cudaMalloc(&G.part, sizeof(double) * 5 * 1216));
    DG_CUDA(cudaMalloc(&G.dsc, sizeof(double) * 8));
  }
  Mlp& net = *G.net[k];
  st = guess_features(net, m->ncell, sh.ncomp, sh.nbc, h, rhs, G.part, G.dsc, s->stream);
  if (st != DG_OK) return st;
  const int64_t need = m->ncell * net.n_out;
  if (need > G.out_cap) {
    if (G.yout) cudaFree(G.yout);
    if (G.target) cudaFree(G.target);
    G.yout = G.target = nullptr;
    DG_CUDA(cudaMalloc(&G.yout, sizeof(float) * need));
    DG_CUDA(cudaMalloc(&G.target, sizeof(float) * need));
    G.out_cap = need;
  }
  st = G.train ? net.forward(m->ncell, G.yout, s->stream) : net.infer(m->ncell, G.yout, s->stream);
  if (st != DG_OK) return st;
  st = guess_apply(m->ncell, sh.ncomp, sh.nbc, h[0], h[1], G.yout, G.dsc, x, s->stream);
  if (st != DG_OK) return st;
  G.predicted = true;
  if (k == 0 && alpha > 0.0) {
    const int64_t n = sh.n;
    if (G.safe_n < n) {
      for (double** p : {&G.xe, &G.dvec, &G.rt}) {
        if (*p) cudaFree(*p);
        *p = nullptr;
      }
      DG_CUDA(cudaMalloc(&G.xe, sizeof(double) * n));
      DG_CUDA(cudaMalloc(&G.dvec, sizeof(double) * n));
      DG_CUDA(cudaMalloc(&G.rt, sizeof(double) * 2 * n));
      G.safe_n = n;
    }
    // theta = <d, b - A xe> / <d, A d> = (<d, b> - <A d, xe>) / <d, A d> (A
    // symmetric): one apply, to the correction only
    st = guess_apply(m->ncell, sh.ncomp, sh.nbc, h[0], h[1], nullptr, nullptr, G.xe, s->stream);
    if (st == DG_OK) st = s->vo.axpby(n, 1.0, x, -1.0, G.xe, G.dvec);
    if (st == DG_OK) st = dg_apply_poisson(s->mesh, alpha, G.dvec, G.rt, s->stream);
    if (st == DG_OK) {
      DG_CUDA(cudaMemcpyAsync(G.rt + n, rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, s->stream));
      st = s->vo.dots(n, 2, G.dvec, G.rt, n, s->vo.scal);       // <d, A d>, <d, b>
    }
    if (st == DG_OK) st = s->vo.dots(n, 1, G.rt, G.xe, n, s->vo.scal + 2);  // <A d, xe>
    if (st != DG_OK) return st;
    launch(theta_axpy_kernel, 1216, 256, 0, s->stream, n, s->vo.scal, G.xe, G.dvec, x);
    count_launch();
    DG_CUDA(cudaGetLastError());
  }
  return DG_OK;
}

// After a solve: one optimiser step on this solve (training mode) and the
// solution into the slot's history.
dg_status finish_guess(dg_solver* s, int slot, int mode, const double* xs) {
  GuessState& G = s->guess;
  if (mode != DG_GUESS_EXTRAP && mode != DG_GUESS_LEARNED) return DG_OK;
  const SysShape sh = shape_of(s, slot);
  const dg_mesh* m = s->mesh;
  double** h = G.hist[slot];
  if (G.predicted && G.train) {
    const int k = (slot & 1) ? 0 : 1;
    Mlp& net = *G.net[k];
    dg_status st = guess_target(m->ncell, sh.ncomp, sh.nbc, h[0], h[1], xs, G.dsc, G.target, s->stream);
    if (st != DG_OK) return st;
    double loss;
    st = net.backward(m->ncell, G.yout, G.target, &loss, s->stream);
    if (st != DG_OK) return st;
    st = net.adam_step(G.lr, s->stream);
    if (st != DG_OK) return st;
    G.last_loss = loss;
    ++G.train_steps;
  }
  G.predicted = false;
  if (!h[3]) {
    for (int a = 0; a < 4; ++a)
      if (!h[a]) DG_CUDA(cudaMalloc(&h[a], sizeof(double) * sh.n));
    G.n[slot] = sh.n;
  }
  double* oldest = h[3];
  h[3] = h[2];
  h[2] = h[1];
  h[1] = h[0];
  h[0] = oldest;
  DG_CUDA(cudaMemcpyAsync(h[0], xs, sizeof(double) * sh.n, cudaMemcpyDeviceToDevice, s->stream));
  if (G.count[slot] < 4) ++G.count[slot];
  return DG_OK;
}

// Momentum predictor of one stage (Eqs. first_stage / second_stage): one
// linear solve with the advecting field in s->ub, or, with fixed_point = K >
// 1, up to K Picard solves, each advected by the previous iterate (the fully
// nonlinear stage), until the relative change of the iterate is below
// fixed_point_tol.  The right-hand side depends on the advecting field only
// through the Dirichlet data's Lax-Friedrichs term, so it is rebuilt only
// when there is wall data.  x = s->ustar holds the guess on entry.
//
// mid = nullptr: the next advecting field is the iterate itself (the
// TR-BDF2 stages); otherwise the midpoint (iterate + mid)/2 (the
// Bell-Colella-Glaz predictor), whose right-hand side depends on the field
// through its explicit advection as well (rebuild_rhs).
dg_status momentum_stage(dg_solver* s, int fixed_point, double fixed_point_tol, int stage,
                         const dg_momentum_coeffs* co, const dg_momentum_rhs* rd,
                         const dg_solve_opts* mo, dg_solve_info* info,
                         const double* mid = nullptr, bool rebuild_rhs = false) {
  dg_status st = dg_solve_stage(s, co, 0.0, s->ub, s->rhs_u, s->ustar, mo, info);
  s->fp_iters[stage] = 1;
  if (st != DG_OK || fixed_point <= 1) return st;
  dg_solve_opts o = *mo;
  o.guess = DG_GUESS_GIVEN;  // each Picard solve starts from the previous iterate
  const int64_t nu = s->nu;
  int it = 1;
  while (it < fixed_point) {
    if (mid) {
      st = s->vo.axpby(nu, 0.5, s->ustar, 0.5, mid, s->ub);
      if (st != DG_OK) return st;
    } else {
      DG_CUDA(cudaMemcpyAsync(s->ub, s->ustar, sizeof(double) * nu, cudaMemcpyDeviceToDevice,
                              s->stream));
    }
    if (rd->uD || rebuild_rhs) {
      st = dg_rhs_momentum(s->mesh, rd, s->rhs_u, s->stream);
      if (st != DG_OK) return st;
    }
    dg_solve_info inf;
    st = dg_solve_stage(s, co, 0.0, s->ub, s->rhs_u, s->ustar, &o, &inf);
    info->iterations += inf.iterations;
    info->res_final = inf.res_final;
    info->status = inf.status;
    ++it;
    if (st != DG_OK) break;
    // change from the previous iterate: ub - it, or 2 ub - mid with a midpoint
    double dd[2];
    st = s->vo.axpby(nu, 1.0, s->ustar, mid ? -2.0 : -1.0, s->ub, s->w);
    if (st == DG_OK && mid) st = s->vo.axpby(nu, 1.0, s->w, 1.0, mid, s->w);
    if (st == DG_OK) st = s->vo.dots_host(nu, 1, s->w, s->w, nu, dd);
    if (st == DG_OK) st = s->vo.dots_host(nu, 1, s->ustar, s->ustar, nu, dd + 1);
    if (st != DG_OK) break;
    if (!std::isfinite(dd[0])) {
      set_error("trbdf2_step: fixed-point iteration diverged");
      st = DG_EBREAKDOWN;
      break;
    }
    if (std::sqrt(dd[0]) < fixed_point_tol * std::max(std::sqrt(dd[1]), 1e-300)) break;
  }
  s->fp_iters[stage] = it;
  return st;
}

}  // namespace
}  // namespace dg

using namespace dg;

extern "C" {

dg_status dg_solver_get_fixed_point(const dg_solver* s, int32_t it[2]) {
  if (!s || !it) {
    set_error("dg_solver_get_fixed_point: bad argument");
    return DG_EINVAL;
  }
  it[0] = s->fp_iters[0];
  it[1] = s->fp_iters[1];
  return DG_OK;
}

dg_status dg_solver_create(dg_mesh* m, double Re, double c, dg_solver** out) {
  if (!m || !out || !(Re > 0.0) || !(c > 0.0)) {
    set_error("dg_solver_create: bad argument");
    return DG_EINVAL;
  }
  *out = nullptr;
  dg_solver* s = new (std::nothrow) dg_solver();
  if (!s) return DG_ENOMEM;
  s->mesh = m;
  s->Re = Re;
  s->c = c;
  s->nus = m->ncell * m->nbu;
  s->nu = s->nus * m->dim;
  s->np = m->ncell * m->nbp;
  dg_status st = DG_OK;
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming) != cudaSuccess) {
    set_error("dg_solver_create: stream or event creation failed");
    st = DG_ECUDA;
  }
  s->vo.stream = s->stream;
  double** vecs_u[] = {&s->w, &s->dinv_u, &s->ub, &s->ustar, &s->ut_old, &s->ut_new, &s->uss,
                       &s->rhs_u, &s->u_g, &s->u_hist, &s->fcomb};
  for (double** v : vecs_u)
    if (st == DG_OK) st = dalloc(s, v, s->nu);
  if (st == DG_OK) st = dalloc(s, &s->diag_s, s->nus);
  if (st == DG_OK) st = dalloc(s, &s->dinv_p, s->np);
  if (st == DG_OK) st = dalloc(s, &s->cgbuf, 5 * s->np);
  if (st == DG_OK) st = dalloc(s, &s->rhs_p, s->np);
  if (st == DG_OK) st = dalloc(s, &s->p_g, s->np);
  if (st == DG_OK) st = dalloc(s, &s->hdev, 768);
  if (st == DG_OK) st = dalloc(s, &s->vo.partial, 1216 * 256);
  if (st == DG_OK) st = dalloc(s, &s->vo.scal, 256);
  if (st == DG_OK && cudaMallocHost(&s->vo.host_scal, sizeof(double) * 1024) != cudaSuccess) {
    set_error("dg_solver_create: pinned host scratch");
    st = DG_ENOMEM;
  }
  if (st == DG_OK) st = ensure_basis(s, 30);
  for (int i = 0; i < 24 && st == DG_OK; ++i)
    if (cudaEventCreate(&s->ev[i]) != cudaSuccess) st = DG_ECUDA;
  if (st != DG_OK) {
    dg_solver_destroy(s);
    return st;
  }
  *out = s;
  return DG_OK;
}

void dg_solver_destroy(dg_solver* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  delete s->mg32;
  delete s->mg64;
  for (int i = 0; i < 24; ++i)
    if (s->ev[i]) cudaEventDestroy(s->ev[i]);
  for (void* a : s->allocs)
    if (a) cudaFree(a);
  if (s->vo.host_scal) cudaFreeHost(s->vo.host_scal);
  if (s->ev_in) cudaEventDestroy(s->ev_in);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

dg_status dg_solve_stage(dg_solver* s, const dg_momentum_coeffs* co, double alpha,
                         const double* ubar, const double* rhs, double* x,
                         const dg_solve_opts* o, dg_solve_info* info) {
  dg_solve_info tmp;
  if (!info) info = &tmp;
  std::memset(info, 0, sizeof(*info));
  if (!s || !rhs || !x || !check_opts(o, "dg_solve_stage")) {
    if (s && o) set_error("dg_solve_stage: bad argument");
    info->status = DG_EINVAL;
    return DG_EINVAL;
  }
  dg_status st = join_caller(s);
  if (st != DG_OK) {
    info->status = st;
    return st;
  }
  if (o->system == DG_SYS_MOMENTUM) {
    if (!co || (co->adv != 0.0 && !ubar)) {
      set_error("dg_solve_stage: momentum solve needs coefficients and ubar");
      info->status = DG_EINVAL;
      return DG_EINVAL;
    }
    st = solve_momentum(s, co, ubar, rhs, x, o, info);
  } else if (o->system == DG_SYS_HELMHOLTZ) {
    st = solve_helmholtz(s, alpha, rhs, x, o, info);
  } else {
    set_error("dg_solve_stage: unknown system");
    st = DG_EINVAL;
  }
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (st == DG_OK && e != cudaSuccess) st = cuda_fail(e, "dg_solve_stage");
  if (st == DG_ENOCONV) set_error("dg_solve_stage: max_iter reached above tolerance");
  if (st == DG_EBREAKDOWN) set_error("dg_solve_stage: non-finite residual or breakdown");
  if (st == DG_ETIMEOUT) set_error("dg_solve_stage: wall-clock limit reached");
  info->status = st;
  return st;
}

dg_status dg_solver_set_stream(dg_solver* s, void* stream) {
  if (!s) {
    set_error("dg_solver_set_stream: null solver");
    return DG_EINVAL;
  }
  s->caller = as_stream(stream);
  return DG_OK;
}

dg_status dg_solver_set_history(dg_solver* s, const double* u_hist) {
  if (!s) {
    set_error("dg_solver_set_history: null solver");
    return DG_EINVAL;
  }
  s->has_pred = false;
  if (!u_hist) {
    s->has_hist = false;
    return DG_OK;
  }
  dg_status st = join_caller(s);
  if (st != DG_OK) return st;
  DG_CUDA(cudaMemcpyAsync(s->u_hist, u_hist, sizeof(double) * s->nu, cudaMemcpyDeviceToDevice,
                          s->stream));
  DG_CUDA(cudaStreamSynchronize(s->stream));
  s->has_hist = true;
  return DG_OK;
}

dg_status trbdf2_step(dg_solver* s, const dg_step_params* prm, double* u, double* p,
                      dg_solve_info info[4]) {
  if (!s || !prm || !u || !p || !(prm->dt > 0.0)) {
    set_error("trbdf2_step: bad argument");
    return DG_EINVAL;
  }
  if (!check_opts(&prm->mom, "trbdf2_step") || !check_opts(&prm->helm, "trbdf2_step"))
    return DG_EINVAL;
  if (prm->fixed_point > 1 && !(prm->fixed_point_tol > 0.0)) {
    set_error("trbdf2_step: fixed_point > 1 needs fixed_point_tol > 0");
    return DG_EINVAL;
  }
  if (join_caller(s) != DG_OK) return DG_ECUDA;
  dg_solve_info loc[4];
  if (!info) info = loc;
  std::memset(info, 0, sizeof(dg_solve_info) * 4);
  dg_mesh* m = s->mesh;
  VecOps& vo = s->vo;
  const cudaStream_t st_ = s->stream;
  const int64_t nu = s->nu, np = s->np;
  const double g = prm->gamma > 0.0 ? prm->gamma : 2.0 - std::sqrt(2.0);
  const double dt = prm->dt;
  const double a31 = (1.0 - g) / (2.0 * (2.0 - g)), a32 = a31, a33 = 1.0 / (2.0 - g);
  dg_solve_opts mo = prm->mom, ho = prm->helm;
  mo.system = DG_SYS_MOMENTUM;
  ho.system = DG_SYS_HELMHOLTZ;
  // the step prepares every guess itself (previous level, extrapolation or
  // learned), so the solves start from the vector they are handed
  if (mo.guess != DG_GUESS_ZERO) mo.guess = DG_GUESS_GIVEN;
  if (ho.guess != DG_GUESS_ZERO) ho.guess = DG_GUESS_GIVEN;
  dg_status st;
#define STEP(call)                  \
  do {                              \
    st = (call);                    \
    if (st != DG_OK) return st;     \
  } while (0)
  Tracer tr{s};
  tr.mark(0);
  if (!s->has_hist) {
    DG_CUDA(cudaMemcpyAsync(s->u_hist, u, sizeof(double) * nu, cudaMemcpyDeviceToDevice, st_));
    s->has_hist = true;
  }
  // ---------------- stage 1: momentum predictor (Eq. first_stage) -------
  if (prm->extrapolate) {
    const double c1 = g / (2.0 * (1.0 - g));
    STEP(vo.axpby(nu, 1.0 + c1, u, -c1, s->u_hist, s->ub));
  } else {
    DG_CUDA(cudaMemcpyAsync(s->ub, u, sizeof(double) * nu, cudaMemcpyDeviceToDevice, st_));
  }
  dg_momentum_coeffs co1 = {1.0 / (g * dt), 1.0 / (2.0 * s->Re), 0.5};
  dg_momentum_rhs r1;
  std::memset(&r1, 0, sizeof(r1));
  r1.mass = co1.mass;
  r1.u_mass = u;
  r1.n_terms = 1;
  r1.visc[0] = co1.visc;
  r1.adv[0] = co1.adv;
  r1.w[0] = u;
  // the explicit advection is advected by ubar_1, or by u^n itself in the
  // fully nonlinear form
  r1.wbar[0] = prm->fixed_point > 1 ? u : s->ub;
  r1.p = p;
  r1.uD = prm->uD_stage1;
  r1.dir_visc = co1.visc;
  r1.dir_adv = co1.adv;
  r1.ubar = s->ub;
  if (prm->f_n && prm->f_ng) {
    STEP(vo.axpby(nu, 0.5, prm->f_n, 0.5, prm->f_ng, s->fcomb));
    r1.f = s->fcomb;
  }
  STEP(dg_rhs_momentum(m, &r1, s->rhs_u, st_));
  if (mo.guess != DG_GUESS_ZERO)
    DG_CUDA(cudaMemcpyAsync(s->ustar, u, sizeof(double) * nu, cudaMemcpyDeviceToDevice, st_));
  tr.mark(1);
  STEP(prepare_guess(s, 0, prm->mom.guess, s->rhs_u, s->ustar));
  tr.mark(2);
  STEP(momentum_stage(s, prm->fixed_point, prm->fixed_point_tol, 0, &co1, &r1, &mo, &info[0]));
  tr.mark(1);
  STEP(finish_guess(s, 0, prm->mom.guess, s->ustar));
  tr.mark(3);
  // ---------------- stage 1: projection (Eq. helmholtz2a) ---------------
  const double tau1 = g * dt, alpha1 = 1.0 / (s->c * s->c * tau1 * tau1);
  // u~(p^n) into ut_old, u** = u* + tau u~(p^n) in the same pass
  STEP(project_fused(m, p, s->ut_old, s->ustar, tau1, nullptr, s->uss, st_));
  STEP(dg_rhs_pressure(m, alpha1, tau1, s->uss, p, s->rhs_p, st_));
  if (ho.guess != DG_GUESS_ZERO)
    DG_CUDA(cudaMemcpyAsync(s->p_g, p, sizeof(double) * np, cudaMemcpyDeviceToDevice, st_));
  tr.mark(1);
  STEP(prepare_guess(s, 1, prm->helm.guess, s->rhs_p, s->p_g, alpha1));
  tr.mark(4);
  STEP(dg_solve_stage(s, nullptr, alpha1, nullptr, s->rhs_p, s->p_g, &ho, &info[1]));
  tr.mark(1);
  STEP(finish_guess(s, 1, prm->helm.guess, s->p_g));
  tr.mark(3);
  // u~(p^{n+g}) into ut_new and u^{n+g} = u* - tau (u~new - u~old)
  STEP(project_fused(m, s->p_g, s->ut_new, s->ustar, -tau1, s->ut_old, s->u_g, st_));
  tr.mark(0);
  // ---------------- stage 2: momentum predictor (Eq. second_stage) ------
  if (prm->extrapolate) {
    STEP(vo.axpby(nu, 1.0 / g, s->u_g, -(1.0 - g) / g, u, s->ub));
  } else {
    DG_CUDA(cudaMemcpyAsync(s->ub, s->u_g, sizeof(double) * nu, cudaMemcpyDeviceToDevice, st_));
  }
  dg_momentum_coeffs co2 = {1.0 / ((1.0 - g) * dt), a33 / s->Re, a33};
  dg_momentum_rhs r2;
  std::memset(&r2, 0, sizeof(r2));
  r2.mass = co2.mass;
  r2.u_mass = s->u_g;
  r2.n_terms = 2;
  r2.visc[0] = a32 / s->Re;
  r2.adv[0] = a32;
  r2.w[0] = s->u_g;
  r2.wbar[0] = s->u_g;
  r2.visc[1] = a31 / s->Re;
  r2.adv[1] = a31;
  r2.w[1] = u;
  r2.wbar[1] = u;
  r2.p = s->p_g;
  r2.uD = prm->uD_stage2;
  r2.dir_visc = co2.visc;
  r2.dir_adv = co2.adv;
  r2.ubar = s->ub;
  if (prm->f_n && prm->f_ng && prm->f_n1) {
    STEP(vo.axpby(nu, a31, prm->f_n, a32, prm->f_ng, s->fcomb));
    STEP(vo.axpby(nu, 1.0, s->fcomb, a33, prm->f_n1, s->fcomb));
    r2.f = s->fcomb;
  }
  STEP(dg_rhs_momentum(m, &r2, s->rhs_u, st_));
  if (mo.guess != DG_GUESS_ZERO)
    DG_CUDA(cudaMemcpyAsync(s->ustar, s->u_g, sizeof(double) * nu, cudaMemcpyDeviceToDevice, st_));
  tr.mark(1);
  STEP(prepare_guess(s, 2, prm->mom.guess, s->rhs_u, s->ustar));
  tr.mark(2);
  STEP(momentum_stage(s, prm->fixed_point, prm->fixed_point_tol, 1, &co2, &r2, &mo, &info[2]));
  tr.mark(1);
  STEP(finish_guess(s, 2, prm->mom.guess, s->ustar));
  tr.mark(3);
  // ---------------- stage 2: projection (Eq. helmholtz3a) ---------------
  const double tau2 = (1.0 - g) * dt, alpha2 = 1.0 / (s->c * s->c * tau2 * tau2);
  // u~(p^{n+g}) is stage 1's ut_new (p^{n+g} has not changed since)
  STEP(vo.axpby(nu, 1.0, s->ustar, tau2, s->ut_new, s->uss));
  STEP(dg_rhs_pressure(m, alpha2, tau2, s->uss, s->p_g, s->rhs_p, st_));
  if (ho.guess != DG_GUESS_ZERO)
    DG_CUDA(cudaMemcpyAsync(p, s->p_g, sizeof(double) * np, cudaMemcpyDeviceToDevice, st_));
  // p (in: p^n, no longer needed) receives p^{n+1}
  tr.mark(1);
  STEP(prepare_guess(s, 3, prm->helm.guess, s->rhs_p, p, alpha2));
  tr.mark(4);
  STEP(dg_solve_stage(s, nullptr, alpha2, nullptr, s->rhs_p, p, &ho, &info[3]));
  tr.mark(1);
  STEP(finish_guess(s, 3, prm->helm.guess, p));
  tr.mark(3);
  // history u^{n+g} before u is overwritten with u^{n+1}
  DG_CUDA(cudaMemcpyAsync(s->u_hist, s->u_g, sizeof(double) * nu, cudaMemcpyDeviceToDevice, st_));
  // u~(p^{n+1}) into ut_old (free now) and u^{n+1} = u* - tau (u~(p^{n+1}) - u~(p^{n+g}))
  STEP(project_fused(m, p, s->ut_old, s->ustar, -tau2, s->ut_new, u, st_));
  tr.mark(5);
  DG_CUDA(cudaStreamSynchronize(st_));
  tr.finish();
#undef STEP
  return DG_OK;
}

dg_status dg_projection_step(dg_solver* s, const dg_projection_params* prm, double* u, double* p,
                             dg_solve_info info[2]) {
  if (!s || !prm || !u || !p || !(prm->dt > 0.0) ||
      (prm->scheme != DG_SCHEME_BCG && prm->scheme != DG_SCHEME_BDF2)) {
    set_error("dg_projection_step: bad argument");
    return DG_EINVAL;
  }
  if (!check_opts(&prm->mom, "dg_projection_step") || !check_opts(&prm->helm, "dg_projection_step"))
    return DG_EINVAL;
  if (prm->fixed_point > 1 && !(prm->fixed_point_tol > 0.0)) {
    set_error("dg_projection_step: fixed_point > 1 needs fixed_point_tol > 0");
    return DG_EINVAL;
  }
  if (join_caller(s) != DG_OK) return DG_ECUDA;
  dg_solve_info loc[2];
  if (!info) info = loc;
  std::memset(info, 0, sizeof(dg_solve_info) * 2);
  dg_mesh* m = s->mesh;
  VecOps& vo = s->vo;
  const cudaStream_t st_ = s->stream;
  const int64_t nu = s->nu, np = s->np;
  const double dt = prm->dt;
  const bool bcg = prm->scheme == DG_SCHEME_BCG;
  dg_solve_opts mo = prm->mom, ho = prm->helm;
  mo.system = DG_SYS_MOMENTUM;
  ho.system = DG_SYS_HELMHOLTZ;
  if (mo.guess != DG_GUESS_ZERO) mo.guess = DG_GUESS_GIVEN;
  dg_status st;
#define STEP(call)              \
  do {                          \
    st = (call);                \
    if (st != DG_OK) return st; \
  } while (0)
  if (!s->has_hist) {  // u^{n-1} = u^n before the first step
    DG_CUDA(cudaMemcpyAsync(s->u_hist, u, sizeof(double) * nu, cudaMemcpyDeviceToDevice, st_));
    s->has_hist = true;
  }
  if (!bcg && !s->u_pred) STEP(dalloc(s, &s->u_pred, nu));
  // ---------------- momentum predictor ----------------
  dg_momentum_coeffs co;
  dg_momentum_rhs r;
  std::memset(&r, 0, sizeof(r));
  if (bcg) {  // Eq. momentum_BCG: Crank-Nicolson with the midpoint advecting field
    co = {1.0 / dt, 1.0 / (2.0 * s->Re), 0.5};
    if (prm->fixed_point > 1)
      DG_CUDA(cudaMemcpyAsync(s->ub, u, sizeof(double) * nu, cudaMemcpyDeviceToDevice, st_));
    else
      STEP(vo.axpby(nu, 1.5, u, -0.5, s->u_hist, s->ub));
    r.mass = co.mass;
    r.u_mass = u;
    r.n_terms = 1;
    r.visc[0] = co.visc;
    r.adv[0] = co.adv;
    r.w[0] = u;
    r.wbar[0] = s->ub;
    if (prm->f_n && prm->f_n1) {
      STEP(vo.axpby(nu, 0.5, prm->f_n, 0.5, prm->f_n1, s->fcomb));
      r.f = s->fcomb;
    }
  } else {  // Eq. momentum_HI: BDF2 with the previous predicted velocity as field
    co = {1.5 / dt, 1.0 / s->Re, 1.0};
    DG_CUDA(cudaMemcpyAsync(s->ub, s->has_pred ? s->u_pred : u, sizeof(double) * nu,
                            cudaMemcpyDeviceToDevice, st_));
    STEP(vo.axpby(nu, 4.0, u, -1.0, s->u_hist, s->uss));
    r.mass = 1.0 / (2.0 * dt);
    r.u_mass = s->uss;
    r.f = prm->f_n1;
  }
  r.p = p;
  r.uD = prm->uD;
  r.dir_visc = co.visc;
  r.dir_adv = co.adv;
  r.ubar = s->ub;
  STEP(dg_rhs_momentum(m, &r, s->rhs_u, st_));
  if (mo.guess != DG_GUESS_ZERO)
    DG_CUDA(cudaMemcpyAsync(s->ustar, u, sizeof(double) * nu, cudaMemcpyDeviceToDevice, st_));
  if (bcg)
    STEP(momentum_stage(s, prm->fixed_point, prm->fixed_point_tol, 0, &co, &r, &mo, &info[0], u,
                        true));
  else
    STEP(momentum_stage(s, 1, 0.0, 0, &co, &r, &mo, &info[0]));
  s->fp_iters[1] = 1;
  // ---------------- projection ----------------
  if (bcg) {  // Eq. helmholtz_BCG: the pressure increment
    const double alpha = 1.0 / (s->c * s->c * dt * dt);
    DG_CUDA(cudaMemsetAsync(s->p_g, 0, sizeof(double) * np, st_));
    STEP(dg_rhs_pressure(m, alpha, dt, s->ustar, s->p_g, s->rhs_p, st_));
    ho.guess = DG_GUESS_ZERO;
    STEP(dg_solve_stage(s, nullptr, alpha, nullptr, s->rhs_p, s->p_g, &ho, &info[1]));
    DG_CUDA(cudaMemcpyAsync(s->u_hist, u, sizeof(double) * nu, cudaMemcpyDeviceToDevice, st_));
    STEP(project_fused(m, s->p_g, s->ut_new, s->ustar, -dt, nullptr, u, st_));
    STEP(vo.axpby(np, 1.0, p, 1.0, s->p_g, p));
  } else {  // Eq. helmholtz_HI with tau = 2 dt / 3
    const double tau = 2.0 * dt / 3.0, alpha = 1.0 / (s->c * s->c * tau * tau);
    STEP(project_fused(m, p, s->ut_old, s->ustar, tau, nullptr, s->uss, st_));
    STEP(dg_rhs_pressure(m, alpha, tau, s->uss, p, s->rhs_p, st_));
    if (ho.guess != DG_GUESS_ZERO) {
      ho.guess = DG_GUESS_GIVEN;
      DG_CUDA(cudaMemcpyAsync(s->p_g, p, sizeof(double) * np, cudaMemcpyDeviceToDevice, st_));
    }
    STEP(dg_solve_stage(s, nullptr, alpha, nullptr, s->rhs_p, s->p_g, &ho, &info[1]));
    DG_CUDA(cudaMemcpyAsync(s->u_pred, s->ustar, sizeof(double) * nu, cudaMemcpyDeviceToDevice, st_));
    s->has_pred = true;
    DG_CUDA(cudaMemcpyAsync(s->u_hist, u, sizeof(double) * nu, cudaMemcpyDeviceToDevice, st_));
    STEP(project_fused(m, s->p_g, s->ut_new, s->ustar, -tau, s->ut_old, u, st_));
    DG_CUDA(cudaMemcpyAsync(p, s->p_g, sizeof(double) * np, cudaMemcpyDeviceToDevice, st_));
  }
  DG_CUDA(cudaStreamSynchronize(st_));
#undef STEP
  return DG_OK;
}

dg_status dg_solver_set_tracing(dg_solver* s, int32_t on) {
  if (!s) {
    set_error("dg_solver_set_tracing: null solver");
    return DG_EINVAL;
  }
  s->tracing = on != 0;
  for (double& x : s->phase_ms) x = 0.0;
  s->traced_steps = 0;
  return DG_OK;
}

dg_status dg_solver_get_trace(const dg_solver* s, double phase_ms[6], int64_t* steps) {
  if (!s || !phase_ms) {
    set_error("dg_solver_get_trace: bad argument");
    return DG_EINVAL;
  }
  for (int i = 0; i < 6; ++i) phase_ms[i] = s->phase_ms[i];
  if (steps) *steps = s->traced_steps;
  return DG_OK;
}

dg_status dg_guess_configure(dg_solver* s, const dg_guess_opts* o) {
  if (!s || !o || o->hidden < 8 || o->hidden > 1024 || !(o->lr > 0.0f) || o->systems < 0 ||
      o->systems > 3) {
    set_error("dg_guess_configure: bad argument");
    return DG_EINVAL;
  }
  GuessState& G = s->guess;
  G.enable = o->enable ? 1 : 0;
  G.train = o->train ? 1 : 0;
  G.systems = o->systems;
  G.lr = o->lr;
  if (!G.net[0] && !G.net[1]) {
    G.hidden = o->hidden;
    G.seed = o->seed;
  }
  return DG_OK;
}

dg_status dg_guess_get_stats(const dg_solver* s, dg_guess_stats* st) {
  if (!s || !st) {
    set_error("dg_guess_get_stats: bad argument");
    return DG_EINVAL;
  }
  st->train_steps = s->guess.train_steps;
  st->last_loss = s->guess.last_loss;
  for (int i = 0; i < 4; ++i) st->history[i] = s->guess.count[i];
  return DG_OK;
}

}  // extern "C"

// Checkpoint (version 2): u^{n-1+gamma}, the stage histories of the guesses
// and the learned-guess networks with their optimiser state.
namespace {
bool put(FILE* f, const void* p, size_t n) { return std::fwrite(p, 1, n, f) == n; }
bool get(FILE* f, void* p, size_t n) { return std::fread(p, 1, n, f) == n; }

template <typename T>
bool put_dev(FILE* f, const T* d, int64_t n) {
  std::vector<T> h(n);
  if (n > 0 && cudaMemcpy(h.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return false;
  return put(f, h.data(), sizeof(T) * n);
}
template <typename T>
bool get_dev(FILE* f, T* d, int64_t n) {
  std::vector<T> h(n);
  if (!get(f, h.data(), sizeof(T) * n)) return false;
  return n == 0 || cudaMemcpy(d, h.data(), sizeof(T) * n, cudaMemcpyHostToDevice) == cudaSuccess;
}
}  // namespace

extern "C" {

dg_status dg_solver_save(const dg_solver* s, const char* path) {
  if (!s || !path) {
    set_error("dg_solver_save: bad argument");
    return DG_EINVAL;
  }
  DG_CUDA(cudaStreamSynchronize(s->stream));
  FILE* f = std::fopen(path, "wb");
  if (!f) {
    set_error(std::string("dg_solver_save: cannot open ") + path);
    return DG_EINVAL;
  }
  const GuessState& G = s->guess;
  const char magic[8] = {'D', 'G', 'T', 'R', 'B', 'D', 'F', '2'};
  int64_t hdr[4] = {2, s->nu, s->np, s->has_hist ? 1 : 0};
  bool ok = put(f, magic, 8) && put(f, hdr, sizeof(hdr)) && put_dev(f, s->u_hist, s->nu);
  for (int sl = 0; sl < 4 && ok; ++sl) {
    int64_t c[2] = {G.count[sl], G.n[sl]};
    ok = put(f, c, sizeof(c));
    for (int a = 0; a < G.count[sl] && ok; ++a) ok = put_dev(f, G.hist[sl][a], G.n[sl]);
  }
  for (int k = 0; k < 2 && ok; ++k) {
    const Mlp* n = G.net[k];
    int64_t d[6] = {n ? 1 : 0, n ? n->n_in : 0, n ? n->hidden : 0, n ? n->n_out : 0,
                    n ? n->adam_t : 0, n ? n->nparam : 0};
    ok = put(f, d, sizeof(d));
    if (n && ok) ok = put_dev(f, n->w, n->nparam) && put_dev(f, n->m1, n->nparam) &&
                      put_dev(f, n->m2, n->nparam);
  }
  int64_t tail[2] = {G.train_steps, 0};
  ok = ok && put(f, tail, sizeof(tail));
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) {
    set_error("dg_solver_save: write failed");
    return DG_EINVAL;
  }
  return DG_OK;
}

dg_status dg_solver_load(dg_solver* s, const char* path) {
  if (!s || !path) {
    set_error("dg_solver_load: bad argument");
    return DG_EINVAL;
  }
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    set_error(std::string("dg_solver_load: cannot open ") + path);
    return DG_EINVAL;
  }
  char magic[8];
  int64_t hdr[4];
  bool ok = get(f, magic, 8) && std::memcmp(magic, "DGTRBDF2", 8) == 0 && get(f, hdr, sizeof(hdr)) &&
            hdr[0] == 2 && hdr[1] == s->nu && hdr[2] == s->np && get_dev(f, s->u_hist, s->nu);
  GuessState& G = s->guess;
  for (int sl = 0; sl < 4 && ok; ++sl) {
    int64_t c[2];
    ok = get(f, c, sizeof(c)) && c[0] >= 0 && c[0] <= 4;
    if (!ok) break;
    const SysShape sh = shape_of(s, sl);
    if (c[0] > 0 && c[1] != sh.n) {
      ok = false;
      break;
    }
    for (int a = 0; a < 4 && c[0] > 0; ++a)
      if (!G.hist[sl][a] && cudaMalloc(&G.hist[sl][a], sizeof(double) * sh.n) != cudaSuccess) ok = false;
    for (int a = 0; a < c[0] && ok; ++a) ok = get_dev(f, G.hist[sl][a], sh.n);
    G.count[sl] = (int)c[0];
    G.n[sl] = sh.n;
  }
  for (int k = 0; k < 2 && ok; ++k) {
    int64_t d[6];
    ok = get(f, d, sizeof(d));
    if (!ok || !d[0]) continue;
    if (!G.net[k]) {
      G.hidden = (int)d[2];
      G.net[k] = new (std::nothrow) Mlp();
      ok = G.net[k] && G.net[k]->init((int)d[1], (int)d[2], (int)d[3], 1, s->stream) == DG_OK;
    }
    Mlp* n = G.net[k];
    ok = ok && n->n_in == d[1] && n->hidden == d[2] && n->n_out == d[3] && n->nparam == d[5] &&
         get_dev(f, n->w, n->nparam) && get_dev(f, n->m1, n->nparam) && get_dev(f, n->m2, n->nparam);
    if (ok) {
      n->adam_t = d[4];
      ok = n->sync_bf16(s->stream) == DG_OK && cudaStreamSynchronize(s->stream) == cudaSuccess;
    }
  }
  int64_t tail[2];
  ok = ok && get(f, tail, sizeof(tail));
  std::fclose(f);
  if (!ok) {
    set_error("dg_solver_load: not a checkpoint of this mesh");
    return DG_EINVAL;
  }
  G.train_steps = tail[0];
  s->has_hist = hdr[3] != 0;
  return DG_OK;
}

}  // extern "C"
