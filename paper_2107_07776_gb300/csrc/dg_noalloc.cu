// dg_solve_helmholtz_noalloc: the pressure Helmholtz solve of dg_solve_stage
// (flexible CG, Jacobi or no preconditioning) for callers that must not
// allocate device memory -- code that runs inside a fixed memory budget set
// up front (embedded or real-time loops), host code that may not call into
// the CUDA allocator at that point (between a caller's own stream-ordered
// allocations, or inside a framework that owns the device heap through its
// own caching allocator), or callers without a dg_solver at all.
//
// All scratch lives in one file-scope __device__ array of fixed size
// (kScratchDoubles doubles, about 12.6 MB), which every GPU that loads the
// library holds until the process exits.  Host code cannot use the array's
// name as a device address (it is a host-side stand-in), so the first call on
// each device looks the address up with cudaGetSymbolAddress while that
// device is current and caches it; make that first call before any stream
// capture.  The mesh's device must be the current device (DG_EINVAL
// otherwise), so the scratch, the mesh and the caller's arrays are on one GPU.  Every call shares the array and it keeps the previous call's
// contents: each solve writes every scratch value before reading it, so
// nothing needs clearing, but calls whose work overlaps on the GPU (other
// streams, other host threads) race on the array and must be serialised by
// the caller.  No cudaMalloc, cudaFree, pinned-host allocation or other
// allocating routine is called.
#include <mutex>

#include "dg_krylov.cuh"

namespace {

constexpr int64_t kMaxDofsP = 262144;  // largest pressure system accepted (2^18 DoFs)
constexpr int64_t kPartialDoubles = 1216 * 2;
constexpr int64_t kScalDoubles = 64;
constexpr int64_t kScratchDoubles = 6 * kMaxDofsP + kPartialDoubles + kScalDoubles;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

double* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// device address of the scratch array on the mesh's device, which must be
// the current one (set-up once per device, with that device current)
dg_status scratch_address(int mesh_device, double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return dg::cuda_fail(e, "dg_solve_helmholtz_noalloc: cudaGetDevice");
  if (dev != mesh_device) {
    dg::set_error("dg_solve_helmholtz_noalloc: the current device (" + std::to_string(dev) +
                  ") is not the mesh's device (" + std::to_string(mesh_device) +
                  "); make the mesh's device current first");
    return DG_EINVAL;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    dg::set_error("dg_solve_helmholtz_noalloc: device index out of range");
    return DG_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return dg::cuda_fail(e, "dg_solve_helmholtz_noalloc: cudaGetSymbolAddress");
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return DG_OK;
}

struct NoallocCtx {
  dg_mesh* mesh;
  double alpha;
  cudaStream_t stream;
  dg::VecOps* vo;
  const double* dinv;
  int64_t n;
};

}  // namespace

using namespace dg;

extern "C" dg_status dg_solve_helmholtz_noalloc(dg_mesh* m, double alpha, const double* rhs,
                                                double* x, const dg_solve_opts* o,
                                                dg_solve_info* info, void* stream) {
  dg_solve_info tmp;
  if (!info) info = &tmp;
  info->iterations = 0;
  info->res0 = info->res_final = 0.0;
  info->status = DG_EINVAL;
  if (!m || !rhs || !x || !o || !(o->tol_rel > 0.0) || o->max_iter < 1 ||
      (o->precond != DG_PC_NONE && o->precond != DG_PC_JACOBI) ||
      (o->guess != DG_GUESS_ZERO && o->guess != DG_GUESS_GIVEN)) {
    set_error("dg_solve_helmholtz_noalloc: bad argument (precond NONE or JACOBI, guess ZERO or GIVEN)");
    return DG_EINVAL;
  }
  const int64_t n = m->ncell * m->nbp;
  if (n > kMaxDofsP) {
    set_error("dg_solve_helmholtz_noalloc: " + std::to_string(n) +
              " pressure DoFs exceed the fixed scratch (at most " + std::to_string(kMaxDofsP) +
              "); use dg_solve_stage");
    return DG_EINVAL;
  }
  double* base = nullptr;
  dg_status st = scratch_address(m->device, &base);
  if (st != DG_OK) {
    info->status = st;
    return st;
  }
  cudaStream_t s = as_stream(stream);
  double* dinv = base;
  double* r = base + n;  // r, r_old, z, p, q: consecutive, as cg_solve requires
  static thread_local double host_scal[kScalDoubles];
  VecOps vo;
  vo.stream = s;
  vo.partial = base + 6 * kMaxDofsP;
  vo.scal = vo.partial + kPartialDoubles;
  vo.host_scal = host_scal;
  NoallocCtx ctx{m, alpha, s, &vo, dinv, n};
  NoallocCtx* c = &ctx;
  // one-pointer captures keep std::function's storage inline (no heap)
  LinOp A = [c](const double* in, double* out) {
    return dg_apply_poisson(c->mesh, c->alpha, in, out, c->stream);
  };
  LinOp J = [c](const double* in, double* out) { return c->vo->mul(c->n, c->dinv, in, out); };
  const LinOp* P = nullptr;
  if (o->guess == DG_GUESS_ZERO) {
    cudaError_t e = cudaMemsetAsync(x, 0, sizeof(double) * n, s);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "dg_solve_helmholtz_noalloc");
      info->status = st;
      return st;
    }
  }
  if (o->precond == DG_PC_JACOBI) {
    st = poisson_diagonal(m, alpha, dinv, s);
    if (st == DG_OK) st = vo.invert(n, dinv, n, dinv);
    if (st != DG_OK) {
      info->status = st;
      return st;
    }
    P = &J;
  }
  st = cg_solve(vo, n, A, P, rhs, x, r, r + n, r + 2 * n, r + 3 * n, r + 4 * n, o->tol_rel,
                o->max_iter, o->timeout_s, info);
  cudaError_t e = cudaStreamSynchronize(s);
  if (st == DG_OK && e != cudaSuccess) st = cuda_fail(e, "dg_solve_helmholtz_noalloc");
  if (st == DG_ENOCONV) set_error("dg_solve_helmholtz_noalloc: max_iter reached above tolerance");
  if (st == DG_EBREAKDOWN) set_error("dg_solve_helmholtz_noalloc: non-finite residual or breakdown");
  if (st == DG_ETIMEOUT) set_error("dg_solve_helmholtz_noalloc: wall-clock limit reached");
  info->status = st;
  return st;
}
