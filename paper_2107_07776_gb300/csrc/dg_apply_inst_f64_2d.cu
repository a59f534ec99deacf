// Instantiation unit of the operator kernel: FP64 storage, native FP64 arithmetic, 2D.
#include "dg_apply_kernel.cuh"

namespace dg {

dg_status launch_f64_2d(int variant, int N, bool adv, const OpArgs<double>& a, const Tab1D<double>& tb,
               const double* ub, const double* src, double* dst, cudaStream_t s) {
  return adv ? launch_dim<double, double, 2, true>(variant, N, a, tb, ub, src, dst, s)
             : launch_dim<double, double, 2, false>(variant, N, a, tb, ub, src, dst, s);
}

}  // namespace dg
