// Instantiation unit of the operator kernel: FP64 storage, float-float arithmetic, 2D.
#include "dg_apply_kernel.cuh"

namespace dg {

dg_status launch_df_2d(int variant, int N, bool adv, const OpArgs<double>& a, const Tab1D<df64>& tb,
               const double* ub, const double* src, double* dst, cudaStream_t s) {
  return adv ? launch_dim<double, df64, 2, true>(variant, N, a, tb, ub, src, dst, s)
             : launch_dim<double, df64, 2, false>(variant, N, a, tb, ub, src, dst, s);
}

}  // namespace dg
