// Instantiation unit of the general-geometry operator kernel: storage double,
// arithmetic df64, 2D.
#include "dg_general_kernel.cuh"

namespace dg {

dg_status gen_df_2d(int kind, int N, const GenArgs<double>& a, const Tab1D<df64>& tb,
                      const double* ub, const double* src, double* dst, cudaStream_t s) {
  return launch_general_dim<double, df64, 2>(kind, N, a, tb, ub, src, dst, s);
}

}  // namespace dg
