// Instantiation unit of the operator kernel: FP32 storage and arithmetic, 2D.
#include "dg_apply_kernel.cuh"

namespace dg {

dg_status launch_f32_2d(int variant, int N, bool adv, const OpArgs<float>& a, const Tab1D<float>& tb,
               const float* ub, const float* src, float* dst, cudaStream_t s) {
  return adv ? launch_dim<float, float, 2, true>(variant, N, a, tb, ub, src, dst, s)
             : launch_dim<float, float, 2, false>(variant, N, a, tb, ub, src, dst, s);
}

}  // namespace dg
