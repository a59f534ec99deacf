// Instantiation unit of the general-geometry operator kernel: storage float,
// arithmetic float, 3D.
#include "dg_general_kernel.cuh"

namespace dg {

dg_status gen_f32_3d(int kind, int N, const GenArgs<float>& a, const Tab1D<float>& tb,
                      const float* ub, const float* src, float* dst, cudaStream_t s) {
  return launch_general_dim<float, float, 3>(kind, N, a, tb, ub, src, dst, s);
}

}  // namespace dg
