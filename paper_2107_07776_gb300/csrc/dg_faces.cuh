// Face numbering of the structured mesh for the face-once kernels: the faces
// normal to axis a form layers along a (n_a layers on a periodic axis, the
// layer l between cells l-1 and l with wrap-around; n_a + 1 on a walled axis,
// layers 0 and n_a on the walls), times the cells of the other axes.  Faces
// of axis 0 come first, then axis 1, then axis 2; within an axis the index
// runs x fastest with the axis replaced by its layers.
#pragma once

#include <stdint.h>

namespace dg {

// number of face layers along axis a: periodic n_a, walled n_a + 1
__host__ __device__ __forceinline__ int face_layers(int n, int per) { return per ? n : n + 1; }

// faces normal to axis a (layers x the other axes' cells)
__host__ __device__ __forceinline__ int64_t faces_of_axis(int a, const int n[3], const int per[3]) {
  int64_t f = face_layers(n[a], per[a]);
  for (int b = 0; b < 3; ++b)
    if (b != a) f *= n[b];
  return f;
}

// linear index of the face at layer l along axis a with the tangential cell
// coordinates of c (x fastest, the axis a dimension replaced by its layers)
__device__ __forceinline__ int64_t face_index(int a, int l, const int c[3], const int n[3],
                                              const int per[3]) {
  const int d0 = a == 0 ? face_layers(n[0], per[0]) : n[0];
  const int d1 = a == 1 ? face_layers(n[1], per[1]) : n[1];
  const int f0 = a == 0 ? l : c[0], f1 = a == 1 ? l : c[1], f2 = a == 2 ? l : c[2];
  return f0 + (int64_t)d0 * (f1 + (int64_t)d1 * f2);
}

}  // namespace dg
