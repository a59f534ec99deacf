// Metric terms of trilinear (non-affine) cells, precomputed once per mesh
// (dg_geom.cu) and read by the general-geometry kernels.
//
// Every cell K is the image of [0,1]^d under the multilinear map of its 2^d
// lattice vertices; J = dx/dxi, Ji = J^-1 (Ji[a][r] = dxi_a/dx_r).  With the
// collocated nodal basis all integrals are sums over the Gauss-Legendre
// nodes, so an integrand needs only these per-point factors:
//
//   volume, per node q of a space with quadrature weight w_q:
//     G[a][b] = w_q det J Sum_r Ji[a][r] Ji[b][r]   (diffusion metric, symmetric)
//     W       = w_q det J                           (mass weight)
//     B[a][r] = w_q det J Ji[a][r]                  (velocity space only: maps
//               physical vectors to reference contravariant components, used
//               by advection, gradient and divergence terms)
//   face f = 2a + s of K (xi_a = s), per face point t:
//     dS      = w_t |det J Ji[a][.]|                (surface weight)
//     n[r]    = outward unit normal of K             (velocity space only)
//     cown[b] = Sum_r Ji[b][r] n[r] on K             (d/dn = cown . grad_ref)
//     cnb[b]  = Sum_r Ji'[b][r] n[r] on the neighbour K' at the same point
//               (its reference coordinate xi_a = 1 - s; 0 on walls)
//   per face: gpen = |Gamma|/|K| (wall) or (|Gamma|/|K| + |Gamma|/|K'|)/2
//     (interior), with |Gamma|, |K| by the (k+2)-point Gauss rule; the kernels
//     multiply by (k+1)^2 (velocity) or k^2 (pressure) for the SIP penalty.
//
// Layouts: volume [cell][field][node], face [cell][face][field][point], so a
// CTA's threads (one per node or face point) read each field coalesced.
#pragma once

#include "dg_common.cuh"

namespace dg {

template <int DIM>
struct GeomCount {
  static constexpr int NG = DIM * (DIM + 1) / 2;   // symmetric metric entries
  static constexpr int NVU = NG + 1 + DIM * DIM;   // velocity volume fields: G, W, B
  static constexpr int NVP = NG + 1;               // pressure volume fields: G, W
  static constexpr int NFU = 1 + 3 * DIM;          // velocity face fields: dS, n, cown, cnb
  static constexpr int NFP = 1 + 2 * DIM;          // pressure face fields: dS, cown, cnb
};

// index of G[a][b] in the packed upper triangle (row-major, a <= b)
__host__ __device__ __forceinline__ constexpr int sym_index(int dim, int a, int b) {
  return (a < b ? a : b) * dim - (a < b ? a : b) * ((a < b ? a : b) - 1) / 2 + (a < b ? b - a : a - b);
}

// Builds the metric arrays of a non-affine mesh (velocity terms only when
// `velocity` is set: multigrid levels need the pressure terms only).
dg_status build_geometry(dg_mesh* m, bool velocity, cudaStream_t s);
void free_geometry(dg_mesh* m);

// stage right-hand sides and diagonals on trilinear cells (dg_general_rhs.cu)
dg_status general_explicit(const dg_mesh* m, int mode, double visc, double adv, const double* w,
                           const double* wb, double* rhs, cudaStream_t s);
dg_status general_mass_grad(const dg_mesh* m, double mass, const double* um, const double* f,
                            const double* p, double* rhs, cudaStream_t s);
dg_status general_pressure_rhs(const dg_mesh* m, double alpha, double inv_tau, const double* uss,
                               const double* p_old, double* rhs, cudaStream_t s);
dg_status general_project(const dg_mesh* m, const double* p, double* ut, cudaStream_t s);
dg_status general_diag(const dg_mesh* m, bool pressure, double mass, double visc, double adv,
                       const double* ub, double* diag, bool fp32, cudaStream_t s);

}  // namespace dg
