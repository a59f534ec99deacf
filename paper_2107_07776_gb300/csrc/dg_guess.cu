// Learned initial guess for the Krylov solves of the TR-BDF2 stages (a
// project addition; the paper uses the plain previous-level guess).
//
// Network: per-cell MLP n_in -> h -> h -> h -> n_out with SiLU between layers.
// Inputs are the cell's DoFs of the last four solutions of the same stage
// system, as the newest value and its first, second and third backward time
// differences, and of the right-hand side, each block scaled by 1/RMS of it;
// the output, times the RMS of the second difference (the size of the error
// of linear extrapolation), is added to the linear extrapolation
// 2 x_{k-1} - x_{k-2}.  The last layer starts at zero,
// so an untrained network returns exactly the extrapolated guess, and the
// Krylov solve still runs to its tolerance whatever the network predicts.
//
// Numerics: BF16 inputs, weights and hidden activations, FP32 accumulation
// and FP32 master weights / pre-activations / gradients, Adam.  All products
// run in one tensor-core GEMM kernel (mma.sync m16n8k16 BF16 -> FP32) with
// strided operands, so forward, input-gradient and weight-gradient products
// (the latter split over rows with a fixed-order second pass) share it.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dg_guess.cuh"

namespace dg {

namespace {

struct GemmDesc {
  int64_t M, N, K;
  const void* A;
  int64_t sam, sak;
  int abf;  // A is BF16 (else FP32)
  const void* B;
  int64_t sbk, sbn;
  int bbf;
  float* C;  // FP32 output (or split partials)
  int64_t scm, scn;
  __nv_bfloat16* Cb;  // BF16 output
  int64_t sbm_, sbn_;
  float* Z;  // FP32 pre-activation output
  int64_t szm, szn;
  const float* bias;
  int act;  // 0 none, 1 SiLU
  int64_t kchunk;
  int64_t pstride;  // > 0: split mode, partial z written at C + z * pstride
};

__device__ __forceinline__ float ld_any(const void* p, int64_t off, int bf) {
  return bf ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[off])
            : reinterpret_cast<const float*>(p)[off];
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }

// C[M x N] = A[M x K] B[K x N] (+ bias, activation); 64 x 64 tile per CTA,
// 4 warps of 32 x 32, K steps of 32 staged in shared memory as BF16.
__global__ void __launch_bounds__(128) gemm_bf16_kernel(const __grid_constant__ GemmDesc d) {
  pdl_entry();
  __shared__ __align__(16) __nv_bfloat16 As[64][40];
  __shared__ __align__(16) __nv_bfloat16 Bs[64][40];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const int wm = warp >> 1, wn = warp & 1;
  const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
  const int64_t kbeg = (int64_t)blockIdx.z * d.kchunk;
  const int64_t kend = kbeg + d.kchunk < d.K ? kbeg + d.kchunk : d.K;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;
  for (int64_t k0 = kbeg; k0 < kend; k0 += 32) {
    for (int idx = tid; idx < 64 * 32; idx += 128) {
      int mm, kk;
      if (d.sak == 1) {
        mm = idx >> 5;
        kk = idx & 31;
      } else {
        kk = idx >> 6;
        mm = idx & 63;
      }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      float v = 0.0f;
      if (gm < d.M && gk < kend) v = ld_any(d.A, gm * d.sam + gk * d.sak, d.abf);
      As[mm][kk] = __float2bfloat16_rn(v);
    }
    for (int idx = tid; idx < 64 * 32; idx += 128) {
      int nn, kk;
      if (d.sbk == 1) {
        nn = idx >> 5;
        kk = idx & 31;
      } else {
        kk = idx >> 6;
        nn = idx & 63;
      }
      const int64_t gn = n0 + nn, gk = k0 + kk;
      float v = 0.0f;
      if (gn < d.N && gk < kend) v = ld_any(d.B, gk * d.sbk + gn * d.sbn, d.bbf);
      Bs[nn][kk] = __float2bfloat16_rn(v);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 32; kk += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int r = wm * 32 + mi * 16;
        a[mi][0] = *reinterpret_cast<const uint32_t*>(&As[r + g][kk + 2 * t]);
        a[mi][1] = *reinterpret_cast<const uint32_t*>(&As[r + g + 8][kk + 2 * t]);
        a[mi][2] = *reinterpret_cast<const uint32_t*>(&As[r + g][kk + 2 * t + 8]);
        a[mi][3] = *reinterpret_cast<const uint32_t*>(&As[r + g + 8][kk + 2 * t + 8]);
      }
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int c = wn * 32 + ni * 8;
        b[ni][0] = *reinterpret_cast<const uint32_t*>(&Bs[c + g][kk + 2 * t]);
        b[ni][1] = *reinterpret_cast<const uint32_t*>(&Bs[c + g][kk + 2 * t + 8]);
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], a[mi], b[ni]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t row = m0 + wm * 32 + mi * 16 + g + (q >> 1) * 8;
        const int64_t col = n0 + wn * 32 + ni * 8 + 2 * t + (q & 1);
        if (row >= d.M || col >= d.N) continue;
        float v = acc[mi][ni][q];
        if (d.pstride > 0) {
          d.C[(int64_t)blockIdx.z * d.pstride + row * d.scm + col * d.scn] = v;
          continue;
        }
        if (d.bias) v += d.bias[col];
        if (d.Z) d.Z[row * d.szm + col * d.szn] = v;
        if (d.act == 1) v = silu(v);
        if (d.C) d.C[row * d.scm + col * d.scn] = v;
        if (d.Cb) d.Cb[row * d.sbm_ + col * d.sbn_] = __float2bfloat16_rn(v);
      }
}

// ---- fused inference: all four layers in one kernel ----
// Each CTA keeps the whole network (BF16 weights, padded rows) in shared
// memory and walks over tiles of 16 rows per warp; a warp's activations stay
// in its own 16 shared-memory rows between layers (only __syncwarp needed),
// the accumulators in registers (16 column tiles of m16n8).  Same rounding
// points as the layer-by-layer path: BF16 inputs, weights and hidden
// activations, FP32 accumulation, bias added after the accumulation.
struct InferDesc {
  int64_t M;
  int n_in, n_out, kp, nop;  // kp: n_in rounded up to 16; nop: n_out rounded up to 8
  const __nv_bfloat16* X;    // [M x n_in]
  const __nv_bfloat16* wb;   // W_l[out][in], packed as in Mlp
  const float* w;            // FP32 master parameters (biases)
  int64_t woff[4], boff[4];
  float* y;                  // [M x n_out]
};

constexpr int kInferHidden = 128;
constexpr int kInferLdh = kInferHidden + 8;  // padded row of a hidden layer

// shared memory of the fused inference kernel with `warps` warps: the four
// weight matrices plus a 16-row activation tile per warp
__host__ __device__ inline int64_t infer_smem_elems(int kp, int nop, int warps) {
  const int s1 = kp + 8, sa = (kp > kInferHidden ? kp : kInferHidden) + 8;
  return (int64_t)kInferHidden * s1 + 2LL * kInferHidden * kInferLdh + (int64_t)nop * kInferLdh +
         (int64_t)warps * 16 * sa;
}

template <int kInferWarps>
__global__ void __launch_bounds__(kInferWarps * 32) mlp_infer_kernel(const __grid_constant__ InferDesc d) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16* sm = reinterpret_cast<__nv_bfloat16*>(smem_raw);
  constexpr int H = kInferHidden, LH = kInferLdh;
  const int s1 = d.kp + 8, sa = (d.kp > H ? d.kp : H) + 8;
  __nv_bfloat16* W1 = sm;
  __nv_bfloat16* W2 = W1 + (int64_t)H * s1;
  __nv_bfloat16* W3 = W2 + (int64_t)H * LH;
  __nv_bfloat16* W4 = W3 + (int64_t)H * LH;
  __nv_bfloat16* act = W4 + (int64_t)d.nop * LH;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const __nv_bfloat16 z16 = __float2bfloat16_rn(0.0f);
  for (int idx = tid; idx < H * d.kp; idx += nthr) {
    const int n = idx / d.kp, k = idx % d.kp;
    W1[n * s1 + k] = k < d.n_in ? d.wb[d.woff[0] + (int64_t)n * d.n_in + k] : z16;
  }
  // the hidden layers (the bulk of the weights) as 16-byte vectors when their
  // packed rows are 16-byte aligned, else element by element
  const bool vec = ((reinterpret_cast<uintptr_t>(d.wb + d.woff[1]) |
                     reinterpret_cast<uintptr_t>(d.wb + d.woff[2])) & 15u) == 0;
  if (vec) {
    for (int idx = tid; idx < H * H / 8; idx += nthr) {
      const int n = idx / (H / 8), k = (idx % (H / 8)) * 8;
      *reinterpret_cast<uint4*>(&W2[n * LH + k]) =
          *reinterpret_cast<const uint4*>(&d.wb[d.woff[1] + (int64_t)n * H + k]);
      *reinterpret_cast<uint4*>(&W3[n * LH + k]) =
          *reinterpret_cast<const uint4*>(&d.wb[d.woff[2] + (int64_t)n * H + k]);
    }
  } else {
    for (int idx = tid; idx < H * H; idx += nthr) {
      const int n = idx / H, k = idx % H;
      W2[n * LH + k] = d.wb[d.woff[1] + idx];
      W3[n * LH + k] = d.wb[d.woff[2] + idx];
    }
  }
  for (int idx = tid; idx < d.nop * H; idx += nthr) {
    const int n = idx / H, k = idx % H;
    W4[n * LH + k] = n < d.n_out ? d.wb[d.woff[3] + (int64_t)n * H + k] : z16;
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  __nv_bfloat16* A = act + (int64_t)warp * 16 * sa;
  const bool vecx = d.n_in % 8 == 0 && (reinterpret_cast<uintptr_t>(d.X) & 15u) == 0;
  const int64_t tile = 16 * kInferWarps;
  for (int64_t r0 = (int64_t)blockIdx.x * tile; r0 < d.M; r0 += (int64_t)gridDim.x * tile) {
    const int64_t wr0 = r0 + warp * 16;
    if (vecx) {  // rows of 8-element multiples: 16-byte chunks, never across rows
      const int cpr = d.n_in / 8;
      for (int idx = lane; idx < 16 * cpr; idx += 32) {
        const int rr = idx / cpr, k = (idx % cpr) * 8;
        const int64_t row = wr0 + rr;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (row < d.M) v = *reinterpret_cast<const uint4*>(&d.X[row * d.n_in + k]);
        *reinterpret_cast<uint4*>(&A[rr * sa + k]) = v;
      }
      for (int idx = lane; idx < 16 * (d.kp - d.n_in); idx += 32) {
        const int rr = idx / (d.kp - d.n_in), k = d.n_in + idx % (d.kp - d.n_in);
        A[rr * sa + k] = z16;
      }
    } else {
      for (int idx = lane; idx < 16 * d.kp; idx += 32) {
        const int rr = idx / d.kp, k = idx % d.kp;
        const int64_t row = wr0 + rr;
        A[rr * sa + k] = (row < d.M && k < d.n_in) ? d.X[row * d.n_in + k] : z16;
      }
    }
    __syncwarp();
    for (int l = 0; l < 4; ++l) {
      const __nv_bfloat16* W = l == 0 ? W1 : (l == 1 ? W2 : (l == 2 ? W3 : W4));
      const int ldw = l == 0 ? s1 : LH;
      const int K = l == 0 ? d.kp : H;
      const int ntiles = l == 3 ? d.nop / 8 : H / 8;
      float acc[H / 8][4];
#pragma unroll
      for (int nt = 0; nt < H / 8; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[nt][q] = 0.0f;
      for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a[4];
        a[0] = *reinterpret_cast<const uint32_t*>(&A[g * sa + k0 + 2 * t]);
        a[1] = *reinterpret_cast<const uint32_t*>(&A[(g + 8) * sa + k0 + 2 * t]);
        a[2] = *reinterpret_cast<const uint32_t*>(&A[g * sa + k0 + 2 * t + 8]);
        a[3] = *reinterpret_cast<const uint32_t*>(&A[(g + 8) * sa + k0 + 2 * t + 8]);
#pragma unroll
        for (int nt = 0; nt < H / 8; ++nt) {
          if (nt >= ntiles) break;
          uint32_t bq[2];
          bq[0] = *reinterpret_cast<const uint32_t*>(&W[(nt * 8 + g) * ldw + k0 + 2 * t]);
          bq[1] = *reinterpret_cast<const uint32_t*>(&W[(nt * 8 + g) * ldw + k0 + 2 * t + 8]);
          mma_bf16(acc[nt], a, bq);
        }
      }
      __syncwarp();  // every lane has read this layer's input rows
      const float* bias = d.w + d.boff[l];
#pragma unroll
      for (int nt = 0; nt < H / 8; ++nt) {
        if (nt >= ntiles) break;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int rr = g + (q >> 1) * 8, col = nt * 8 + 2 * t + (q & 1);
          if (l < 3) {
            A[rr * sa + col] = __float2bfloat16_rn(silu(acc[nt][q] + bias[col]));
          } else if (col < d.n_out && wr0 + rr < d.M) {
            d.y[(wr0 + rr) * d.n_out + col] = acc[nt][q] + bias[col];
          }
        }
      }
      __syncwarp();
    }
  }
}

unsigned gridn(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// out[i] = sum_z part[z * n + i], fixed order
__global__ void split_reduce_kernel(int64_t n, int nz, const float* __restrict__ part,
                                    float* __restrict__ out) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int z = 0; z < nz; ++z) s += part[(int64_t)z * n + i];
    out[i] = s;
  }
}

// dz = 2 (y - t) / count, loss partials sum (y - t)^2 (double), fixed order
__global__ void __launch_bounds__(256) out_grad_kernel(int64_t n, float scale, const float* __restrict__ y,
                                                       const float* __restrict__ t, float* __restrict__ dz,
                                                       double* __restrict__ part) {
  pdl_entry();
  __shared__ double s[256];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float e = y[i] - t[i];
    dz[i] = scale * e;
    acc += (double)e * (double)e;
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// dz = dh * silu'(z); dzb = bf16(dz)
__global__ void silu_back_kernel(int64_t n, const float* __restrict__ dh, const float* __restrict__ z,
                                 float* __restrict__ dz) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float zz = z[i];
    const float sg = 1.0f / (1.0f + expf(-zz));
    dz[i] = dh[i] * sg * (1.0f + zz * (1.0f - sg));
  }
}

__global__ void to_bf16_kernel(int64_t n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

// column sums of a row-major [rows x cols] matrix, one block per column
__global__ void __launch_bounds__(256) col_sum_kernel(int64_t rows, int cols, const float* __restrict__ a,
                                                      float* __restrict__ out) {
  pdl_entry();
  __shared__ float s[256];
  const int c = blockIdx.x;
  float acc = 0.0f;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) acc += a[r * cols + c];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) s[threadIdx.x] += s[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = s[0];
}

__global__ void adam_kernel(int64_t n, float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m1, float* __restrict__ m2, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.0f - b1) * gi;
    const float v = b2 * m2[i] + (1.0f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    w[i] -= lr * (a * c1) / (sqrtf(v * c2) + eps);
  }
}

// ---- solver-side feature kernels (system vectors are [comp][cell][node]) ----
// The four stored solutions enter as their value and backward time
// differences (an invertible re-encoding that keeps the small differences
// representable in BF16): d0 = x1, d1 = x1 - x2, d2 = x1 - 2 x2 + x3,
// d3 = x1 - 3 x2 + 3 x3 - x4, each scaled by the inverse of its RMS.
// X[c][j*nbs + i] = d_j * is[j] (j < 4), X[c][4*nbs + i] = b * is[4]
__global__ void features_kernel(int64_t ncell, int ncomp, int nbc, const double* __restrict__ h0,
                                const double* __restrict__ h1, const double* __restrict__ h2,
                                const double* __restrict__ h3, const double* __restrict__ b,
                                const double* __restrict__ dsc, __nv_bfloat16* __restrict__ X) {
  pdl_entry();
  const double is0 = dsc[0], is1 = dsc[1], is2 = dsc[2], is3 = dsc[3], isb = dsc[4];
  const int nbs = ncomp * nbc;
  const int64_t total = ncell * nbs;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = k / nbs;
    const int i = (int)(k % nbs);
    const int comp = i / nbc, node = i % nbc;
    const int64_t o = ((int64_t)comp * ncell + c) * nbc + node;
    const double x1 = h0[o], x2 = h1[o], x3 = h2[o], x4 = h3[o];
    __nv_bfloat16* row = X + c * (int64_t)(5 * nbs);
    row[i] = __float2bfloat16_rn((float)(x1 * is0));
    row[nbs + i] = __float2bfloat16_rn((float)((x1 - x2) * is1));
    row[2 * nbs + i] = __float2bfloat16_rn((float)((x1 - 2.0 * x2 + x3) * is2));
    row[3 * nbs + i] = __float2bfloat16_rn((float)((x1 - 3.0 * x2 + 3.0 * x3 - x4) * is3));
    row[4 * nbs + i] = __float2bfloat16_rn((float)(b[o] * isb));
  }
}

// sums of squares of d0..d3 (as above) and of b, per block (fixed order)
__global__ void __launch_bounds__(256) hist_norms_kernel(int64_t n, const double* __restrict__ h0,
                                                         const double* __restrict__ h1,
                                                         const double* __restrict__ h2,
                                                         const double* __restrict__ h3,
                                                         const double* __restrict__ b,
                                                         double* __restrict__ part) {
  pdl_entry();
  __shared__ double s[5][256];
  double a[5] = {0, 0, 0, 0, 0};
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double x1 = h0[k], x2 = h1[k], x3 = h2[k], x4 = h3[k];
    const double d[5] = {x1, x1 - x2, x1 - 2.0 * x2 + x3, x1 - 3.0 * x2 + 3.0 * x3 - x4, b[k]};
    for (int j = 0; j < 5; ++j) a[j] += d[j] * d[j];
  }
  for (int j = 0; j < 5; ++j) s[j][threadIdx.x] = a[j];
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int j = 0; j < 5; ++j) s[j][threadIdx.x] += s[j][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int j = 0; j < 5; ++j) part[blockIdx.x * 5 + j] = s[j][0];
}

// block RMS values of the features from the partial sums (one warp per
// feature block, fixed lane assignment and reduction tree): dsc[0..4] inverse scales, dsc[5] the output scale (the
// second difference's RMS, else the first's, else the level's), dsc[6] its
// inverse
__global__ void __launch_bounds__(160) guess_scales_kernel(int nb, int64_t n, const double* __restrict__ part,
                                                           double* __restrict__ dsc) {
  pdl_entry();
  __shared__ double rms[5];
  const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;  // one warp per block j
  double a = 0.0;
  for (int i = lane; i < nb; i += 32) a += part[i * 5 + j];  // fixed assignment and order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) rms[j] = sqrt(a / (double)n);
  __syncthreads();
  if (threadIdx.x < 5) {
    const double r = rms[threadIdx.x];
    dsc[threadIdx.x] = 1.0 / (r > 0.0 && isfinite(r) ? r : 1.0);
  }
  if (threadIdx.x == 0) {
    const double s0 = rms[0] > 0.0 && isfinite(rms[0]) ? rms[0] : 1.0;
    const double so = rms[2] > 0.0 ? rms[2] : (rms[1] > 0.0 ? rms[1] : s0);
    dsc[5] = so;
    dsc[6] = 1.0 / so;
  }
}

// x = 2 h0 - h1 + dsc[5] * y  (y == nullptr: plain extrapolation)
__global__ void apply_guess_kernel(int64_t ncell, int ncomp, int nbc, const double* __restrict__ h0,
                                   const double* __restrict__ h1, const float* __restrict__ y,
                                   const double* __restrict__ dsc, double* __restrict__ x) {
  pdl_entry();
  const double so = y ? dsc[5] : 0.0;
  const int nbs = ncomp * nbc;
  const int64_t total = ncell * nbs;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = k / nbs;
    const int i = (int)(k % nbs);
    const int comp = i / nbc, node = i % nbc;
    const int64_t o = ((int64_t)comp * ncell + c) * nbc + node;
    double v = 2.0 * h0[o] - h1[o];
    if (y) v += so * (double)y[c * nbs + i];
    x[o] = v;
  }
}

// t = (x* - (2 h0 - h1)) / so in network layout
__global__ void target_kernel(int64_t ncell, int ncomp, int nbc, const double* __restrict__ h0,
                              const double* __restrict__ h1, const double* __restrict__ xs,
                              const double* __restrict__ dsc, float* __restrict__ t) {
  pdl_entry();
  const double iso = dsc[6];
  const int nbs = ncomp * nbc;
  const int64_t total = ncell * nbs;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = k / nbs;
    const int i = (int)(k % nbs);
    const int comp = i / nbc, node = i % nbc;
    const int64_t o = ((int64_t)comp * ncell + c) * nbc + node;
    t[c * nbs + i] = (float)((xs[o] - (2.0 * h0[o] - h1[o])) * iso);
  }
}

__global__ void f32_to_bf16_rows_kernel(int64_t n, const float* __restrict__ a,
                                        __nv_bfloat16* __restrict__ b) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

dg_status gemm(const GemmDesc& d0, int64_t ksplit, cudaStream_t s) {
  GemmDesc d = d0;
  if (d.M <= 0 || d.N <= 0 || d.K <= 0) return DG_OK;
  d.kchunk = ksplit > 1 ? ((d.K + ksplit - 1) / ksplit + 31) / 32 * 32 : d.K;
  const int64_t nz = (d.K + d.kchunk - 1) / d.kchunk;
  dim3 grid((unsigned)((d.N + 63) / 64), (unsigned)((d.M + 63) / 64), (unsigned)nz);
  if (grid.y > 65535 || nz > 65535) {
    set_error("learned guess: GEMM grid too large");
    return DG_EINVAL;
  }
  launch(gemm_bf16_kernel, grid, 128, 0, s, d); count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

uint64_t splitmix(uint64_t& st) {
  uint64_t z = (st += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

// ------------------------------------------------------------------ Mlp
Mlp::~Mlp() {
  void* ps[] = {w, g, m1, m2, wb, xb, z[0], z[1], z[2], z[3], hb[0], hb[1], hb[2], dz, dzb, dh,
                part, loss_part};
  for (void* p : ps)
    if (p) cudaFree(p);
  if (host_loss) cudaFreeHost(host_loss);
}

dg_status Mlp::init(int ni, int h, int no, uint64_t seed, cudaStream_t s) {
  n_in = ni;
  hidden = h;
  n_out = no;
  dims[0] = ni;
  dims[1] = dims[2] = dims[3] = h;
  dims[4] = no;
  int64_t off = 0;
  for (int l = 0; l < 4; ++l) {
    woff[l] = off;
    off += (int64_t)dims[l + 1] * dims[l];
    boff[l] = off;
    off += dims[l + 1];
  }
  nparam = off;
  std::vector<float> hw(nparam, 0.0f);
  uint64_t st = seed;
  for (int l = 0; l < 3; ++l) {  // Glorot-uniform layers 1-3; the output layer starts at zero
    const double lim = std::sqrt(6.0 / (dims[l] + dims[l + 1]));
    for (int64_t i = 0; i < (int64_t)dims[l + 1] * dims[l]; ++i) {
      const double u = (double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
      hw[woff[l] + i] = (float)((2.0 * u - 1.0) * lim);
    }
  }
  DG_CUDA(cudaMalloc(&w, sizeof(float) * nparam));
  DG_CUDA(cudaMalloc(&g, sizeof(float) * nparam));
  DG_CUDA(cudaMalloc(&m1, sizeof(float) * nparam));
  DG_CUDA(cudaMalloc(&m2, sizeof(float) * nparam));
  DG_CUDA(cudaMalloc(&wb, sizeof(__nv_bfloat16) * nparam));
  DG_CUDA(cudaMemcpyAsync(w, hw.data(), sizeof(float) * nparam, cudaMemcpyHostToDevice, s));
  DG_CUDA(cudaMemsetAsync(m1, 0, sizeof(float) * nparam, s));
  DG_CUDA(cudaMemsetAsync(m2, 0, sizeof(float) * nparam, s));
  DG_CUDA(cudaMallocHost(&host_loss, sizeof(double) * 1216));
  DG_CUDA(cudaMalloc(&loss_part, sizeof(double) * 1216));
  dg_status stt = sync_bf16(s);
  if (stt != DG_OK) return stt;
  // hw is a host buffer that goes out of scope on return: the copy must finish
  DG_CUDA(cudaStreamSynchronize(s));
  return DG_OK;
}

dg_status Mlp::sync_bf16(cudaStream_t s) {
  launch(f32_to_bf16_rows_kernel, gridn(nparam), 256, 0, s, nparam, w, wb); count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status Mlp::reserve(int64_t rows, cudaStream_t s) {
  (void)s;
  if (rows <= cap) return DG_OK;
  void* ps[] = {xb, z[0], z[1], z[2], z[3], hb[0], hb[1], hb[2], dz, dzb, dh, part};
  for (void* p : ps)
    if (p) cudaFree(p);
  cap = rows;
  const int64_t wmax = hidden > n_out ? hidden : n_out;
  DG_CUDA(cudaMalloc(&xb, sizeof(__nv_bfloat16) * cap * n_in));
  for (int l = 0; l < 4; ++l) DG_CUDA(cudaMalloc(&z[l], sizeof(float) * cap * dims[l + 1]));
  for (int l = 0; l < 3; ++l) DG_CUDA(cudaMalloc(&hb[l], sizeof(__nv_bfloat16) * cap * hidden));
  DG_CUDA(cudaMalloc(&dz, sizeof(float) * cap * wmax));
  DG_CUDA(cudaMalloc(&dzb, sizeof(__nv_bfloat16) * cap * wmax));
  DG_CUDA(cudaMalloc(&dh, sizeof(float) * cap * hidden));
  // weight-gradient partials: up to 64 row splits of the largest layer
  const int64_t maxw = (int64_t)hidden * (n_in > hidden ? n_in : hidden) +
                       (int64_t)n_out * hidden;
  part_cap = 64 * maxw;
  DG_CUDA(cudaMalloc(&part, sizeof(float) * part_cap));
  return DG_OK;
}

// Inference only: the fused kernel when the network fits in shared memory
// (hidden width 128), else the layer-by-layer GEMMs.
dg_status Mlp::infer(int64_t M, float* y, cudaStream_t s) {
  const int kp = (n_in + 15) / 16 * 16, nop = (n_out + 7) / 8 * 8;
  int dev = 0, max_optin = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // 16 warps per CTA (one CTA per SM covers 16 x 16 rows per SM and pass)
  // when their activation tiles fit next to the weights, else 8
  const int64_t bytes16 = 2 * infer_smem_elems(kp, nop, 16), bytes8 = 2 * infer_smem_elems(kp, nop, 8);
  const int warps = bytes16 <= max_optin ? 16 : 8;
  const int64_t bytes = warps == 16 ? bytes16 : bytes8;
  if (hidden != kInferHidden || nop > kInferHidden || bytes > max_optin) return forward(M, y, s);
  if (M <= 0) return DG_OK;
  void (*kern)(InferDesc) = warps == 16 ? mlp_infer_kernel<16> : mlp_infer_kernel<8>;
  DG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  int per_sm = 0;
  DG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, bytes));
  const int64_t tiles = (M + 16 * warps - 1) / (16 * warps);
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sms * std::max(1, per_sm)));
  InferDesc d;
  d.M = M;
  d.n_in = n_in;
  d.n_out = n_out;
  d.kp = kp;
  d.nop = nop;
  d.X = xb;
  d.wb = wb;
  d.w = w;
  for (int l = 0; l < 4; ++l) {
    d.woff[l] = woff[l];
    d.boff[l] = boff[l];
  }
  d.y = y;
  launch(kern, (unsigned)grid, warps * 32, bytes, s, d);
  count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status Mlp::forward(int64_t M, float* y, cudaStream_t s) {
  for (int l = 0; l < 4; ++l) {
    GemmDesc d;
    std::memset(&d, 0, sizeof(d));
    d.M = M;
    d.N = dims[l + 1];
    d.K = dims[l];
    d.A = l == 0 ? (const void*)xb : (const void*)hb[l - 1];
    d.sam = dims[l];
    d.sak = 1;
    d.abf = 1;
    d.B = wb + woff[l];  // W_l[out][in]: B(k = in, n = out)
    d.sbk = 1;
    d.sbn = dims[l];
    d.bbf = 1;
    d.bias = w + boff[l];
    d.Z = z[l];
    d.szm = dims[l + 1];
    d.szn = 1;
    if (l < 3) {
      d.act = 1;
      d.Cb = hb[l];
      d.sbm_ = hidden;
      d.sbn_ = 1;
    } else {
      d.C = y;
      d.scm = n_out;
      d.scn = 1;
    }
    dg_status st = gemm(d, 1, s);
    if (st != DG_OK) return st;
  }
  return DG_OK;
}

dg_status Mlp::backward(int64_t M, const float* y, const float* t, double* loss, cudaStream_t s) {
  const int64_t nout = M * n_out;
  const int nb = (int)std::min<int64_t>(1216, std::max<int64_t>(1, (nout + 1023) / 1024));
  launch(out_grad_kernel, nb, 256, 0, s, nout, (float)(2.0 / (double)nout), y, t, dz, loss_part); count_launch();
  DG_CUDA(cudaGetLastError());
  for (int l = 3; l >= 0; --l) {
    const int64_t no = dims[l + 1], ni = dims[l];
    launch(to_bf16_kernel, gridn(M * no), 256, 0, s, M * no, dz, dzb); count_launch();
    // dW_l[out][in] = sum_m dz[m][out] h_{l-1}[m][in], rows split for parallelism
    int64_t ksplit = std::min<int64_t>(64, std::max<int64_t>(1, M / 2048));
    while (ksplit > 1 && ksplit * no * ni > part_cap) --ksplit;
    GemmDesc d;
    std::memset(&d, 0, sizeof(d));
    d.M = no;
    d.N = ni;
    d.K = M;
    d.A = dzb;
    d.sam = 1;
    d.sak = no;
    d.abf = 1;
    d.B = l == 0 ? (const void*)xb : (const void*)hb[l - 1];
    d.sbk = ni;
    d.sbn = 1;
    d.bbf = 1;
    const int64_t kchunk = ksplit > 1 ? ((M + ksplit - 1) / ksplit + 31) / 32 * 32 : M;
    const int64_t nz = (M + kchunk - 1) / kchunk;
    d.C = nz > 1 ? part : g + woff[l];
    d.scm = ni;
    d.scn = 1;
    if (nz > 1) d.pstride = no * ni;
    dg_status st = gemm(d, ksplit, s);
    if (st != DG_OK) return st;
    if (nz > 1) {
      launch(split_reduce_kernel, gridn(no * ni), 256, 0, s, no * ni, (int)nz, part, g + woff[l]); count_launch();
    }
    launch(col_sum_kernel, (unsigned)no, 256, 0, s, M, (int)no, dz, g + boff[l]); count_launch();
    DG_CUDA(cudaGetLastError());
    if (l == 0) break;
    // dh[m][in] = sum_out dz[m][out] W_l[out][in]
    GemmDesc e;
    std::memset(&e, 0, sizeof(e));
    e.M = M;
    e.N = ni;
    e.K = no;
    e.A = dzb;
    e.sam = no;
    e.sak = 1;
    e.abf = 1;
    e.B = wb + woff[l];
    e.sbk = ni;
    e.sbn = 1;
    e.bbf = 1;
    e.C = dh;
    e.scm = ni;
    e.scn = 1;
    st = gemm(e, 1, s);
    if (st != DG_OK) return st;
    launch(silu_back_kernel, gridn(M * ni), 256, 0, s, M * ni, dh, z[l - 1], dz); count_launch();
    DG_CUDA(cudaGetLastError());
  }
  if (loss) {
    DG_CUDA(cudaMemcpyAsync(host_loss, loss_part, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    double acc = 0.0;
    for (int i = 0; i < nb; ++i) acc += host_loss[i];
    *loss = acc / (double)nout;
  }
  return DG_OK;
}

dg_status Mlp::adam_step(float lr, cudaStream_t s) {
  ++adam_t;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = (float)(1.0 / (1.0 - std::pow((double)b1, (double)adam_t)));
  const float c2 = (float)(1.0 / (1.0 - std::pow((double)b2, (double)adam_t)));
  launch(adam_kernel, gridn(nparam), 256, 0, s, nparam, w, g, m1, m2, lr, b1, b2, 1e-8f, c1, c2); count_launch();
  DG_CUDA(cudaGetLastError());
  return sync_bf16(s);
}

GuessState::~GuessState() {
  delete net[0];
  delete net[1];
  if (part) cudaFree(part);
  if (dsc) cudaFree(dsc);
  for (auto& sl : hist)
    for (double* p : sl)
      if (p) cudaFree(p);
  if (yout) cudaFree(yout);
  if (target) cudaFree(target);
  if (xe) cudaFree(xe);
  if (dvec) cudaFree(dvec);
  if (rt) cudaFree(rt);
}

dg_status mlp_forward_backward(int64_t M, int n_in, int hidden, int n_out, const float* weights,
                               const float* X, const float* T, float* Y, float* loss,
                               float* grad, cudaStream_t s) {
  Mlp net;
  dg_status st = net.init(n_in, hidden, n_out, 1, s);
  if (st != DG_OK) return st;
  DG_CUDA(cudaMemcpyAsync(net.w, weights, sizeof(float) * net.nparam, cudaMemcpyDeviceToDevice, s));
  st = net.sync_bf16(s);
  if (st != DG_OK) return st;
  st = net.reserve(M, s);
  if (st != DG_OK) return st;
  launch(f32_to_bf16_rows_kernel, gridn(M * n_in), 256, 0, s, M * n_in, X, net.xb); count_launch();
  DG_CUDA(cudaGetLastError());
  st = net.forward(M, Y, s);
  if (st != DG_OK) return st;
  if (T) {
    double l = 0.0;
    st = net.backward(M, Y, T, &l, s);
    if (st != DG_OK) return st;
    if (loss) *loss = (float)l;
    if (grad) DG_CUDA(cudaMemcpyAsync(grad, net.g, sizeof(float) * net.nparam, cudaMemcpyDeviceToDevice, s));
  }
  DG_CUDA(cudaStreamSynchronize(s));
  return DG_OK;
}

dg_status mlp_infer(int64_t M, int n_in, int hidden, int n_out, const float* weights,
                    const float* X, float* Y, cudaStream_t s) {
  Mlp net;
  dg_status st = net.init(n_in, hidden, n_out, 1, s);
  if (st != DG_OK) return st;
  DG_CUDA(cudaMemcpyAsync(net.w, weights, sizeof(float) * net.nparam, cudaMemcpyDeviceToDevice, s));
  st = net.sync_bf16(s);
  if (st != DG_OK) return st;
  st = net.reserve(M, s);
  if (st != DG_OK) return st;
  launch(f32_to_bf16_rows_kernel, gridn(M * n_in), 256, 0, s, M * n_in, X, net.xb); count_launch();
  DG_CUDA(cudaGetLastError());
  st = net.infer(M, Y, s);
  if (st != DG_OK) return st;
  DG_CUDA(cudaStreamSynchronize(s));
  return DG_OK;
}

// ------------------------------------------------------------------ solver glue
dg_status guess_features(Mlp& net, int64_t ncell, int ncomp, int nbc, double* const h[4],
                         const double* b, double* part, double* dsc, cudaStream_t s) {
  dg_status st = net.reserve(ncell, s);
  if (st != DG_OK) return st;
  const int64_t n = ncell * ncomp * nbc;
  const int nb = (int)std::min<int64_t>(1216, std::max<int64_t>(1, (n + 1023) / 1024));
  launch(hist_norms_kernel, nb, 256, 0, s, n, h[0], h[1], h[2], h[3], b, part); count_launch();
  launch(guess_scales_kernel, 1, 160, 0, s, nb, n, part, dsc); count_launch();
  launch(features_kernel, gridn(n), 256, 0, s, ncell, ncomp, nbc, h[0], h[1], h[2], h[3], b, dsc,
                                           net.xb); count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status guess_apply(int64_t ncell, int ncomp, int nbc, const double* h0, const double* h1,
                      const float* y, const double* dsc, double* x, cudaStream_t s) {
  launch(apply_guess_kernel, gridn(ncell * ncomp * nbc), 256, 0, s, ncell, ncomp, nbc, h0, h1, y, dsc, x); count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

dg_status guess_target(int64_t ncell, int ncomp, int nbc, const double* h0, const double* h1,
                       const double* xs, const double* dsc, float* t, cudaStream_t s) {
  launch(target_kernel, gridn(ncell * ncomp * nbc), 256, 0, s, ncell, ncomp, nbc, h0, h1, xs, dsc, t); count_launch();
  DG_CUDA(cudaGetLastError());
  return DG_OK;
}

}  // namespace dg

extern "C" dg_status dg_mlp_infer(int64_t M, int32_t n_in, int32_t hidden, int32_t n_out,
                                  const float* weights, const float* X, float* Y, void* stream) {
  if (M < 1 || n_in < 1 || hidden < 1 || n_out < 1 || !weights || !X || !Y) {
    dg::set_error("dg_mlp_infer: bad argument");
    return DG_EINVAL;
  }
  return dg::mlp_infer(M, n_in, hidden, n_out, weights, X, Y, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" dg_status dg_mlp_forward_backward(int64_t M, int32_t n_in, int32_t hidden, int32_t n_out,
                                             const float* weights, const float* X, const float* T,
                                             float* Y, float* loss, float* grad, void* stream) {
  if (M < 1 || n_in < 1 || hidden < 1 || n_out < 1 || !weights || !X || !Y) {
    dg::set_error("dg_mlp_forward_backward: bad argument");
    return DG_EINVAL;
  }
  return dg::mlp_forward_backward(M, n_in, hidden, n_out, weights, X, T, Y, loss, grad,
                                  reinterpret_cast<cudaStream_t>(stream));
}
