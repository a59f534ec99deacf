// Learned initial guess for the stage solves: per-cell MLP (see dg_guess.cu).
#pragma once

#include <cuda_bf16.h>

#include <vector>

#include "dg_common.cuh"

namespace dg {

// One fully connected network n_in -> h -> h -> h -> n_out with SiLU between
// layers; FP32 master weights, BF16 copies for the tensor-core GEMMs, Adam.
struct Mlp {
  int n_in = 0, hidden = 0, n_out = 0;
  int dims[5] = {0, 0, 0, 0, 0};
  int64_t woff[4] = {0, 0, 0, 0}, boff[4] = {0, 0, 0, 0}, nparam = 0;
  float* w = nullptr;            // master parameters (packed W1 b1 W2 b2 W3 b3 W4 b4)
  float* g = nullptr;            // gradients
  float* m1 = nullptr;           // Adam moments
  float* m2 = nullptr;
  __nv_bfloat16* wb = nullptr;   // BF16 copies of the weight matrices (same packing, biases unused)
  int64_t adam_t = 0;
  // activations for up to cap rows
  int64_t cap = 0;
  __nv_bfloat16* xb = nullptr;   // inputs [cap x n_in]
  float* z[4] = {nullptr, nullptr, nullptr, nullptr};           // pre-activations
  __nv_bfloat16* hb[3] = {nullptr, nullptr, nullptr};          // hidden activations
  float* dz = nullptr;           // [cap x max(h, n_out)] FP32
  __nv_bfloat16* dzb = nullptr;  // BF16 copy of dz
  float* dh = nullptr;           // [cap x h] FP32
  float* part = nullptr;         // split reductions
  int64_t part_cap = 0;
  double* loss_part = nullptr;
  double* host_loss = nullptr;

  ~Mlp();
  dg_status init(int n_in, int hidden, int n_out, uint64_t seed, cudaStream_t s);
  dg_status reserve(int64_t rows, cudaStream_t s);
  dg_status sync_bf16(cudaStream_t s);
  // Y = f(X) for M rows; X given as BF16 in xb (already filled) -> y [M x n_out]
  dg_status forward(int64_t M, float* y, cudaStream_t s);
  // the same output without keeping activations for a backward pass (one
  // fused launch when the network fits in shared memory)
  dg_status infer(int64_t M, float* y, cudaStream_t s);
  // gradients of mean((Y - T)^2) after forward(); loss returned if non-null
  dg_status backward(int64_t M, const float* y, const float* t, double* loss, cudaStream_t s);
  dg_status adam_step(float lr, cudaStream_t s);
};

// Learned-guess state of a solver: one net per system kind, histories of the
// last four solutions of each (stage, system) slot.
struct GuessState {
  int enable = 0, train = 0, systems = 1, hidden = 128;
  float lr = 1e-3f;
  uint64_t seed = 1;
  Mlp* net[2] = {nullptr, nullptr};    // 0: pressure, 1: momentum
  double* hist[4][4] = {};             // [slot][age], slot = 2*(stage-1) + (system: 0 mom, 1 helm)
  int count[4] = {0, 0, 0, 0};
  int64_t n[4] = {0, 0, 0, 0};
  float* yout = nullptr;               // [rows x n_out] network output
  float* target = nullptr;             // [rows x n_out] training target
  int64_t out_cap = 0;
  double* part = nullptr;              // norm partials (device)
  double* dsc = nullptr;               // device: inverse input scales, output scale, its inverse
  bool predicted = false;
  double last_loss = 0.0;
  int64_t train_steps = 0;
  // Helmholtz safeguard: the extrapolated guess, the learned correction and
  // the residual / operator image used to weight it (pressure-space vectors)
  double* xe = nullptr;
  double* dvec = nullptr;
  double* rt = nullptr;  // [2 n]: b - A xe, then A d
  int64_t safe_n = 0;
  ~GuessState();
};

// solver glue: features of one stage system from its history (h[0] newest)
// and right-hand side, with the block scales and the output scale computed
// on the device into dsc (no host round trip); the guess x = 2 h0 - h1 +
// dsc[5] y; the training target.
dg_status guess_features(Mlp& net, int64_t ncell, int ncomp, int nbc, double* const h[4],
                         const double* b, double* part, double* dsc, cudaStream_t s);
dg_status guess_apply(int64_t ncell, int ncomp, int nbc, const double* h0, const double* h1,
                      const float* y, const double* dsc, double* x, cudaStream_t s);
dg_status guess_target(int64_t ncell, int ncomp, int nbc, const double* h0, const double* h1,
                       const double* xs, const double* dsc, float* t, cudaStream_t s);

// entries of the tests' checks: see dg_mlp_forward_backward, dg_mlp_infer
dg_status mlp_infer(int64_t M, int n_in, int hidden, int n_out, const float* weights,
                    const float* X, float* Y, cudaStream_t s);
dg_status mlp_forward_backward(int64_t M, int n_in, int hidden, int n_out, const float* weights,
                               const float* X, const float* T, float* Y, float* loss, float* grad,
                               cudaStream_t s);

}  // namespace dg
