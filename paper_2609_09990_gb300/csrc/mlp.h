// Learned Davidson preconditioner network (see kernels_mlp.cu).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace gbd {

constexpr int kMlpF = 8;
constexpr int kMlpH = 128;
constexpr int kMlpParams = kMlpH * kMlpF + kMlpH + kMlpH + 1;   // W1, b1, w2, b2

// per-iteration scalars of the feature map
struct MlpScalars {
  double theta;     // Ritz value
  double rnorm;     // ||r||
  double den_rms;   // RMS of (d - theta) over the vector
  double iter;      // Davidson iteration
};

void launch_mlp_precond(const double* r, const double* d, const MlpScalars& s, int64_t n, const void* w16, double* t,
                        int* bad, cudaStream_t st);
void launch_mlp_features(const double* r, const double* d, const MlpScalars& s, int64_t n, float* X,
                         cudaStream_t st);
void launch_mlp_forward(const float* X, int64_t n, const float* p, float* g, cudaStream_t st);
int mlp_grad_blocks(int64_t n);
// grad_and_loss: kMlpParams gradient entries then the loss
// loss = sum w (g - y)^2 / W + lam mean(g^2)
void launch_mlp_grad(const float* X, const float* y, const float* w, int64_t n, double inv_W, double lam,
                     const float* p, double* partial, int nblk, double* grad_and_loss, cudaStream_t st);
// strength of the prior towards the Jacobi step used in training
constexpr double kMlpPrior = 0.5;
void launch_mlp_adam(float* p, float* m, float* v, const double* grad, float lr, int step, void* p16,
                     cudaStream_t st);
void launch_mlp_to_half(const float* p, void* p16, cudaStream_t st);

}  // namespace gbd
