// Learned Davidson preconditioner: a pointwise two-layer MLP (F = 8 features
// -> 128 ReLU units -> 1) that rescales the Jacobi step element by element,
//   t_i = -r_i / (d_i - theta) * (1 + clip(g_i, -0.9, 4)).
// FP16 weights, FP32 arithmetic.  Inference is fused with the feature
// computation and the preconditioner; training uses per-block partial
// gradients (deterministic), an FP64 reduction and Adam.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "mlp.h"

namespace gbd {

namespace {

constexpr int kF = kMlpF, kH = kMlpH;

struct Weights {
  float W1[kH][kF];
  float b1[kH];
  float w2[kH];
  float b2;
};

__device__ void load_weights(Weights& w, const __half* p) {
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
    float v = __half2float(p[i]);
    if (i < kH * kF) w.W1[i / kF][i % kF] = v;
    else if (i < kH * kF + kH) w.b1[i - kH * kF] = v;
    else if (i < kH * kF + 2 * kH) w.w2[i - kH * kF - kH] = v;
    else w.b2 = v;
  }
  __syncthreads();
}

__device__ void load_weights_f32(Weights& w, const float* p) {
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
    float v = p[i];
    if (i < kH * kF) w.W1[i / kF][i % kF] = v;
    else if (i < kH * kF + kH) w.b1[i - kH * kF] = v;
    else if (i < kH * kF + 2 * kH) w.w2[i - kH * kF - kH] = v;
    else w.b2 = v;
  }
  __syncthreads();
}

__device__ __forceinline__ float net(const Weights& w, const float* f) {
  float g = w.b2;
#pragma unroll 4
  for (int j = 0; j < kH; ++j) {
    float z = w.b1[j];
#pragma unroll
    for (int q = 0; q < kF; ++q) z = fmaf(w.W1[j][q], f[q], z);
    g = fmaf(w.w2[j], fmaxf(z, 0.f), g);
  }
  return g;
}

// features of one element (the same formulas as the CPU reference)
__device__ __forceinline__ void feat(double r, double d, const MlpScalars& s, float* f) {
  const double den = d - s.theta;
  f[0] = (float)(den / s.den_rms);
  f[1] = (float)(r / s.rnorm);
  f[2] = (float)(fabs(r) / s.rnorm);
  f[3] = (float)log(fabs(den) + 1e-12);
  f[4] = (float)log(s.rnorm);
  f[5] = (float)(s.iter / 32.0);
  f[6] = den > 0 ? 1.f : (den < 0 ? -1.f : 0.f);
  f[7] = 1.f;
}

__global__ void precond_kernel(const double* __restrict__ r, const double* __restrict__ d, MlpScalars s, int64_t n,
                               const __half* __restrict__ p, double* __restrict__ t, int* bad) {
  __shared__ Weights w;
  load_weights(w, p);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float f[kF];
    feat(r[i], d[i], s, f);
    const float g = fminf(fmaxf(net(w, f), -0.9f), 4.f);   // the range of the training targets
    double den = d[i] - s.theta;
    if (fabs(den) < 1e-8) den = den >= 0.0 ? 1e-8 : -1e-8;
    const double v = -r[i] / den * (1.0 + (double)g);
    if (!isfinite(v)) *bad = 1;
    t[i] = v;
  }
}

__global__ void forward_kernel(const float* __restrict__ X, int64_t n, const float* __restrict__ p,
                               float* __restrict__ g) {
  __shared__ Weights w;
  load_weights_f32(w, p);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    g[i] = net(w, X + i * kF);
}

__global__ void features_kernel(const double* __restrict__ r, const double* __restrict__ d, MlpScalars s,
                                int64_t n, float* __restrict__ X) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    feat(r[i], d[i], s, X + i * kF);
}

// loss = sum w (g - y)^2 / W + lam_n sum g^2 (lam_n = lam / n: a prior
// towards g = 0, the Jacobi step); per-block partial gradients
// partial layout per block: [W1 (H*F) | b1 (H) | w2 (H) | b2 | loss]
constexpr int kTile = 256;
__global__ void grad_kernel(const float* __restrict__ X, const float* __restrict__ y, const float* __restrict__ wt,
                            int64_t n, double inv_W, double lam_n, const float* __restrict__ p,
                            double* __restrict__ partial) {
  __shared__ Weights w;
  __shared__ float xs[kTile][kF];
  __shared__ float dg[kTile];
  __shared__ float red[kTile];
  load_weights_f32(w, p);
  const int j = threadIdx.x;   // hidden unit handled in phase 2 (j < kH)
  float aW1[kF] = {0}, ab1 = 0, aw2 = 0;
  float adg = 0, aloss = 0;
  for (int64_t e0 = (int64_t)blockIdx.x * kTile; e0 < n; e0 += (int64_t)gridDim.x * kTile) {
    // phase 1: forward for element e0 + threadIdx.x
    const int64_t e = e0 + threadIdx.x;
    if (e < n) {
#pragma unroll
      for (int q = 0; q < kF; ++q) xs[threadIdx.x][q] = X[e * kF + q];
      const float g = net(w, xs[threadIdx.x]);
      const float diff = g - y[e];
      dg[threadIdx.x] = (float)(2.0 * inv_W) * wt[e] * diff + (float)(2.0 * lam_n) * g;
      aloss += (float)inv_W * wt[e] * diff * diff + (float)lam_n * g * g;
    } else {
      dg[threadIdx.x] = 0.f;
#pragma unroll
      for (int q = 0; q < kF; ++q) xs[threadIdx.x][q] = 0.f;
    }
    __syncthreads();
    if (j < kH) {
      const int cnt = (int)((n - e0) < kTile ? (n - e0) : kTile);
      for (int i = 0; i < cnt; ++i) {
        float z = w.b1[j];
#pragma unroll
        for (int q = 0; q < kF; ++q) z = fmaf(w.W1[j][q], xs[i][q], z);
        const float gi = dg[i];
        if (z > 0.f) {
          aw2 = fmaf(gi, z, aw2);
          const float dh = gi * w.w2[j];
#pragma unroll
          for (int q = 0; q < kF; ++q) aW1[q] = fmaf(dh, xs[i][q], aW1[q]);
          ab1 += dh;
        }
      }
    }
    if (threadIdx.x == 0) {
      const int cnt = (int)((n - e0) < kTile ? (n - e0) : kTile);
      for (int i = 0; i < cnt; ++i) adg += dg[i];
    }
    __syncthreads();
  }
  double* out = partial + (int64_t)blockIdx.x * (kMlpParams + 1);
  if (j < kH) {
#pragma unroll
    for (int q = 0; q < kF; ++q) out[j * kF + q] = aW1[q];
    out[kH * kF + j] = ab1;
    out[kH * kF + kH + j] = aw2;
  }
  red[threadIdx.x] = aloss;
  __syncthreads();
  for (int st = kTile / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[kMlpParams - 1] = adg;
    out[kMlpParams] = red[0];
  }
}

__global__ void reduce_partials(const double* __restrict__ partial, int nblk, double* __restrict__ out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= kMlpParams; k += gridDim.x * blockDim.x) {
    double s = 0;
    for (int b = 0; b < nblk; ++b) s += partial[(int64_t)b * (kMlpParams + 1) + k];
    out[k] = s;
  }
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const double* __restrict__ grad, float lr, float b1, float b2, float eps, int step,
                            __half* __restrict__ p16) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kMlpParams; k += gridDim.x * blockDim.x) {
    const float g = (float)grad[k];
    m[k] = b1 * m[k] + (1.f - b1) * g;
    v[k] = b2 * v[k] + (1.f - b2) * g * g;
    const float mh = m[k] / (1.f - powf(b1, (float)step));
    const float vh = v[k] / (1.f - powf(b2, (float)step));
    p[k] -= lr * mh / (sqrtf(vh) + eps);
    p16[k] = __float2half_rn(p[k]);
  }
}

__global__ void to_half_kernel(const float* __restrict__ p, __half* __restrict__ h) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kMlpParams; k += gridDim.x * blockDim.x)
    h[k] = __float2half_rn(p[k]);
}

int grid_n(int64_t n, int t) {
  int64_t b = (n + t - 1) / t;
  if (b > 152 * 8) b = 152 * 8;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

void launch_mlp_precond(const double* r, const double* d, const MlpScalars& s, int64_t n, const void* w16, double* t,
                        int* bad, cudaStream_t st) {
  precond_kernel<<<grid_n(n, 256), 256, 0, st>>>(r, d, s, n, (const __half*)w16, t, bad);
}

void launch_mlp_features(const double* r, const double* d, const MlpScalars& s, int64_t n, float* X,
                         cudaStream_t st) {
  features_kernel<<<grid_n(n, 256), 256, 0, st>>>(r, d, s, n, X);
}

void launch_mlp_forward(const float* X, int64_t n, const float* p, float* g, cudaStream_t st) {
  forward_kernel<<<grid_n(n, 256), 256, 0, st>>>(X, n, p, g);
}

int mlp_grad_blocks(int64_t n) {
  int64_t b = (n + kTile - 1) / kTile;
  if (b > 152 * 2) b = 152 * 2;
  return (int)(b < 1 ? 1 : b);
}

void launch_mlp_grad(const float* X, const float* y, const float* w, int64_t n, double inv_W, double lam,
                     const float* p, double* partial, int nblk, double* grad_and_loss, cudaStream_t st) {
  grad_kernel<<<nblk, kTile, 0, st>>>(X, y, w, n, inv_W, n > 0 ? lam / (double)n : 0.0, p, partial);
  reduce_partials<<<(kMlpParams + 256) / 256, 256, 0, st>>>(partial, nblk, grad_and_loss);
}

void launch_mlp_adam(float* p, float* m, float* v, const double* grad, float lr, int step, void* p16,
                     cudaStream_t st) {
  adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(p, m, v, grad, lr, 0.9f, 0.999f, 1e-8f, step, (__half*)p16);
}

void launch_mlp_to_half(const float* p, void* p16, cudaStream_t st) {
  to_half_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(p, (__half*)p16);
}

}  // namespace gbd
