// Learned Davidson preconditioner: data recording inside Davidson, training
// on the device, storage, and the pieces the test interface exposes.
//
// Data: while a solve runs with the diagonal preconditioner, each Davidson
// iteration j of a step stores, at up to 2048 fixed sample positions i,
// r_i, d_i and the current Ritz vector x_j,i together with theta, ||r|| and
// the RMS of (d - theta).  When the step has converged, x_conv at the same
// positions gives e = x_conv - x_j (sign-aligned), and each sample becomes a
// feature row, a target y and a weight w (same formulas as the CPU
// reference): the network learns the element-wise rescaling of the Jacobi
// step that points it at the converged vector.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "engine.h"
#include "mlp.h"

namespace gbd {

namespace {
void features_host(double r, double d, const MlpScalars& s, float* f) {
  const double den = d - s.theta;
  f[0] = (float)(den / s.den_rms);
  f[1] = (float)(r / s.rnorm);
  f[2] = (float)(std::fabs(r) / s.rnorm);
  f[3] = (float)std::log(std::fabs(den) + 1e-12);
  f[4] = (float)std::log(s.rnorm);
  f[5] = (float)(s.iter / 32.0);
  f[6] = den > 0 ? 1.f : (den < 0 ? -1.f : 0.f);
  f[7] = 1.f;
}
}  // namespace

void Engine::record_iteration(const double* r_dev, const double* diag_dev, const double* x_dev, const MlpScalars& s) {
  const int64_t n = psi_size;
  const int S = (int)std::min<int64_t>(n, 2048);
  if (rec_idx.size() != (size_t)S || rec_n != n) {
    rec_idx.resize(S);
    for (int i = 0; i < S; ++i) rec_idx[i] = (int64_t)((double)i * n / S);
    rec_n = n;
  }
  Rec R;
  R.s = s;
  R.r.resize(S);
  R.d.resize(S);
  R.x.resize(S);
  // few scattered elements: gather on the host side of three small copies
  std::vector<double> hr(n), hd(n), hx(n);
  CK(cudaMemcpyAsync(hr.data(), r_dev, n * sizeof(double), cudaMemcpyDeviceToHost, stream));
  CK(cudaMemcpyAsync(hd.data(), diag_dev, n * sizeof(double), cudaMemcpyDeviceToHost, stream));
  CK(cudaMemcpyAsync(hx.data(), x_dev, n * sizeof(double), cudaMemcpyDeviceToHost, stream));
  sync();
  for (int i = 0; i < S; ++i) {
    R.r[i] = hr[rec_idx[i]];
    R.d[i] = hd[rec_idx[i]];
    R.x[i] = hx[rec_idx[i]];
  }
  rec_iters.push_back(std::move(R));
}

void Engine::record_converged(const double* x_dev) {
  if (rec_iters.empty()) return;
  const int64_t n = psi_size;
  std::vector<double> hx(n);
  CK(cudaMemcpyAsync(hx.data(), x_dev, n * sizeof(double), cudaMemcpyDeviceToHost, stream));
  sync();
  const int S = (int)rec_idx.size();
  std::vector<double> xc(S);
  for (int i = 0; i < S; ++i) xc[i] = hx[rec_idx[i]];
  for (const Rec& R : rec_iters) {
    double dot = 0;
    for (int i = 0; i < S; ++i) dot += xc[i] * R.x[i];
    const double sg = dot < 0 ? -1.0 : 1.0;
    std::vector<double> tj(S), e(S);
    double te = 0, ee = 0;
    for (int i = 0; i < S; ++i) {
      double den = R.d[i] - R.s.theta;
      if (std::fabs(den) < 1e-8) den = den >= 0 ? 1e-8 : -1e-8;
      tj[i] = -R.r[i] / den;
      e[i] = sg * xc[i] - R.x[i];
      te += tj[i] * e[i];
      ee += e[i] * e[i];
    }
    if (!(ee > 1e-30)) continue;
    const double a = te / ee;
    for (int i = 0; i < S; ++i) {
      const double tji = std::fabs(tj[i]) > 1e-300 ? tj[i] : 1e-300;
      const double ratio = a * e[i] / tji;
      const double y = std::min(4.0, std::max(-0.9, ratio - 1.0));
      const double w = tj[i] * tj[i] / (1.0 + (ratio - 1.0) * (ratio - 1.0));
      if (!std::isfinite(y) || !std::isfinite(w)) continue;
      float f[kMlpF];
      features_host(R.r[i], R.d[i], R.s, f);
      bool ok = true;
      for (float v : f) ok = ok && std::isfinite(v);
      if (!ok) continue;
      data_X.insert(data_X.end(), f, f + kMlpF);
      data_y.push_back((float)y);
      data_w.push_back((float)w);
    }
  }
  rec_iters.clear();
}

// full-batch Adam on the recorded data; returns the final loss
double Engine::train_precond(int epochs, double lr, uint64_t seed) {
  const int64_t n = (int64_t)data_y.size();
  if (n == 0) throw Error(-6, "no recorded preconditioner data");
  // normalise the weights so that the loss is an average
  double W = 0;
  for (float w : data_w) W += w;
  float* X = dalloc<float>((size_t)n * kMlpF);
  float* y = dalloc<float>(n);
  float* w = dalloc<float>(n);
  CK(cudaMemcpyAsync(X, data_X.data(), data_X.size() * sizeof(float), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(y, data_y.data(), n * sizeof(float), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(w, data_w.data(), n * sizeof(float), cudaMemcpyHostToDevice, stream));
  // initial weights: small random first layer, zero output layer (g = 0:
  // the network starts as the Jacobi step)
  std::vector<float> p0(kMlpParams, 0.f);
  std::mt19937_64 g(seed);
  std::normal_distribution<double> nd(0.0, 1.0);
  for (int i = 0; i < kMlpH * kMlpF; ++i) p0[i] = (float)(nd(g) / std::sqrt((double)kMlpF));
  for (int j = 0; j < kMlpH; ++j) p0[kMlpH * kMlpF + j] = 0.01f;
  float* p = dalloc<float>(kMlpParams);
  float* m = dalloc<float>(kMlpParams);
  float* v = dalloc<float>(kMlpParams);
  CK(cudaMemcpyAsync(p, p0.data(), kMlpParams * sizeof(float), cudaMemcpyHostToDevice, stream));
  CK(cudaMemsetAsync(m, 0, kMlpParams * sizeof(float), stream));
  CK(cudaMemsetAsync(v, 0, kMlpParams * sizeof(float), stream));
  if (!mlp_w16) mlp_w16 = dalloc<uint16_t>(kMlpParams);
  const int nblk = mlp_grad_blocks(n);
  double* partial = dalloc<double>((size_t)nblk * (kMlpParams + 1));
  double* grad = dalloc<double>(kMlpParams + 1);
  for (int ep = 1; ep <= epochs; ++ep) {
    launch_mlp_grad(X, y, w, n, 1.0 / W, kMlpPrior, p, partial, nblk, grad, stream);
    launch_mlp_adam(p, m, v, grad, (float)lr, ep, mlp_w16, stream);
    stats.launches += 3;
  }
  double loss = 0;
  launch_mlp_grad(X, y, w, n, 1.0 / W, kMlpPrior, p, partial, nblk, grad, stream);
  CK(cudaMemcpyAsync(&loss, grad + kMlpParams, sizeof(double), cudaMemcpyDeviceToHost, stream));
  mlp_f32.resize(kMlpParams);
  CK(cudaMemcpyAsync(mlp_f32.data(), p, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, stream));
  sync();
  CK(cudaGetLastError());
  for (void* q : {(void*)X, (void*)y, (void*)w, (void*)p, (void*)m, (void*)v, (void*)partial, (void*)grad}) dfree(q);
  mlp_loaded = true;
  return loss;
}

void Engine::set_precond_weights(const float* params) {
  mlp_f32.assign(params, params + kMlpParams);
  float* p = dalloc<float>(kMlpParams);
  CK(cudaMemcpyAsync(p, params, kMlpParams * sizeof(float), cudaMemcpyHostToDevice, stream));
  if (!mlp_w16) mlp_w16 = dalloc<uint16_t>(kMlpParams);
  launch_mlp_to_half(p, mlp_w16, stream);
  sync();
  dfree(p);
  mlp_loaded = true;
}

void Engine::mlp_loss_grad(const float* X, const float* y, const float* w, int64_t n, const float* params,
                           double lam, double* loss, double* grad) {
  double W = 0;
  for (int64_t i = 0; i < n; ++i) W += w[i];
  float* dX = dalloc<float>((size_t)n * kMlpF);
  float* dy = dalloc<float>(n);
  float* dw = dalloc<float>(n);
  float* dp = dalloc<float>(kMlpParams);
  CK(cudaMemcpyAsync(dX, X, (size_t)n * kMlpF * sizeof(float), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(dy, y, n * sizeof(float), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(dw, w, n * sizeof(float), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(dp, params, kMlpParams * sizeof(float), cudaMemcpyHostToDevice, stream));
  const int nblk = mlp_grad_blocks(n);
  double* partial = dalloc<double>((size_t)nblk * (kMlpParams + 1));
  double* out = dalloc<double>(kMlpParams + 1);
  launch_mlp_grad(dX, dy, dw, n, 1.0 / W, lam, dp, partial, nblk, out, stream);
  stats.launches += 2;
  std::vector<double> h(kMlpParams + 1);
  CK(cudaMemcpyAsync(h.data(), out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, stream));
  sync();
  CK(cudaGetLastError());
  std::memcpy(grad, h.data(), kMlpParams * sizeof(double));
  *loss = h[kMlpParams];
  for (void* q : {(void*)dX, (void*)dy, (void*)dw, (void*)dp, (void*)partial, (void*)out}) dfree(q);
}

void Engine::mlp_apply(const double* r, const double* d, double theta, double iter, int64_t n, double* t) {
  if (!mlp_loaded) throw Error(-6, "no preconditioner weights");
  double sd = 0, sdd = 0, rr = 0;
  for (int64_t i = 0; i < n; ++i) {
    const double den = d[i] - theta;
    sdd += den * den;
    rr += r[i] * r[i];
  }
  (void)sd;
  MlpScalars s{theta, std::sqrt(rr) + 1e-300, std::sqrt(sdd / std::max<int64_t>(n, 1)) + 1e-300, iter};
  double* dr = dalloc<double>(n);
  double* dd = dalloc<double>(n);
  double* dt = dalloc<double>(n);
  int* bad = dalloc<int>(1);
  CK(cudaMemcpyAsync(dr, r, n * sizeof(double), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(dd, d, n * sizeof(double), cudaMemcpyHostToDevice, stream));
  CK(cudaMemsetAsync(bad, 0, sizeof(int), stream));
  launch_mlp_precond(dr, dd, s, n, mlp_w16, dt, bad, stream);
  stats.launches++;
  CK(cudaMemcpyAsync(t, dt, n * sizeof(double), cudaMemcpyDeviceToHost, stream));
  sync();
  CK(cudaGetLastError());
  for (void* q : {(void*)dr, (void*)dd, (void*)dt, (void*)bad}) dfree(q);
}

// file: "GBDMLP1\n", int32 F, int32 H, kMlpParams float32 (master copy)
void Engine::save_precond(const char* path) const {
  if (!mlp_loaded || mlp_f32.size() != (size_t)kMlpParams) throw Error(-6, "no preconditioner weights to save");
  FILE* f = std::fopen(path, "wb");
  if (!f) throw Error(-1, "cannot open preconditioner file for writing");
  const char magic[8] = {'G', 'B', 'D', 'M', 'L', 'P', '1', '\n'};
  int32_t dims[2] = {kMlpF, kMlpH};
  bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(dims, 4, 2, f) == 2 &&
            std::fwrite(mlp_f32.data(), 4, kMlpParams, f) == (size_t)kMlpParams;
  std::fclose(f);
  if (!ok) throw Error(-1, "short write of the preconditioner file");
}

void Engine::load_precond(const char* path) {
  FILE* f = std::fopen(path, "rb");
  if (!f) throw Error(-1, "cannot open preconditioner file");
  char magic[8];
  int32_t dims[2];
  std::vector<float> p(kMlpParams);
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "GBDMLP1\n", 8) == 0 &&
            std::fread(dims, 4, 2, f) == 2 && dims[0] == kMlpF && dims[1] == kMlpH &&
            std::fread(p.data(), 4, kMlpParams, f) == (size_t)kMlpParams;
  std::fclose(f);
  if (!ok) throw Error(-1, "not a preconditioner file of this network shape");
  for (float v : p)
    if (!std::isfinite(v)) throw Error(-1, "preconditioner file holds non-finite weights");
  set_precond_weights(p.data());
}

}  // namespace gbd
