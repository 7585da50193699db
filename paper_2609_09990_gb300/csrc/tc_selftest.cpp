// Self-test of the tensor-core grouped GEMM on random panels: conversion
// kernel -> panels -> tc_gemm (FP64 transposed output) against an FP64 host
// product of the decoded panel values (BF16 / TF32) or of the original FP64
// values (TF32x3).  Exposed as gbd_tc_selftest for the GPU tests.
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "../../include/gbdmrg_test.h"
#include "tc_gemm.h"

namespace gbd {
}

namespace {

float bf16_to_float(uint16_t v) {
  uint32_t u = (uint32_t)v << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

}  // namespace

extern "C" int gbd_tc_selftest(int32_t device, int32_t prec, int32_t M, int32_t N, int32_t K, int32_t nterms,
                               uint64_t seed, double* max_err, double* max_ref) {
  using namespace gbd;
  if (prec < 0 || prec > 3 || M < 1 || N < 1 || N > 4096 || K < 1 || nterms < 1 || !max_err || !max_ref)
    return GBD_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return GBD_ERR_CUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const bool bfp = prec == kBF16 || prec == kBF16x3, split = prec == kTF32x3 || prec == kBF16x3;
  const int eb = bfp ? 2 : 4;
  const int kstep = bfp ? 16 : 8;
  const int Kp = (K + kstep - 1) / kstep * kstep;
  const int64_t pitchA = ((int64_t)Kp * nterms + 63) / 64 * 64 + 64;
  const int64_t pitchB = (Kp + 63) / 64 * 64;
  const int64_t rowsA = M, rowsB = (int64_t)N * nterms;
  std::mt19937_64 g(seed);
  std::normal_distribution<double> nd;
  std::vector<double> A((size_t)M * Kp * nterms, 0.0), B((size_t)nterms * N * Kp, 0.0);
  for (int t = 0; t < nterms; ++t)
    for (int i = 0; i < M; ++i)
      for (int k = 0; k < K; ++k) A[((size_t)i * nterms + t) * Kp + k] = nd(g);
  for (int t = 0; t < nterms; ++t)
    for (int j = 0; j < N; ++j)
      for (int k = 0; k < K; ++k) B[((size_t)t * N + j) * Kp + k] = nd(g);
  // device buffers
  double *dA = nullptr, *dB = nullptr, *dC = nullptr;
  void *pa[2] = {nullptr, nullptr}, *pb[2] = {nullptr, nullptr};
  int* derr = nullptr;
  TcConv* dconv = nullptr;
  TcTile* dtiles = nullptr;
  TcTerm* dterms = nullptr;
  int rc = GBD_OK;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == GBD_OK) rc = GBD_ERR_CUDA;
  };
  ck(cudaMalloc(&dA, A.size() * 8));
  ck(cudaMalloc(&dB, B.size() * 8));
  ck(cudaMalloc(&dC, (size_t)M * N * 8));
  for (int h = 0; h < (split ? 2 : 1); ++h) {
    ck(cudaMalloc(&pa[h], rowsA * pitchA * eb));
    ck(cudaMalloc(&pb[h], rowsB * pitchB * eb));
    ck(cudaMemset(pa[h], 0, rowsA * pitchA * eb));
    ck(cudaMemset(pb[h], 0, rowsB * pitchB * eb));
  }
  ck(cudaMalloc(&derr, sizeof(int)));
  ck(cudaMemset(derr, 0, sizeof(int)));
  if (rc != GBD_OK) goto out;
  {
    ck(cudaMemcpy(dA, A.data(), A.size() * 8, cudaMemcpyHostToDevice));
    ck(cudaMemcpy(dB, B.data(), B.size() * 8, cudaMemcpyHostToDevice));
    // A panel: row i, term t at columns [t*Kp, t*Kp+Kp); B panel: rows t*N+j
    std::vector<TcConv> conv;
    for (int t = 0; t < nterms; ++t) {
      conv.push_back({dA + (size_t)t * Kp, 1.0, M, Kp, Kp * nterms, 0, t * Kp, 0});
      conv.push_back({dB + (size_t)t * N * Kp, 1.0, N, Kp, Kp, 0, 0, 0});
    }
    std::vector<TcConv> ca, cb;
    for (size_t i = 0; i < conv.size(); ++i) (i % 2 ? cb : ca).push_back(conv[i]);
    for (int t = 0; t < nterms; ++t) cb[t].r0 = t * N;
    ck(cudaMalloc(&dconv, conv.size() * sizeof(TcConv)));
    ck(cudaMemcpy(dconv, ca.data(), ca.size() * sizeof(TcConv), cudaMemcpyHostToDevice));
    launch_tc_convert(dconv, (int)ca.size(), prec, pa[0], pa[1], pitchA, 0);
    ck(cudaDeviceSynchronize());
    ck(cudaMemcpy(dconv, cb.data(), cb.size() * sizeof(TcConv), cudaMemcpyHostToDevice));
    launch_tc_convert(dconv, (int)cb.size(), prec, pb[0], pb[1], pitchB, 0);
    ck(cudaDeviceSynchronize());
    // tiles: 128-row M tiles x 256-column N tiles; output C^T (N x M, ld M)
    std::vector<TcTile> tiles;
    std::vector<TcTerm> terms;
    for (int m0 = 0; m0 < M; m0 += 128)
      for (int n0 = 0; n0 < N; n0 += 256) {
        TcTile T{};
        T.t0 = (int)terms.size();
        int nv = std::min(256, N - n0);
        for (int t = 0; t < nterms; ++t) terms.push_back({t * Kp, 0, t * N + n0, Kp, t % 3 == 2 ? 1 : 0, 0, 0, 0});
        T.t1 = (int)terms.size();
        T.m0 = m0;
        T.m_valid = std::min(128, M - m0);
        T.n_mma = (nv + 15) / 16 * 16;
        T.n_valid = nv;
        int bs = 0;
        while ((16 << bs) < T.n_mma) ++bs;
        T.bsel = bs;
        T.mode = kTcSigma;
        T.beta = 0;
        T.ld = M;
        T.out = (int64_t)n0 * M;
        tiles.push_back(T);
      }
    ck(cudaMalloc(&dtiles, tiles.size() * sizeof(TcTile)));
    ck(cudaMalloc(&dterms, terms.size() * sizeof(TcTerm)));
    ck(cudaMemcpy(dtiles, tiles.data(), tiles.size() * sizeof(TcTile), cudaMemcpyHostToDevice));
    ck(cudaMemcpy(dterms, terms.data(), terms.size() * sizeof(TcTerm), cudaMemcpyHostToDevice));
    TcMaps maps;
    std::memset(&maps, 0, sizeof(maps));
    for (int h = 0; h < (split ? 2 : 1); ++h) {
      if (!tc_encode_panel(&maps.a[h], eb, pa[h], pitchA, rowsA, 128)) rc = GBD_ERR_CUDA;
      for (int s = 0; s < 5; ++s)
        if (!tc_encode_panel(&maps.b[h][s], eb, pb[h], pitchB, rowsB, 16u << s)) rc = GBD_ERR_CUDA;
    }
    if (rc != GBD_OK) goto out;
    TcLaunch L{dtiles, dterms, (int)tiles.size(), prec, nullptr, nullptr, dC, derr, nullptr, nullptr, nullptr, 256,
               tc_stages(prec, 256)};
    if (!launch_tc_gemm(maps, L, sms, 0)) rc = GBD_ERR_CUDA;
    ck(cudaGetLastError());
    ck(cudaDeviceSynchronize());
    int herr = 0;
    ck(cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost));
    if (rc != GBD_OK) goto out;
    if (herr) { rc = GBD_ERR_TIMEOUT; goto out; }
    std::vector<double> Ct((size_t)M * N);
    ck(cudaMemcpy(Ct.data(), dC, Ct.size() * 8, cudaMemcpyDeviceToHost));
    // decoded operands
    std::vector<double> Ad(A.size()), Bd(B.size());
    if (split) {
      Ad = A;
      Bd = B;
    } else {
      std::vector<uint8_t> ha(rowsA * pitchA * eb), hb(rowsB * pitchB * eb);
      ck(cudaMemcpy(ha.data(), pa[0], ha.size(), cudaMemcpyDeviceToHost));
      ck(cudaMemcpy(hb.data(), pb[0], hb.size(), cudaMemcpyDeviceToHost));
      auto dec = [&](const std::vector<uint8_t>& v, int64_t idx) -> double {
        if (eb == 2) {
          uint16_t u;
          std::memcpy(&u, &v[idx * 2], 2);
          return bf16_to_float(u);
        }
        float f;
        std::memcpy(&f, &v[idx * 4], 4);
        return f;
      };
      for (int t = 0; t < nterms; ++t)
        for (int i = 0; i < M; ++i)
          for (int k = 0; k < Kp; ++k) Ad[((size_t)i * nterms + t) * Kp + k] = dec(ha, (int64_t)i * pitchA + t * Kp + k);
      for (int t = 0; t < nterms; ++t)
        for (int j = 0; j < N; ++j)
          for (int k = 0; k < Kp; ++k) Bd[((size_t)t * N + j) * Kp + k] = dec(hb, (int64_t)(t * N + j) * pitchB + k);
    }
    double me = 0, mr = 0;
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < N; ++j) {
        double s = 0;
        for (int t = 0; t < nterms; ++t) {
          double st = 0;
          for (int k = 0; k < Kp; ++k) st += Ad[((size_t)i * nterms + t) * Kp + k] * Bd[((size_t)t * N + j) * Kp + k];
          s += (t % 3 == 2) ? -st : st;
        }
        me = std::max(me, std::fabs(Ct[(size_t)j * M + i] - s));
        mr = std::max(mr, std::fabs(s));
      }
    *max_err = me;
    *max_ref = mr;
  }
out:
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dC);
  for (int h = 0; h < 2; ++h) {
    cudaFree(pa[h]);
    cudaFree(pb[h]);
  }
  cudaFree(derr);
  cudaFree(dconv);
  cudaFree(dtiles);
  cudaFree(dterms);
  return rc;
}

// Dense throughput of tc_gemm_kernel: one M x N x K product (operands made
// of a constant byte pattern: the values do not matter for timing), 128 x 256
// tiles, launched `reps` times after one warm-up; CUDA events around the
// timed launches.  flops = 2 M N K per launch (TF32x3 / BF16x3 execute three
// MMAs per product and are reported by the same algorithmic count).
extern "C" int gbd_tc_rate(int32_t device, int32_t prec, int32_t M, int32_t N, int32_t K, int32_t reps,
                           double* tflops, double* ms_per_launch) {
  using namespace gbd;
  if (prec < 0 || prec > 3 || M < 128 || N < 256 || K < 64 || reps < 1 || !tflops || !ms_per_launch ||
      M % 128 || N % 256 || K % 64)
    return GBD_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return GBD_ERR_CUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const bool bfp = prec == kBF16 || prec == kBF16x3, split = prec == kTF32x3 || prec == kBF16x3;
  const int eb = bfp ? 2 : 4;
  double *dA = nullptr, *dB = nullptr, *dC = nullptr;
  void *pa[2] = {nullptr, nullptr}, *pb[2] = {nullptr, nullptr};
  int* derr = nullptr;
  TcConv* dconv = nullptr;
  TcTile* dtiles = nullptr;
  TcTerm* dterms = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = GBD_OK;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == GBD_OK) rc = e == cudaErrorMemoryAllocation ? GBD_ERR_OOM : GBD_ERR_CUDA;
  };
  // FP64 sources of 128 rows x K, converted repeatedly into the panels
  ck(cudaMalloc(&dA, (size_t)128 * K * 8));
  ck(cudaMalloc(&dC, (size_t)M * N * 8));
  for (int h = 0; h < (split ? 2 : 1); ++h) {
    ck(cudaMalloc(&pa[h], (size_t)M * K * eb));
    ck(cudaMalloc(&pb[h], (size_t)N * K * eb));
  }
  ck(cudaMalloc(&derr, sizeof(int)));
  ck(cudaMemset(derr, 0, sizeof(int)));
  ck(cudaEventCreate(&e0));
  ck(cudaEventCreate(&e1));
  if (rc != GBD_OK) goto out;
  {
    ck(cudaMemset(dA, 0x3F, (size_t)128 * K * 8));   // every double 0x3F3F... (about 4.8e-4)
    std::vector<TcConv> ca, cb;
    for (int r = 0; r < M; r += 128) ca.push_back({dA, 1.0, 128, K, K, r, 0, 0});
    for (int r = 0; r < N; r += 128) cb.push_back({dA, 1.0, 128, K, K, r, 0, 0});
    ck(cudaMalloc(&dconv, std::max(ca.size(), cb.size()) * sizeof(TcConv)));
    ck(cudaMemcpy(dconv, ca.data(), ca.size() * sizeof(TcConv), cudaMemcpyHostToDevice));
    launch_tc_convert(dconv, (int)ca.size(), prec, pa[0], pa[1], K, 0);
    ck(cudaDeviceSynchronize());
    ck(cudaMemcpy(dconv, cb.data(), cb.size() * sizeof(TcConv), cudaMemcpyHostToDevice));
    launch_tc_convert(dconv, (int)cb.size(), prec, pb[0], pb[1], K, 0);
    ck(cudaDeviceSynchronize());
    std::vector<TcTile> tiles;
    std::vector<TcTerm> terms;
    for (int m0 = 0; m0 < M; m0 += 128)
      for (int n0 = 0; n0 < N; n0 += 256) {
        TcTile T{};
        T.t0 = (int)terms.size();
        terms.push_back({0, 0, n0, K, 0, 0, 0, 0});
        T.t1 = (int)terms.size();
        T.m0 = m0;
        T.m_valid = 128;
        T.n_mma = 256;
        T.n_valid = 256;
        T.bsel = 4;
        T.mode = kTcSigma;
        T.beta = 0;
        T.ld = M;
        T.out = (int64_t)n0 * M;
        tiles.push_back(T);
      }
    ck(cudaMalloc(&dtiles, tiles.size() * sizeof(TcTile)));
    ck(cudaMalloc(&dterms, terms.size() * sizeof(TcTerm)));
    ck(cudaMemcpy(dtiles, tiles.data(), tiles.size() * sizeof(TcTile), cudaMemcpyHostToDevice));
    ck(cudaMemcpy(dterms, terms.data(), terms.size() * sizeof(TcTerm), cudaMemcpyHostToDevice));
    TcMaps maps;
    std::memset(&maps, 0, sizeof(maps));
    for (int h = 0; h < (split ? 2 : 1); ++h) {
      if (!tc_encode_panel(&maps.a[h], eb, pa[h], K, M, 128)) rc = GBD_ERR_CUDA;
      for (int s = 0; s < 5; ++s)
        if (!tc_encode_panel(&maps.b[h][s], eb, pb[h], K, N, 16u << s)) rc = GBD_ERR_CUDA;
    }
    if (rc != GBD_OK) goto out;
    TcLaunch L{dtiles, dterms, (int)tiles.size(), prec, nullptr, nullptr, dC, derr, nullptr, nullptr, nullptr, 256,
               tc_stages(prec, 256)};
    if (!launch_tc_gemm(maps, L, sms, 0)) rc = GBD_ERR_CUDA;   // warm-up
    ck(cudaEventRecord(e0, 0));
    for (int r = 0; r < reps && rc == GBD_OK; ++r)
      if (!launch_tc_gemm(maps, L, sms, 0)) rc = GBD_ERR_CUDA;
    ck(cudaEventRecord(e1, 0));
    ck(cudaGetLastError());
    ck(cudaDeviceSynchronize());
    int herr = 0;
    ck(cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost));
    if (rc != GBD_OK) goto out;
    if (herr) { rc = GBD_ERR_TIMEOUT; goto out; }
    float ms = 0;
    ck(cudaEventElapsedTime(&ms, e0, e1));
    *ms_per_launch = ms / reps;
    *tflops = 2.0 * M * (double)N * K / (*ms_per_launch * 1e-3) / 1e12;
  }
out:
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dC);
  for (int h = 0; h < 2; ++h) {
    cudaFree(pa[h]);
    cudaFree(pb[h]);
  }
  cudaFree(derr);
  cudaFree(dconv);
  cudaFree(dtiles);
  cudaFree(dterms);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return rc;
}

// Failure detection of the tensor-core kernels without a fault: a bounded
// mbarrier wait on a barrier that is never completed returns with the
// error flag raised; the same wait with an arrival succeeds.
extern "C" int gbd_wait_selftest(int32_t device, int32_t arrive, int32_t* err_flag, int32_t* waited_ok) {
  using namespace gbd;
  if (!err_flag || !waited_ok) return GBD_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return GBD_ERR_CUDA;
  int* d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(int)) != cudaSuccess) return GBD_ERR_OOM;
  int rc = GBD_OK, h[2] = {0, 0};
  if (cudaMemset(d, 0, 2 * sizeof(int)) != cudaSuccess || !bounded_wait_probe(arrive, d, d + 1, 0) ||
      cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = GBD_ERR_CUDA;
  cudaFree(d);
  *err_flag = h[0];
  *waited_ok = h[1];
  return rc;
}
