// A grouped FP64 GEMM plan (GemmPlan: outputs C = sum_t alpha op(A) op(B))
// run on the tensor cores instead of the FP64 units: the environment
// update's two contractions (L' = U^T (Lenl U) and its mirror) are bulk
// contractions like the sigma's, and GB300 runs FP64 at ~1.3 TFLOP/s.
//
// Every distinct operand block is converted once into a K-blocked panel
// (pitch one 128-byte box row; a block of R rows and K columns takes
// ceil(K / W) groups of R rows), the TF32x3 (or BF16x3) hi/lo split of the
// accurate sigma tier.  The kernel computes D = A_p B_p^T with both panels
// K-major; the C^T epilogue makes that the row-major C when the A panel holds
// op(B)^T (rows = columns of C) and the B panel holds op(A) (rows = rows of
// C).  An output whose summed K exceeds kc is split into chunks accumulated
// in FP32 partial slots and summed in FP64 in a fixed order (tc_reduce), as
// in the sigma: no FP32 accumulation runs longer than kc.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

#include "engine.h"
#include "tc_gemm.h"

namespace gbd {

namespace {
inline int bsel_of(int n) {
  int b = 0;
  while ((16 << b) < n) ++b;
  return b;
}
}  // namespace

void Engine::run_tc(GemmPlan& p, int prec) {
  if (p.outs.empty()) return;
  const bool split = prec == kTF32x3 || prec == kBF16x3;
  const bool bfp = prec == kBF16 || prec == kBF16x3;
  const int eb = bfp ? 2 : 4;
  const int W = 128 / eb;                 // elements per box row (panel pitch)
  const int kstep = bfp ? 16 : 8;         // MMA K step
  const int64_t kc = split ? 512 : 2048;  // longest FP32 accumulation (multiple of W)
  const int ncap = 128;
  // ---- operand blocks, each converted once: (source, rows, K, ld, trans,
  //      scale) -> first panel row; a block takes ceil(K / W) groups of rows
  struct Blk { int64_t row0; int rows; };
  using Key = std::tuple<const double*, int, int, int, int, double>;
  std::map<Key, Blk> mapA, mapB;
  std::vector<TcConv> convA, convB;
  int64_t rowsA = 0, rowsB = 0;
  auto block = [&](std::map<Key, Blk>& mp, std::vector<TcConv>& conv, int64_t& rows, const double* src, int R,
                   int K, int ld, int trans, double scale) -> Blk {
    Key key{src, R, K, ld, trans, scale};
    auto it = mp.find(key);
    if (it != mp.end()) return it->second;
    Blk b{rows, R};
    const int64_t nblk = (K + W - 1) / W;
    rows += nblk * R;
    if (rows > INT32_MAX / 2) throw Error(-2, "tensor-core GEMM plan: operand panel too large");
    // trans: element (r, k) = src[k * ld + r]; otherwise src[r * ld + k]
    check_range(src, trans ? K : R, trans ? R : K, ld, "tensor-core GEMM operand");
    conv.push_back({src, scale, R, K, ld, (int32_t)b.row0, 0, R, trans});
    mp.emplace(key, b);
    return b;
  };
  std::vector<TcTile> tiles;
  std::vector<TcTerm> terms;
  std::vector<TcRed> red;
  int64_t slot = 0, red_total = 0;
  double* base = nullptr;
  for (const GemmOut& o : p.outs)
    if (o.M > 0 && o.N > 0 && (!base || o.C < base)) base = o.C;
  for (const GemmOut& o : p.outs) {
    if (o.M <= 0 || o.N <= 0) continue;
    if (o.beta != 0) throw Error(-6, "tensor-core GEMM plan: accumulating outputs are not supported");
    // the term pieces of this output (each at most kc of K)
    const int t0 = (int)terms.size();
    int64_t ktot = 0;
    for (int t = o.t0; t < o.t1; ++t) {
      const GemmTerm& g = p.terms[t];
      if (g.K <= 0) continue;
      const bool ta = g.flags & 1, tb = g.flags & 2;
      const double mag = std::fabs(g.alpha);
      const bool unit = mag == 1.0;
      // A panel: op(B)^T, N rows; B panel: op(A), M rows (alpha folded in
      // unless it is a sign)
      const Blk a = block(mapA, convA, rowsA, g.B, o.N, g.K, g.ldb, tb ? 0 : 1, 1.0);
      const Blk b = block(mapB, convB, rowsB, g.A, o.M, g.K, g.lda, ta ? 1 : 0, unit ? 1.0 : g.alpha);
      const int neg = unit && g.alpha < 0 ? 1 : 0;
      for (int64_t k0 = 0; k0 < g.K; k0 += kc) {
        const int64_t kb = k0 / W;
        const int k = (int)std::min<int64_t>(kc, g.K - k0);
        TcTerm tm{0, (int32_t)(a.row0 + kb * a.rows), (int32_t)(b.row0 + kb * b.rows),
                  (k + kstep - 1) / kstep * kstep, neg, 0, a.rows, b.rows};
        terms.push_back(tm);
        ktot += tm.k;
      }
    }
    const int t1 = (int)terms.size();
    const int64_t out = o.C - base;
    for (int nA = 0; nA < o.N; nA += 128)
      for (int mB = 0; mB < o.M; mB += ncap) {
        TcTile T{};
        T.t0 = t0;
        T.t1 = t1;
        T.m0 = nA;
        T.m_valid = std::min(128, o.N - nA);
        T.n0 = mB;
        T.n_valid = std::min(ncap, o.M - mB);
        T.n_mma = (T.n_valid + 15) / 16 * 16;
        T.bsel = bsel_of(T.n_mma);
        T.mode = kTcSigma;
        T.beta = 0;
        T.ld = o.ldc;
        T.out = out + (int64_t)mB * o.ldc;
        if (ktot <= kc) {
          tiles.push_back(T);
          continue;
        }
        // split K: chunks of whole pieces into FP32 slots, summed in FP64
        TcRed R{T.out, slot, red_total, T.ld, T.m0, T.m_valid, T.n_valid, T.n_mma, 0};
        red_total += (int64_t)T.m_valid * T.n_valid;
        int t = t0;
        while (t < t1) {
          TcTile Cc = T;
          Cc.t0 = t;
          int64_t k = 0;
          while (t < t1 && (t == Cc.t0 || k + terms[t].k <= kc)) k += terms[t++].k;
          Cc.t1 = t;
          Cc.mode = kTcPart;
          Cc.out = slot;
          Cc.ld = 128;
          slot += (int64_t)128 * T.n_mma;
          R.nslot++;
          tiles.push_back(Cc);
        }
        red.push_back(R);
      }
  }
  if (tiles.empty()) return;
  rowsA = std::max<int64_t>(rowsA, 128);
  rowsB = std::max<int64_t>(rowsB, 256);
  // ---- panels (zeroed: K padding and rows past a block read zeros) and conversions
  const int nh = split ? 2 : 1;
  void* pa[2] = {nullptr, nullptr};
  void* pb[2] = {nullptr, nullptr};
  for (int h = 0; h < nh; ++h) {
    pa[h] = dalloc<uint8_t>((size_t)rowsA * W * eb);
    pb[h] = dalloc<uint8_t>((size_t)rowsB * W * eb);
    CK(cudaMemsetAsync(pa[h], 0, (size_t)rowsA * W * eb, stream));
    CK(cudaMemsetAsync(pb[h], 0, (size_t)rowsB * W * eb, stream));
  }
  for (int side = 0; side < 2; ++side) {
    std::vector<TcConv>& cv = side ? convB : convA;
    if (cv.empty()) continue;
    TcConv* d = dalloc<TcConv>(cv.size());
    h2d(d, cv.data(), cv.size() * sizeof(TcConv));
    void** pan = side ? pb : pa;
    launch_tc_convert(d, (int)cv.size(), prec, pan[0], pan[1], W, stream);
    stats.launches++;
    CK(cudaGetLastError());
    dfree(d);
  }
  TcMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int h = 0; h < nh; ++h) {
    bool ok = tc_encode_panel(&maps.a[h], eb, pa[h], W, rowsA, 128);
    for (int b = 0; b < 5 && ok; ++b) ok = tc_encode_panel(&maps.b[h][b], eb, pb[h], W, rowsB, 16u << b);
    if (!ok) throw Error(-3, "tensor map encoding failed");
  }
  TcTile* dt = dalloc<TcTile>(tiles.size());
  TcTerm* dm = dalloc<TcTerm>(std::max<size_t>(terms.size(), 1));
  h2d(dt, tiles.data(), tiles.size() * sizeof(TcTile));
  h2d(dm, terms.data(), terms.size() * sizeof(TcTerm));
  float* part = slot ? dalloc<float>((size_t)slot) : nullptr;
  TcRed* dr = red.empty() ? nullptr : dalloc<TcRed>(red.size());
  if (dr) h2d(dr, red.data(), red.size() * sizeof(TcRed));
  if (!d_env_err) {
    d_env_err = dalloc<int>(1);
    CK(cudaMemsetAsync(d_env_err, 0, sizeof(int), stream));
  }
  TcLaunch L{dt, dm, (int)tiles.size(), prec, nullptr, nullptr, base, d_env_err, part, nullptr, nullptr, ncap,
             tc_stages(prec, ncap)};
  if (!launch_tc_gemm(maps, L, num_sms, stream)) throw Error(-3, "invalid tensor-core launch configuration");
  stats.launches++;
  if (dr) {
    launch_tc_reduce(dr, (int)red.size(), red_total, part, base, stream);
    stats.launches++;
  }
  CK(cudaGetLastError());
  env_tc_pending = true;   // the bounded-wait flag is read after the next synchronisation
  for (int h = 0; h < nh; ++h) {
    dfree(pa[h]);
    dfree(pb[h]);
  }
  for (void* q : {(void*)dt, (void*)dm, (void*)part, (void*)dr})
    if (q) dfree(q);
}

}  // namespace gbd

namespace gbd {

// Self-test of run_tc against the FP64 grouped GEMM on random operands: two
// outputs (M x N and a smaller one sharing the first term's A block), nterms
// terms each of K columns with transposition flags `flags` (1 transA, 2
// transB) and alternating signs; max |C_tc - C_fp64| and max |C_fp64|.
void Engine::gemm_tc_selftest(int M, int N, int K, int nterms, int flags, int prec, uint64_t seed, double* max_err,
                              double* max_ref) {
  const bool ta = flags & 1, tb = flags & 2;
  uint64_t st = seed * 0x9E3779B97F4A7C15ull + 1;
  auto rnd = [&]() {
    st ^= st >> 12;
    st ^= st << 25;
    st ^= st >> 27;
    return (double)((st * 0x2545F4914F6CDD1Dull) >> 11) / 9007199254740992.0 - 0.5;
  };
  const int lda = (ta ? M : K) + 3, ldb = (tb ? K : N) + 5;
  const size_t asz = (size_t)(ta ? K : M) * lda, bsz = (size_t)(tb ? N : K) * ldb;
  std::vector<double> hA(asz * nterms), hB(bsz * nterms);
  for (double& v : hA) v = rnd();
  for (double& v : hB) v = rnd();
  double* A = dalloc<double>(hA.size());
  double* B = dalloc<double>(hB.size());
  const int ldc = N + 7;
  const int M2 = std::max(1, M / 3), N2 = std::max(1, N / 2);
  const size_t csz = (size_t)M * ldc + (size_t)M2 * N2;
  double* C1 = dalloc<double>(csz);
  double* C2 = dalloc<double>(csz);
  h2d(A, hA.data(), hA.size() * sizeof(double));
  h2d(B, hB.data(), hB.size() * sizeof(double));
  CK(cudaMemsetAsync(C1, 0, csz * sizeof(double), stream));
  CK(cudaMemsetAsync(C2, 0, csz * sizeof(double), stream));
  auto plan = [&](double* C, GemmPlan& p) {
    p.add_out(C, ldc, M, N, 0);
    for (int t = 0; t < nterms; ++t)
      p.add_term(A + asz * t, lda, B + bsz * t, ldb, K, flags, t % 2 ? -1.0 : 1.0);
    // second output: the first term's operands on a corner, scaled by 0.5
    p.add_out(C + (size_t)M * ldc, N2, M2, N2, 0);
    p.add_term(A, lda, B, ldb, K, flags, 0.5);
  };
  GemmPlan p1, p2;
  plan(C1, p1);
  plan(C2, p2);
  check(p1);
  run_tc(p1, prec);
  upload(p2);
  run(p2);
  release(p2);
  std::vector<double> h1(csz), h2(csz);
  CK(cudaMemcpyAsync(h1.data(), C1, csz * sizeof(double), cudaMemcpyDeviceToHost, stream));
  CK(cudaMemcpyAsync(h2.data(), C2, csz * sizeof(double), cudaMemcpyDeviceToHost, stream));
  sync();
  double me = 0, mr = 0;
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < N; ++j) {
      me = std::max(me, std::fabs(h1[(size_t)i * ldc + j] - h2[(size_t)i * ldc + j]));
      mr = std::max(mr, std::fabs(h2[(size_t)i * ldc + j]));
    }
  for (size_t e = (size_t)M * ldc; e < csz; ++e) {
    me = std::max(me, std::fabs(h1[e] - h2[e]));
    mr = std::max(mr, std::fabs(h2[e]));
  }
  *max_err = me;
  *max_ref = mr;
  for (void* q : {(void*)A, (void*)B, (void*)C1, (void*)C2}) dfree(q);
  sync();
}

}  // namespace gbd
