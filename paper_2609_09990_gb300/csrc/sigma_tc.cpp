// Reduced-precision sigma build on the tensor cores.
//
// The same two stages as the FP64 path (stage A  Y_b = psi Renl[b]^T,
// stage B  sigma = sum_b Lenl[b] Y_b), run by the tcgen05 grouped GEMM on
// panels: the two-site state, the enlarged-operator sub-blocks and the Y^T
// intermediate are stored in BF16, TF32 or TF32 hi/lo with every K range
// starting at a multiple of 16 columns and zero padded.  Stage A writes Y^T
// straight into the stage-B operand panel; stage B accumulates sigma in FP32
// (TMEM) and stores it as FP64.  The enlarged operators and environments
// stay FP64; only the matvec inside Davidson changes precision.
#include <algorithm>
#include <climits>
#include <cstring>
#include <map>

#include "engine.h"
#include "tc_gemm.h"

namespace gbd {

int tc_smem_bytes(int prec);

struct TcPlan {
  int prec = 0, eb = 2;
  void *psi[2] = {nullptr, nullptr}, *rs[2] = {nullptr, nullptr}, *ls[2] = {nullptr, nullptr},
       *yt[2] = {nullptr, nullptr};
  int64_t psi_pitch = 0, rs_pitch = 0, ls_pitch = 0, yt_pitch = 0;
  TcPsiSector* d_sec = nullptr;
  int nsec = 0;
  TcTile* d_tiles[2] = {nullptr, nullptr};
  TcTerm* d_terms[2] = {nullptr, nullptr};
  int ntiles[2] = {0, 0};
  TcMaps maps[2];
  int* d_err = nullptr;
  double flops_alg = 0, flops_exec = 0;
};

namespace {
inline int64_t up16(int64_t x) { return (x + 15) / 16 * 16; }
inline int64_t up64(int64_t x) { return std::max<int64_t>(64, (x + 63) / 64 * 64); }
inline int bsel_for(int n) {
  int b = 0;
  while ((16 << b) < n) ++b;
  return b;
}
}  // namespace

TcPlan* Engine::tc_build(const EnlOp& lenl, const EnlOp& renl, int prec) {
  TcPlan* P = new TcPlan();
  P->prec = prec;
  P->eb = prec == kBF16 ? 2 : 4;
  const int nh = prec == kTF32x3 ? 2 : 1;
  const int nq = EL.n();
  // ---- psi panel: rows E_L(Q) stacked, columns E_R(Q) with padded sub-ranges
  std::vector<int64_t> psi_row(nq);
  std::vector<std::array<int, 4>> cpadR(nq), cpadL(nq);
  int64_t rows = 0, wmax = 0, wlmax = 0;
  std::vector<TcPsiSector> sec(nq);
  for (int q = 0; q < nq; ++q) {
    psi_row[q] = rows;
    rows += EL.dim[q];
    int64_t w = 0, wl = 0;
    for (int s = 0; s < 4; ++s) {
      cpadR[q][s] = (int)w;
      if (ER.soff[q][s] >= 0) w += up16(ER.sdim[q][s]);
      cpadL[q][s] = (int)wl;
      if (EL.soff[q][s] >= 0) wl += up16(EL.sdim[q][s]);
    }
    wmax = std::max(wmax, w);
    wlmax = std::max(wlmax, wl);
    TcPsiSector& S = sec[q];
    S.src_off = psi_off[q];
    S.rows = EL.dim[q];
    S.cols = ER.dim[q];
    S.r0 = (int32_t)psi_row[q];
    for (int s = 0; s < 4; ++s) {
      S.cbreak[s] = ER.soff[q][s] >= 0 ? ER.soff[q][s] : INT_MAX;
      S.cpad[s] = cpadR[q][s];
    }
  }
  P->psi_pitch = up64(wmax);
  const int64_t psi_rows = std::max<int64_t>(rows, 1);
  // ---- sub-block panels
  auto sub_panel = [&](const EnlOp& op, std::vector<int64_t>& rowof, int64_t& pitch) {
    int64_t r = 0, w = 0;
    rowof.resize(op.subs.size());
    for (size_t i = 0; i < op.subs.size(); ++i) {
      rowof[i] = r;
      r += op.subs[i].rows;
      w = std::max<int64_t>(w, up16(op.subs[i].cols));
    }
    pitch = up64(w);
    return std::max<int64_t>(r, 1);
  };
  std::vector<int64_t> rs_row, ls_row;
  const int64_t rs_rows = sub_panel(renl, rs_row, P->rs_pitch);
  const int64_t ls_rows = sub_panel(lenl, ls_row, P->ls_pitch);
  // ---- Y blocks (b, Qin) -> rows E_R(Qout) of the Y^T panel
  std::map<std::pair<int, int>, std::vector<int>> rby, lout;
  std::map<std::pair<int, int>, int> lhas;
  for (size_t i = 0; i < renl.subs.size(); ++i) rby[{renl.subs[i].b, renl.subs[i].qin}].push_back((int)i);
  for (size_t i = 0; i < lenl.subs.size(); ++i) {
    lhas[{lenl.subs[i].b, lenl.subs[i].qin}] = 1;
    lout[{lenl.subs[i].qout, lenl.subs[i].sout}].push_back((int)i);
  }
  std::map<std::pair<int, int>, int64_t> ybase;
  int64_t yrows = 0;
  for (auto& kv : rby) {
    if (!lhas.count(kv.first)) continue;
    int qout = renl.subs[kv.second[0]].qout;
    ybase[kv.first] = yrows;
    yrows += ER.dim[qout];
  }
  P->yt_pitch = up64(wlmax);
  yrows = std::max<int64_t>(yrows, 1);
  // ---- allocate and zero the panels
  for (int h = 0; h < nh; ++h) {
    P->psi[h] = dalloc<uint8_t>((size_t)(psi_rows * P->psi_pitch * P->eb));
    P->rs[h] = dalloc<uint8_t>((size_t)(rs_rows * P->rs_pitch * P->eb));
    P->ls[h] = dalloc<uint8_t>((size_t)(ls_rows * P->ls_pitch * P->eb));
    P->yt[h] = dalloc<uint8_t>((size_t)(yrows * P->yt_pitch * P->eb));
    CK(cudaMemsetAsync(P->psi[h], 0, psi_rows * P->psi_pitch * P->eb, stream));
    CK(cudaMemsetAsync(P->rs[h], 0, rs_rows * P->rs_pitch * P->eb, stream));
    CK(cudaMemsetAsync(P->ls[h], 0, ls_rows * P->ls_pitch * P->eb, stream));
    CK(cudaMemsetAsync(P->yt[h], 0, yrows * P->yt_pitch * P->eb, stream));
  }
  // ---- convert the sub-blocks (once per step)
  auto convert = [&](const EnlOp& op, const std::vector<int64_t>& rowof, void** panel, int64_t pitch) {
    std::vector<TcConv> tasks;
    for (size_t i = 0; i < op.subs.size(); ++i) {
      const EnlSub& s = op.subs[i];
      check_range(s.ptr, s.rows, s.cols, s.cols, "tc convert source");
      tasks.push_back({s.ptr, s.sign, s.rows, s.cols, s.cols, (int32_t)rowof[i], 0});
    }
    if (tasks.empty()) return;
    TcConv* d = dalloc<TcConv>(tasks.size());
    CK(cudaMemcpyAsync(d, tasks.data(), tasks.size() * sizeof(TcConv), cudaMemcpyHostToDevice, stream));
    launch_tc_convert(d, (int)tasks.size(), prec, panel[0], panel[1], pitch, stream);
    stats.launches++;
    CK(cudaGetLastError());
    sync();
    dfree(d);
  };
  convert(renl, rs_row, P->rs, P->rs_pitch);
  convert(lenl, ls_row, P->ls, P->ls_pitch);
  P->nsec = nq;
  P->d_sec = dalloc<TcPsiSector>(std::max(nq, 1));
  CK(cudaMemcpyAsync(P->d_sec, sec.data(), nq * sizeof(TcPsiSector), cudaMemcpyHostToDevice, stream));
  // ---- stage A tiles: Y_b(Qin)[:, (so, q_r')] = sum psi(Qin)[:, (si, q_r)] Rsub^T
  std::vector<TcTile> tiles;
  std::vector<TcTerm> terms;
  for (auto& kv : rby) {
    auto yb = ybase.find(kv.first);
    if (yb == ybase.end()) continue;
    const int qin = kv.first.second;
    const int qout = renl.subs[kv.second[0]].qout;
    for (int so = 0; so < 4; ++so) {
      if (ER.soff[qout][so] < 0) continue;
      const int N = ER.sdim[qout][so];
      for (int m0 = 0; m0 < EL.dim[qin]; m0 += 128)
        for (int n0 = 0; n0 < N; n0 += 256) {
          TcTile T{};
          T.t0 = (int)terms.size();
          for (int i : kv.second) {
            const EnlSub& s = renl.subs[i];
            if (s.sout != so) continue;
            terms.push_back({cpadR[qin][s.sin], (int32_t)psi_row[qin], (int32_t)(rs_row[i] + n0),
                             (int32_t)up16(s.cols), 0, 0});
            P->flops_alg += m0 == 0 && n0 == 0 ? 2.0 * EL.dim[qin] * N * s.cols : 0.0;
          }
          T.t1 = (int)terms.size();
          T.m0 = m0;
          T.m_valid = std::min(128, EL.dim[qin] - m0);
          const int nv = std::min(256, N - n0);
          T.n_mma = (int)up16(nv);
          T.n_valid = nv;
          T.bsel = bsel_for(T.n_mma);
          T.mode = kTcYT;
          T.beta = 0;
          T.ld = (int32_t)P->yt_pitch;
          T.out = yb->second + ER.soff[qout][so] + n0;
          for (int s = 0; s < 4; ++s) {
            T.rbreak[s] = EL.soff[qin][s] >= 0 ? EL.soff[qin][s] : INT_MAX;
            T.rpad[s] = cpadL[qin][s];
          }
          for (int t = T.t0; t < T.t1; ++t) P->flops_exec += 2.0 * 128 * T.n_mma * terms[t].k;
          tiles.push_back(T);
        }
    }
  }
  auto upload_tiles = [&](int which) {
    P->ntiles[which] = (int)tiles.size();
    std::stable_sort(tiles.begin(), tiles.end(),
                     [](const TcTile& a, const TcTile& b) { return (a.t1 - a.t0) > (b.t1 - b.t0); });
    P->d_tiles[which] = dalloc<TcTile>(std::max<size_t>(tiles.size(), 1));
    P->d_terms[which] = dalloc<TcTerm>(std::max<size_t>(terms.size(), 1));
    if (!tiles.empty())
      CK(cudaMemcpyAsync(P->d_tiles[which], tiles.data(), tiles.size() * sizeof(TcTile), cudaMemcpyHostToDevice,
                         stream));
    if (!terms.empty())
      CK(cudaMemcpyAsync(P->d_terms[which], terms.data(), terms.size() * sizeof(TcTerm), cudaMemcpyHostToDevice,
                         stream));
    sync();
    tiles.clear();
    terms.clear();
  };
  upload_tiles(0);
  // ---- stage B tiles: sigma(Qout)[rows (q_l', so), E_R tile] = sum Y^T Lsub^T
  for (int q = 0; q < nq; ++q)
    for (int so = 0; so < 4; ++so) {
      if (EL.soff[q][so] < 0) continue;
      const int N = EL.sdim[q][so];
      auto it = lout.find({q, so});
      for (int m0 = 0; m0 < ER.dim[q]; m0 += 128)
        for (int n0 = 0; n0 < N; n0 += 256) {
          TcTile T{};
          T.t0 = (int)terms.size();
          if (it != lout.end())
            for (int i : it->second) {
              const EnlSub& s = lenl.subs[i];
              auto yb = ybase.find({s.b, s.qin});
              if (yb == ybase.end()) continue;
              terms.push_back({cpadL[s.qin][s.sin], (int32_t)yb->second, (int32_t)(ls_row[i] + n0),
                               (int32_t)up16(s.cols), 0, 0});
              P->flops_alg += m0 == 0 && n0 == 0 ? 2.0 * ER.dim[q] * N * s.cols : 0.0;
            }
          T.t1 = (int)terms.size();
          T.m0 = m0;
          T.m_valid = std::min(128, ER.dim[q] - m0);
          const int nv = std::min(256, N - n0);
          T.n_mma = (int)up16(nv);
          T.n_valid = nv;
          T.bsel = bsel_for(T.n_mma);
          T.mode = kTcSigma;
          T.beta = 0;
          T.ld = ER.dim[q];
          T.out = psi_off[q] + (int64_t)(EL.soff[q][so] + n0) * ER.dim[q];
          for (int t = T.t0; t < T.t1; ++t) P->flops_exec += 2.0 * 128 * T.n_mma * terms[t].k;
          tiles.push_back(T);
        }
    }
  upload_tiles(1);
  // ---- tensor maps
  std::memset(P->maps, 0, sizeof(P->maps));
  for (int h = 0; h < nh; ++h) {
    bool ok = tc_encode_panel(&P->maps[0].a[h], P->eb, P->psi[h], P->psi_pitch, psi_rows, 128) &&
              tc_encode_panel(&P->maps[1].a[h], P->eb, P->yt[h], P->yt_pitch, yrows, 128);
    for (int b = 0; b < 5 && ok; ++b)
      ok = tc_encode_panel(&P->maps[0].b[h][b], P->eb, P->rs[h], P->rs_pitch, rs_rows, 16u << b) &&
           tc_encode_panel(&P->maps[1].b[h][b], P->eb, P->ls[h], P->ls_pitch, ls_rows, 16u << b);
    if (!ok) {
      tc_free(P);
      throw Error(-3, "tensor map encoding failed");
    }
  }
  P->d_err = dalloc<int>(1);
  CK(cudaMemsetAsync(P->d_err, 0, sizeof(int), stream));
  sync();
  return P;
}

void Engine::tc_free(TcPlan* P) {
  if (!P) return;
  for (int h = 0; h < 2; ++h)
    for (void* p : {P->psi[h], P->rs[h], P->ls[h], P->yt[h]})
      if (p) dfree(p);
  for (int w = 0; w < 2; ++w) {
    if (P->d_tiles[w]) dfree(P->d_tiles[w]);
    if (P->d_terms[w]) dfree(P->d_terms[w]);
  }
  if (P->d_sec) dfree(P->d_sec);
  if (P->d_err) dfree(P->d_err);
  delete P;
}

// y = H_eff x with the tensor-core stages (every sub-block's coefficient is
// folded into its converted panel rows, so no term carries a sign) (x, y: FP64 two-site vectors)
void Engine::tc_apply(TcPlan* P, const double* x, double* y) {
  settle();
  CK(cudaEventRecord(ev0, stream));
  launch_tc_convert_psi(x, P->d_sec, P->nsec, psi_size, P->prec, P->psi[0], P->psi[1], P->psi_pitch, stream);
  TcLaunch A{P->d_tiles[0], P->d_terms[0], P->ntiles[0], P->prec, P->yt[0], P->yt[1], nullptr, P->d_err};
  launch_tc_gemm(P->maps[0], A, num_sms, stream);
  TcLaunch B{P->d_tiles[1], P->d_terms[1], P->ntiles[1], P->prec, nullptr, nullptr, y, P->d_err};
  launch_tc_gemm(P->maps[1], B, num_sms, stream);
  CK(cudaEventRecord(ev1, stream));
  CK(cudaMemcpyAsync(tc_err_host, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, stream));
  stats.launches += 3;
  CK(cudaGetLastError());
  sigma_pending = 2;
  stats.sigma_flops += P->flops_alg;
  stats.sigma_flops_exec += P->flops_exec;
  stats.n_sigma++;
  stats.n_sigma_tc++;
  stats.tc_flops += P->flops_alg;
}

}  // namespace gbd
