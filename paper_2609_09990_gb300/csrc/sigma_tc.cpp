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
#include <atomic>
#include <array>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

#include "engine.h"
#include "linalg_host.h"
#include "tc_gemm.h"

namespace gbd {


struct TcPlan {
  int prec = 0, eb = 2;
  TcTune tune;
  void *psi[2] = {nullptr, nullptr}, *rs[2] = {nullptr, nullptr}, *ls[2] = {nullptr, nullptr},
       *yt[2] = {nullptr, nullptr};
  int64_t psi_pitch = 0, rs_pitch = 0, ls_pitch = 0, yt_pitch = 0;
  TcPsiSector* d_sec = nullptr;
  int nsec = 0;
  TcTile* d_tiles[2] = {nullptr, nullptr};
  TcTerm* d_terms[2] = {nullptr, nullptr};
  int ntiles[2] = {0, 0};
  TcMaps maps[2];
  float* part = nullptr;         // split-K partial slots of stage B
  TcYRow* d_yrows = nullptr;      // stage A: where the stacked Renl rows of each member go in Y^T
  int32_t* d_ymem = nullptr;      // stage A: member of every stacked row
  double *xin = nullptr, *yout = nullptr;   // fixed sigma input/output of the replayed graph
  GraphSeq graph;
  TcRed* d_red = nullptr;
  int nred = 0;
  int64_t red_total = 0;
  int64_t kc = 0;                // split-K chunk length (summed K of whole terms)
  int* d_err = nullptr;
  double flops_alg = 0, flops_exec = 0;
  // algorithmic HBM bytes of one sigma: the Renl and Lenl sub-blocks once,
  // the Y^T sections that some Lenl sub-block reads written once and read
  // once, psi read and sigma written in FP64
  double bytes_alg = 0;
  // the same split by stage (A, B), and the bytes the TMA boxes of each
  // stage request from L2, by operand (A box, B box): whole boxes of 128
  // B wide and 128 (A) or 16 << bsel (B) rows per K step
  double alg_st[2] = {0, 0}, box_st[2][2] = {{0, 0}, {0, 0}};
  // the valid rows x K of those boxes (no padding of rows, K or box width)
  double dense_st[2][2] = {{0, 0}, {0, 0}};
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

TcPlan* Engine::tc_build(const EnlOp& lenl, const EnlOp& renl, int prec, TcTune tune) {
  TcPlan* P = new TcPlan();
  P->prec = prec;
  P->tune = tune;
  P->eb = prec == kBF16 || prec == kBF16x3 ? 2 : 4;
  const int nh = prec == kTF32x3 || prec == kBF16x3 ? 2 : 1;
  const int nq = EL.n();
  double tph = now_ms();
  auto phase = [&](int i) {
    const double t = now_ms();
    stats.tcb_ms[i] += t - tph;
    tph = t;
  };
  // ---- psi panel: rows E_L(Q) stacked, columns E_R(Q) with padded sub-ranges
  std::vector<int64_t> psi_row(nq);
  std::vector<std::array<int, 4>> cpadR(nq), cpadL(nq);
  int64_t rows = 0, wmax = 0;
  std::vector<TcPsiSector> sec(nq);
  std::vector<int> wlq(nq);   // padded width of E_L(q)
  for (int q = 0; q < nq; ++q) {
    psi_row[q] = rows;
    int64_t w = 0, wl = 0;
    for (int s = 0; s < 4; ++s) {
      cpadR[q][s] = (int)w;
      if (ER.soff[q][s] >= 0) w += up16(ER.sdim[q][s]);
      cpadL[q][s] = (int)wl;
      if (EL.soff[q][s] >= 0) wl += up16(EL.sdim[q][s]);
    }
    wlq[q] = (int)wl;
    rows += wl;   // psi rows in padded E_L positions (zero rows in the padding)
    wmax = std::max(wmax, w);
    TcPsiSector& S = sec[q];
    S.src_off = psi_off[q];
    S.rows = EL.dim[q];
    S.cols = ER.dim[q];
    S.r0 = (int32_t)psi_row[q];
    for (int s = 0; s < 4; ++s) {
      S.cbreak[s] = ER.soff[q][s] >= 0 ? ER.soff[q][s] : INT_MAX;
      S.cpad[s] = cpadR[q][s];
      S.rbreak[s] = EL.soff[q][s] >= 0 ? EL.soff[q][s] : INT_MAX;
      S.rpad[s] = cpadL[q][s];
    }
  }
  P->psi_pitch = up64(wmax);
  const int64_t psi_rows = std::max<int64_t>(rows, 256);   // >= the largest B box
  // ---- K layout of stage B.  For output sector q the contraction runs
  //      over the column sections (b, qin, sin) that some Lenl[b] sub-block
  //      (qin, sin -> q, sout) reads, in the order (b, qin, sin), each
  //      section up16(cols) wide: K_q in all.  Y^T(q) (rows E_R(q)) and the
  //      Lenl panel of q (rows E_L(q): every s_out section at its offset,
  //      zero where Lenl[b] has no sub-block into it) are stored K-blocked:
  //      block j holds columns [jW, (j+1)W) of every row, one W-element
  //      panel row each (W = one 128-byte box row).  A stage-B tile then
  //      streams dense boxes down the blocks, and the rows a 128-row box
  //      reads beyond E_R(q) are the next block's, which it reads next.
  //      Only the sections some sub-block reads are written by stage A.
  const int W = 128 / P->eb;
  int nb = 0;
  for (const EnlSub& s : renl.subs) nb = std::max(nb, s.b + 1);
  for (const EnlSub& s : lenl.subs) nb = std::max(nb, s.b + 1);
  std::vector<int> rfirst((size_t)nb * nq, -1);   // first Renl sub of (b, qin)
  for (size_t i = 0; i < renl.subs.size(); ++i) {
    int& f = rfirst[(size_t)renl.subs[i].b * nq + renl.subs[i].qin];
    if (f < 0) f = (int)i;
  }
  std::vector<int32_t> koff((size_t)nb * nq * 4, -1);   // K offset of section (b, qin, sin) in K_qout
  std::vector<char> yuse((size_t)nb * nq, 0);            // (b, qin) has a section in use
  std::vector<int64_t> Kq(nq, 0), yrow0(nq, 0);
  // K groups of output sector q: sections read by only the s_out section g
  // of E_L(q) form group g (0..3), sections read by several form group 4;
  // each group starts at a K-block boundary.  gk[q][g] = first K, gk[q][g+1]
  // bounds it (aligned up).  Stage B multiplies Y^T(q) by one Lenl panel per
  // s_out section over group s_out and group 4 only, so the panel holds the
  // rows of that section alone (no zero rows of other sections).
  std::vector<std::array<int64_t, 6>> gk(nq);
  std::vector<std::array<int64_t, 5>> glen(nq);
  std::vector<std::array<int64_t, 4>> lrow0s(nq), kqs(nq);   // Lenl panel of (q, s_out): first row, K length
  std::vector<int64_t> lrow0(nq, -1);                        // unsplit sector: one panel over E_L(q)
  std::vector<int> smask((size_t)nb * nq * 4, 0);          // s_out sections reading a section
  // split sectors: E_L(q) of at least tc_sout_min rows (smaller ones keep one
  // panel over all of E_L(q): their zero rows cost less than more, smaller
  // tiles); an unsplit sector has all its sections in group 0
  std::vector<char> spl(nq, 0);
  for (int q = 0; q < nq; ++q) spl[q] = EL.dim[q] >= tc_sout_min;
  std::vector<int8_t> kgroup;   // group of every listed section (filled once its s_out mask is complete)
  auto group_of = [&](int32_t key) { return (int)kgroup[key]; };
  auto upW = [&](int64_t x) { return (x + W - 1) / W * W; };
  int64_t yrows = 0, ls_rows = 0;
  {
    std::vector<std::vector<int32_t>> secs((size_t)nq);
    for (const EnlSub& s : lenl.subs) {
      const size_t bq = (size_t)s.b * nq + s.qin, key = bq * 4 + s.sin;
      if (s.cols != EL.sdim[s.qin][s.sin] || s.rows != EL.sdim[s.qout][s.sout])
        throw Error(-3, "enlarged-operator sub-block does not match its sections");
      if (rfirst[bq] < 0) continue;   // no Y block
      if (renl.subs[rfirst[bq]].qout != s.qout) throw Error(-3, "Lenl and Renl channels disagree on the sector");
      smask[key] |= 1 << s.sout;
      if (koff[key] != -1) continue;   // already listed
      koff[key] = -2;
      secs[s.qout].push_back((int32_t)key);
    }
    kgroup.assign(smask.size(), 0);
    for (int q = 0; q < nq; ++q)
      if (spl[q])
        for (int32_t key : secs[q]) {
          const int m = smask[key];
          kgroup[key] = (int8_t)((m & (m - 1)) ? 4 : __builtin_ctz(m));
        }
    for (int q = 0; q < nq; ++q) {
      // (group, b, qin, sin) order
      std::sort(secs[q].begin(), secs[q].end(), [&](int32_t x, int32_t y) {
        const int gx = group_of(x), gy = group_of(y);
        return gx != gy ? gx < gy : x < y;
      });
      int64_t k = 0;
      size_t i = 0;
      for (int g = 0; g < 5; ++g) {
        k = upW(k);
        gk[q][g] = k;
        for (; i < secs[q].size() && group_of(secs[q][i]) == g; ++i) {
          const int32_t key = secs[q][i];
          koff[key] = (int32_t)k;
          yuse[key / 4] = 1;
          const int qin = (key / 4) % nq, sin = key % 4;
          k += up16(EL.sdim[qin][sin]);
          // Y^T(q) section written by stage A and read by stage B
          const double yb = (double)P->eb * nh * ER.dim[q] * EL.sdim[qin][sin];
          P->bytes_alg += 2.0 * yb;
          P->alg_st[0] += yb;
          P->alg_st[1] += yb;
        }
        glen[q][g] = k - gk[q][g];
      }
      gk[q][5] = upW(k);
      Kq[q] = k;
      const int64_t nblk = gk[q][5] / W;
      yrow0[q] = yrows;
      yrows += nblk * ER.dim[q];
      for (int so = 0; so < 4; ++so) {
        lrow0s[q][so] = -1;
        kqs[q][so] = 0;
      }
      if (!spl[q]) {
        lrow0[q] = ls_rows;
        ls_rows += nblk * EL.dim[q];
        continue;
      }
      for (int so = 0; so < 4; ++so) {
        if (EL.soff[q][so] < 0 || (glen[q][so] == 0 && glen[q][4] == 0)) continue;
        kqs[q][so] = upW(glen[q][so]) + upW(glen[q][4]);
        lrow0s[q][so] = ls_rows;
        ls_rows += kqs[q][so] / W * EL.sdim[q][so];
      }
    }
  }
  P->yt_pitch = W;
  P->ls_pitch = W;
  yrows = std::max<int64_t>(yrows, 128);
  ls_rows = std::max<int64_t>(ls_rows, 256);
  // ---- stage A operand: the Renl sub-blocks with the same (qin, qout, so)
  //      and the same set of input local states si, stacked over b (rows
  //      m(so) per b), one 16-aligned column section per si.  Every stacked
  //      row is one row of Y^T, so a 128-row A box covers many channels b.
  //      The B operand (psi rows of qin) and the column sections depend on
  //      (qin, set of si) only, so members with different (qout, so) share
  //      a group; each member's run record sends its stacked rows, and each
  //      column section of them, to their place in the K-blocked Y^T(Qout).
  struct AGroup {
    int qin, mask;
    std::vector<std::array<int, 4>> mem;   // per member: sub index for each si (-1: none)
    std::vector<int> b, qout, so;
    std::vector<int64_t> roff;             // first stacked row of each member (from row0)
    int64_t rows = 0, row0 = 0;
    std::array<int, 4> col{};
  };
  std::vector<AGroup> groups;
  std::vector<TcYRow> yrowtab;
  std::vector<int32_t> ymem;
  int64_t rs_rows = 0, rs_width = 0;
  {
    // (b, qin) with a Y block in use -> compact index; (that index, so) -> subs per si
    std::vector<int> bq_of((size_t)nb * nq, -1);
    int nbq = 0;
    for (size_t bq = 0; bq < yuse.size(); ++bq)
      if (yuse[bq]) bq_of[bq] = nbq++;
    std::vector<std::array<int, 4>> bso((size_t)nbq * 4, std::array<int, 4>{-1, -1, -1, -1});
    std::vector<int> bq_key((size_t)nbq);
    for (size_t bq = 0; bq < yuse.size(); ++bq)
      if (bq_of[bq] >= 0) bq_key[bq_of[bq]] = (int)bq;
    for (size_t i = 0; i < renl.subs.size(); ++i) {
      const EnlSub& s = renl.subs[i];
      const int c = bq_of[(size_t)s.b * nq + s.qin];
      if (c < 0) continue;
      int& slot = bso[(size_t)c * 4 + s.sout][s.sin];
      if (slot >= 0) throw Error(-3, "duplicate enlarged-operator sub-block");
      slot = (int)i;
    }
    std::vector<int> gidx((size_t)nq * 16, -1);   // (qin, mask) -> group
    for (size_t key = 0; key < bso.size(); ++key) {
      const std::array<int, 4>& m = bso[key];
      int mask = 0, any = -1;
      for (int si = 0; si < 4; ++si)
        if (m[si] >= 0) {
          mask |= 1 << si;
          any = m[si];
        }
      if (!mask) continue;
      const int so = (int)(key % 4), bq = bq_key[key / 4];
      const int qin = bq % nq, b = bq / nq;
      const int qout = renl.subs[any].qout;
      int& g = gidx[(size_t)qin * 16 + mask];
      if (g < 0) {
        g = (int)groups.size();
        AGroup ng;
        ng.qin = qin;
        ng.mask = mask;
        groups.push_back(ng);
      }
      AGroup& G = groups[g];
      G.mem.push_back(m);
      G.b.push_back(b);
      G.qout.push_back(qout);
      G.so.push_back(so);
      G.roff.push_back(G.rows);
      G.rows += ER.sdim[qout][so];
    }
    for (AGroup& g : groups) {
      g.row0 = rs_rows;
      int64_t w = 0;
      for (int si = 0; si < 4; ++si) {
        g.col[si] = (int)w;
        if (g.mask >> si & 1) w += up16(ER.sdim[g.qin][si]);
      }
      rs_width = std::max(rs_width, w);
      for (size_t bi = 0; bi < g.b.size(); ++bi) {
        const int q = g.qout[bi], mso = ER.sdim[q][g.so[bi]];
        TcYRow R{};
        R.base = (yrow0[q] + ER.soff[q][g.so[bi]]) * (int64_t)W;
        R.stride = (int32_t)(ER.dim[q] * W);
        for (int s = 0; s < 4; ++s) R.koff[s] = koff[((size_t)g.b[bi] * nq + g.qin) * 4 + s];
        R.first = (int32_t)(g.row0 + g.roff[bi]);
        ymem.insert(ymem.end(), (size_t)mso, (int32_t)yrowtab.size());
        yrowtab.push_back(R);
      }
      rs_rows += g.rows;
    }
  }
  P->rs_pitch = up64(rs_width);
  rs_rows = std::max<int64_t>(rs_rows, 128);
  phase(0);   // host: layouts, groups, run records
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
  auto convert = [&](const EnlOp& op, const std::vector<int64_t>& rowof, const std::vector<int64_t>& colof,
                     const std::vector<int32_t>* kstride, void** panel, int64_t pitch) {
    // task lists of contiguous blocks of sub-blocks on the host pool,
    // concatenated in block order (the same list as a serial pass)
    const size_t nsub = op.subs.size();
    const int nblk = (int)std::min<size_t>(16, (nsub + 2047) / 2048);
    std::vector<std::vector<TcConv>> part((size_t)std::max(nblk, 1));
    std::atomic<int> bad(0);
    auto work = [&](int bb) {
      const size_t i0 = nsub * bb / nblk, i1 = nsub * (bb + 1) / nblk;
      std::vector<TcConv>& out = part[bb];
      out.reserve(i1 - i0);
      AllocCache cache;
      for (size_t i = i0; i < i1; ++i) {
        const EnlSub& s = op.subs[i];
        if (rowof[i] < 0) continue;   // not used by any product
        const bool ok = s.trans ? in_allocation(s.ptr, s.cols, s.rows, s.rows, cache)
                                : in_allocation(s.ptr, s.rows, s.cols, s.cols, cache);
        if (!ok) {
          bad = 1;
          return;
        }
        out.push_back({s.ptr, s.sign, s.rows, s.cols, s.trans ? s.rows : s.cols, (int32_t)rowof[i],
                       (int32_t)colof[i], kstride ? (*kstride)[i] : 0, s.trans});
      }
    };
    if (nblk > 1) host_parallel_for(nblk, work);
    else if (nblk == 1) work(0);
    if (bad) throw Error(-6, "plan check: tc convert source outside its allocation");
    std::vector<TcConv> tasks;
    size_t ntask = 0;
    for (const auto& v : part) ntask += v.size();
    tasks.reserve(ntask);
    for (const auto& v : part) tasks.insert(tasks.end(), v.begin(), v.end());
    if (tasks.empty()) return;
    TcConv* d = dalloc<TcConv>(tasks.size());
    h2d(d, tasks.data(), tasks.size() * sizeof(TcConv));
    launch_tc_convert(d, (int)tasks.size(), prec, panel[0], panel[1], pitch, stream);
    stats.launches++;
    CK(cudaGetLastError());
    dfree(d);   // stream-ordered: after the conversion
  };
  {
    std::vector<int64_t> r0(renl.subs.size(), -1), c0(renl.subs.size(), 0);
    for (const AGroup& g : groups)
      for (size_t bi = 0; bi < g.b.size(); ++bi)
        for (int si = 0; si < 4; ++si) {
          const int i = g.mem[bi][si];
          if (i < 0) continue;
          r0[i] = g.row0 + g.roff[bi];
          c0[i] = g.col[si];
        }
    convert(renl, r0, c0, nullptr, P->rs, P->rs_pitch);
  }
  {
    // Lenl sub-block (qin, sin -> q, sout): rows at E_L(q) offset of sout in
    // every K block of q, columns from the K offset of its section
    std::vector<int64_t> r0(lenl.subs.size(), -1), c0(lenl.subs.size(), 0);
    std::vector<int32_t> ks(lenl.subs.size(), 0);
    for (size_t i = 0; i < lenl.subs.size(); ++i) {
      const EnlSub& s = lenl.subs[i];
      const int32_t key = (int32_t)(((size_t)s.b * nq + s.qin) * 4 + s.sin);
      const int32_t k = koff[key];
      if (k < 0) continue;
      const int q = s.qout, g = group_of(key);
      if (!spl[q]) {   // rows at the E_L(q) offset of sout in every K block of q
        r0[i] = lrow0[q] + EL.soff[q][s.sout];
        c0[i] = k;
        ks[i] = EL.dim[q];
        continue;
      }
      // panel (qout, sout): group sout first, then group 4
      r0[i] = lrow0s[q][s.sout];
      c0[i] = g == 4 ? upW(glen[q][s.sout]) + (k - gk[q][4]) : k - gk[q][s.sout];
      ks[i] = EL.sdim[q][s.sout];
    }
    convert(lenl, r0, c0, &ks, P->ls, P->ls_pitch);
  }
  if (!yrowtab.empty()) {
    P->d_yrows = dalloc<TcYRow>(yrowtab.size());
    P->d_ymem = dalloc<int32_t>(ymem.size());
    h2d(P->d_yrows, yrowtab.data(), yrowtab.size() * sizeof(TcYRow));
    h2d(P->d_ymem, ymem.data(), ymem.size() * sizeof(int32_t));
  }
  P->nsec = nq;
  P->d_sec = dalloc<TcPsiSector>(std::max(nq, 1));
  h2d(P->d_sec, sec.data(), nq * sizeof(TcPsiSector));
  phase(1);   // panels allocated, zeroed and converted
  // ---- stage A tiles: Y^T rows (b, so part of E_R(qout)) x E_L(qin)
  //      columns = sum over si  Rsub(b; si -> so) psi(qin)[:, si part]^T
  std::vector<TcTile> tiles;
  std::vector<TcTerm> terms;
  std::vector<int32_t> term_k;   // unpadded K of every term (byte counts only)
  for (const AGroup& g : groups) {
    const int64_t grows = g.rows;
    for (size_t bi = 0; bi < g.b.size(); ++bi) {
      const int mso = ER.sdim[g.qout[bi]][g.so[bi]];
      for (int si = 0; si < 4; ++si)
        if (g.mem[bi][si] >= 0) {
          P->flops_alg += 2.0 * EL.dim[g.qin] * mso * ER.sdim[g.qin][si];
          P->bytes_alg += (double)P->eb * nh * mso * ER.sdim[g.qin][si];           // Renl sub-block
          P->alg_st[0] += (double)P->eb * nh * mso * ER.sdim[g.qin][si];
        }
    }
    // one term list per group, shared by its tiles; consecutive si whose
    // sections are adjacent in both panels form one term (the same MMAs in
    // the same order, with fewer, fuller boxes)
    const int gt0 = (int)terms.size();
    for (int si = 0; si < 4; ++si)
      if (g.mask >> si & 1) {
        const int w = (int)up16(ER.sdim[g.qin][si]);
        if ((int)terms.size() > gt0) {
          TcTerm& t = terms.back();
          if (t.ax + t.k == g.col[si] && t.bx + t.k == cpadR[g.qin][si]) {
            t.k += w;
            term_k.back() += ER.sdim[g.qin][si];
            continue;
          }
        }
        term_k.push_back(ER.sdim[g.qin][si]);
        terms.push_back({g.col[si], (int32_t)g.row0, (int32_t)psi_row[g.qin], w, 0, cpadR[g.qin][si], 0, 0});
      }
    const int gt1 = (int)terms.size();
    for (int64_t m0 = 0; m0 < grows; m0 += 128)
      for (int n0 = 0; n0 < wlq[g.qin]; n0 += tune.ncap[0]) {
        TcTile T{};
        T.t0 = gt0;
        T.t1 = gt1;
        T.m0 = (int32_t)m0;
        T.m_valid = (int32_t)std::min<int64_t>(128, grows - m0);
        const int nv = std::min(tune.ncap[0], wlq[g.qin] - n0);   // a multiple of 16
        T.n_mma = (int)up16(nv);
        T.n_valid = nv;
        T.bsel = bsel_for(T.n_mma);
        T.mode = kTcYTblk;
        T.beta = 0;
        T.ld = (int32_t)P->yt_pitch;
        T.out = g.row0 + m0;
        T.n0 = n0;
        for (int s = 0; s < 4; ++s) T.rbreak[s] = cpadL[g.qin][s];   // column sections of E_L(qin)
        for (int t = T.t0; t < T.t1; ++t) P->flops_exec += 2.0 * 128 * T.n_mma * terms[t].k;
        tiles.push_back(T);
      }
  }
  // stage A: most expensive tiles first (tc_order_a 0) or the N tiles of each
  // Renl-stack block together (1); stage B: by the keys, in the
  // priority tc_order names (tiles that read the same boxes adjacent, so
  // that they run at the same time on neighbouring SMs and share the boxes
  // through L2)
  std::vector<std::array<int, 5>> bkey;
  auto upload_tiles = [&](int which) {
    P->ntiles[which] = (int)tiles.size();
    // the persistent CTAs stride over the list, so consecutive tiles run together
    std::vector<double> cost(tiles.size());
    std::vector<int> order(tiles.size());
    for (size_t i = 0; i < tiles.size(); ++i) {
      double c = 0;
      for (int t = tiles[i].t0; t < tiles[i].t1; ++t) c += terms[t].k;
      cost[i] = c * tiles[i].n_mma + 4096.0;   // + per-tile fixed cost (epilogue)
      order[i] = (int)i;
    }
    if (which == 1 && bkey.size() == tiles.size()) {
      // bkey holds (q, m0, chunk, 0, n0); the order names the priority
      static const int perm[3][5] = {{0, 1, 2, 3, 4}, {0, 2, 1, 3, 4}, {0, 3, 2, 4, 1}};
      const int* pm = perm[tc_order];
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        for (int i = 0; i < 5; ++i)
          if (bkey[a][pm[i]] != bkey[b][pm[i]]) return bkey[a][pm[i]] < bkey[b][pm[i]];
        return false;
      });
    } else if (which == 0 && tc_order_a == 1) {
      // the N tiles of one 128-row block of the Renl stack (same out row)
      // adjacent, so they run together and read its A boxes from DRAM
      // once; blocks by their summed cost, most expensive first
      std::map<int64_t, double> bcost;
      for (size_t i = 0; i < tiles.size(); ++i) bcost[tiles[i].out] += cost[i];
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const double ca = bcost[tiles[a].out], cb = bcost[tiles[b].out];
        if (ca != cb) return ca > cb;
        if (tiles[a].out != tiles[b].out) return tiles[a].out < tiles[b].out;
        return tiles[a].n0 < tiles[b].n0;
      });
    } else
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    {
      std::vector<TcTile> sorted(tiles.size());
      for (size_t i = 0; i < order.size(); ++i) sorted[i] = tiles[order[i]];
      tiles.swap(sorted);
    }
    {
      const int kstep = 128 / P->eb;
      for (const TcTile& T : tiles)
        for (int t = T.t0; t < T.t1; ++t) {
          const double steps = (double)((terms[t].k + kstep - 1) / kstep) * nh;
          P->box_st[which][0] += steps * 128 * 128;
          P->box_st[which][1] += steps * (16 << T.bsel) * 128;
          P->dense_st[which][0] += (double)T.m_valid * term_k[t] * P->eb * nh;
          P->dense_st[which][1] += (double)T.n_valid * term_k[t] * P->eb * nh;
        }
    }
    P->d_tiles[which] = dalloc<TcTile>(std::max<size_t>(tiles.size(), 1));
    P->d_terms[which] = dalloc<TcTerm>(std::max<size_t>(terms.size(), 1));
    h2d(P->d_tiles[which], tiles.data(), tiles.size() * sizeof(TcTile));
    h2d(P->d_terms[which], terms.data(), terms.size() * sizeof(TcTerm));
    tiles.clear();
    terms.clear();
    term_k.clear();
  };
  phase(2);   // host: stage A tiles
  upload_tiles(0);
  phase(3);   // upload
  // ---- stage B tiles: sigma(q)[E_L(q) rows, E_R(q) tile] = Lenl panel of q
  //      x Y^T(q)^T over K_q: one dense product per output sector, its K
  //      cut into chunks of kc (multiples of W) that are separate terms
  for (const EnlSub& s : lenl.subs)
    if (koff[((size_t)s.b * nq + s.qin) * 4 + s.sin] >= 0) {
      P->flops_alg += 2.0 * ER.dim[s.qout] * s.rows * s.cols;
      P->bytes_alg += (double)P->eb * nh * s.rows * s.cols;                       // Lenl sub-block
      P->alg_st[1] += (double)P->eb * nh * s.rows * s.cols;
    }
  // chunk length: the summed K x columns over all output tiles, shared out
  // over ~4 tiles per SM, within [256, 512] (split types) or [256, 2048].
  // It depends on the sizes only, never on the tuned tile shape, so the
  // tile shape never changes the arithmetic.
  int64_t kc = 0;
  {
    int64_t work = 0;
    for (int q = 0; q < nq; ++q)
      if (EL.dim[q] > 0 && ER.dim[q] > 0) work += (int64_t)((ER.dim[q] + 127) / 128) * Kq[q] * EL.dim[q];
    kc = work / ((int64_t)4 * num_sms * 256);
    kc = (kc + 63) / 64 * 64;
    kc = std::max<int64_t>(256, std::min<int64_t>(nh == 2 ? 512 : 2048, kc));
    P->kc = kc;
  }
  // sections of sigma that no product reaches are written as zeros by the
  // reduction (tasks without slots)
  std::vector<TcRed> zero_red;
  for (int q = 0; q < nq; ++q) {
    if (EL.dim[q] <= 0 || ER.dim[q] <= 0) continue;
    if (!spl[q]) {
      // one product over all of E_L(q) and K_q
      const int N = EL.dim[q];
      const int ot0 = (int)terms.size();
      for (int64_t k0 = 0; k0 < Kq[q]; k0 += kc) {
        const int64_t blk = k0 / W, k = std::min<int64_t>(kc, Kq[q] - k0);
        term_k.push_back((int32_t)k);
        terms.push_back({0, (int32_t)(yrow0[q] + blk * ER.dim[q]), (int32_t)(lrow0[q] + blk * EL.dim[q]), (int32_t)k,
                         0, 0, ER.dim[q], EL.dim[q]});
      }
      const int ot1 = (int)terms.size();
      for (int m0 = 0; m0 < ER.dim[q]; m0 += 128)
        for (int n0 = 0; n0 < N; n0 += tune.ncap[1]) {
          TcTile T{};
          T.t0 = ot0;
          T.t1 = ot1;
          T.n0 = n0;
          T.m0 = m0;
          T.m_valid = std::min(128, ER.dim[q] - m0);
          const int nv = std::min(tune.ncap[1], N - n0);
          T.n_mma = (int)up16(nv);
          T.n_valid = nv;
          T.bsel = bsel_for(T.n_mma);
          T.mode = kTcSigma;
          T.beta = 0;
          T.ld = ER.dim[q];
          T.out = psi_off[q] + (int64_t)n0 * ER.dim[q];
          P->flops_exec += 2.0 * 128 * T.n_mma * (double)Kq[q];
          tiles.push_back(T);
          bkey.push_back({q * 4, m0, 0, 0, n0});   // chunk index filled by the split
        }
      continue;
    }
    for (int so = 0; so < 4; ++so) {
      if (EL.soff[q][so] < 0) continue;
      const int N = EL.sdim[q][so];
      const int64_t out0 = psi_off[q] + (int64_t)EL.soff[q][so] * ER.dim[q];
      if (lrow0s[q][so] < 0) {
        for (int m0 = 0; m0 < ER.dim[q]; m0 += 128)
          zero_red.push_back({out0, 0, 0, ER.dim[q], m0, std::min(128, ER.dim[q] - m0), N, 0, 0});
        continue;
      }
      // one term list per (q, s_out): group s_out, then group 4, in chunks
      // of at most kc starting on K-block boundaries
      const int ot0 = (int)terms.size();
      auto add_range = [&](int64_t kabs, int64_t len, int64_t kpanel) {
        for (int64_t k0 = 0; k0 < len; k0 += kc) {
          const int64_t k = std::min<int64_t>(kc, len - k0);
          const int64_t yblk = (kabs + k0) / W, pblk = (kpanel + k0) / W;
          term_k.push_back((int32_t)k);
          terms.push_back({0, (int32_t)(yrow0[q] + yblk * ER.dim[q]), (int32_t)(lrow0s[q][so] + pblk * N),
                           (int32_t)k, 0, 0, ER.dim[q], N});
        }
      };
      add_range(gk[q][so], glen[q][so], 0);
      add_range(gk[q][4], glen[q][4], upW(glen[q][so]));
      const int ot1 = (int)terms.size();
      double ksum = 0;
      for (int t = ot0; t < ot1; ++t) ksum += terms[t].k;
      for (int m0 = 0; m0 < ER.dim[q]; m0 += 128)
        for (int n0 = 0; n0 < N; n0 += tune.ncap[1]) {
          TcTile T{};
          T.t0 = ot0;
          T.t1 = ot1;
          T.n0 = n0;
          T.m0 = m0;
          T.m_valid = std::min(128, ER.dim[q] - m0);
          const int nv = std::min(tune.ncap[1], N - n0);
          T.n_mma = (int)up16(nv);
          T.n_valid = nv;
          T.bsel = bsel_for(T.n_mma);
          T.mode = kTcSigma;
          T.beta = 0;
          T.ld = ER.dim[q];
          T.out = out0 + (int64_t)n0 * ER.dim[q];
          P->flops_exec += 2.0 * 128 * T.n_mma * ksum;
          tiles.push_back(T);
          // key (q s_out, m0, chunk, -, n0): by default the n tiles of one
          // (q, s_out, m0, chunk) read the same Y^T boxes and run together
          bkey.push_back({q * 4 + so, m0, 0, 0, n0});   // chunk index filled by the split
        }
    }
  }
  // ---- split K: a stage-B tile with more than one chunk becomes one tile
  //      per chunk writing an FP32 partial slot, summed in FP64 by
  //      tc_reduce.  The chunks fill the SMs when sigma has few output
  //      tiles, and they bound the length of every FP32 accumulation in
  //      TMEM (its rounding error grows with that length).
  {
    std::vector<TcTile> split;
    std::vector<std::array<int, 5>> skey;
    std::vector<TcRed> red;
    int64_t slot = 0, red_total = 0;
    for (size_t ti = 0; ti < tiles.size(); ++ti) {
      const TcTile& T = tiles[ti];
      int64_t ktot = 0;
      for (int t = T.t0; t < T.t1; ++t) ktot += terms[t].k;
      if (ktot <= kc) {
        split.push_back(T);
        skey.push_back(bkey[ti]);
        continue;
      }
      TcRed R{T.out, slot, red_total, T.ld, T.m0, T.m_valid, T.n_valid, T.n_mma, 0};
      red_total += (int64_t)T.m_valid * T.n_valid;
      int t = T.t0;
      while (t < T.t1) {
        TcTile Cc = T;
        Cc.t0 = t;
        int64_t k = 0;
        while (t < T.t1 && (t == Cc.t0 || k + terms[t].k <= kc)) k += terms[t++].k;
        Cc.t1 = t;
        Cc.mode = kTcPart;
        Cc.out = slot;
        Cc.ld = 128;
        slot += (int64_t)128 * T.n_mma;
        std::array<int, 5> kk = bkey[ti];
        kk[2] = R.nslot;
        skey.push_back(kk);
        R.nslot++;
        split.push_back(Cc);
      }
      red.push_back(R);
    }
    for (TcRed z : zero_red) {
      z.e0 = red_total;
      red_total += (int64_t)z.m_valid * z.n_valid;
      red.push_back(z);
    }
    tiles.swap(split);
    bkey.swap(skey);
    P->nred = (int)red.size();
    P->red_total = red_total;
    if (!red.empty()) {
      P->part = dalloc<float>((size_t)slot);
      P->d_red = dalloc<TcRed>(red.size());
      h2d(P->d_red, red.data(), red.size() * sizeof(TcRed));
    }
  }
  phase(2);   // host: stage B tiles and split K
  upload_tiles(1);
  phase(3);
  P->bytes_alg += 2.0 * 8.0 * psi_size;                                          // psi in, sigma out
  P->alg_st[0] += 8.0 * psi_size;
  P->alg_st[1] += 8.0 * psi_size;
  // ---- tensor maps
  std::memset(P->maps, 0, sizeof(P->maps));
  for (int h = 0; h < nh; ++h) {
    bool ok = tc_encode_panel(&P->maps[0].a[h], P->eb, P->rs[h], P->rs_pitch, rs_rows, 128) &&
              tc_encode_panel(&P->maps[1].a[h], P->eb, P->yt[h], P->yt_pitch, yrows, 128);
    for (int b = 0; b < 5 && ok; ++b)
      ok = tc_encode_panel(&P->maps[0].b[h][b], P->eb, P->psi[h], P->psi_pitch, psi_rows, 16u << b) &&
           tc_encode_panel(&P->maps[1].b[h][b], P->eb, P->ls[h], P->ls_pitch, ls_rows, 16u << b);
    if (!ok) {
      tc_free(P);
      throw Error(-3, "tensor map encoding failed");
    }
  }
  phase(4);   // tensor maps
  P->d_err = dalloc<int>(1);
  CK(cudaMemsetAsync(P->d_err, 0, sizeof(int), stream));
  return P;
}

// Autotuner of the numerics-neutral tile shape: on the first plan of a
// shape class (precision, size of the two-site state, number of Renl
// sub-blocks), every N cap in {256, 128, 64} is built and its stage A and
// stage B launches are timed separately on the current two-site state (one
// untimed run, then the best of two); each stage keeps its fastest cap.
TcPlan* Engine::tc_plan(const EnlOp& lenl, const EnlOp& renl, int prec) {
  const double t0 = now_ms();
  TcPlan* P = tc_plan_impl(lenl, renl, prec);
  stats.tc_build_ms += now_ms() - t0;
  return P;
}

TcPlan* Engine::tc_plan_impl(const EnlOp& lenl, const EnlOp& renl, int prec) {
  if (tc_fixed_cap) return tc_build(lenl, renl, prec, TcTune{{tc_fixed_cap, tc_fixed_cap}});
  if (!autotune) return tc_build(lenl, renl, prec, TcTune());
  // shape class: operand type, size of the two-site state, number of Renl
  // sub-blocks, and how that size is spread over the sectors (the effective
  // number of sectors (sum_Q w_Q)^2 / sum_Q w_Q^2, w_Q = E_L(Q) E_R(Q)): a
  // state of the same size in a few large sectors tiles differently from one
  // spread over many small ones
  auto lg = [](double x) { return (int64_t)std::lround(2.0 * std::log2(std::max(x, 1.0))); };
  double w1 = 0, w2 = 0;
  for (int q = 0; q < EL.n(); ++q) {
    const double w = (double)EL.dim[q] * ER.dim[q];
    w1 += w;
    w2 += w * w;
  }
  const int64_t ka = lg((double)psi_size), kb = lg((double)renl.subs.size()), ks = lg(w2 > 0 ? w1 * w1 / w2 : 1.0);
  const int64_t key = ((int64_t)prec << 48) | (ka << 32) | (kb << 16) | ks;
  auto it = tuned.find(key);
  if (it != tuned.end()) return tc_build(lenl, renl, prec, it->second);
  // a class within two half-octave buckets of a tuned one in every feature
  // takes its shape (sizes drift from sweep to sweep; tuning again would
  // cost more than it gains)
  for (const auto& kv : tuned) {
    const int64_t p2 = kv.first >> 48, a2 = (kv.first >> 32) & 0xFFFF, b2 = (kv.first >> 16) & 0xFFFF,
                  s2 = kv.first & 0xFFFF;
    if (p2 == prec && std::llabs(a2 - ka) <= 2 && std::llabs(b2 - kb) <= 2 && std::llabs(s2 - ks) <= 2) {
      tuned[key] = kv.second;
      return tc_build(lenl, renl, prec, kv.second);
    }
  }
  cudaEvent_t e[4];
  for (auto& x : e) CK(cudaEventCreate(&x));
  double* y = dalloc<double>(psi_size);
  TcTune best;
  float bt[2] = {1e30f, 1e30f};
  for (int c : {256, 128, 64}) {
    TcPlan* P = tc_build(lenl, renl, prec, TcTune{{c, c}});
    for (int rep = 0; rep < 3; ++rep) {
      launch_tc_convert_psi(psi, P->d_sec, P->nsec, psi_size, P->prec, P->psi[0], P->psi[1], P->psi_pitch, stream);
      TcLaunch A{P->d_tiles[0], P->d_terms[0], P->ntiles[0], P->prec, P->yt[0], P->yt[1], nullptr, P->d_err,
                 nullptr, P->d_yrows, P->d_ymem, c, tc_stages(prec, c)};
      TcLaunch B{P->d_tiles[1], P->d_terms[1], P->ntiles[1], P->prec, nullptr, nullptr, y, P->d_err, P->part,
                 nullptr, nullptr, c, tc_stages(prec, c)};
      CK(cudaEventRecord(e[0], stream));
      bool ok = launch_tc_gemm(P->maps[0], A, num_sms, stream);
      CK(cudaEventRecord(e[1], stream));
      ok = ok && launch_tc_gemm(P->maps[1], B, num_sms, stream);
      launch_tc_reduce(P->d_red, P->nred, P->red_total, P->part, y, stream);
      CK(cudaEventRecord(e[2], stream));
      if (!ok) throw Error(-3, "invalid tensor-core launch configuration");
      CK(cudaEventSynchronize(e[2]));
      float ta = 0, tb = 0;
      CK(cudaEventElapsedTime(&ta, e[0], e[1]));
      CK(cudaEventElapsedTime(&tb, e[1], e[2]));
      if (rep == 0) continue;
      if (ta < bt[0]) { bt[0] = ta; best.ncap[0] = c; }
      if (tb < bt[1]) { bt[1] = tb; best.ncap[1] = c; }
    }
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    sync();
    tc_free(P);
    if (herr) throw Error(-5, "tensor-core pipeline wait timed out");
    stats.autotune_trials++;
  }
  dfree(y);
  for (auto& x : e) cudaEventDestroy(x);
  tuned[key] = best;
  return tc_build(lenl, renl, prec, best);
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
  if (P->part) dfree(P->part);
  if (P->d_yrows) dfree(P->d_yrows);
  if (P->d_ymem) dfree(P->d_ymem);
  if (P->xin) dfree(P->xin);
  if (P->yout) dfree(P->yout);
  Engine::drop(P->graph);
  if (P->d_red) dfree(P->d_red);
  if (P->d_err) dfree(P->d_err);
  delete P;
}

// y = H_eff x with the tensor-core stages (every sub-block's coefficient is
// folded into its converted panel rows, so no term carries a sign) (x, y: FP64 two-site vectors)
void Engine::tc_apply(TcPlan* P, const double* x, double* y) {
  settle();
  CK(cudaEventRecord(ev0, stream));
  auto launches = [&](const double* xi, double* yo) {
    launch_tc_convert_psi(xi, P->d_sec, P->nsec, psi_size, P->prec, P->psi[0], P->psi[1], P->psi_pitch, stream);
    // external event nodes when captured (they time every replay), plain
    // records otherwise
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(stream, &cs));
    const unsigned evf = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
    CK(cudaEventRecordWithFlags(evg0, stream, evf));
    TcLaunch A{P->d_tiles[0], P->d_terms[0], P->ntiles[0], P->prec, P->yt[0], P->yt[1], nullptr, P->d_err,
               nullptr, P->d_yrows, P->d_ymem, P->tune.ncap[0], tc_stages(P->prec, P->tune.ncap[0])};
    TcLaunch B{P->d_tiles[1], P->d_terms[1], P->ntiles[1], P->prec, nullptr, nullptr, yo, P->d_err, P->part,
               nullptr, nullptr, P->tune.ncap[1], tc_stages(P->prec, P->tune.ncap[1])};
    bool ok = launch_tc_gemm(P->maps[0], A, num_sms, stream);
    CK(cudaEventRecordWithFlags(evgm, stream, evf));
    ok = ok && launch_tc_gemm(P->maps[1], B, num_sms, stream);
    if (!ok) throw Error(-3, "invalid tensor-core launch configuration");
    CK(cudaEventRecordWithFlags(evg1, stream, evf));
    launch_tc_reduce(P->d_red, P->nred, P->red_total, P->part, yo, stream);
  };
  if (use_graphs) {
    // the graph reads and writes fixed buffers
    if (!P->xin) {
      P->xin = dalloc<double>(psi_size);
      P->yout = dalloc<double>(psi_size);
    }
    CK(cudaMemcpyAsync(P->xin, x, psi_size * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    replay(P->graph, [&]() { launches(P->xin, P->yout); });
    CK(cudaMemcpyAsync(y, P->yout, psi_size * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  } else {
    launches(x, y);
  }
  CK(cudaEventRecord(ev1, stream));
  CK(cudaMemcpyAsync(tc_err_host, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, stream));
  stats.launches += P->nred ? 4 : 3;
  CK(cudaGetLastError());
  sigma_pending = 2;
  stats.sigma_flops += P->flops_alg;
  stats.sigma_flops_exec += P->flops_exec;
  stats.n_sigma++;
  stats.n_sigma_tc++;
  stats.tc_flops += P->flops_alg;
  stats.tc_bytes += P->bytes_alg;
  for (int s = 0; s < 2; ++s) {
    stats.tc_dense_st[s][0] += P->dense_st[s][0];
    stats.tc_dense_st[s][1] += P->dense_st[s][1];
    stats.tc_alg_st[s] += P->alg_st[s];
    stats.tc_box_st[s][0] += P->box_st[s][0];
    stats.tc_box_st[s][1] += P->box_st[s][1];
  }
  stats.tc_flops_p[P->prec] += P->flops_alg;
  stats.last_tc_prec = P->prec;
}

}  // namespace gbd
