// Excited states by penalty deflation (Sec. "Excited states: dual-penalty
// deflation and NACMEs"): the lower converged states stay resident and are
// projected into every two-site optimisation through overlap environments.
//
// For a stored state |j> with site tensors S_i (its own bonds and sectors)
// and the current MPS (left-canonical A_i left of the two sites,
// right-canonical B_i right of them):
//   OL_j[k](q)   = <left basis of bond k, sector q | left part of |j>>
//                = sum_s A_{k-1}(q)[s]^T OL_j[k-1](q - s) S_{k-1}(q)[s]
//   OR_j[k](q)   = sum_s B_k(q)[s] OR_j[k+1](q + s) S_k(q)[s]^T
//   phi_j(Q)     = [OL_j[k] S_k](Q) . [S_{k+1} OR_j[k+2]^T](Q)
// in the two-site layout of sector Q (rows E_L(Q), columns E_R(Q)), so that
// phi_j = the projection of |j> onto the current two-site space, whatever
// the gauge of the stored MPS.  The two-site problem becomes
//   (H_eff + w sum_j phi_j phi_j^T) x = theta x,
// and its diagonal H_eff,ii + w sum_j phi_j,i^2 (the deflation-aware
// diagonal of the preconditioner family).  Every contraction is a grouped
// FP64 GEMM checked against its allocations before launch.
//
// The paper's dual penalty lambda S_z^2 + mu (N - N_el)^2 (Eq. dualpen) is
// zero inside the (N_alpha, N_beta) sector this solver is blocked by, so it
// has no counterpart here.
#include <algorithm>
#include <cmath>

#include "engine.h"

namespace gbd {

void Engine::free_ov(Ov& o) {
  if (o.d) dfree(o.d);
  o = Ov();
}

void Engine::clear_states() {
  for (auto& v : OLv)
    for (auto& o : v) free_ov(o);
  for (auto& v : ORv)
    for (auto& o : v) free_ov(o);
  OLv.clear();
  ORv.clear();
  for (auto& st : defl) {
    for (auto& s : st.fl) free_site(s);
    for (auto& s : st.fr) free_site(s);
  }
  defl.clear();
}

// zeroed blocks (current sector x stored sector) for the sectors of the
// current bond that the stored state also has
void Engine::ov_make(int j, int bond, Ov& o) {
  free_ov(o);
  const Bond& bc = bonds[bond];
  const Bond& bs = defl[j].bonds[bond];
  o.off.assign(bc.nsec(), -1);
  o.rows.assign(bc.nsec(), 0);
  o.cols.assign(bc.nsec(), 0);
  int64_t tot = 0;
  for (int i = 0; i < bc.nsec(); ++i) {
    const int js = bs.find(bc.na[i], bc.nb[i]);
    if (js < 0) continue;
    o.off[i] = tot;
    o.rows[i] = bc.dim[i];
    o.cols[i] = bs.dim[js];
    tot += (int64_t)bc.dim[i] * bs.dim[js];
  }
  o.size = tot;
  const int64_t alloc = std::max<int64_t>(tot, 1);
  o.d = dalloc<double>(alloc);
  CK(cudaMemsetAsync(o.d, 0, alloc * sizeof(double), stream));
}

// the current MPS, every site in both layouts (a copy through the host; once
// per stored state)
void Engine::store_state() {
  Stored st;
  st.bonds = bonds;
  st.fl.resize(n);
  st.fr.resize(n);
  for (int i = 0; i < n; ++i) {
    const Site& S = sites[i];
    Site L0, L1;
    layout_site(i, 0, L0);
    layout_site(i, 1, L1);
    if (S.size != (S.layout == 0 ? L0.size : L1.size)) throw Error(-6, "stored state: site size mismatch");
    std::vector<double> h(std::max<int64_t>(S.size, 1));
    CK(cudaMemcpyAsync(h.data(), S.d, S.size * sizeof(double), cudaMemcpyDeviceToHost, stream));
    sync();
    std::vector<double> fl(std::max<int64_t>(L0.size, 1), 0.0), fr(std::max<int64_t>(L1.size, 1), 0.0);
    const Bond& bl = bonds[i];
    const Bond& br = bonds[i + 1];
    const Space lsp = left_space(bl, bond_qs(br));    // fused-left row sections, by sector of bond i+1
    const Space rsp = right_space(br, bond_qs(bl));   // fused-right column sections, by sector of bond i
    // element ((s, a), c) of block Q (fused-left) = element (a, (s, c)) of block q = Q - s (fused-right)
    for (int jr = 0; jr < br.nsec(); ++jr)
      for (int s = 0; s < 4; ++s) {
        if (lsp.soff[jr][s] < 0) continue;
        const int jl = lsp.ssec[jr][s];
        const int ml = bl.dim[jl], mr = br.dim[jr];
        const int rso = rsp.soff[jl][s];
        if (rso < 0) throw Error(-6, "stored state: inconsistent site sections");
        for (int a = 0; a < ml; ++a)
          for (int c = 0; c < mr; ++c) {
            const int64_t ifl = L0.off[jr] + (int64_t)(lsp.soff[jr][s] + a) * mr + c;
            const int64_t ifr = L1.off[jl] + (int64_t)a * rsp.dim[jl] + rso + c;
            if (S.layout == 0) fr[ifr] = h[ifl];
            else fl[ifl] = h[ifr];
          }
      }
    if (S.layout == 0) std::copy(h.begin(), h.begin() + S.size, fl.begin());
    else std::copy(h.begin(), h.begin() + S.size, fr.begin());
    st.fl[i] = L0;
    st.fr[i] = L1;
    st.fl[i].d = dalloc<double>(std::max<int64_t>(L0.size, 1));
    st.fr[i].d = dalloc<double>(std::max<int64_t>(L1.size, 1));
    CK(cudaMemcpyAsync(st.fl[i].d, fl.data(), L0.size * sizeof(double), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(st.fr[i].d, fr.data(), L1.size * sizeof(double), cudaMemcpyHostToDevice, stream));
    sync();
  }
  defl.push_back(std::move(st));
}

// OL at bond 0 and OR at bond n are the 1 x 1 identity; OR at bonds n-1 .. 2
// from the right-canonical sites of the freshly initialised MPS
void Engine::ov_init() {
  const int nj = (int)defl.size();
  for (auto& v : OLv)
    for (auto& o : v) free_ov(o);
  for (auto& v : ORv)
    for (auto& o : v) free_ov(o);
  OLv.assign(nj, std::vector<Ov>(n + 1));
  ORv.assign(nj, std::vector<Ov>(n + 1));
  const double one = 1.0;
  for (int j = 0; j < nj; ++j) {
    ov_make(j, 0, OLv[j][0]);
    ov_make(j, n, ORv[j][n]);
    if (OLv[j][0].size != 1 || ORv[j][n].size != 1) throw Error(-6, "stored state: boundary bonds differ");
    CK(cudaMemcpyAsync(OLv[j][0].d, &one, sizeof(double), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(ORv[j][n].d, &one, sizeof(double), cudaMemcpyHostToDevice, stream));
    sync();
    for (int b = n - 1; b >= 2; --b) ov_update_right(j, b);
  }
}

void Engine::ov_update_left(int j, int k) {
  const Stored& st = defl[j];
  const Site& A = sites[k];
  if (A.layout != 0) throw Error(-6, "overlap update: site is not fused-left");
  const Bond& bc0 = bonds[k];
  const Bond& bc1 = bonds[k + 1];
  const Bond& bs0 = st.bonds[k];
  const Bond& bs1 = st.bonds[k + 1];
  const Ov& in = OLv[j][k];
  Ov& out = OLv[j][k + 1];
  ov_make(j, k + 1, out);
  const Space lsc = left_space(bc0, bond_qs(bc1));
  const Space lss = left_space(bs0, bond_qs(bs1));
  const Site& S = st.fl[k];
  struct TB { int i1, s, i0; int64_t off; };
  std::vector<TB> tbs;
  int64_t tsize = 0;
  for (int i1 = 0; i1 < bc1.nsec(); ++i1) {
    if (out.off[i1] < 0) continue;
    const int j1 = bs1.find(bc1.na[i1], bc1.nb[i1]);
    for (int s = 0; s < 4; ++s) {
      if (lsc.soff[i1][s] < 0 || lss.soff[j1][s] < 0) continue;
      const int i0 = lsc.ssec[i1][s];
      if (in.off[i0] < 0) continue;
      tbs.push_back({i1, s, i0, tsize});
      tsize += (int64_t)bc0.dim[i0] * bs1.dim[j1];
    }
  }
  double* T = dalloc<double>(std::max<int64_t>(tsize, 1));
  GemmPlan p1, p2;
  // T(i1, s) = OL[k](q) S_k(Q)[s]   (m_cur(q) x m_j(Q))
  for (const TB& t : tbs) {
    const int j1 = bs1.find(bc1.na[t.i1], bc1.nb[t.i1]);
    const int mj1 = bs1.dim[j1];
    p1.add_out(T + t.off, mj1, bc0.dim[t.i0], mj1, 0);
    p1.add_term(in.d + in.off[t.i0], in.cols[t.i0], S.d + S.off[j1] + (int64_t)lss.soff[j1][t.s] * mj1, mj1,
                in.cols[t.i0], 0, 1.0);
  }
  // OL[k+1](Q) = sum_s A_k(Q)[s]^T T(Q, s)
  for (int i1 = 0; i1 < bc1.nsec(); ++i1) {
    if (out.off[i1] < 0) continue;
    const int mj1 = out.cols[i1], mc1 = bc1.dim[i1];
    p2.add_out(out.d + out.off[i1], mj1, mc1, mj1, 0);
    for (const TB& t : tbs)
      if (t.i1 == i1)
        p2.add_term(A.d + A.off[i1] + (int64_t)lsc.soff[i1][t.s] * mc1, mc1, T + t.off, mj1, bc0.dim[t.i0], 1,
                    1.0);
  }
  upload(p1);
  upload(p2);
  run(p1);
  run(p2);
  sync();
  release(p1);
  release(p2);
  dfree(T);
}

void Engine::ov_update_right(int j, int b) {
  const Stored& st = defl[j];
  const Site& B = sites[b];
  if (B.layout != 1) throw Error(-6, "overlap update: site is not fused-right");
  const Bond& bc0 = bonds[b];
  const Bond& bc1 = bonds[b + 1];
  const Bond& bs0 = st.bonds[b];
  const Bond& bs1 = st.bonds[b + 1];
  const Ov& in = ORv[j][b + 1];
  Ov& out = ORv[j][b];
  ov_make(j, b, out);
  const Space rsc = right_space(bc1, bond_qs(bc0));
  const Space rss = right_space(bs1, bond_qs(bs0));
  const Site& S = st.fr[b];
  struct TB { int i0, s, i1; int64_t off; };
  std::vector<TB> tbs;
  int64_t tsize = 0;
  for (int i0 = 0; i0 < bc0.nsec(); ++i0) {
    if (out.off[i0] < 0) continue;
    const int j0 = bs0.find(bc0.na[i0], bc0.nb[i0]);
    for (int s = 0; s < 4; ++s) {
      if (rsc.soff[i0][s] < 0 || rss.soff[j0][s] < 0) continue;
      const int i1 = rsc.ssec[i0][s];
      if (in.off[i1] < 0) continue;
      tbs.push_back({i0, s, i1, tsize});
      tsize += (int64_t)bc1.dim[i1] * bs0.dim[j0];
    }
  }
  double* T = dalloc<double>(std::max<int64_t>(tsize, 1));
  GemmPlan p1, p2;
  // T(i0, s) = OR[b+1](q + s) S_b(q)[s]^T   (m_cur(q + s) x m_j(q))
  for (const TB& t : tbs) {
    const int j0 = bs0.find(bc0.na[t.i0], bc0.nb[t.i0]);
    const int mj0 = bs0.dim[j0];
    p1.add_out(T + t.off, mj0, bc1.dim[t.i1], mj0, 0);
    p1.add_term(in.d + in.off[t.i1], in.cols[t.i1], S.d + S.off[j0] + rss.soff[j0][t.s], rss.dim[j0],
                in.cols[t.i1], 2, 1.0);
  }
  // OR[b](q) = sum_s B_b(q)[s] T(q, s)
  for (int i0 = 0; i0 < bc0.nsec(); ++i0) {
    if (out.off[i0] < 0) continue;
    const int mj0 = out.cols[i0];
    p2.add_out(out.d + out.off[i0], mj0, bc0.dim[i0], mj0, 0);
    for (const TB& t : tbs)
      if (t.i0 == i0)
        p2.add_term(B.d + B.off[i0] + rsc.soff[i0][t.s], rsc.dim[i0], T + t.off, mj0, bc1.dim[t.i1], 0, 1.0);
  }
  upload(p1);
  upload(p2);
  run(p1);
  run(p2);
  sync();
  release(p1);
  release(p2);
  dfree(T);
}

// phi_j for every stored state at the two sites (k, k+1), into phi
// (n_stored x psi_size, zero where a state has no weight)
void Engine::deflation_vectors(int k, double* phi) {
  const int nj = (int)defl.size();
  CK(cudaMemsetAsync(phi, 0, (size_t)nj * psi_size * sizeof(double), stream));
  for (int j = 0; j < nj; ++j) {
    const Stored& st = defl[j];
    const Bond& bs0 = st.bonds[k];
    const Bond& bs1 = st.bonds[k + 1];
    const Bond& bs2 = st.bonds[k + 2];
    const Ov& OL = OLv[j][k];
    const Ov& OR = ORv[j][k + 2];
    const Space lss = left_space(bs0, bond_qs(bs1));
    const Space rss = right_space(bs2, bond_qs(bs1));
    const Site& SL = st.fl[k];
    const Site& SR = st.fr[k + 1];
    std::vector<int64_t> t1off(EL.n(), -1), t2off(EL.n(), -1);
    int64_t t1size = 0, t2size = 0;
    for (int iq = 0; iq < EL.n(); ++iq) {
      const int jQ = bs1.find(EL.qa[iq], EL.qb[iq]);
      if (jQ < 0) continue;
      t1off[iq] = t1size;
      t2off[iq] = t2size;
      t1size += (int64_t)EL.dim[iq] * bs1.dim[jQ];
      t2size += (int64_t)bs1.dim[jQ] * ER.dim[iq];
    }
    double* T1 = dalloc<double>(std::max<int64_t>(t1size, 1));
    double* T2 = dalloc<double>(std::max<int64_t>(t2size, 1));
    CK(cudaMemsetAsync(T1, 0, std::max<int64_t>(t1size, 1) * sizeof(double), stream));
    CK(cudaMemsetAsync(T2, 0, std::max<int64_t>(t2size, 1) * sizeof(double), stream));
    GemmPlan p1, p2, p3;
    double* out = phi + (int64_t)j * psi_size;
    for (int iq = 0; iq < EL.n(); ++iq) {
      if (t1off[iq] < 0) continue;
      const int jQ = bs1.find(EL.qa[iq], EL.qb[iq]);
      const int mQ = bs1.dim[jQ];
      // T1(Q), rows E_L(Q): section s1 = OL[k](q_l) S_k(Q)[s1]
      for (int s1 = 0; s1 < 4; ++s1) {
        if (EL.soff[iq][s1] < 0 || lss.soff[jQ][s1] < 0) continue;
        const int i0 = EL.ssec[iq][s1];
        if (OL.off[i0] < 0) continue;
        p1.add_out(T1 + t1off[iq] + (int64_t)EL.soff[iq][s1] * mQ, mQ, EL.sdim[iq][s1], mQ, 0);
        p1.add_term(OL.d + OL.off[i0], OL.cols[i0], SL.d + SL.off[jQ] + (int64_t)lss.soff[jQ][s1] * mQ, mQ,
                    OL.cols[i0], 0, 1.0);
      }
      // T2(Q), columns E_R(Q): section s2 = S_{k+1}(Q)[s2] OR[k+2](q_r)^T
      for (int s2 = 0; s2 < 4; ++s2) {
        if (ER.soff[iq][s2] < 0 || rss.soff[jQ][s2] < 0) continue;
        const int i2 = ER.ssec[iq][s2];
        if (OR.off[i2] < 0) continue;
        p2.add_out(T2 + t2off[iq] + ER.soff[iq][s2], ER.dim[iq], mQ, ER.sdim[iq][s2], 0);
        p2.add_term(SR.d + SR.off[jQ] + rss.soff[jQ][s2], rss.dim[jQ], OR.d + OR.off[i2], OR.cols[i2],
                    OR.cols[i2], 2, 1.0);
      }
      // phi(Q) = T1(Q) T2(Q)
      p3.add_out(out + psi_off[iq], ER.dim[iq], EL.dim[iq], ER.dim[iq], 0);
      p3.add_term(T1 + t1off[iq], mQ, T2 + t2off[iq], ER.dim[iq], mQ, 0, 1.0);
    }
    upload(p1);
    upload(p2);
    upload(p3);
    run(p1);
    run(p2);
    run(p3);
    sync();
    release(p1);
    release(p2);
    release(p3);
    dfree(T1);
    dfree(T2);
  }
}

}  // namespace gbd
