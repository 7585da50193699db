// One- and two-particle RDMs contracted through the MPS itself (paper:
// device k-RDMs of the converged MPS, Sec. "The DMRG-QD-NEVPT2 energy"),
//   gamma_pq = sum_s <a+_ps a_qs>,  Gamma_pqrs = sum_st <a+_ps a+_rt a_st a_qs>,
// at a cost polynomial in n and M (no determinant expansion).
//
// Jordan-Wigner form.  With the modes ordered 0a, 0b, 1a, 1b, ... every
// ladder operator is a tensor product of 4 x 4 site matrices: the parity P
// on the sites before its own, its local ladder matrix on its own site (a
// beta operator carrying the parity of its site's alpha mode), I after.  A
// product of ladder operators is then a tensor product whose matrix on site
// x is the ordered product of what each factor puts there.  Cut at bond b,
//   <psi| O_left (x) O_right |psi> = sum_q sum_ij L_b[O_left](q'<-q)_ij R_b[O_right](q'<-q)_ij
// for an MPS in any gauge, L_b and R_b contracting bra and ket over the
// sites before and after the bond.
//
// Each element is cut after the site of its second operator in site order
// (after the first when the last three share one site), so that its left
// part has at most one operator before the cut site and its right part
// operators on at most two sites.  Every site matrix of a part is scaled to
// a canonical sign (first nonzero entry +1); the tuple of canonical
// matrices names an environment channel and the product of the scales
// stays with the element.  A channel has one parent (its tuple without the
// site next to the neighbouring bond) and one site matrix Y:
//   L_{x+1}[c] = sum_{s',s} Y[s',s] X_{s'}^T L_x[parent] X_s,
//   R_x[c]     = sum_{s',s} Y[s',s] X_{s'} R_{x+1}[parent] X_s^T,
// X_s(q, r) the site tensor's block of local state s: two grouped FP64 GEMM
// launches per site (parent blocks times X_s, then the X_{s'} products).
// The channels that elements use at a bond are stored grouped by their
// quantum-number shift and by sector, so all their Frobenius products at
// that bond are one split-K GEMM per shift class.  FP64 throughout.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <unordered_map>

#include "engine.h"

namespace gbd {

namespace opstr {

using Mat4 = std::array<int, 16>;   // <s'|op|s> at [s' * 4 + s]; local states 0, a, b, ab

Mat4 mat_ident() {
  Mat4 m{};
  for (int i = 0; i < 4; ++i) m[i * 5] = 1;
  return m;
}
Mat4 mat_parity() {
  Mat4 m{};
  m[0] = 1;
  m[5] = -1;
  m[10] = -1;
  m[15] = 1;
  return m;
}
// t = 0: a+_alpha, 1: a+_beta, 2: a_alpha, 3: a_beta; |ab> = a+_a a+_b |0>,
// so a_beta |ab> = -|a>
Mat4 mat_ladder(int t) {
  Mat4 a{};
  if (t == 0 || t == 2) {
    a[0 * 4 + 1] = 1;    // |a>  -> |0>
    a[2 * 4 + 3] = 1;    // |ab> -> |b>
  } else {
    a[0 * 4 + 2] = 1;    // |b>  -> |0>
    a[1 * 4 + 3] = -1;   // |ab> -> -|a>
  }
  if (t >= 2) return a;
  Mat4 c{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) c[i * 4 + j] = a[j * 4 + i];
  return c;
}
Mat4 mat_mul(const Mat4& x, const Mat4& y) {
  Mat4 z{};
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 4; ++k) {
      if (!x[i * 4 + k]) continue;
      for (int j = 0; j < 4; ++j) z[i * 4 + j] += x[i * 4 + k] * y[k * 4 + j];
    }
  return z;
}
// scale to the first nonzero entry +1; returns the scale (0: zero matrix)
int canon(Mat4& m) {
  for (int i = 0; i < 16; ++i)
    if (m[i]) {
      const int lam = m[i];
      if (lam != 1 && lam != -1) throw Error(-6, "RDM: site matrix entry outside {-1, 0, 1}");
      if (lam < 0)
        for (auto& v : m) v = -v;
      return lam;
    }
  return 0;
}
int32_t mkey(const Mat4& m) {
  int32_t k = 0;
  for (int i = 0; i < 16; ++i) k = k * 3 + (m[i] + 1);
  return k;
}
Mat4 unkey(int32_t k) {
  Mat4 m{};
  for (int i = 15; i >= 0; --i) {
    m[i] = k % 3 - 1;
    k /= 3;
  }
  return m;
}
// particle shift (alpha, beta) of a nonzero site matrix that maps local
// states to local states of one fixed shift
std::pair<int, int> mshift(const Mat4& m) {
  for (int so = 0; so < 4; ++so)
    for (int si = 0; si < 4; ++si)
      if (m[so * 4 + si]) return {QA[so] - QA[si], QB[so] - QB[si]};
  return {0, 0};
}
// the row s' of the nonzero entry in column s (-1 if none); ladder products
// are signed partial permutations, so there is at most one
int col_row(const Mat4& m, int s) {
  for (int so = 0; so < 4; ++so)
    if (m[so * 4 + s]) return so;
  return -1;
}

struct Chan {
  int parent = -1;      // channel at the neighbouring bond (left: b - 1, right: b + 1)
  int32_t y = 0;        // key of the site matrix between the two bonds
  int da = 0, db = 0;   // block (q' <- q): q' = q + (da, db) in bond (left-block) labels
  int cls = -1, row = -1;   // product class at this bond and row inside it
};
struct Side {
  std::vector<Chan> ch;
  std::unordered_map<std::string, int> idx;
};

int reg_left(std::vector<Side>& L, const int32_t* keys, int b) {
  std::string k((const char*)keys, sizeof(int32_t) * (size_t)b);
  auto it = L[b].idx.find(k);
  if (it != L[b].idx.end()) return it->second;
  Chan c;
  if (b > 0) {
    c.parent = reg_left(L, keys, b - 1);
    c.y = keys[b - 1];
    const Chan& p = L[b - 1].ch[c.parent];
    const auto d = mshift(unkey(c.y));
    c.da = p.da + d.first;
    c.db = p.db + d.second;
  }
  const int id = (int)L[b].ch.size();
  L[b].ch.push_back(c);
  L[b].idx.emplace(std::move(k), id);
  return id;
}

int reg_right(std::vector<Side>& R, const int32_t* keys, int b, int n) {
  std::string k((const char*)(keys + b), sizeof(int32_t) * (size_t)(n - b));
  auto it = R[b].idx.find(k);
  if (it != R[b].idx.end()) return it->second;
  Chan c;
  if (b < n) {
    c.parent = reg_right(R, keys, b + 1, n);
    c.y = keys[b];
    const Chan& p = R[b + 1].ch[c.parent];
    const auto d = mshift(unkey(c.y));
    c.da = p.da - d.first;
    c.db = p.db - d.second;
  }
  const int id = (int)R[b].ch.size();
  R[b].ch.push_back(c);
  R[b].idx.emplace(std::move(k), id);
  return id;
}

struct Elem {
  int bond, lc, rc;
  double lam;
  int64_t out;   // < n^2: gamma index; else n^2 + Gamma index; -1: the norm
};

// shift classes of one bond: rows on each side and the split-K layout of G
struct BondProd {
  std::map<std::pair<int, int>, int> cls_of;
  std::vector<std::pair<int, int>> shift;
  std::vector<std::vector<int>> lrows, rrows;   // channels in row order
  std::vector<int64_t> gbase;                   // first partial of the class in G
  std::vector<int> nsplit;
};

// environment blocks of one bond: off[ch * nsec + q] (-1: absent)
struct CEnv {
  int nsec = 0;
  std::vector<int64_t> off;
  double* d = nullptr;
  int64_t size = 0;
  int64_t at(int ch, int q) const { return off[(size_t)ch * nsec + q]; }
};


// one operator product per element; see the file comment for the cut
struct StringSet {
  int n;
  std::vector<Side> Ls, Rs;
  std::vector<Elem> elems;
  std::vector<BondProd> prod;
  Mat4 I4, P4;
  int32_t keyI, keyP;
  std::vector<int32_t> keys;
  // elems[0] is the norm <psi|psi> (no factor, cut at bond 1)
  explicit StringSet(int n_) : n(n_), Ls(n_ + 1), Rs(n_ + 1), prod(n_ + 1), keys(n_) {
    I4 = mat_ident();
    P4 = mat_parity();
    keyI = mkey(I4);
    keyP = mkey(P4);
    add(nullptr, nullptr, nullptr, 0, -1);
  }
  // factors in product order: site, site matrix, odd (a fermionic factor,
  // parity P on every site before its own); out tags the element.  False
  // when the product vanishes identically.
  bool add(const int* pos, const Mat4* mats, const char* odd, int nops, int64_t out) {
    // distinct sites and the cut k (the left part holds sites <= k)
    int site[16], mult[16], nd = 0;
    for (int i = 0; i < nops; ++i) {
      int j = 0;
      while (j < nd && site[j] != pos[i]) ++j;
      if (j == nd) {
        site[nd] = pos[i];
        mult[nd++] = 0;
      }
      mult[j]++;
    }
    for (int a = 0; a < nd; ++a)
      for (int b = a + 1; b < nd; ++b)
        if (site[b] < site[a]) {
          std::swap(site[a], site[b]);
          std::swap(mult[a], mult[b]);
        }
    int k = 0;
    if (nd == 1 || nd == 2) k = site[0];
    else if (nd == 3) k = mult[0] >= 2 ? site[0] : site[1];
    else if (nd == 4) k = site[1];
    else if (nd > 4) throw Error(-6, "operator string on more than four sites");
    double lam = 1.0;
    for (int x = 0; x < n; ++x) {
      int after = 0, here = 0;
      for (int i = 0; i < nops; ++i) {
        after += odd[i] && pos[i] > x;
        here += pos[i] == x;
      }
      if (!here) {
        keys[x] = (after & 1) ? keyP : keyI;
        continue;
      }
      Mat4 m = I4;
      for (int i = 0; i < nops; ++i) {
        if (x < pos[i]) {
          if (odd[i]) m = mat_mul(m, P4);
        } else if (x == pos[i]) {
          m = mat_mul(m, mats[i]);
        }
      }
      const int sgn = canon(m);
      if (sgn == 0) return false;
      lam *= sgn;
      keys[x] = mkey(m);
    }
    const int b = k + 1;
    const int lc = reg_left(Ls, keys.data(), b);
    const int rc = reg_right(Rs, keys.data(), b, n);
    const Chan& L = Ls[b].ch[lc];
    const Chan& R = Rs[b].ch[rc];
    if (L.da != R.da || L.db != R.db) throw Error(-6, "operator string does not conserve the particle numbers");
    elems.push_back({b, lc, rc, lam, out});
    return true;
  }
};

}  // namespace opstr

using namespace opstr;

// Values <psi|O|psi> / <psi|psi> of the registered strings, in the order of
// S.elems (elems[0], the norm itself, gives 1).
std::vector<double> Engine::eval_strings(StringSet& S) {
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<Side>& Ls = S.Ls;
  std::vector<Side>& Rs = S.Rs;
  std::vector<BondProd>& prod = S.prod;
  // product classes and rows
  for (const Elem& e : S.elems) {
    BondProd& P = prod[e.bond];
    Chan& L = Ls[e.bond].ch[e.lc];
    Chan& R = Rs[e.bond].ch[e.rc];
    auto key = std::make_pair(L.da, L.db);
    auto it = P.cls_of.find(key);
    int c;
    if (it == P.cls_of.end()) {
      c = (int)P.shift.size();
      P.cls_of[key] = c;
      P.shift.push_back(key);
      P.lrows.emplace_back();
      P.rrows.emplace_back();
    } else {
      c = it->second;
    }
    if (L.row < 0) {
      L.cls = c;
      L.row = (int)P.lrows[c].size();
      P.lrows[c].push_back(e.lc);
    }
    if (R.row < 0) {
      R.cls = c;
      R.row = (int)P.rrows[c].size();
      P.rrows[c].push_back(e.rc);
    }
  }
  // split-K layout of the products: the output tiles of all classes of a
  // bond share one launch; K is split until that launch has about four
  // 32 x 32 tiles per SM, each split keeping at least 2048 of K
  int64_t gsize = 0;
  for (int b = 1; b <= n; ++b) {
    BondProd& P = prod[b];
    const Bond& bd = bonds[b];
    std::vector<int64_t> ksum(P.shift.size(), 0), tiles(P.shift.size(), 0);
    int64_t tiles_all = 0;
    for (size_t c = 0; c < P.shift.size(); ++c) {
      for (int q = 0; q < bd.nsec(); ++q) {
        const int qo = bd.find(bd.na[q] + P.shift[c].first, bd.nb[q] + P.shift[c].second);
        if (qo >= 0) ksum[c] += (int64_t)bd.dim[qo] * bd.dim[q];
      }
      tiles[c] = (int64_t)((P.lrows[c].size() + 31) / 32) * ((P.rrows[c].size() + 31) / 32);
      tiles_all += tiles[c];
    }
    const int64_t want = (4 * (int64_t)num_sms + std::max<int64_t>(tiles_all, 1) - 1) / std::max<int64_t>(tiles_all, 1);
    for (size_t c = 0; c < P.shift.size(); ++c) {
      const int ns = (int)std::max<int64_t>(1, std::min<int64_t>({64, ksum[c] / 2048, want}));
      P.gbase.push_back(gsize);
      P.nsplit.push_back(ns);
      gsize += (int64_t)ns * P.lrows[c].size() * P.rrows[c].size();
    }
  }

  // ---- environments
  int64_t live = 0, peak = 0;
  auto alloc_env = [&](int b, const Side& S, bool left, CEnv& E) {
    const Bond& bd = bonds[b];
    const BondProd& P = prod[b];
    E.nsec = bd.nsec();
    E.off.assign(S.ch.size() * (size_t)E.nsec, -1);
    int64_t tot = 0;
    if (b >= 1)
      for (size_t c = 0; c < P.shift.size(); ++c) {
        const auto& rows = left ? P.lrows[c] : P.rrows[c];
        for (int q = 0; q < E.nsec; ++q) {
          const int qo = bd.find(bd.na[q] + P.shift[c].first, bd.nb[q] + P.shift[c].second);
          if (qo < 0) continue;
          const int64_t blk = (int64_t)bd.dim[qo] * bd.dim[q];
          for (size_t r = 0; r < rows.size(); ++r) E.off[(size_t)rows[r] * E.nsec + q] = tot + (int64_t)r * blk;
          tot += (int64_t)rows.size() * blk;
        }
      }
    for (size_t ch = 0; ch < S.ch.size(); ++ch) {
      if (S.ch[ch].row >= 0 && b >= 1) continue;
      for (int q = 0; q < E.nsec; ++q) {
        const int qo = bd.find(bd.na[q] + S.ch[ch].da, bd.nb[q] + S.ch[ch].db);
        if (qo < 0) continue;
        E.off[ch * (size_t)E.nsec + q] = tot;
        tot += (int64_t)bd.dim[qo] * bd.dim[q];
      }
    }
    E.size = tot;
    E.d = dalloc<double>(tot);
    CK(cudaMemsetAsync(E.d, 0, std::max<int64_t>(tot, 1) * sizeof(double), stream));
    live += tot * (int64_t)sizeof(double);
    peak = std::max(peak, live);
  };
  auto free_cenv = [&](CEnv& E) {
    if (E.d) dfree(E.d);
    live -= E.size * (int64_t)sizeof(double);
    E.d = nullptr;
    E.size = 0;
  };
  auto seed = [&](CEnv& E) {   // the one 1 x 1 block of a boundary bond
    static const double one = 1.0;
    for (int64_t o : E.off)
      if (o >= 0) h2d(E.d + o, &one, sizeof(double));
  };
  // L_{x+1} from L_x through site x
  auto left_step = [&](int x, const CEnv& Ep, CEnv& Ec) {
    const Bond& bl = bonds[x];
    const Bond& br = bonds[x + 1];
    const Side& Sp = Ls[x];
    const Side& Sc = Ls[x + 1];
    const int ns = bl.nsec();
    std::vector<std::array<char, 4>> need(Sp.ch.size(), std::array<char, 4>{0, 0, 0, 0});
    std::vector<Mat4> Y(Sc.ch.size());
    for (size_t c = 0; c < Sc.ch.size(); ++c) {
      Y[c] = unkey(Sc.ch[c].y);
      for (int s = 0; s < 4; ++s)
        if (col_row(Y[c], s) >= 0) need[Sc.ch[c].parent][s] = 1;
    }
    // T[p, s, q] = L_x[p](q' <- q) X_s(q, r): m_q' x m_r
    std::vector<int64_t> toff(Sp.ch.size() * 4 * (size_t)ns, -1);
    int64_t tsz = 0;
    for (size_t p = 0; p < Sp.ch.size(); ++p)
      for (int s = 0; s < 4; ++s) {
        if (!need[p][s]) continue;
        for (int q = 0; q < ns; ++q) {
          if (Ep.at((int)p, q) < 0) continue;
          const int r = br.find(bl.na[q] + QA[s], bl.nb[q] + QB[s]);
          if (r < 0) continue;
          const int qo = bl.find(bl.na[q] + Sp.ch[p].da, bl.nb[q] + Sp.ch[p].db);
          toff[(p * 4 + s) * ns + q] = tsz;
          tsz += (int64_t)bl.dim[qo] * br.dim[r];
        }
      }
    double* T = dalloc<double>(tsz);
    live += tsz * (int64_t)sizeof(double);
    peak = std::max(peak, live);
    GemmPlan g1, g2;
    for (size_t p = 0; p < Sp.ch.size(); ++p)
      for (int s = 0; s < 4; ++s)
        for (int q = 0; q < ns; ++q) {
          const int64_t to = toff[(p * 4 + s) * ns + q];
          if (to < 0) continue;
          const int r = br.find(bl.na[q] + QA[s], bl.nb[q] + QB[s]);
          const int qo = bl.find(bl.na[q] + Sp.ch[p].da, bl.nb[q] + Sp.ch[p].db);
          int ld = 0;
          const double* X = site_block(x, q, s, ld);
          g1.add_out(T + to, br.dim[r], bl.dim[qo], br.dim[r], 0);
          g1.add_term(Ep.d + Ep.at((int)p, q), bl.dim[q], X, ld, bl.dim[q], 0, 1.0);
        }
    for (size_t c = 0; c < Sc.ch.size(); ++c) {
      const Chan& C = Sc.ch[c];
      const Chan& Pc = Sp.ch[C.parent];
      for (int r = 0; r < br.nsec(); ++r) {
        const int64_t eo = Ec.at((int)c, r);
        if (eo < 0) continue;
        const int ro = br.find(br.na[r] + C.da, br.nb[r] + C.db);
        g2.add_out(Ec.d + eo, br.dim[r], br.dim[ro], br.dim[r], 0);
        for (int s = 0; s < 4; ++s) {
          const int so = col_row(Y[c], s);
          if (so < 0) continue;
          const int q = bl.find(br.na[r] - QA[s], br.nb[r] - QB[s]);
          if (q < 0) continue;
          const int64_t to = toff[((size_t)C.parent * 4 + s) * ns + q];
          if (to < 0) continue;
          const int qo = bl.find(bl.na[q] + Pc.da, bl.nb[q] + Pc.db);
          if (br.find(bl.na[qo] + QA[so], bl.nb[qo] + QB[so]) != ro) throw Error(-6, "RDM: left channel shift mismatch");
          int ld = 0;
          const double* Xo = site_block(x, qo, so, ld);
          g2.add_term(Xo, ld, T + to, br.dim[r], bl.dim[qo], 1, (double)Y[c][so * 4 + s]);
        }
      }
    }
    upload(g1);
    run(g1);
    release(g1);
    upload(g2);
    run(g2);
    release(g2);
    live -= tsz * (int64_t)sizeof(double);
    dfree(T);
  };
  // R_x from R_{x+1} through site x
  auto right_step = [&](int x, const CEnv& Ep, CEnv& Ec) {
    const Bond& bl = bonds[x];
    const Bond& br = bonds[x + 1];
    const Side& Sp = Rs[x + 1];
    const Side& Sc = Rs[x];
    const int ns = br.nsec();
    std::vector<std::array<char, 4>> need(Sp.ch.size(), std::array<char, 4>{0, 0, 0, 0});
    std::vector<Mat4> Y(Sc.ch.size());
    for (size_t c = 0; c < Sc.ch.size(); ++c) {
      Y[c] = unkey(Sc.ch[c].y);
      for (int s = 0; s < 4; ++s)
        if (col_row(Y[c], s) >= 0) need[Sc.ch[c].parent][s] = 1;
    }
    // T[p, s, r] = R_{x+1}[p](r' <- r) X_s(q, r)^T: m_r' x m_q
    std::vector<int64_t> toff(Sp.ch.size() * 4 * (size_t)ns, -1);
    int64_t tsz = 0;
    for (size_t p = 0; p < Sp.ch.size(); ++p)
      for (int s = 0; s < 4; ++s) {
        if (!need[p][s]) continue;
        for (int r = 0; r < ns; ++r) {
          if (Ep.at((int)p, r) < 0) continue;
          const int q = bl.find(br.na[r] - QA[s], br.nb[r] - QB[s]);
          if (q < 0) continue;
          const int ro = br.find(br.na[r] + Sp.ch[p].da, br.nb[r] + Sp.ch[p].db);
          toff[(p * 4 + s) * ns + r] = tsz;
          tsz += (int64_t)br.dim[ro] * bl.dim[q];
        }
      }
    double* T = dalloc<double>(tsz);
    live += tsz * (int64_t)sizeof(double);
    peak = std::max(peak, live);
    GemmPlan g1, g2;
    for (size_t p = 0; p < Sp.ch.size(); ++p)
      for (int s = 0; s < 4; ++s)
        for (int r = 0; r < ns; ++r) {
          const int64_t to = toff[(p * 4 + s) * ns + r];
          if (to < 0) continue;
          const int q = bl.find(br.na[r] - QA[s], br.nb[r] - QB[s]);
          const int ro = br.find(br.na[r] + Sp.ch[p].da, br.nb[r] + Sp.ch[p].db);
          int ld = 0;
          const double* X = site_block(x, q, s, ld);
          g1.add_out(T + to, bl.dim[q], br.dim[ro], bl.dim[q], 0);
          g1.add_term(Ep.d + Ep.at((int)p, r), br.dim[r], X, ld, br.dim[r], 2, 1.0);
        }
    for (size_t c = 0; c < Sc.ch.size(); ++c) {
      const Chan& C = Sc.ch[c];
      const Chan& Pc = Sp.ch[C.parent];
      for (int q = 0; q < bl.nsec(); ++q) {
        const int64_t eo = Ec.at((int)c, q);
        if (eo < 0) continue;
        const int qo = bl.find(bl.na[q] + C.da, bl.nb[q] + C.db);
        g2.add_out(Ec.d + eo, bl.dim[q], bl.dim[qo], bl.dim[q], 0);
        for (int s = 0; s < 4; ++s) {
          const int so = col_row(Y[c], s);
          if (so < 0) continue;
          const int r = br.find(bl.na[q] + QA[s], bl.nb[q] + QB[s]);
          if (r < 0) continue;
          const int64_t to = toff[((size_t)C.parent * 4 + s) * ns + r];
          if (to < 0) continue;
          const int ro = br.find(br.na[r] + Pc.da, br.nb[r] + Pc.db);
          if (bl.find(br.na[ro] - QA[so], br.nb[ro] - QB[so]) != qo) throw Error(-6, "RDM: right channel shift mismatch");
          int ld = 0;
          const double* Xo = site_block(x, qo, so, ld);
          g2.add_term(Xo, ld, T + to, bl.dim[q], br.dim[ro], 0, (double)Y[c][so * 4 + s]);
        }
      }
    }
    upload(g1);
    run(g1);
    release(g1);
    upload(g2);
    run(g2);
    release(g2);
    live -= tsz * (int64_t)sizeof(double);
    dfree(T);
  };
  double* G = dalloc<double>(gsize);
  // Frobenius products of the stored channels at bond b: G = L R^T per class
  auto products = [&](int b, const CEnv& EL, const CEnv& ER) {
    const Bond& bd = bonds[b];
    const BondProd& P = prod[b];
    GemmPlan g;
    for (size_t c = 0; c < P.shift.size(); ++c) {
      const int nl = (int)P.lrows[c].size(), nr = (int)P.rrows[c].size();
      std::vector<int> qs;
      int64_t ksum = 0;
      for (int q = 0; q < bd.nsec(); ++q) {
        const int qo = bd.find(bd.na[q] + P.shift[c].first, bd.nb[q] + P.shift[c].second);
        if (qo < 0) continue;
        qs.push_back(q);
        ksum += (int64_t)bd.dim[qo] * bd.dim[q];
      }
      const int nsp = P.nsplit[c];
      size_t qi = 0;
      int64_t done = 0;
      for (int sp = 0; sp < nsp; ++sp) {
        g.add_out(G + P.gbase[c] + (int64_t)sp * nl * nr, nr, nl, nr, 0);
        const int64_t goal = ksum * (sp + 1) / nsp;
        while (qi < qs.size() && (done < goal || sp == nsp - 1)) {
          const int q = qs[qi++];
          const int qo = bd.find(bd.na[q] + P.shift[c].first, bd.nb[q] + P.shift[c].second);
          const int blk = bd.dim[qo] * bd.dim[q];
          g.add_term(EL.d + EL.at(P.lrows[c][0], q), blk, ER.d + ER.at(P.rrows[c][0], q), blk, blk, 2, 1.0);
          done += blk;
        }
      }
    }
    upload(g);
    run(g);
    release(g);
  };

  std::vector<CEnv> Le(n + 1);
  alloc_env(0, Ls[0], true, Le[0]);
  seed(Le[0]);
  // left pass: every bond's environments stay until its products
  for (int x = 0; x < n; ++x) {
    alloc_env(x + 1, Ls[x + 1], true, Le[x + 1]);
    left_step(x, Le[x], Le[x + 1]);
  }
  free_cenv(Le[0]);
  // right pass, with the products at each bond as its right side appears
  CEnv Rn, Rc;
  alloc_env(n, Rs[n], false, Rn);
  seed(Rn);
  products(n, Le[n], Rn);
  free_cenv(Le[n]);
  for (int x = n - 1; x >= 1; --x) {
    alloc_env(x, Rs[x], false, Rc);
    right_step(x, Rn, Rc);
    free_cenv(Rn);
    products(x, Le[x], Rc);
    free_cenv(Le[x]);
    Rn = Rc;
    Rc = CEnv();
  }
  free_cenv(Rn);
  std::vector<double> Gh((size_t)gsize);
  if (gsize > 0) CK(cudaMemcpyAsync(Gh.data(), G, gsize * sizeof(double), cudaMemcpyDeviceToHost, stream));
  sync();
  stats.d2h += gsize * sizeof(double);
  dfree(G);
  // ---- values: the sum of each element's split-K partials, normalised
  std::vector<double> vals(S.elems.size());
  for (size_t i = 0; i < S.elems.size(); ++i) {
    const Elem& e = S.elems[i];
    const BondProd& P = prod[e.bond];
    const Chan& L = Ls[e.bond].ch[e.lc];
    const Chan& R = Rs[e.bond].ch[e.rc];
    const int c = L.cls;
    const int64_t nl = (int64_t)P.lrows[c].size(), nr = (int64_t)P.rrows[c].size();
    double v = 0;
    for (int sp = 0; sp < P.nsplit[c]; ++sp) v += Gh[(size_t)(P.gbase[c] + sp * nl * nr + L.row * nr + R.row)];
    vals[i] = e.lam * v;
  }
  const double nrm2 = vals[0];
  if (!(nrm2 > 0)) throw Error(-4, "MPS has zero norm");
  for (double& v : vals) v /= nrm2;
  stats.rdm_env_bytes = (double)peak;
  stats.rdm_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return vals;
}

// gamma_pq = sum_s <a+_ps a_qs>, Gamma_pqrs = sum_st <a+_ps a+_rt a_st a_qs>
void Engine::rdms(double* rdm1, double* rdm2) {
  stats.rdm_ms = 0;
  const int n2 = n * n;
  StringSet S(n);
  Mat4 lad[4];
  for (int t = 0; t < 4; ++t) lad[t] = mat_ladder(t);
  const char odd[4] = {1, 1, 1, 1};
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q)
      for (int sg = 0; sg < 2; ++sg) {
        const int pos[2] = {p, q};
        const Mat4 m[2] = {lad[sg], lad[2 + sg]};
        S.add(pos, m, odd, 2, (int64_t)p * n + q);
      }
  if (rdm2)
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q)
        for (int r = 0; r < n; ++r)
          for (int s = 0; s < n; ++s)
            for (int sg = 0; sg < 2; ++sg)
              for (int tu = 0; tu < 2; ++tu) {
                const int pos[4] = {p, r, s, q};
                const Mat4 m[4] = {lad[sg], lad[tu], lad[2 + tu], lad[2 + sg]};
                S.add(pos, m, odd, 4, n2 + (((int64_t)p * n + q) * n + r) * n + s);
              }
  const std::vector<double> v = eval_strings(S);
  std::vector<double> g1(n2, 0.0);
  if (rdm2) std::fill(rdm2, rdm2 + (size_t)n2 * n2, 0.0);
  for (size_t i = 1; i < S.elems.size(); ++i) {
    const int64_t o = S.elems[i].out;
    if (o < n2) g1[o] += v[i];
    else rdm2[o - n2] += v[i];
  }
  if (rdm1) std::memcpy(rdm1, g1.data(), n2 * sizeof(double));
}

// One- and two-orbital reduced density matrices (the inputs of the orbital
// entropies and the mutual information that order the lattice, Sec.
// "Cholesky decomposition for the wavefunction", ingredient (ii)):
//   rho[x', x] = <psi| C+_{x'} prod_m (1 - n_m) C_x |psi>
// over the modes m of the orbital (pair), C+_x creating the local state x
// (modes in order, alpha before beta, orbital i before j) and C_x its
// adjoint: the fermionic partial trace with the kept modes moved to the
// front.  Only entries with equal particle numbers in x and x' can be
// nonzero; the others are set to zero.
void Engine::orbital_rdms(double* rho1, double* rho2) {
  stats.rdm_ms = 0;
  StringSet S(n);
  Mat4 lad[4], proj[2];
  for (int t = 0; t < 4; ++t) lad[t] = mat_ladder(t);
  for (int sp = 0; sp < 2; ++sp) {   // 1 - n_alpha, 1 - n_beta
    proj[sp] = mat_ident();
    for (int s = 0; s < 4; ++s)
      if ((sp == 0 ? QA[s] : QB[s]) == 1) proj[sp][s * 5] = 0;
  }
  const int npairs = n * (n - 1) / 2;
  auto emit = [&](const int* orb, int no, const int* xp, const int* x, int64_t out) {
    int pos[12];
    Mat4 m[12];
    char odd[12];
    int k = 0;
    for (int a = 0; a < no; ++a)
      for (int sp = 0; sp < 2; ++sp)
        if ((xp[a] >> sp) & 1) {
          pos[k] = orb[a];
          m[k] = lad[sp];
          odd[k++] = 1;
        }
    for (int a = 0; a < no; ++a)
      for (int sp = 0; sp < 2; ++sp) {
        pos[k] = orb[a];
        m[k] = proj[sp];
        odd[k++] = 0;
      }
    for (int a = no - 1; a >= 0; --a)
      for (int sp = 1; sp >= 0; --sp)
        if ((x[a] >> sp) & 1) {
          pos[k] = orb[a];
          m[k] = lad[2 + sp];
          odd[k++] = 1;
        }
    S.add(pos, m, odd, k, out);
  };
  auto na_of = [](int x) { return x & 1; };
  auto nb_of = [](int x) { return (x >> 1) & 1; };
  for (int i = 0; i < n; ++i)
    for (int x = 0; x < 4; ++x) {
      const int orb[1] = {i}, xx[1] = {x};
      emit(orb, 1, xx, xx, (int64_t)i * 16 + x * 5);
    }
  const int64_t base2 = (int64_t)n * 16;
  int pr = 0;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j, ++pr)
      for (int yp = 0; yp < 16; ++yp)
        for (int y = 0; y < 16; ++y) {
          const int xp[2] = {yp & 3, yp >> 2}, x[2] = {y & 3, y >> 2};
          if (na_of(xp[0]) + na_of(xp[1]) != na_of(x[0]) + na_of(x[1]) ||
              nb_of(xp[0]) + nb_of(xp[1]) != nb_of(x[0]) + nb_of(x[1]))
            continue;
          const int orb[2] = {i, j};
          emit(orb, 2, xp, x, base2 + (int64_t)pr * 256 + yp * 16 + y);
        }
  const std::vector<double> v = eval_strings(S);
  if (rho1) std::fill(rho1, rho1 + (size_t)n * 16, 0.0);
  if (rho2) std::fill(rho2, rho2 + (size_t)npairs * 256, 0.0);
  for (size_t e = 1; e < S.elems.size(); ++e) {
    const int64_t o = S.elems[e].out;
    if (o < base2) {
      if (rho1) rho1[o] = v[e];
    } else if (rho2) {
      rho2[o - base2] = v[e];
    }
  }
}

}  // namespace gbd
