// MPO of the active-space Hamiltonian, built term by term.
//
// The paper applies H as a matrix-product operator so that the d^L operator
// is never formed (Sec. "Cholesky decomposition for the wavefunction", item
// (i)); it does not print the construction.  Ours:
//   H = sum h_pq a+_ps a_qs + 1/2 sum (pq|rs) a+_ps a+_rt a_st a_qs.
// Each operator string is reordered into site order (sign = parity of the
// reordering) and routed through one channel per bond:
//   no operator left of the bond -> I;  none right of it -> H;
//   one operator left, or two left and two right with k <= k_switch
//        -> bare channel labelled by the left operators (no coefficient);
//   otherwise -> complementary channel labelled by the right operators.
// The coefficient is applied on the site where the path first enters a
// complementary or H channel.  Entries whose target channel is odd are
// multiplied by the local parity on their input side, so that all
// contractions downstream are plain tensor products (the Jordan-Wigner signs
// live in the tensors).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <unordered_map>
#include <unordered_set>

#include "gbd_internal.h"

namespace gbd {

namespace {

using Mat4 = std::array<double, 16>;   // row = output state, col = input state

Mat4 identity4() {
  Mat4 m{};
  for (int i = 0; i < 4; ++i) m[i * 4 + i] = 1.0;
  return m;
}

// local fermion operators on [0, a, b, ab] with |ab> = a+_a a+_b |0>
Mat4 local_op(int spin, bool dag) {
  Mat4 m{};
  if (spin == 0) {   // a+_alpha: |0>->|a>, |b>->|ab>
    if (dag) { m[1 * 4 + 0] = 1.0; m[3 * 4 + 2] = 1.0; }
    else     { m[0 * 4 + 1] = 1.0; m[2 * 4 + 3] = 1.0; }
  } else {           // a+_beta: |0>->|b>, |a>->-|ab>
    if (dag) { m[2 * 4 + 0] = 1.0; m[3 * 4 + 1] = -1.0; }
    else     { m[0 * 4 + 2] = 1.0; m[1 * 4 + 3] = -1.0; }
  }
  return m;
}

Mat4 matmul4(const Mat4& x, const Mat4& y) {
  Mat4 r{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0;
      for (int k = 0; k < 4; ++k) s += x[i * 4 + k] * y[k * 4 + j];
      r[i * 4 + j] = s;
    }
  return r;
}

struct Term {
  int nops;
  int code[4];   // sorted op codes: site*4 + spin*2 + (dag ? 0 : 1)
  double coef;
};

inline int op_site(int c) { return c >> 2; }
inline int op_spin(int c) { return (c >> 1) & 1; }
inline bool op_dag(int c) { return (c & 1) == 0; }

// Sort op codes ascending; return the permutation parity (number of
// inversions).  Only distinct spin orbitals are ever exchanged here.
int sort_codes(int* c, int n) {
  int inv = 0;
  for (int i = 1; i < n; ++i) {
    int x = c[i], j = i - 1;
    while (j >= 0 && c[j] > x) { c[j + 1] = c[j]; --j; ++inv; }
    c[j + 1] = x;
  }
  return inv;
}

uint64_t term_key(const int* c, int n) {
  uint64_t k = (uint64_t)n;
  for (int i = 0; i < n; ++i) k = (k << 14) | (uint64_t)c[i];
  return k;
}

Label label_of(const Term& t, int k, int k_switch) {
  int nl = 0;
  while (nl < t.nops && op_site(t.code[nl]) < k) ++nl;
  int nr = t.nops - nl;
  Label L;
  if (nl == 0) { L.kind = 0; return L; }
  if (nr == 0) { L.kind = 1; return L; }
  if (nl == 1 || (nl == 2 && nr == 2 && k <= k_switch)) {
    L.kind = 2; L.nops = nl; L.c0 = t.code[0]; L.c1 = nl > 1 ? t.code[1] : 0;
  } else {
    L.kind = 3; L.nops = nr; L.c0 = t.code[nl]; L.c1 = nr > 1 ? t.code[nl + 1] : 0;
  }
  return L;
}

void label_delta(const Label& L, int& da, int& db, int& par) {
  da = db = 0;
  par = L.nops & 1;
  if (L.kind < 2) { par = 0; return; }
  int codes[2] = {L.c0, L.c1};
  for (int i = 0; i < L.nops; ++i) {
    int d = op_dag(codes[i]) ? 1 : -1;
    if (op_spin(codes[i]) == 0) da += d; else db += d;
  }
  if (L.kind == 3) { da = -da; db = -db; }
}

}  // namespace

void build_mpo(int n, const double* h, const double* eri, int k_switch, Mpo& out) {
  // ---- terms, merged by canonical operator string
  std::unordered_map<uint64_t, size_t> where;
  std::vector<Term> terms;
  where.reserve((size_t)n * n * n * n * 2);
  auto add = [&](double coef, int nops, const int* raw) {
    Term t;
    t.nops = nops;
    for (int i = 0; i < nops; ++i) t.code[i] = raw[i];
    int inv = sort_codes(t.code, nops);
    t.coef = (inv & 1) ? -coef : coef;
    uint64_t key = term_key(t.code, nops);
    auto it = where.find(key);
    if (it == where.end()) { where.emplace(key, terms.size()); terms.push_back(t); }
    else terms[it->second].coef += t.coef;
  };
  auto code = [](int site, int spin, bool dag) { return site * 4 + spin * 2 + (dag ? 0 : 1); };
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) {
      double v = h[p * n + q];
      if (v == 0.0) continue;
      for (int s = 0; s < 2; ++s) {
        int raw[2] = {code(p, s, true), code(q, s, false)};
        add(v, 2, raw);
      }
    }
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q)
      for (int r = 0; r < n; ++r)
        for (int ss = 0; ss < n; ++ss) {
          double v = eri[((size_t)(p * n + q) * n + r) * n + ss];
          if (v == 0.0) continue;
          for (int s = 0; s < 2; ++s)
            for (int t = 0; t < 2; ++t) {
              if ((p == r && s == t) || (q == ss && s == t)) continue;
              int raw[4] = {code(p, s, true), code(r, t, true), code(ss, t, false), code(q, s, false)};
              add(0.5 * v, 4, raw);
            }
        }
  terms.erase(std::remove_if(terms.begin(), terms.end(), [](const Term& t) { return t.coef == 0.0; }),
              terms.end());

  // ---- channel labels per bond
  out.n = n;
  out.k_switch = k_switch;
  out.labels.assign(n + 1, {});
  std::vector<std::unordered_map<uint64_t, int>> index(n + 1);
  {
    std::vector<std::unordered_map<uint64_t, Label>> seen(n + 1);
    for (const Term& t : terms)
      for (int k = 0; k <= n; ++k) {
        Label L = label_of(t, k, k_switch);
        seen[k].emplace(L.key(), L);
      }
    for (int k = 0; k <= n; ++k) {
      std::vector<Label> v;
      for (auto& kv : seen[k]) v.push_back(kv.second);
      std::sort(v.begin(), v.end(), [](const Label& x, const Label& y) { return x.key() < y.key(); });
      out.labels[k] = v;
      for (int i = 0; i < (int)v.size(); ++i) index[k][v[i].key()] = i;
    }
  }
  out.dA.assign(n + 1, {});
  out.dB.assign(n + 1, {});
  out.parity.assign(n + 1, {});
  out.ident_channel.assign(n + 1, -1);
  out.ham_channel.assign(n + 1, -1);
  for (int k = 0; k <= n; ++k) {
    for (int i = 0; i < (int)out.labels[k].size(); ++i) {
      int da, db, par;
      label_delta(out.labels[k][i], da, db, par);
      out.dA[k].push_back(da);
      out.dB[k].push_back(db);
      out.parity[k].push_back(par);
      if (out.labels[k][i].kind == 0) out.ident_channel[k] = i;
      if (out.labels[k][i].kind == 1) out.ham_channel[k] = i;
    }
  }

  // ---- site tensors
  out.W.assign(n, {});
  for (int i = 0; i < n; ++i) {
    std::unordered_map<uint64_t, Mat4> acc;
    acc.reserve(terms.size() / 4 + 16);
    for (const Term& t : terms) {
      Label La = label_of(t, i, k_switch), Lb = label_of(t, i + 1, k_switch);
      int a = index[i][La.key()], b = index[i + 1][Lb.key()];
      Mat4 loc = identity4();
      for (int j = 0; j < t.nops; ++j)
        if (op_site(t.code[j]) == i) loc = matmul4(loc, local_op(op_spin(t.code[j]), op_dag(t.code[j])));
      uint64_t key = ((uint64_t)a << 32) | (uint64_t)b;
      bool applies = (La.kind == 0 || La.kind == 2) && (Lb.kind == 1 || Lb.kind == 3);
      auto it = acc.find(key);
      if (applies) {
        if (it == acc.end()) it = acc.emplace(key, Mat4{}).first;
        for (int e = 0; e < 16; ++e) it->second[e] += t.coef * loc[e];
      } else if (it == acc.end()) {
        acc.emplace(key, loc);
      }
    }
    std::vector<MpoEntry> ent;
    for (auto& kv : acc) {
      int a = (int)(kv.first >> 32), b = (int)(kv.first & 0xffffffffu);
      bool odd = out.parity[i + 1][b] != 0;
      for (int so = 0; so < 4; ++so)
        for (int si = 0; si < 4; ++si) {
          double v = kv.second[so * 4 + si];
          if (odd && PAR[si]) v = -v;   // W P on the input side
          if (v != 0.0) ent.push_back({a, b, so, si, v});
        }
    }
    std::sort(ent.begin(), ent.end(), [](const MpoEntry& x, const MpoEntry& y) {
      if (x.b != y.b) return x.b < y.b;
      if (x.a != y.a) return x.a < y.a;
      if (x.sout != y.sout) return x.sout < y.sout;
      return x.sin < y.sin;
    });
    out.W[i] = std::move(ent);
  }
}

// Hermitian-conjugate channel pairs, certified from the W tensors.  For a
// real MPS, L_b[c]^T = <L|O_c^T|L>: if every left environment at bond k
// satisfies L_k[conj a] = sign_a L_k[a]^T (bond 0: only the identity is
// nonzero), then L_{k+1}[d] = sign L_{k+1}[c]^T whenever W_k's column d
// equals sign times column c with each entry (a, s', s, v) replaced by
// (conj a, s, s', sign_a v).  Right environments follow the same rule on
// W_k's rows from bond n (only the H channel nonzero) down.  Channels whose
// column (row) has no such partner, or whose coefficients differ in the last
// bit, stay unpaired (-1) and are computed; so do self-conjugate ones.
void mpo_conjugates(const Mpo& m, std::vector<std::vector<int>>& cl, std::vector<std::vector<int>>& sl,
                    std::vector<std::vector<int>>& cr, std::vector<std::vector<int>>& sr) {
  const int n = m.n;
  cl.assign(n + 1, {});
  sl.assign(n + 1, {});
  cr.assign(n + 1, {});
  sr.assign(n + 1, {});
  auto self = [&](int bond, std::vector<std::vector<int>>& c, std::vector<std::vector<int>>& sg) {
    const int nc = (int)m.labels[bond].size();
    c[bond].resize(nc);
    sg[bond].assign(nc, 1);
    for (int i = 0; i < nc; ++i) c[bond][i] = i;
  };
  self(0, cl, sl);
  self(n, cr, sr);
  using Ent = std::tuple<int, int, int, double>;   // (channel at the other bond, s_out, s_in, value)
  // entries sorted, first value made positive; sg: the sign taken out
  auto canon = [](std::vector<Ent> v, int& sg) {
    std::sort(v.begin(), v.end());
    sg = 1;
    if (!v.empty() && std::get<3>(v[0]) < 0) {
      sg = -1;
      for (auto& e : v) std::get<3>(e) = -std::get<3>(e);
    }
    return v;
  };
  auto pair_up = [&](const std::vector<std::vector<Ent>>& lines, const std::vector<int>& cprev,
                     const std::vector<int>& sprev, std::vector<int>& cout, std::vector<int>& sout) {
    const int nc = (int)lines.size();
    cout.assign(nc, -1);
    sout.assign(nc, 1);
    std::map<std::vector<Ent>, std::vector<int>> by;
    std::vector<int> sg(nc, 1);
    for (int c = 0; c < nc; ++c) by[canon(lines[c], sg[c])].push_back(c);
    for (int c = 0; c < nc; ++c) {
      if (cout[c] >= 0) continue;
      if (lines[c].empty()) {   // a zero environment
        cout[c] = c;
        continue;
      }
      std::vector<Ent> t;
      bool ok = true;
      for (const Ent& e : lines[c]) {
        const int a = std::get<0>(e);
        if (cprev[a] < 0) {
          ok = false;
          break;
        }
        t.emplace_back(cprev[a], std::get<2>(e), std::get<1>(e), sprev[a] * std::get<3>(e));
      }
      if (!ok) continue;
      int st = 1;
      auto it = by.find(canon(t, st));
      if (it == by.end()) continue;
      for (int d : it->second) {
        if (cout[d] >= 0) continue;
        cout[c] = d;
        cout[d] = c;
        sout[c] = sout[d] = st * sg[d];   // lines[d] = sg[d] st t
        break;
      }
    }
  };
  for (int k = 0; k < n; ++k) {   // left: columns of W_k (bond k -> bond k + 1)
    std::vector<std::vector<Ent>> col(m.labels[k + 1].size());
    for (const MpoEntry& e : m.W[k]) col[e.b].emplace_back(e.a, e.sout, e.sin, e.v);
    pair_up(col, cl[k], sl[k], cl[k + 1], sl[k + 1]);
  }
  for (int k = n - 1; k >= 0; --k) {   // right: rows of W_k (bond k + 1 -> bond k)
    std::vector<std::vector<Ent>> row(m.labels[k].size());
    for (const MpoEntry& e : m.W[k]) row[e.a].emplace_back(e.b, e.sout, e.sin, e.v);
    pair_up(row, cr[k + 1], sr[k + 1], cr[k], sr[k]);
  }
}

}  // namespace gbd
