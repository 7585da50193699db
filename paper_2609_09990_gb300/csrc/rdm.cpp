// One- and two-particle RDMs of the current MPS (paper: device k-RDMs of the
// converged MPS, Sec. "The DMRG-QD-NEVPT2 energy" and Sec. "Computational
// details"):
//   gamma_pq = sum_s <a+_ps a_qs>,  Gamma_pqrs = sum_st <a+_ps a+_rt a_st a_qs>
//            = <E_pq E_rs> - delta_qr gamma_ps.
// The MPS is expanded into the determinant basis |I_a, I_b> (alpha creators,
// then beta creators, strings in colex order addr = sum_i C(o_i, i+1)):
// prefix vectors (sites < h) and suffix vectors (sites >= h) are built by
// grouped GEMMs and multiplied at the middle bond h, then scattered with the
// sign that reorders site-major creators into alpha-first order.  With
// D[pq] = E_pq C (formed in chunks of alpha strings), gamma_pq = C . D[pq]
// and <E_pq E_rs> = D[qp] . D[rs] is one split-K Gram GEMM.  FP64.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "engine.h"

namespace gbd {

void launch_scatter_ci(const double* A, int npref, int nsuf, const int* aP, const int* bP, const signed char* sP,
                       const int* aS, const int* bS, const signed char* sS, double sector_sign, int64_t Nb,
                       double* C, cudaStream_t s);
void launch_apply_e_chunk(const double* C, int64_t Nb, const int* excA, const int* excB, int n2, int ja0, int cs,
                          double* D, cudaStream_t s);
void launch_apply_e_vecs(const double* V, int nv, int64_t Na, int64_t Nb, const int* excA, const int* excB, int n2,
                         int rs, double* out, cudaStream_t s);
int pair_rdm_blocks(int64_t ndet);
void launch_pair_rdm(const double* C, int64_t NaS, int64_t NbS, const uint32_t* strA, const uint32_t* strB,
                     const int* binom, int n, int NaTot, const int* pairs, int npairs, double* partial,
                     cudaStream_t s);

namespace {

double binom_i(int n, int k) {
  if (k < 0 || k > n) return 0;
  double r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return std::round(r);
}

int colex(uint32_t bits, int n) {
  int addr = 0, pos = 0;
  for (int o = 0; o < n; ++o)
    if (bits >> o & 1u) addr += (int)binom_i(o, ++pos);
  return addr;
}

// all k-subsets of n orbitals indexed by colex address
std::vector<uint32_t> strings(int n, int k) {
  std::vector<uint32_t> out((size_t)binom_i(n, k));
  std::vector<int> c(k);
  for (int i = 0; i < k; ++i) c[i] = i;
  while (true) {
    uint32_t b = 0;
    for (int x : c) b |= 1u << x;
    out[colex(b, n)] = b;
    int i = k - 1;
    while (i >= 0 && c[i] == n - k + i) --i;
    if (i < 0) break;
    ++c[i];
    for (int j = i + 1; j < k; ++j) c[j] = c[j - 1] + 1;
  }
  return out;
}

// exc[J * n^2 + p*n + q] = (I + 1) * sign with E_pq |I> = sign |J>, else 0
std::vector<int> excitations(int n, int k) {
  auto str = strings(n, k);
  int n2 = n * n;
  std::vector<int> exc(str.size() * n2, 0);
  for (size_t I = 0; I < str.size(); ++I) {
    uint32_t b = str[I];
    for (int q = 0; q < n; ++q) {
      if (!(b >> q & 1u)) continue;
      int sq = __builtin_popcount(b & ((1u << q) - 1u)) & 1;
      uint32_t rest = b & ~(1u << q);
      for (int p = 0; p < n; ++p) {
        if (rest >> p & 1u) continue;
        int sp = __builtin_popcount(rest & ((1u << p) - 1u)) & 1;
        uint32_t jb = rest | (1u << p);
        int J = colex(jb, n);
        exc[(size_t)J * n2 + p * n + q] = ((sq ^ sp) ? -1 : 1) * ((int)I + 1);
      }
    }
  }
  return exc;
}

}  // namespace

// site block X_i(q, s): m_i(q) x m_{i+1}(q+s), row-major with leading
// dimension ld, inside either site layout; nullptr if q + s is no sector
const double* Engine::site_block(int i, int qi, int s, int& ld) const {
  const Bond& bl = bonds[i];
  const Bond& br = bonds[i + 1];
  const Site& S = sites[i];
  int r = br.find(bl.na[qi] + QA[s], bl.nb[qi] + QB[s]);
  if (r < 0) return nullptr;
  if (S.layout == 1) {
    int coff = 0, cols = 0;
    for (int t = 0; t < 4; ++t) {
      int rr = br.find(bl.na[qi] + QA[t], bl.nb[qi] + QB[t]);
      if (rr < 0) continue;
      if (t < s) coff += br.dim[rr];
      cols += br.dim[rr];
    }
    ld = cols;
    return S.d + S.off[qi] + coff;
  }
  int roff = 0;
  for (int t = 0; t < s; ++t) {
    int jj = bl.find(br.na[r] - QA[t], br.nb[r] - QB[t]);
    if (jj >= 0) roff += bl.dim[jj];
  }
  ld = br.dim[r];
  return S.d + S.off[r] + (int64_t)roff * br.dim[r];
}

// The current MPS expanded into the determinant basis: C[Ia * Nb_str + Ib]
// (device, caller frees), not normalised.
double* Engine::expand_ci(int64_t& Na_str, int64_t& Nb_str) {
  const int h = n / 2;
  Na_str = (int64_t)binom_i(n, Na);
  Nb_str = (int64_t)binom_i(n, Nb);
  const int64_t ndet = Na_str * Nb_str;
  if (ndet > (int64_t)400000000) throw Error(-1, "RDMs need the determinant expansion; too many determinants");
  auto block = [&](int i, int qi, int s, int& ld) { return site_block(i, qi, s, ld); };

  // ---- prefixes (sites < h), rows of P_i(q)
  struct Fix { std::vector<uint32_t> a, b; double* d = nullptr; };
  std::vector<Fix> pre(1);
  pre[0].a = {0};
  pre[0].b = {0};
  pre[0].d = dalloc<double>(1);
  {
    double one = 1.0;
    CK(cudaMemcpyAsync(pre[0].d, &one, sizeof(double), cudaMemcpyHostToDevice, stream));
  }
  for (int i = 0; i < h; ++i) {
    const Bond& bl = bonds[i];
    const Bond& br = bonds[i + 1];
    std::vector<Fix> nx(br.nsec());
    GemmPlan p;
    for (int j = 0; j < br.nsec(); ++j) {
      Fix& f = nx[j];
      std::vector<std::pair<int, int>> parts;   // (parent sector, s)
      for (int s = 0; s < 4; ++s) {
        int qi = bl.find(br.na[j] - QA[s], br.nb[j] - QB[s]);
        if (qi < 0 || pre[qi].a.empty()) continue;
        parts.push_back({qi, s});
        for (size_t t = 0; t < pre[qi].a.size(); ++t) {
          f.a.push_back(pre[qi].a[t] | ((uint32_t)QA[s] << i));
          f.b.push_back(pre[qi].b[t] | ((uint32_t)QB[s] << i));
        }
      }
      if (f.a.empty()) continue;
      int mr = br.dim[j];
      f.d = dalloc<double>(f.a.size() * (size_t)mr);
      int64_t row = 0;
      for (auto& pr : parts) {
        int qi = pr.first, s = pr.second;
        int np = (int)pre[qi].a.size();
        int ld = 0;
        const double* X = block(i, qi, s, ld);
        p.add_out(f.d + row * mr, mr, np, mr, 0);
        p.add_term(pre[qi].d, bl.dim[qi], X, ld, bl.dim[qi], 0, 1.0);
        row += np;
      }
    }
    upload(p);
    run(p);
    release(p);
    for (auto& f : pre) if (f.d) dfree(f.d);
    pre.swap(nx);
  }
  // ---- suffixes (sites >= h), columns of R_i(q)
  std::vector<Fix> suf(bonds[n].nsec());
  {
    int qi = 0;
    suf[qi].a = {0};
    suf[qi].b = {0};
    suf[qi].d = dalloc<double>(1);
    double one = 1.0;
    CK(cudaMemcpyAsync(suf[qi].d, &one, sizeof(double), cudaMemcpyHostToDevice, stream));
  }
  for (int i = n - 1; i >= h; --i) {
    const Bond& bl = bonds[i];
    const Bond& br = bonds[i + 1];
    std::vector<Fix> nx(bl.nsec());
    GemmPlan p;
    for (int j = 0; j < bl.nsec(); ++j) {
      Fix& f = nx[j];
      std::vector<std::pair<int, int>> parts;   // (child sector, s)
      for (int s = 0; s < 4; ++s) {
        int r = br.find(bl.na[j] + QA[s], bl.nb[j] + QB[s]);
        if (r < 0 || suf[r].a.empty()) continue;
        parts.push_back({r, s});
        for (size_t t = 0; t < suf[r].a.size(); ++t) {
          f.a.push_back(suf[r].a[t] | ((uint32_t)QA[s] << i));
          f.b.push_back(suf[r].b[t] | ((uint32_t)QB[s] << i));
        }
      }
      if (f.a.empty()) continue;
      int ncols = (int)f.a.size();
      f.d = dalloc<double>((size_t)bl.dim[j] * ncols);
      int64_t col = 0;
      for (auto& pr : parts) {
        int r = pr.first, s = pr.second;
        int ns = (int)suf[r].a.size();
        int ld = 0;
        const double* X = block(i, j, s, ld);
        p.add_out(f.d + col, ncols, bl.dim[j], ns, 0);
        p.add_term(X, ld, suf[r].d, ns, br.dim[r], 0, 1.0);
        col += ns;
      }
    }
    upload(p);
    run(p);
    release(p);
    for (auto& f : suf) if (f.d) dfree(f.d);
    suf.swap(nx);
  }
  // ---- amplitudes at the middle bond, scattered into C[Ia, Ib]
  double* C = dalloc<double>(ndet);
  CK(cudaMemsetAsync(C, 0, ndet * sizeof(double), stream));
  const Bond& bh = bonds[h];
  for (int j = 0; j < bh.nsec(); ++j) {
    if (pre[j].a.empty() || suf[j].a.empty()) continue;
    int a = bh.na[j], b = bh.nb[j];
    int np = (int)pre[j].a.size(), ns = (int)suf[j].a.size(), m = bh.dim[j];
    double* A = dalloc<double>((size_t)np * ns);
    GemmPlan p;
    p.add_out(A, ns, np, ns, 0);
    p.add_term(pre[j].d, m, suf[j].d, ns, m, 0, 1.0);
    upload(p);
    run(p);
    release(p);
    std::vector<int> aP(np), bP(np), aS(ns), bS(ns);
    std::vector<signed char> sP(np), sS(ns);
    auto addr_from = [&](uint32_t bits, int pos0) {
      int ad = 0, pos = pos0;
      for (int o = 0; o < n; ++o)
        if (bits >> o & 1u) ad += (int)binom_i(o, ++pos);
      return ad;
    };
    auto sign_of = [&](uint32_t ab, uint32_t bb) {
      int ex = 0;
      for (int jj = 0; jj < n; ++jj)
        if (bb >> jj & 1u) ex += __builtin_popcount(ab >> (jj + 1));
      return (signed char)((ex & 1) ? -1 : 1);
    };
    for (int t = 0; t < np; ++t) {
      aP[t] = addr_from(pre[j].a[t], 0);
      bP[t] = addr_from(pre[j].b[t], 0);
      sP[t] = sign_of(pre[j].a[t], pre[j].b[t]);
    }
    for (int t = 0; t < ns; ++t) {
      aS[t] = addr_from(suf[j].a[t], a);
      bS[t] = addr_from(suf[j].b[t], b);
      sS[t] = sign_of(suf[j].a[t], suf[j].b[t]);
    }
    double ssec = ((b * (Na - a)) & 1) ? -1.0 : 1.0;
    int* d_i = dalloc<int>(2 * (size_t)np + 2 * (size_t)ns);
    signed char* d_s = dalloc<signed char>((size_t)np + ns);
    CK(cudaMemcpyAsync(d_i, aP.data(), np * sizeof(int), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(d_i + np, bP.data(), np * sizeof(int), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(d_i + 2 * np, aS.data(), ns * sizeof(int), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(d_i + 2 * np + ns, bS.data(), ns * sizeof(int), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(d_s, sP.data(), np, cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(d_s + np, sS.data(), ns, cudaMemcpyHostToDevice, stream));
    launch_scatter_ci(A, np, ns, d_i, d_i + np, d_s, d_i + 2 * np, d_i + 2 * np + ns, d_s + np, ssec, Nb_str, C,
                      stream);
    stats.launches++;
    CK(cudaGetLastError());
    sync();
    dfree(A);
    dfree(d_i);
    dfree(d_s);
  }
  for (auto& f : pre) if (f.d) dfree(f.d);
  for (auto& f : suf) if (f.d) dfree(f.d);
  return C;
}

void Engine::rdms_ci(double* rdm1, double* rdm2) {
  int64_t Na_str = 0, Nb_str = 0;
  double* C = expand_ci(Na_str, Nb_str);
  const int64_t ndet = Na_str * Nb_str;
  // ---- D[pq] = E_pq C in chunks of alpha strings; gamma and <E E> by GEMM
  const int n2 = n * n;
  auto excA = excitations(n, Na), excB = excitations(n, Nb);
  int* d_excA = dalloc<int>(excA.size());
  int* d_excB = dalloc<int>(excB.size());
  CK(cudaMemcpyAsync(d_excA, excA.data(), excA.size() * sizeof(int), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(d_excB, excB.data(), excB.size() * sizeof(int), cudaMemcpyHostToDevice, stream));
  int64_t budget = (int64_t)1 << 27;   // doubles per D chunk (1 GiB)
  int cs = (int)std::max<int64_t>(1, std::min<int64_t>(Na_str, budget / ((int64_t)n2 * Nb_str)));
  double* D = dalloc<double>((size_t)n2 * cs * Nb_str);
  const int SPLIT = 32;
  double* Mp = dalloc<double>((size_t)SPLIT * n2 * n2);
  double* gp = dalloc<double>((size_t)SPLIT * n2);
  bool first = true;
  for (int ja0 = 0; ja0 < Na_str; ja0 += cs) {
    int c = (int)std::min<int64_t>(cs, Na_str - ja0);
    launch_apply_e_chunk(C, Nb_str, d_excA, d_excB, n2, ja0, c, D, stream);
    stats.launches++;
    CK(cudaGetLastError());
    int64_t K = (int64_t)c * Nb_str;
    int parts = (int)std::min<int64_t>(SPLIT, std::max<int64_t>(1, K / 4096));
    int64_t step = (K + parts - 1) / parts;
    GemmPlan p;
    const double* Cchunk = C + (int64_t)ja0 * Nb_str;
    for (int s = 0; s < SPLIT; ++s) {
      int64_t k0 = (int64_t)s * step, k1 = std::min<int64_t>(K, k0 + step);
      p.add_out(Mp + (size_t)s * n2 * n2, n2, n2, n2, first ? 0 : 1);
      if (s < parts && k1 > k0) p.add_term(D + k0, (int)K, D + k0, (int)K, (int)(k1 - k0), 2, 1.0);
      p.add_out(gp + (size_t)s * n2, 1, n2, 1, first ? 0 : 1);
      if (s < parts && k1 > k0) p.add_term(D + k0, (int)K, Cchunk + k0, 1, (int)(k1 - k0), 0, 1.0);
    }
    upload(p);
    run(p);
    release(p);
    first = false;
  }
  // sum the split-K partials and read back
  double* Msum = dalloc<double>((size_t)n2 * n2 + n2);
  AxpyPlan ax;
  ax.outs.push_back({Msum, (int64_t)n2 * n2, 0, 0});
  for (int s = 0; s < SPLIT; ++s) ax.terms.push_back({Mp + (size_t)s * n2 * n2, 1.0});
  ax.outs.back().t1 = (int)ax.terms.size();
  ax.outs.push_back({Msum + (size_t)n2 * n2, (int64_t)n2, (int)ax.terms.size(), 0});
  for (int s = 0; s < SPLIT; ++s) ax.terms.push_back({gp + (size_t)s * n2, 1.0});
  ax.outs.back().t1 = (int)ax.terms.size();
  upload(ax);
  run(ax);
  release(ax);
  int nblk = reduction_blocks(ndet);
  double* partial = dalloc<double>(nblk);
  double* nrm_d = dalloc<double>(1);
  launch_multi_dot(C, ndet, 1, C, ndet, nrm_d, partial, nblk, stream);
  stats.launches += 2;
  std::vector<double> Mh((size_t)n2 * n2 + n2);
  double nrm2 = 0;
  CK(cudaMemcpyAsync(Mh.data(), Msum, Mh.size() * sizeof(double), cudaMemcpyDeviceToHost, stream));
  CK(cudaMemcpyAsync(&nrm2, nrm_d, sizeof(double), cudaMemcpyDeviceToHost, stream));
  sync();
  stats.d2h += (Mh.size() + 1) * sizeof(double);
  for (void* q : {(void*)C, (void*)d_excA, (void*)d_excB, (void*)D, (void*)Mp, (void*)gp, (void*)Msum,
                  (void*)partial, (void*)nrm_d})
    dfree(q);
  if (!(nrm2 > 0)) throw Error(-4, "MPS has zero norm in the determinant expansion");
  const double* M = Mh.data();
  const double* g = Mh.data() + (size_t)n2 * n2;
  std::vector<double> g1(n2);
  for (int i = 0; i < n2; ++i) g1[i] = g[i] / nrm2;
  if (rdm1) std::memcpy(rdm1, g1.data(), n2 * sizeof(double));
  if (rdm2)
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q)
        for (int r = 0; r < n; ++r)
          for (int s = 0; s < n; ++s) {
            double v = M[(size_t)(q * n + p) * n2 + r * n + s] / nrm2;
            if (q == r) v -= g1[p * n + s];
            rdm2[(((size_t)p * n + q) * n + r) * n + s] = v;
          }
}

// ---------------------------------------------------------------- 3-RDM
// Gamma3_pqrstu = sum_{s,t,v} <a+_ps a+_rt a+_tv a_uv a_st a_qs> (Sec.
// "Computational details": one- through three-particle RDMs on the device)
// from products of excitation operators,
//   <E_pq E_rs E_tu> = Gamma3_pqrstu + d_qt Gamma_purs + d_st Gamma_pqru
//                      + d_qr Gamma_pstu + d_qr d_st gamma_pu,
// and <E_pq E_rs E_tu> = D[qp] . (E_rs D[tu]) with D[tu] = E_tu C: for each
// rs, the n^2 vectors E_rs D[tu] and one split-K Gram GEMM against D.  FP64.
void Engine::rdm3(double* out) {
  int64_t NaS = 0, NbS = 0;
  double* C = expand_ci(NaS, NbS);
  const int64_t ndet = NaS * NbS;
  const int n2 = n * n;
  if (ndet > (int64_t)0x7fffffff || 2.0 * n2 * (double)ndet * sizeof(double) > 64e9) {
    dfree(C);
    throw Error(-1, "3-RDM: the determinant expansion needs 2 n^2 vectors of the determinant length (at most 64 GB)");
  }
  auto excA = excitations(n, Na), excB = excitations(n, Nb);
  int* d_excA = dalloc<int>(excA.size());
  int* d_excB = dalloc<int>(excB.size());
  CK(cudaMemcpyAsync(d_excA, excA.data(), excA.size() * sizeof(int), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(d_excB, excB.data(), excB.size() * sizeof(int), cudaMemcpyHostToDevice, stream));
  double* D = dalloc<double>((size_t)n2 * ndet);
  double* F = dalloc<double>((size_t)n2 * ndet);
  launch_apply_e_chunk(C, NbS, d_excA, d_excB, n2, 0, (int)NaS, D, stream);
  stats.launches++;
  CK(cudaGetLastError());
  const int SPLIT = 32;
  const int parts = (int)std::min<int64_t>(SPLIT, std::max<int64_t>(1, ndet / 4096));
  const int64_t step = (ndet + parts - 1) / parts;
  double* Mp = dalloc<double>((size_t)parts * n2 * n2);
  double* M3 = dalloc<double>((size_t)n2 * n2 * n2);
  double* M2 = dalloc<double>((size_t)n2 * n2 + n2);
  // Gram of D against a set of n2 vectors W (D . W^T), split over K and summed
  // in a fixed order into dst
  auto gram = [&](const double* W, int ldw_is_vec, double* dst, int ncols) {
    GemmPlan p;
    for (int s = 0; s < parts; ++s) {
      const int64_t k0 = (int64_t)s * step, k1 = std::min<int64_t>(ndet, k0 + step);
      p.add_out(Mp + (size_t)s * n2 * ncols, ncols, n2, ncols, 0);
      if (k1 > k0) p.add_term(D + k0, (int)ndet, W + k0, ldw_is_vec ? 1 : (int)ndet, (int)(k1 - k0),
                              ldw_is_vec ? 0 : 2, 1.0);
    }
    upload(p);
    run(p);
    release(p);
    AxpyPlan ax;
    ax.outs.push_back({dst, (int64_t)n2 * ncols, 0, 0});
    for (int s = 0; s < parts; ++s) ax.terms.push_back({Mp + (size_t)s * n2 * ncols, 1.0});
    ax.outs.back().t1 = (int)ax.terms.size();
    upload(ax);
    run(ax);
    release(ax);
  };
  gram(D, 0, M2, n2);            // <E_qp C | E_rs C>
  gram(C, 1, M2 + (size_t)n2 * n2, 1);   // <E_qp C | C>
  for (int rs = 0; rs < n2; ++rs) {
    launch_apply_e_vecs(D, n2, NaS, NbS, d_excA, d_excB, n2, rs, F, stream);
    stats.launches++;
    CK(cudaGetLastError());
    gram(F, 0, M3 + (size_t)rs * n2 * n2, n2);
  }
  int nblk = reduction_blocks(ndet);
  double* partial = dalloc<double>(nblk);
  double* nrm_d = dalloc<double>(1);
  launch_multi_dot(C, ndet, 1, C, ndet, nrm_d, partial, nblk, stream);
  stats.launches += 2;
  std::vector<double> h3((size_t)n2 * n2 * n2), h2((size_t)n2 * n2 + n2);
  double nrm2 = 0;
  CK(cudaMemcpyAsync(h3.data(), M3, h3.size() * sizeof(double), cudaMemcpyDeviceToHost, stream));
  CK(cudaMemcpyAsync(h2.data(), M2, h2.size() * sizeof(double), cudaMemcpyDeviceToHost, stream));
  CK(cudaMemcpyAsync(&nrm2, nrm_d, sizeof(double), cudaMemcpyDeviceToHost, stream));
  sync();
  stats.d2h += (h3.size() + h2.size() + 1) * sizeof(double);
  for (void* q : {(void*)C, (void*)d_excA, (void*)d_excB, (void*)D, (void*)F, (void*)Mp, (void*)M3, (void*)M2,
                  (void*)partial, (void*)nrm_d})
    dfree(q);
  if (!(nrm2 > 0)) throw Error(-4, "MPS has zero norm in the determinant expansion");
  // gamma_pq = <E_pq> = <E_qp C | C>; Gamma_pqrs = <E_pq E_rs> - d_qr gamma_ps
  std::vector<double> g1(n2), g2((size_t)n2 * n2);
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) g1[p * n + q] = h2[(size_t)n2 * n2 + q * n + p] / nrm2;
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q)
      for (int r = 0; r < n; ++r)
        for (int s2 = 0; s2 < n; ++s2) {
          double v = h2[(size_t)(q * n + p) * n2 + r * n + s2] / nrm2;
          if (q == r) v -= g1[p * n + s2];
          g2[(size_t)(p * n + q) * n2 + r * n + s2] = v;
        }
  auto G2 = [&](int p, int q, int r, int s2) { return g2[(size_t)(p * n + q) * n2 + r * n + s2]; };
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q)
      for (int r = 0; r < n; ++r)
        for (int s2 = 0; s2 < n; ++s2)
          for (int t = 0; t < n; ++t)
            for (int u = 0; u < n; ++u) {
              double v = h3[((size_t)(r * n + s2) * n2 + q * n + p) * n2 + t * n + u] / nrm2;
              if (q == t) v -= G2(p, u, r, s2);
              if (s2 == t) v -= G2(p, q, r, u);
              if (q == r) v -= G2(p, s2, t, u);
              if (q == r && s2 == t) v -= g1[p * n + u];
              out[((((size_t)(p * n + q) * n + r) * n + s2) * n + t) * n + u] = v;
            }
}

// ---------------------------------------------------------------- orbital RDMs
// One- and two-orbital reduced density matrices (the inputs of the orbital
// entropies and the mutual information that order the lattice, Sec.
// "Cholesky decomposition for the wavefunction", ingredient (ii)): rho_ij
// from the determinant expansion by pair_rdm_kernel (fermionic partial trace
// with the pair's modes moved to the front), rho_i as its partial trace.
void Engine::orbital_rdms_ci(double* rho1, double* rho2) {
  int64_t NaS = 0, NbS = 0;
  double* C = expand_ci(NaS, NbS);
  const int64_t ndet = NaS * NbS;
  const int npairs = n * (n - 1) / 2;
  auto sa = strings(n, Na), sb = strings(n, Nb);
  std::vector<int> binom(33 * 33, 0), pairs;
  for (int o = 0; o <= 32; ++o)
    for (int k = 0; k <= 32; ++k) binom[o * 33 + k] = k <= o ? (int)binom_i(o, k) : 0;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) pairs.insert(pairs.end(), {i, j});
  uint32_t* d_sa = dalloc<uint32_t>(sa.size());
  uint32_t* d_sb = dalloc<uint32_t>(sb.size());
  int* d_binom = dalloc<int>(binom.size());
  int* d_pairs = dalloc<int>(std::max<size_t>(pairs.size(), 1));
  CK(cudaMemcpyAsync(d_sa, sa.data(), sa.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(d_sb, sb.data(), sb.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(d_binom, binom.data(), binom.size() * sizeof(int), cudaMemcpyHostToDevice, stream));
  if (!pairs.empty())
    CK(cudaMemcpyAsync(d_pairs, pairs.data(), pairs.size() * sizeof(int), cudaMemcpyHostToDevice, stream));
  const int nb = pair_rdm_blocks(ndet);
  double* partial = dalloc<double>((size_t)std::max(npairs, 1) * nb * 26);
  if (npairs > 0) {
    launch_pair_rdm(C, NaS, NbS, d_sa, d_sb, d_binom, n, Na, d_pairs, npairs, partial, stream);
    stats.launches++;
    CK(cudaGetLastError());
  }
  int nblk = reduction_blocks(ndet);
  double* red = dalloc<double>(nblk);
  double* nrm_d = dalloc<double>(1);
  launch_multi_dot(C, ndet, 1, C, ndet, nrm_d, red, nblk, stream);
  stats.launches += 2;
  std::vector<double> hp((size_t)std::max(npairs, 1) * nb * 26);
  double nrm2 = 0;
  CK(cudaMemcpyAsync(hp.data(), partial, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, stream));
  CK(cudaMemcpyAsync(&nrm2, nrm_d, sizeof(double), cudaMemcpyDeviceToHost, stream));
  sync();
  for (void* q : {(void*)C, (void*)d_sa, (void*)d_sb, (void*)d_binom, (void*)d_pairs, (void*)partial, (void*)red,
                  (void*)nrm_d})
    dfree(q);
  if (!(nrm2 > 0)) throw Error(-4, "MPS has zero norm in the determinant expansion");
  // slots -> (local states): sector (na, nb), variants u (alpha on i / on j
  // when na = 1), v (beta likewise), k = u * nbv + v
  struct Sec { int na, nb, base; };
  const Sec secs[9] = {{0, 0, 0}, {0, 2, 1}, {2, 0, 2}, {2, 2, 3}, {1, 0, 4}, {1, 2, 7}, {0, 1, 10}, {2, 1, 13},
                       {1, 1, 16}};
  auto local = [](int na, int nb, int u, int v) {
    int ai, aj, bi, bj;
    if (na == 1) { ai = u == 0; aj = u == 1; } else { ai = aj = na / 2; }
    if (nb == 1) { bi = v == 0; bj = v == 1; } else { bi = bj = nb / 2; }
    return ai + 2 * bi + 4 * (aj + 2 * bj);
  };
  std::vector<double> r2((size_t)std::max(npairs, 1) * 256, 0.0);
  for (int pr = 0; pr < npairs; ++pr) {
    double slot[26] = {0};
    for (int b = 0; b < nb; ++b)
      for (int t = 0; t < 26; ++t) slot[t] += hp[((size_t)pr * nb + b) * 26 + t];
    double* R = r2.data() + (size_t)pr * 256;
    for (const Sec& sc : secs) {
      const int nav = sc.na == 1 ? 2 : 1, nbv = sc.nb == 1 ? 2 : 1, d = nav * nbv;
      int x[4];
      for (int u = 0, k = 0; u < nav; ++u)
        for (int v = 0; v < nbv; ++v, ++k) x[k] = local(sc.na, sc.nb, u, v);
      int t = sc.base;
      for (int a = 0; a < d; ++a)
        for (int b = a; b < d; ++b, ++t) {
          R[x[a] * 16 + x[b]] = slot[t] / nrm2;
          R[x[b] * 16 + x[a]] = slot[t] / nrm2;
        }
    }
  }
  if (rho2) std::memcpy(rho2, r2.data(), (size_t)npairs * 256 * sizeof(double));
  if (rho1) {
    // rho_i = tr_j rho_ij for a pair containing i (j > i: trace the high
    // index; i = n-1: pair (0, n-1), trace the low one)
    for (int i = 0; i < n; ++i) {
      double* o = rho1 + (size_t)i * 16;
      std::fill(o, o + 16, 0.0);
      if (n < 2) continue;
      const bool low = i < n - 1;
      const int a = low ? i : 0, b = low ? n - 1 : i;
      const int pr = a * n - a * (a + 1) / 2 + (b - a - 1);
      const double* R = r2.data() + (size_t)pr * 256;
      for (int x = 0; x < 4; ++x)
        for (int y = 0; y < 4; ++y)
          for (int z = 0; z < 4; ++z)
            o[x * 4 + y] += low ? R[(x + 4 * z) * 16 + (y + 4 * z)] : R[(z + 4 * x) * 16 + (z + 4 * y)];
    }
  }
}

}  // namespace gbd
