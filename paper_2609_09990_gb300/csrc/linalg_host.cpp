// Small dense FP64 linear algebra on the host: the Rayleigh-Ritz
// eigenproblem of Davidson (k <= ~24) and the per-sector reduced density
// matrices of the decimation step (edges of a few hundred).
//
// Symmetric eigensolver: Householder reduction to tridiagonal form followed
// by the implicit-shift QL iteration (Wilkinson & Reinsch, Handbook for
// Automatic Computation II, 1971), written from the algorithm's description.
#include <algorithm>
#include <array>
#include <cmath>
#include <numeric>
#include <vector>

#include "linalg_host.h"

namespace gbd {

namespace {
// [0, count) in nblk contiguous blocks, on the host pool when par; every
// element is handled by exactly one block in the serial order
template <class F>
void blocks(bool par, int count, F&& f) {
  if (!par || count < 64) {
    f(0, count);
    return;
  }
  // block edges on multiples of 8 doubles (64-byte lines): no two threads
  // write the same cache line of a row
  const int nblk = std::min(16, count / 32);
  auto edge = [&](int b) { return b == nblk ? count : (int)((int64_t)count * b / nblk) / 8 * 8; };
  host_parallel_for(nblk, [&](int b) { f(edge(b), edge(b + 1)); });
}
constexpr int kParallelEig = 160;   // matrices at least this large split their O(n^2) loops
}  // namespace

// Householder tridiagonalisation of A (n x n symmetric, row-major):
// d, e the diagonal and sub-diagonal of T = Q^T A Q, Q = H_0 H_1 ... H_{n-3}
// with H_k = I - beta_k v_k v_k^T acting on rows k+1 .. n-1 (v_k empty and
// beta_k = 0 for an identity step)
static void tridiagonalize(int n, const double* A, bool par, std::vector<double>& d, std::vector<double>& e,
                           std::vector<std::vector<double>>& refl, std::vector<double>& beta_l) {
  // only the lower triangle of the working copy is read and updated
  std::vector<double> a(A, A + (size_t)n * n);
  d.assign(n, 0.0);
  e.assign(n, 0.0);
  refl.clear();
  beta_l.clear();
  std::vector<double> p, pp;
  for (int k = 0; k + 2 < n; ++k) {
    int m = n - k - 1;
    std::vector<double> v(m);
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) { v[i] = a[(size_t)(k + 1 + i) * n + k]; nrm += v[i] * v[i]; }
    nrm = std::sqrt(nrm);
    double alpha = v[0] > 0 ? -nrm : nrm;
    double vv = 0.0;
    v[0] -= alpha;
    for (int i = 0; i < m; ++i) vv += v[i] * v[i];
    if (vv == 0.0 || nrm == 0.0) {
      refl.push_back({});
      beta_l.push_back(0.0);
      continue;
    }
    double beta = 2.0 / vv;
    // p = beta * A22 v from the lower triangle: row i contributes
    // A_ij v_j to p_i and A_ij v_i to p_j (j < i).  Row blocks of equal
    // triangle area, each with its own accumulator, summed in block order.
    const int nblk = (par && m >= 256) ? std::min(16, m / 32) : 1;
    auto edge = [&](int bb) { return bb >= nblk ? m : (int)(m * std::sqrt((double)bb / nblk)); };
    pp.assign((size_t)nblk * m, 0.0);
    auto rows = [&](int bb) {
      double* acc = &pp[(size_t)bb * m];
      for (int i = edge(bb); i < edge(bb + 1); ++i) {
        const double* row = &a[(size_t)(k + 1 + i) * n + k + 1];
        const double vi = v[i];
        double s = 0.0;
        for (int j = 0; j < i; ++j) {
          s += row[j] * v[j];
          acc[j] += row[j] * vi;
        }
        acc[i] += s + row[i] * vi;
      }
    };
    if (nblk > 1) host_parallel_for(nblk, rows);
    else rows(0);
    p.assign(m, 0.0);
    for (int bb = 0; bb < nblk; ++bb)
      for (int i = 0; i < m; ++i) p[i] += pp[(size_t)bb * m + i];
    for (int i = 0; i < m; ++i) p[i] *= beta;
    double K = 0.0;
    for (int i = 0; i < m; ++i) K += v[i] * p[i];
    K *= 0.5 * beta;
    for (int i = 0; i < m; ++i) p[i] -= K * v[i];   // w
    // A22 -= v w^T + w v^T on the lower triangle
    auto upd = [&](int bb) {
      for (int i = edge(bb); i < edge(bb + 1); ++i) {
        double* row = &a[(size_t)(k + 1 + i) * n + k + 1];
        const double vi = v[i], wi = p[i];
        for (int j = 0; j <= i; ++j) row[j] -= vi * p[j] + wi * v[j];
      }
    };
    if (nblk > 1) host_parallel_for(nblk, upd);
    else upd(0);
    a[(size_t)(k + 1) * n + k] = alpha;
    for (int i = 1; i < m; ++i) a[(size_t)(k + 1 + i) * n + k] = 0.0;
    refl.push_back(v);
    beta_l.push_back(beta);
  }
  for (int i = 0; i < n; ++i) d[i] = a[(size_t)i * n + i];
  for (int i = 0; i + 1 < n; ++i) e[i] = a[(size_t)(i + 1) * n + i];
}

// implicit QL on the tridiagonal (d, e) (Wilkinson & Reinsch): d becomes
// the eigenvalues (unsorted); rot, if given, receives (row, s, c) of every
// rotation in order, which applied to the columns of Q give the
// eigenvectors.  An off-diagonal element is negligible when it is below eps
// relative to its neighbours or below eps * ||T|| (backward-stable absolute
// deflation; density matrices have many eigenvalues near zero where a purely
// relative test stalls).  0, or -1 without convergence.
static int ql_iterate(int n, std::vector<double>& d, std::vector<double>& e,
                      std::vector<std::array<double, 3>>* rot) {
  const double eps = 2.220446049250313e-16;
  double anorm = 0.0;
  for (int i = 0; i < n; ++i) anorm = std::max(anorm, std::fabs(d[i]) + std::fabs(e[i]) + (i ? std::fabs(e[i - 1]) : 0.0));
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    while (true) {
      int m = l;
      for (; m < n - 1; ++m) {
        double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
        if (std::fabs(e[m]) <= eps * dd || std::fabs(e[m]) <= eps * anorm) break;
      }
      if (m == l) break;
      if (++iter > 200) return -1;
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
      double s = 1.0, c = 1.0, p = 0.0;
      int i = m - 1;
      bool early = false;
      for (; i >= l; --i) {
        double f = s * e[i], b = c * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= p;
          e[m] = 0.0;
          early = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
        if (rot) rot->push_back({(double)i, s, c});
      }
      if (early) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  return 0;
}

// A: n x n symmetric, row-major.  On return w ascending, Z column j = eigvec j.
// Large matrices run the row / column loops of each phase in parallel
// blocks; every element sees the same operations in the same order.
int sym_eig(int n, const double* A, double* w, double* Z) {
  if (n <= 0) return 0;
  const bool par = n >= kParallelEig;
  std::vector<double> d, e;
  std::vector<std::vector<double>> refl;
  std::vector<double> beta_l;
  tridiagonalize(n, A, par, d, e, refl, beta_l);
  // ---- Q = H_0 H_1 ... H_{n-3}, built from the right; each column block
  // of z takes every reflector in turn (the columns are independent)
  std::vector<double> z((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) z[(size_t)i * n + i] = 1.0;
  blocks(par, n, [&](int j0, int j1) {
    std::vector<double> t(n, 0.0);
    for (int k = (int)refl.size() - 1; k >= 0; --k) {
      if (beta_l[k] == 0.0) continue;
      const std::vector<double>& v = refl[k];
      const int m = (int)v.size(), o = k + 1;
      // z[o:, cols] -= beta v (v^T z[o:, cols])
      for (int j = j0; j < j1; ++j) t[j] = 0.0;
      for (int i = 0; i < m; ++i) {
        const double* row = &z[(size_t)(o + i) * n];
        for (int j = j0; j < j1; ++j) t[j] += v[i] * row[j];
      }
      for (int i = 0; i < m; ++i) {
        double* row = &z[(size_t)(o + i) * n];
        const double f = beta_l[k] * v[i];
        for (int j = j0; j < j1; ++j) row[j] -= f * t[j];
      }
    }
  });
  // ---- implicit QL on (d, e), rotating the columns of z, kept transposed
  // (zt row j = column j of z) so that a rotation touches two contiguous rows
  std::vector<double> zt((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) zt[(size_t)j * n + i] = z[(size_t)i * n + j];
  std::vector<std::array<double, 3>> rot;   // (row, s, c) of every QL rotation, in order
  if (ql_iterate(n, d, e, &rot) != 0) return -1;
  // every rotation of the QL iterations, in order, on column blocks of zt
  // (the recurrences for d and e never read the eigenvectors)
  blocks(par, n, [&](int k0, int k1) {
    for (const auto& R : rot) {
      double* zi = &zt[(size_t)R[0] * n];
      double* zi1 = zi + n;
      const double rs = R[1], rc = R[2];
      for (int k = k0; k < k1; ++k) {
        const double zf = zi1[k];
        zi1[k] = rs * zi[k] + rc * zf;
        zi[k] = rc * zi[k] - rs * zf;
      }
    }
  });
  // ---- sort ascending
  std::vector<int> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return d[x] < d[y]; });
  for (int j = 0; j < n; ++j) {
    w[j] = d[ord[j]];
    const double* src = &zt[(size_t)ord[j] * n];
    for (int i = 0; i < n; ++i) Z[(size_t)i * n + j] = src[i];
  }
  return 0;
}

// Rows of M (m x c, m <= c) -> M = Lo Q with Q orthonormal rows (Gram-Schmidt
// applied twice per row).  Lo is m x m lower triangular.
int row_orthonormalize(int m, int c, double* M, double* Lo) {
  std::fill(Lo, Lo + (size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) {
    double* mi = M + (size_t)i * c;
    for (int pass = 0; pass < 2; ++pass) {
      for (int j = 0; j < i; ++j) {
        const double* qj = M + (size_t)j * c;
        double r = 0.0;
        for (int t = 0; t < c; ++t) r += qj[t] * mi[t];
        for (int t = 0; t < c; ++t) mi[t] -= r * qj[t];
        Lo[(size_t)i * m + j] += r;
      }
    }
    double nrm = 0.0;
    for (int t = 0; t < c; ++t) nrm += mi[t] * mi[t];
    nrm = std::sqrt(nrm);
    if (nrm < 1e-300) return -1;
    for (int t = 0; t < c; ++t) mi[t] /= nrm;
    Lo[(size_t)i * m + i] = nrm;
  }
  return 0;
}

}  // namespace gbd
