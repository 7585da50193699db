// Internal data structures of the DMRG sweep engine (host + device).
//
// Quantum numbers: every bond k (0..n) is labelled by the particle numbers
// q = (N_alpha, N_beta) of the left block (sites < k).  Local site states are
// [0, alpha, beta, alpha+beta] with quantum numbers QA/QB below.
//
// Layouts (all row-major FP64 on the device unless stated):
//   environment block  (channel a, sector q_in) -> m(q_in + delta_a) x m(q_in)
//   two-site state     one dense block per middle sector Q of bond k+1:
//                      rows = enlarged left  E_L(Q) = concat_s (q_l = Q - s, s)
//                      cols = enlarged right E_R(Q) = concat_s (s, q_r = Q + s)
//   left-canonical A_k fused-left per sector Q of bond k+1: m_EL(Q) x m_{k+1}(Q)
//   right-canonical B_k fused-right per sector q of bond k: m_k(q) x m_ER(q)
#pragma once

#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

namespace gbd {

constexpr int QA[4] = {0, 1, 0, 1};
constexpr int QB[4] = {0, 0, 1, 1};
constexpr int PAR[4] = {0, 1, 1, 0};

inline int qkey(int a, int b) { return a * 64 + b; }

// sector index by (N_alpha, N_beta), both in [0, 63]: a dense 64 x 64 table
struct QIndex {
  std::vector<int> t;
  void clear() { t.assign(64 * 64, -1); }
  void set(int a, int b, int v) {
    if (t.empty()) clear();
    t[a * 64 + b] = v;
  }
  int get(int a, int b) const {
    if (a < 0 || b < 0 || a > 63 || b > 63 || t.empty()) return -1;
    return t[a * 64 + b];
  }
};

struct Bond {
  std::vector<int> na, nb, dim;   // sorted by (na, nb)
  std::vector<int64_t> off;        // prefix offsets of dims
  QIndex idx;
  void finalize();
  int find(int a, int b) const { return idx.get(a, b); }
  int nsec() const { return (int)na.size(); }
  int64_t total() const { return off.empty() ? 0 : off.back(); }
};

// ---------------------------------------------------------------- MPO
// Channel labels: kind 0 = I, 1 = H, 2 = bare (left operators fixed),
// 3 = complementary (right operators fixed); up to two operator codes
// code = site*4 + spin*2 + (creator ? 0 : 1).  key orders labels.
struct Label {
  int kind = 0, nops = 0, c0 = 0, c1 = 0;
  uint64_t key() const {
    return ((uint64_t)kind << 40) | ((uint64_t)nops << 32) | ((uint64_t)c0 << 16) | (uint64_t)c1;
  }
};

struct MpoEntry {       // one nonzero local matrix element of W_i[a,b]
  int a, b, sout, sin;
  double v;
};

struct Mpo {
  int n = 0, k_switch = 0;
  std::vector<std::vector<Label>> labels;          // per bond
  std::vector<std::vector<int>> dA, dB, parity;    // per bond per channel
  std::vector<std::vector<MpoEntry>> W;            // per site, dressed, sorted by (b, a, sout, sin)
  std::vector<int> ident_channel;                  // per bond: index of 'I' (-1 if absent)
  std::vector<int> ham_channel;                    // per bond: index of 'H' (-1 if absent)
};

void build_mpo(int n, const double* h, const double* eri, int k_switch, Mpo& out);
// certified Hermitian-conjugate channel pairs per bond: cl/cr[bond][c] = the
// partner d with L[d] = sl[c] L[c]^T (R[d] = sr[c] R[c]^T), c itself for a
// self-conjugate or zero channel, -1 when none is certified
void mpo_conjugates(const Mpo& m, std::vector<std::vector<int>>& cl, std::vector<std::vector<int>>& sl,
                    std::vector<std::vector<int>>& cr, std::vector<std::vector<int>>& sr);

// ---------------------------------------------------------------- grouped GEMM
// C[out] = beta * C + sum_terms alpha * op(A) op(B), op = transpose if flag.
struct GemmTerm {
  const double* A;
  const double* B;
  int32_t lda, ldb, K, flags;   // flags: 1 = transA, 2 = transB
  double alpha;
};
struct GemmOut {
  double* C;
  int32_t ldc, M, N;
  int32_t t0, t1;   // term range
  int32_t beta;     // 0 = overwrite, 1 = accumulate
  int32_t pad;
};
struct GemmTile {
  int32_t out, tm, tn, pad;
};

struct GemmPlan {       // host side lists plus their device copies
  std::vector<GemmTerm> terms;
  std::vector<GemmOut> outs;
  std::vector<GemmTile> tiles;   // 32 x 32 register-blocked tiles
  std::vector<GemmTile> flat;    // {out, -1, first element, 0}: 256 elements, one per thread
  GemmTerm* d_terms = nullptr;
  GemmOut* d_outs = nullptr;
  GemmTile* d_tiles = nullptr;
  GemmTile* d_flat = nullptr;
  double flops = 0.0;       // 2 m n k summed over terms
  void clear() { terms.clear(); outs.clear(); tiles.clear(); flat.clear(); flops = 0.0; }
  int add_out(double* C, int ldc, int M, int N, int beta) {
    GemmOut o{C, ldc, M, N, (int)terms.size(), (int)terms.size(), beta, 0};
    outs.push_back(o);
    return (int)outs.size() - 1;
  }
  void add_term(const double* A, int lda, const double* B, int ldb, int K, int flags, double alpha) {
    GemmTerm t{A, B, lda, ldb, K, flags, alpha};
    terms.push_back(t);
    GemmOut& o = outs.back();
    o.t1 = (int)terms.size();
    flops += 2.0 * o.M * o.N * K;
  }
};

// Block axpy: out[i] = sum_j coef_j * src_j[i] over equally sized blocks.
struct AxpyTerm { const double* src; double coef; };
struct AxpyOut { double* dst; int64_t len; int32_t t0, t1; };
struct AxpyPlan {
  std::vector<AxpyTerm> terms;
  std::vector<AxpyOut> outs;
  std::vector<int64_t> cstart;   // first work chunk of every output (upload fills it)
  AxpyTerm* d_terms = nullptr;
  AxpyOut* d_outs = nullptr;
  int64_t* d_cstart = nullptr;
  int64_t nchunks = 0;
  double bytes = 0;              // 8 (terms + 1) len summed over the outputs
  void clear() { terms.clear(); outs.clear(); cstart.clear(); nchunks = 0; bytes = 0; }
};
constexpr int kAxpyChunk = 1024;   // output elements per work chunk of the block axpy

// ---------------------------------------------------------------- kernels (kernels.cu)
void launch_gemm_f64(const GemmPlan& p, cudaStream_t s);
void launch_axpy(const AxpyPlan& p, cudaStream_t s);
void launch_set_identity(double* d, int m, cudaStream_t s);
// dst = sign * src^T for blocks src (rows x cols, row-major, dense); one
// 32 x 32 tile per item
struct TransTask { const double* src; double* dst; int32_t rows, cols; double sign; };
struct TransTile { int32_t task, r0, c0, pad; };
void launch_block_transpose(const TransTask* tasks, const TransTile* tiles, int ntiles, cudaStream_t s);
// Davidson vector ops (vectors V_j = V + j * stride)
void launch_multi_dot(const double* V, int64_t stride, int k, const double* x, int64_t n, double* out_dev,
                      double* partial, int nblk, cudaStream_t s);
void launch_lincomb(double* out, const double* V, int64_t stride, const double* coef_dev, int k, int64_t n,
                    int accumulate, cudaStream_t s, double coef_scale = 1.0);
void launch_normalize(const double* t, const double* nrm2_dev, int64_t n, double* out, cudaStream_t s);
// *out = max_i |x_i| (out is overwritten)
void launch_absmax(const double* x, int64_t n, double* out, cudaStream_t s);
void launch_residual_precond(const double* x, const double* sx, const double* diag, double theta, int64_t n,
                             double* r, double* t, double* partial, int nblk, double* out_dev, cudaStream_t s);
void launch_scale(double* x, double a, int64_t n, cudaStream_t s);
// out = K^-1 (scale v) - (x . K^-1 scale v)/(x . K^-1 x) K^-1 x with K = the
// guarded d - theta (x . out = 0): the Olsen correction for v = r, scale -1,
// and the preconditioner of the inner PCG.  Three launches, no host sync;
// partial holds 2 * nblk doubles, sums_dev 2.
void launch_projected_precond(const double* v, const double* x, const double* diag, double theta, double scale,
                              int64_t n, double* out, double* partial, int nblk, double* sums_dev, cudaStream_t s);
// y = a x + b y
void launch_axpby(double* y, double a, const double* x, double b, int64_t n, cudaStream_t s);
// d[i] += w sum_j phi[j * n + i]^2 (j < k)
void launch_add_sq(double* d, const double* phi, int k, int64_t n, double w, cudaStream_t s);
int reduction_blocks(int64_t n);

}  // namespace gbd
