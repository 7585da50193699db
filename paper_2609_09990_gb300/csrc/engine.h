// Sweep engine: the host-side planner and driver of the device kernels.
#pragma once

#include <array>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "gbd_internal.h"
#include "mlp.h"

namespace gbd {

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define CK(x)                                                                                      \
  do {                                                                                             \
    cudaError_t e_ = (x);                                                                          \
    if (e_ != cudaSuccess)                                                                         \
      throw Error(e_ == cudaErrorMemoryAllocation ? -2 : -3,                                      \
                  std::string(#x) + ": " + cudaGetErrorString(e_) + " (line " +                  \
                      std::to_string(__LINE__) + ")");                                             \
  } while (0)


// Enlarged space over a list of sectors Q: E_L(Q) = concat_s (Q - s) from a
// left bond, or E_R(Q) = concat_s (Q + s) from a right bond.
struct Space {
  std::vector<int> qa, qb, dim;
  std::vector<std::array<int, 4>> soff, ssec, sdim;
  QIndex idx;
  int find(int a, int b) const { return idx.get(a, b); }
  int n() const { return (int)qa.size(); }
};

struct Env {          // operator blocks (channel, q_in) of one bond
  int nch = 0, nsec = 0;
  std::vector<int64_t> off;   // nch * nsec, -1 if absent
  std::vector<int> rows, cols;
  double* d = nullptr;
  int64_t size = 0;
  bool valid = false;
  int64_t at(int ch, int sec) const { return off[(size_t)ch * nsec + sec]; }
};

struct EnlSub {       // one sub-block of an enlarged operator
  int b, qin, sin, qout, sout, rows, cols;
  const double* ptr;
  int64_t own_off;    // >= 0: offset into the owned buffer (resolved later)
  double sign;
  int trans = 0;      // 1: the block is sign * (the cols x rows block at ptr)^T (a conjugate channel's)
};
struct EnlOp {
  std::vector<EnlSub> subs;
  double* own = nullptr;
  int64_t own_size = 0;
};

struct Site {         // device tensor of one site; layout 0 = fused-left, 1 = fused-right
  double* d = nullptr;
  int64_t size = 0;
  int layout = 1;
  std::vector<int64_t> off;   // per sector of the key bond (right bond for FL, left bond for FR)
};

struct Weight { double lam; int key, idx, j; };
std::vector<Weight> select_states(std::vector<Weight> w, int M, double cutoff, double tie, double* total,
                                  double max_disc = 0.0, int m_min = 1);
std::vector<Bond> initial_bond_dims(int n, int Na, int Nb, int M);

struct Stats {
  double sigma_flops = 0, sigma_ms = 0, env_flops = 0, env_ms = 0, enl_ms = 0, step_ms = 0;
  double trunc_ms = 0, davidson_ms = 0;
  double sigma_flops_exec = 0, tc_ms = 0, tc_flops = 0, last_residual = 0;
  int64_t n_sigma_tc = 0;
  int64_t n_sigma = 0, n_steps = 0, launches = 0, h2d = 0, d2h = 0;
  int64_t davidson_iters = 0, precond_fallbacks = 0;
  int64_t inner_matvecs = 0;   // sigma builds inside the inner PCG corrections
  int64_t tier_iters[3] = {0, 0, 0};
  double max_final_residual = 0, sum_final_residual = 0;   // over Davidson solves
  int64_t n_solves = 0, n_above_tol = 0;   // Davidson solves, and those that ended with ||r|| >= tol
  double sweep_max_residual = 0;           // largest final ||r|| of the current (or last) sweep
  int64_t graph_launches = 0, autotune_trials = 0;
  double tc_gemm_ms_st[2] = {0, 0};   // tc_gemm_kernel time by stage (A, B)
  double tc_alg_st[2] = {0, 0}, tc_box_st[2][2] = {{0, 0}, {0, 0}}, tc_dense_st[2][2] = {{0, 0}, {0, 0}};   // per stage: algorithmic, TMA box bytes (A, B)
  double tc_gemm_ms = 0, tc_bytes = 0;   // tc_gemm_kernel launches only; algorithmic bytes of the TC sigma builds
  double tc_flops_p[4] = {0, 0, 0, 0}, tc_gemm_ms_p[4] = {0, 0, 0, 0};   // by operand type (BF16, TF32, TF32x3, BF16x3)
  int last_tc_prec = 0;
  double tc_build_ms = 0;   // host wall time building tensor-core plans (incl. autotuning)
  double enl_host_ms = 0, diag_ms = 0;   // host part of the enlarged operators; the H_eff diagonal
  double trunc_rho_ms = 0, trunc_eig_ms = 0;   // decimation: density matrices to the host; host eigensolves
  double env_wall_ms = 0;   // environment update: upload (plan checks) + kernels, wall
  double enl_dev_ms = 0, enl_bytes = 0;   // block-axpy launches of the enlarged operators: device time, bytes
  double tcb_ms[5] = {0, 0, 0, 0, 0};   // plan-build phases: layout/groups, panels, tiles, upload, maps
  double rdm_ms = 0, rdm_env_bytes = 0;   // last rdms(): wall time, peak bytes of its environments
  double h2d_wait_ms = 0;   // host time waiting for a staging-ring region (its earlier copy still queued)
  void add(const Stats& o) {   // sum of the additive counters (batched solves)
    sigma_flops += o.sigma_flops; sigma_ms += o.sigma_ms; env_flops += o.env_flops; env_ms += o.env_ms;
    enl_ms += o.enl_ms; step_ms += o.step_ms; trunc_ms += o.trunc_ms; davidson_ms += o.davidson_ms;
    sigma_flops_exec += o.sigma_flops_exec; tc_ms += o.tc_ms; tc_flops += o.tc_flops;
    n_sigma_tc += o.n_sigma_tc; n_sigma += o.n_sigma; n_steps += o.n_steps; launches += o.launches;
    h2d += o.h2d; d2h += o.d2h; davidson_iters += o.davidson_iters; precond_fallbacks += o.precond_fallbacks;
    inner_matvecs += o.inner_matvecs;
    for (int i = 0; i < 3; ++i) tier_iters[i] += o.tier_iters[i];
    max_final_residual = std::max(max_final_residual, o.max_final_residual);
    sum_final_residual += o.sum_final_residual;
    n_solves += o.n_solves;
    n_above_tol += o.n_above_tol;
    sweep_max_residual = std::max(sweep_max_residual, o.sweep_max_residual);
    graph_launches += o.graph_launches; autotune_trials += o.autotune_trials;
    for (int s = 0; s < 2; ++s) {
      tc_gemm_ms_st[s] += o.tc_gemm_ms_st[s];
      tc_alg_st[s] += o.tc_alg_st[s];
      tc_box_st[s][0] += o.tc_box_st[s][0];
      tc_box_st[s][1] += o.tc_box_st[s][1];
      tc_dense_st[s][0] += o.tc_dense_st[s][0];
      tc_dense_st[s][1] += o.tc_dense_st[s][1];
    }
    tc_gemm_ms += o.tc_gemm_ms; tc_bytes += o.tc_bytes; tc_build_ms += o.tc_build_ms; enl_host_ms += o.enl_host_ms; diag_ms += o.diag_ms;
    trunc_rho_ms += o.trunc_rho_ms; trunc_eig_ms += o.trunc_eig_ms; env_wall_ms += o.env_wall_ms;
    enl_dev_ms += o.enl_dev_ms; enl_bytes += o.enl_bytes;
    rdm_ms += o.rdm_ms; rdm_env_bytes = std::max(rdm_env_bytes, o.rdm_env_bytes);
    h2d_wait_ms += o.h2d_wait_ms;
    for (int i = 0; i < 5; ++i) tcb_ms[i] += o.tcb_ms[i];
    for (int i = 0; i < 4; ++i) { tc_flops_p[i] += o.tc_flops_p[i]; tc_gemm_ms_p[i] += o.tc_gemm_ms_p[i]; }
    max_discarded = std::max(max_discarded, o.max_discarded);
  }   // Davidson iterations: low-precision tier, TF32x3 tier, FP64
  double max_discarded = 0;
};

struct Schedule {
  std::vector<int> M;
  std::vector<double> tol;
  int max_iter = 100, max_space = 24, precision = 0, precond = 0, refine = 0;
  uint64_t seed = 1;
  double cutoff = 1e-12, tie = 1e-10;
};

struct TcPlan;
double now_ms();   // steady-clock wall time
// host threads of the engine's parallel loops on the calling thread (0 = default)
void set_host_threads(int n);

struct TcTune {     // numerics-neutral tile shape of the tensor-core sigma
  int ncap[2] = {256, 256};   // largest N tile of stage A and of stage B (64, 128, 256)
};

struct GraphSeq {   // one captured launch sequence (see Engine::replay)
  cudaGraphExec_t exec = nullptr;
  int calls = 0;
};

namespace opstr {
struct StringSet;
}

class Engine {
 public:
  explicit Engine(int device);
  ~Engine();
  void prepare(int n, int n_elec, int two_sz, int n_chol, const double* h, const double* chol,
               double e_core, const Schedule& sch);
  void init_state();       // initial MPS and environments
  double sweep(int s);     // returns the Ritz value of the last step
  double final_energy();
  // spin-summed 1-/2-RDMs of the current MPS, contracted through the MPS
  // (operator-string environments; rdm_mps.cpp)
  void rdms(double* rdm1, double* rdm2);
  // the same from the determinant expansion (at most 4e8 determinants)
  void rdms_ci(double* rdm1, double* rdm2);
  // spin-summed 3-RDM [n^6] of the current MPS (determinant expansion;
  // needs 2 n^2 determinant-length vectors on the device)
  void rdm3(double* out);
  // one- and two-orbital reduced density matrices of the current MPS:
  // rho1 [n][4][4], rho2 [n(n-1)/2][16][16] for the pairs (i<j) in
  // lexicographic order (local basis of orbital i: |0>, |a>, |b>, |ab> =
  // c+_a^x c+_b^y |vac>, index x + 2y; pair basis index x_i + 4 x_j with the
  // modes of i before those of j), contracted through the MPS (rdm_mps.cpp)
  void orbital_rdms(double* rho1, double* rho2);
  // the same from the determinant expansion
  void orbital_rdms_ci(double* rho1, double* rho2);
  // values <psi|O|psi> / <psi|psi> of many Jordan-Wigner operator strings
  // through operator-string environments (rdm_mps.cpp)
  std::vector<double> eval_strings(opstr::StringSet& S);
  // excited states by penalty deflation: the converged lower states stay
  // resident (both site layouts) and enter every two-site step through
  // overlap environments; sigma gains w sum_j phi_j (phi_j . x) and the
  // diagonal w sum_j phi_j^2, phi_j = the stored state j projected onto the
  // current two-site basis
  void store_state();        // keep the current MPS as a deflated state
  void clear_states();
  void ov_init();            // after init_state: overlap environments of every stored state
  double defl_w = 0.0;       // penalty weight w (Ha)
  // per-bond adaptive bond dimension: discarded-weight target per decimation
  // (0: fixed M) and the smallest bond kept under it
  double adapt_disc = 0.0;
  int adapt_mmin = 1;
  int n_stored() const { return (int)defl.size(); }
  // a device copy of the MPS with the centre at bond (0,1) (after
  // init_state or a full sweep), and the return to it: sites and bonds are
  // copied back and the environments rebuilt, so that several sweeps can
  // start from one state
  void save_state();
  void restore_state();
  bool has_saved_state() const { return !snap_sites.empty(); }
  // debug / test hooks
  void set_mps(const int* nsec, const int* sectors, const double* data, int center);
  int64_t two_site_size(int k);
  void apply_heff(int k, const double* in, double* out, double* diag_out, int prec = 0);
  double run_step(int k, int dir, int M, double tol, double* tau, std::vector<double>* kept);
  void bond_sectors(int bond, std::vector<int>& out) const;
  int mpo_bond_dim(int bond) const { return (int)mpo.labels[bond].size(); }
  std::vector<uint64_t> mpo_labels(int bond) const;
  void env_block(int side, int bond, int channel, int sector, std::vector<double>& out, int& rows, int& cols);
  void multi_dot(const double* V, int64_t stride, int k, const double* x, int64_t n, double* out_host);

  // learned preconditioner
  void record_iteration(const double* r_dev, const double* diag_dev, const double* x_dev, const MlpScalars& s);
  void record_converged(const double* x_dev);
  double train_precond(int epochs, double lr, uint64_t seed);
  void set_precond_weights(const float* params);
  void mlp_loss_grad(const float* X, const float* y, const float* w, int64_t n, const float* params, double lam,
                     double* loss,
                     double* grad);
  void mlp_apply(const double* r, const double* d, double theta, double iter, int64_t n, double* t);
  void save_precond(const char* path) const;
  void load_precond(const char* path);
  bool recording = false;
  bool mlp_loaded = false;
  bool use_graphs = true;     // replay the sigma launch sequences as CUDA graphs
  bool autotune = true;       // pick the tensor-core tile shape per shape class by timing
  int tc_fixed_cap = 0;       // > 0: that N cap for every tensor-core plan (no tuning)
  int pcg_steps = 4;          // inner PCG (preconditioner 3): at most this many matvecs per correction
  double pcg_rel_tol = 0.1;   // ... stopping when |residual| < pcg_rel_tol |r|
  int tc_order = 1;           // stage-B tile order: 0 (q,m0,chunk,n0), 1 (q,chunk,m0,n0), 2 (q,chunk,n0,m0)
  int tc_order_a = 0;         // stage-A tile order: 0 most expensive first, 1 Renl-stack blocks together
  int tc_sout_min = 160;      // stage B: output sectors with E_L(q) >= this many rows split by s_out section
  int tier2 = 2;              // operands of the accurate tier: 2 = TF32x3, 3 = BF16x3 (TcPrec)
  // environment updates of the sweep steps of reduced-precision schedules:
  // -1 = FP64 (default), else on the tensor cores with these operands
  // (TcPrec).  Environments built outside the steps (initial state, saved
  // state, installed MPS, the reported energy) are always FP64.
  int env_prec = -1;
  bool env_tc_used = false;   // the right environments hold tensor-core updates
  bool force_fp64_env = false;
  // certified Hermitian-conjugate channel pairs of the MPO (mpo_conjugates):
  // an environment update computes one channel of each pair and transposes
  // it into the other (env_conj = false: every channel computed)
  std::vector<std::vector<int>> conj_l, sign_l, conj_r, sign_r;
  bool env_conj = true;
  bool env_derived(int bond, int c, bool left) const;
  // sub-blocks of the derived channels of an enlarged operator: the
  // transposes of their partners' (bond: the channels' bond)
  void append_conjugates(EnlOp& op, int bond, bool left) const;
  void env_transposes(Env& out, int bond, bool left);
  // stopping of the accurate tier: a plateau (no 30 % drop over 3
  // iterations) ends it below tier2_floor_mult * u2 * max(1, |theta|);
  // hard_stag_iters > 0: no 30 % drop over that many iterations ends it at
  // any level
  double tier2_floor_mult = 1.0;
  int hard_stag_iters = 8;
  int64_t tc_min_two_site = 4096;   // smaller two-site states: reduced-precision schedules use FP64
  // tier-1 (BF16/TF32) Davidson iterations and steps of the current and the
  // previous sweep: a warm sweep whose predecessor averaged < 2 tier-1
  // iterations per step skips tier 1 (its plan would cost more than it saves)
  int64_t t1_iters_cur = 0, t1_steps_cur = 0, t1_iters_prev = -1, t1_steps_prev = 0;
  bool skip_tier1 = false;
  const std::vector<float>& precond_weights() const { return mlp_f32; }
  int64_t n_samples() const { return (int64_t)data_y.size(); }

  Stats stats;
  std::vector<double> sweep_E;
  int n = 0, Na = 0, Nb = 0;
  double e_core = 0;
  Schedule sched;
  bool prepared = false;

 private:
  int device;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t evg0 = nullptr, evg1 = nullptr;   // around the tensor-core GEMM launches of one sigma
  cudaEvent_t evgm = nullptr;                    // between its stage A and stage B
  std::vector<double> h, eri;
  Mpo mpo;
  std::vector<Bond> bonds;
  std::vector<Site> sites;
  std::vector<Env> Lenv, Renv;
  std::vector<Bond> snap_bonds;   // save_state()
  std::vector<Site> snap_sites;
  void free_snapshot();

  // ---- deflated states and their overlap environments
  struct Ov {                       // <current basis | stored basis> on one bond, per current sector
    std::vector<int64_t> off;       // -1: the stored state has no such sector
    std::vector<int> rows, cols;
    double* d = nullptr;
    int64_t size = 0;
  };
  struct Stored {
    std::vector<Bond> bonds;
    std::vector<Site> fl, fr;       // every site fused-left and fused-right
  };
  std::vector<Stored> defl;
  std::vector<std::vector<Ov>> OLv, ORv;   // [state][bond]
  double* defl_phi = nullptr;       // n_stored x psi_size at the current step
  void free_ov(Ov& o);
  void ov_make(int j, int bond, Ov& o);
  void ov_update_left(int j, int k);    // OLv[j][k+1] from OLv[j][k] and sites[k] (fused-left)
  void ov_update_right(int j, int b);   // ORv[j][b] from ORv[j][b+1] and sites[b] (fused-right)
  void deflation_vectors(int k, double* phi);

  // ---- current two-site step state
  int cur_k = -1;
  Space EL, ER;
  std::vector<int64_t> psi_off;
  int64_t psi_size = 0;
  double* psi = nullptr;

  std::map<uintptr_t, size_t> allocs;   // live device allocations (base -> bytes)
  mutable uintptr_t chk_base = 0;       // last allocation a range check matched
  mutable size_t chk_size = 0;
  int num_sms = 152;
  template <class T>
  T* dalloc(size_t n) {
    void* p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMallocAsync(&p, n * sizeof(T), stream);
    if (e != cudaSuccess) throw Error(-2, std::string("device allocation failed: ") + cudaGetErrorString(e));
    allocs[(uintptr_t)p] = n * sizeof(T);
    return (T*)p;
  }
  void check_range(const void* p, int64_t rows, int64_t cols, int64_t ld, const char* what) const;
  // the same test without the shared cache (safe on several host threads
  // while nothing is allocated or freed): false if the block leaves every
  // live allocation
  struct AllocCache { uintptr_t base = 0; size_t size = 0; };
  bool in_allocation(const void* p, int64_t rows, int64_t cols, int64_t ld, AllocCache& c) const;
  const double* site_block(int i, int qi, int s, int& ld) const;
  void check(const GemmPlan& p) const;
  void check(const AxpyPlan& p) const;
  void dfree(void* p);
  void upload(GemmPlan& p);
  void release(GemmPlan& p);
  void upload(AxpyPlan& p);
  void release(AxpyPlan& p);
  void run(GemmPlan& p);
  void run(AxpyPlan& p);
  void sync();
  void settle();
  // Host-to-device copies of plans and small tensors go through a pinned
  // staging ring, so that they neither wait for the stream (as copies from
  // pageable memory do) nor need a synchronisation before the host buffer
  // is reused: the bytes are copied into the ring at once, and a region is
  // reused only after the event recorded behind its copy has completed.
  // Copies larger than a quarter of the ring take the pageable path.
  uint8_t* pin_ring = nullptr;
  size_t pin_cap = 0;
  uint64_t pin_pos = 0;                    // bytes staged so far (absolute position)
  struct PinUse { uint64_t start, end; cudaEvent_t ev; };
  std::deque<PinUse> pin_inflight;
  std::vector<cudaEvent_t> ev_pool;        // timing-disabled events for the ring
  cudaEvent_t pool_event();
  void h2d(void* dst, const void* src, size_t bytes);
  // environment-update launches timed by event pairs, read after the next
  // stream synchronisation (no synchronisation of their own)
  struct EnvTimer { cudaEvent_t a, b; double* acc; };   // acc: the stats counter the time goes to
  std::vector<EnvTimer> env_timers;
  std::vector<cudaEvent_t> timer_pool;     // timing events for env_timers
  void drain_timers();
  void timed_env_launch(GemmPlan& p1, GemmPlan& p2);
  // a GemmPlan (every output overwritten) on the tensor cores, operands in
  // precision prec (TcPrec), split-K FP64 sums (gemm_tc.cpp)
  void run_tc(GemmPlan& p, int prec);
  int* d_env_err = nullptr;      // bounded-wait flag of the tensor-core environment updates
  bool env_tc_pending = false;   // such launches since the last check of the flag
  EnvTimer timer_begin(double* acc);
  void timer_end(EnvTimer t);
  int sigma_pending = 0;          // 1: FP64 sigma, 2: tensor-core sigma awaiting accounting
  int* tc_err_host = nullptr;     // pinned copy of the tensor-core error flag

  void free_env(Env& e);
  void make_env(int bond, Env& e);
  Space left_space(const Bond& bl, const std::vector<std::pair<int, int>>& Qs) const;
  Space right_space(const Bond& br, const std::vector<std::pair<int, int>>& Qs) const;
  std::vector<std::pair<int, int>> bond_qs(const Bond& b) const;
  void layout_site(int i, int layout, Site& s) const;
  void free_site(Site& s);
  void build_lenl(int k, const Env& Lk, const Space& el, EnlOp& op, AxpyPlan& ax);
  void build_renl(int i, const Env& Ri1, const Space& er, EnlOp& op, AxpyPlan& ax);
  void finish_enl(EnlOp& op, AxpyPlan& ax);
  void free_enl(EnlOp& op);
  void env_update_left(const EnlOp& lenl, const Space& el, const Site& A, const Bond& bnew, Env& out);
  void env_update_right(const EnlOp& renl, const Space& er, const Site& B, const Bond& bnew, Env& out);
  void setup_two_site(int k);
  void form_psi(int k, int pattern);
  struct Sigma;
  void plan_sigma(const EnlOp& lenl, const EnlOp& renl, Sigma& sg);
  void sigma(Sigma& sg, const double* x, double* y);
  void compute_diag(const EnlOp& lenl, const EnlOp& renl, double* diag);
  // stag_rel > 0: stop on stagnation (reduced-precision operators); see the definition
  double davidson(const std::function<void(const double*, double*)>& op, const double* diag, double tol,
                  int max_iter, int max_space, double stag_rel);
  // the Davidson solve of one step in schedule precision `precision` with at
  // most `refine` FP64 iterations; the Ritz vector is left in psi
  double solve_tiers(Sigma& sg, const double* diag, double tol, int precision, int refine, bool& planned);
  void free_sigma(Sigma& sg, bool planned);
  struct CanonMap { int64_t src, dst; int rows, cols, ld; };
  std::vector<CanonMap> canonical_maps(int k) const;
  void to_fused(const std::vector<CanonMap>& maps, const double* in, double* out) const;
  void from_fused(const std::vector<CanonMap>& maps, const double* in, double* out) const;
  void inner_pcg(const std::function<void(const double*, double*)>& op, const double* diag, const double* xr,
                 const double* rr_vec, double th, double* tout, double* cg, double* partial, int nblk, double* dsums);
  TcPlan* tc_build(const EnlOp& lenl, const EnlOp& renl, int prec, TcTune tune = TcTune());
  TcPlan* tc_plan(const EnlOp& lenl, const EnlOp& renl, int prec);   // tc_build with the tuned shape
  TcPlan* tc_plan_impl(const EnlOp& lenl, const EnlOp& renl, int prec);
  std::map<int64_t, TcTune> tuned;
  void tc_apply(TcPlan* p, const double* x, double* y);
  void tc_free(TcPlan* p);
  void truncate(int k, int dir, int M, double* tau, std::vector<double>* kept);
  // A fixed launch sequence on `stream`: run directly on its first use,
  // captured into a CUDA graph on the second, replayed from then on.
  template <class F>
  void replay(GraphSeq& g, F&& launches) {
    if (!use_graphs || g.calls++ == 0) {
      launches();
      return;
    }
    if (!g.exec) {
      cudaGraph_t graph;
      CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
      launches();
      CK(cudaStreamEndCapture(stream, &graph));
      cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
      cudaGraphDestroy(graph);
      CK(e);
    }
    CK(cudaGraphLaunch(g.exec, stream));
    stats.graph_launches++;
  }
  static void drop(GraphSeq& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.calls = 0;
  }
  double step(int k, int dir, int M, double tol, double* tau, std::vector<double>* kept);

 public:
  // Davidson at the current centre k in the given schedule precision
  // without decimation or environment update: Ritz value, and the FP64
  // Rayleigh quotient and FP64 residual norm of the resulting vector
  void probe_step(int k, int precision, int refine, double tol, double* theta, double* e64, double* r64);
  void gemm_tc_selftest(int M, int N, int K, int nterms, int flags, int prec, uint64_t seed, double* max_err,
                        double* max_ref);
  // the inner-PCG correction of the Davidson solver at centre k with the
  // FP64 sigma and the step's own H_eff diagonal, from host x, r and theta
  void pcg_selftest(int k, const double* x_host, const double* r_host, double theta, double* t_host,
                    int64_t* matvecs);

 private:
  void init_mps(uint64_t seed, int M);
  double* expand_ci(int64_t& Na_str, int64_t& Nb_str);
  void build_right_envs(int from_k);
  void build_left_envs(int to_k);
  struct Rec {
    MlpScalars s;
    std::vector<double> r, d, x;
  };
  std::vector<Rec> rec_iters;
  std::vector<int64_t> rec_idx;
  int64_t rec_n = 0;
  std::vector<float> data_X, data_y, data_w, mlp_f32;
  uint16_t* mlp_w16 = nullptr;
};

}  // namespace gbd
