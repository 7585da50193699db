// C ABI of the sweep engine: argument validation, error codes, and the
// translation of exceptions into status codes (none crosses the boundary).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#include "../../include/gbdmrg.h"
#include "../../include/gbdmrg_test.h"
#include "engine.h"
#include "linalg_host.h"
#include "tc_gemm.h"

namespace gbd {
double mps_init_value(uint64_t seed, int site, int na, int nb, int s, int row, int col);
}

struct gbd_ctx {
  int device = 0;
  std::unique_ptr<gbd::Engine> eng;
  std::string err;
  int batch_workers = 0;
  bool graphs = true;
  gbd::Stats batch_stats;   // summed over the workers of the last batched solve
};

namespace {

int fail(gbd_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

template <class F>
int guarded(gbd_ctx* c, F&& f) {
  if (!c) return GBD_ERR_ARG;
  try {
    c->err.clear();
    return f();
  } catch (const gbd::Error& e) {
    return fail(c, e.code, e.what());
  } catch (const std::bad_alloc&) {
    return fail(c, GBD_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(c, GBD_ERR_CUDA, e.what());
  }
}

int validate(gbd_ctx* c, const gbd_problem* p, const gbd_schedule* s) {
  if (!p || !s) return fail(c, GBD_ERR_ARG, "problem or schedule is NULL");
  int n = p->n_orb;
  if (n < 2 || n > 32) return fail(c, GBD_ERR_ARG, "n_orb must be in [2, 32]");
  if (p->n_elec < 0 || p->n_elec > 2 * n) return fail(c, GBD_ERR_ARG, "n_elec outside [0, 2 n_orb]");
  if (((p->n_elec - p->two_sz) % 2) != 0) return fail(c, GBD_ERR_ARG, "n_elec and two_sz parity differ");
  int lim = std::min(p->n_elec, 2 * n - p->n_elec);
  if (std::abs(p->two_sz) > lim) return fail(c, GBD_ERR_ARG, "|two_sz| too large for n_elec");
  if (p->n_chol < 0) return fail(c, GBD_ERR_ARG, "n_chol < 0");
  if (!p->h || (p->n_chol > 0 && !p->chol)) return fail(c, GBD_ERR_ARG, "h or chol is NULL");
  if (!std::isfinite(p->e_core)) return fail(c, GBD_ERR_ARG, "e_core not finite");
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double a = p->h[i * n + j], b = p->h[j * n + i];
      if (!std::isfinite(a)) return fail(c, GBD_ERR_ARG, "h has NaN/Inf");
      if (std::fabs(a - b) > 1e-12) return fail(c, GBD_ERR_ARG, "h is not symmetric");
    }
  for (int Q = 0; Q < p->n_chol; ++Q)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double a = p->chol[((size_t)Q * n + i) * n + j], b = p->chol[((size_t)Q * n + j) * n + i];
        if (!std::isfinite(a)) return fail(c, GBD_ERR_ARG, "chol has NaN/Inf");
        if (std::fabs(a - b) > 1e-12) return fail(c, GBD_ERR_ARG, "chol slice is not symmetric");
      }
  if (s->n_sweeps < 1 || !s->bond_dim || !s->davidson_tol) return fail(c, GBD_ERR_ARG, "empty sweep schedule");
  for (int i = 0; i < s->n_sweeps; ++i) {
    if (s->bond_dim[i] < 1) return fail(c, GBD_ERR_ARG, "bond_dim < 1");
    if (!(s->davidson_tol[i] > 0) || !std::isfinite(s->davidson_tol[i]))
      return fail(c, GBD_ERR_ARG, "davidson_tol must be positive");
  }
  if (s->davidson_max_iter < 0 || s->davidson_max_subspace < 0) return fail(c, GBD_ERR_ARG, "negative Davidson limit");
  if (s->davidson_max_subspace != 0 && s->davidson_max_subspace < 5)
    return fail(c, GBD_ERR_ARG, "davidson_max_subspace must be >= 5");
  if (s->precision != GBD_FP64 && s->precision != GBD_TF32 && s->precision != GBD_BF16)
    return fail(c, GBD_ERR_ARG, "unknown precision");
  if (s->fp64_refine < 0) return fail(c, GBD_ERR_ARG, "fp64_refine < 0");
  if (s->preconditioner < GBD_PRECOND_DIAG || s->preconditioner > GBD_PRECOND_PCG)
    return fail(c, GBD_ERR_ARG, "unknown preconditioner");
  if (s->svd_cutoff < 0 || !std::isfinite(s->svd_cutoff)) return fail(c, GBD_ERR_ARG, "svd_cutoff invalid");
  return GBD_OK;
}

gbd::Schedule to_schedule(const gbd_schedule* s) {
  gbd::Schedule out;
  for (int i = 0; i < s->n_sweeps; ++i) {
    out.M.push_back(s->bond_dim[i]);
    out.tol.push_back(s->davidson_tol[i]);
  }
  out.max_iter = s->davidson_max_iter > 0 ? s->davidson_max_iter : 100;
  out.max_space = s->davidson_max_subspace > 0 ? s->davidson_max_subspace : 24;
  out.precision = s->precision;
  out.precond = s->preconditioner;
  out.seed = s->seed;
  out.cutoff = s->svd_cutoff > 0 ? s->svd_cutoff : 1e-12;
  out.refine = s->fp64_refine;
  return out;
}

// estimated cost of one active space: n_orb x M_max^3 x sweeps
double problem_cost(const gbd_problem& p, const gbd_schedule& s) {
  int mmax = 1;
  for (int k = 0; k < s.n_sweeps; ++k) mmax = std::max(mmax, s.bond_dim[k]);
  return (double)p.n_orb * mmax * (double)mmax * mmax * s.n_sweeps;
}

int setup(gbd_ctx* c, const gbd_problem* p, const gbd_schedule* s) {
  int rc = validate(c, p, s);
  if (rc != GBD_OK) return rc;
  if (!c->eng) c->eng.reset(new gbd::Engine(c->device));
  c->eng->prepare(p->n_orb, p->n_elec, p->two_sz, p->n_chol, p->h, p->chol, p->e_core, to_schedule(s));
  return GBD_OK;
}

}  // namespace

extern "C" {

int gbd_create(gbd_ctx** ctx, int device_ordinal) {
  if (!ctx) return GBD_ERR_ARG;
  *ctx = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return GBD_ERR_CUDA;
  if (device_ordinal < 0 || device_ordinal >= ndev) return GBD_ERR_ARG;
  gbd_ctx* c = new (std::nothrow) gbd_ctx;
  if (!c) return GBD_ERR_OOM;
  c->device = device_ordinal;
  *ctx = c;
  return GBD_OK;
}

void gbd_destroy(gbd_ctx* ctx) {
  if (!ctx) return;
  try {
    ctx->eng.reset();
  } catch (...) {
  }
  delete ctx;
}

const char* gbd_last_error(const gbd_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

namespace {
// the whole schedule of one prepared problem on engine e
void run_solve(gbd::Engine& e, const gbd_problem* p, const gbd_schedule* s, gbd_result* r) {
  e.init_state();
  for (int i = 0; i < s->n_sweeps; ++i) {
    double en = e.sweep(i);
    if (r->sweep_energies) r->sweep_energies[i] = en + p->e_core;
  }
  r->energy = e.final_energy() + p->e_core;
  if (r->rdm1 || r->rdm2) e.rdms(r->rdm1, r->rdm2);
  r->max_discarded_weight = e.stats.max_discarded;
  r->n_matvec = e.stats.n_sigma;
  r->status = GBD_OK;
}
}  // namespace

int gbd_solve(gbd_ctx* ctx, const gbd_problem* p, const gbd_schedule* s, gbd_result* r) {
  return guarded(ctx, [&]() {
    if (!r) return fail(ctx, GBD_ERR_ARG, "result is NULL");
    int rc = setup(ctx, p, s);
    if (rc != GBD_OK) return rc;
    gbd::Engine& e = *ctx->eng;
    if (s->preconditioner == GBD_PRECOND_LEARNED && !e.mlp_loaded)
      return fail(ctx, GBD_ERR_STATE, "learned preconditioner requested but no weights are loaded");
    run_solve(e, p, s, r);
    return GBD_OK;
  });
}

int gbd_solve_states(gbd_ctx* ctx, const gbd_problem* p, const gbd_schedule* s, int32_t n_states, double penalty,
                     double target_s2, int32_t max_extra, gbd_result* results, double* s2, int32_t* n_found) {
  return guarded(ctx, [&]() {
    if (!results || !s2 || !n_found) return fail(ctx, GBD_ERR_ARG, "results, s2 or n_found is NULL");
    if (n_states < 1 || max_extra < 0) return fail(ctx, GBD_ERR_ARG, "n_states < 1 or max_extra < 0");
    if (!(penalty > 0) || !std::isfinite(penalty) || !std::isfinite(target_s2))
      return fail(ctx, GBD_ERR_ARG, "penalty must be positive and finite");
    *n_found = 0;
    int rc = setup(ctx, p, s);
    if (rc != GBD_OK) return rc;
    gbd::Engine& e = *ctx->eng;
    if (s->preconditioner == GBD_PRECOND_LEARNED && !e.mlp_loaded)
      return fail(ctx, GBD_ERR_STATE, "learned preconditioner requested but no weights are loaded");
    const int n = p->n_orb;
    const uint64_t seed0 = e.sched.seed;
    e.defl_w = penalty;
    std::vector<double> g1((size_t)n * n), g2((size_t)n * n * n * n), se((size_t)s->n_sweeps);
    int found = 0;
    for (int a = 0; a < n_states + max_extra && found < n_states; ++a) {
      e.sched.seed = seed0 + (uint64_t)a;
      e.init_state();
      e.ov_init();
      for (int i = 0; i < s->n_sweeps; ++i) se[i] = e.sweep(i) + p->e_core;
      const double energy = e.final_energy() + p->e_core;
      e.rdms(g1.data(), g2.data());
      // <S^2> = -1/2 sum_pq Gamma_pqqp - N^2/4 + N
      double t = 0;
      for (int pp = 0; pp < n; ++pp)
        for (int q = 0; q < n; ++q) t += g2[(((size_t)pp * n + q) * n + q) * n + pp];
      const double N = p->n_elec;
      const double v = -0.5 * t - N * N / 4.0 + N;
      if (target_s2 < 0 || std::fabs(v - target_s2) < 0.1) {
        gbd_result& r = results[found];
        r.energy = energy;
        if (r.sweep_energies) std::copy(se.begin(), se.end(), r.sweep_energies);
        if (r.rdm1) std::copy(g1.begin(), g1.end(), r.rdm1);
        if (r.rdm2) std::copy(g2.begin(), g2.end(), r.rdm2);
        r.max_discarded_weight = e.stats.max_discarded;
        r.n_matvec = e.stats.n_sigma;
        r.status = GBD_OK;
        s2[found] = v;
        ++found;
        *n_found = found;
      }
      if (found < n_states) e.store_state();
    }
    e.clear_states();
    e.sched.seed = seed0;
    if (found < n_states) return fail(ctx, GBD_ERR_NOCONV, "fewer roots of the target <S^2> than requested");
    return GBD_OK;
  });
}

int gbd_set_batch_workers(gbd_ctx* ctx, int32_t workers) {
  if (!ctx || workers < 0) return GBD_ERR_ARG;
  ctx->batch_workers = workers;
  return GBD_OK;
}

int gbd_solve_batched(gbd_ctx* ctx, int32_t n, const gbd_problem* problems, const gbd_schedule* schedules,
                      gbd_result* results) {
  return guarded(ctx, [&]() {
    if (n < 0) return fail(ctx, GBD_ERR_ARG, "n < 0");
    if (n == 0) return GBD_OK;
    if (!problems || !schedules || !results) return fail(ctx, GBD_ERR_ARG, "problems, schedules or results is NULL");
    bool learned = false;
    for (int i = 0; i < n; ++i) {
      int rc = validate(ctx, &problems[i], &schedules[i]);
      if (rc != GBD_OK) return fail(ctx, rc, "problem " + std::to_string(i) + ": " + ctx->err);
      learned |= schedules[i].preconditioner == GBD_PRECOND_LEARNED;
    }
    const std::vector<float>* weights = nullptr;
    if (learned) {
      if (!ctx->eng || !ctx->eng->mlp_loaded)
        return fail(ctx, GBD_ERR_STATE, "learned preconditioner requested but no weights are loaded");
      weights = &ctx->eng->precond_weights();
    }
    for (int i = 0; i < n; ++i) results[i].status = GBD_ERR_STATE;   // until solved
    // most expensive first (longest-processing-time order)
    std::vector<int> order(n);
    std::vector<double> cost(n);
    for (int i = 0; i < n; ++i) cost[i] = problem_cost(problems[i], schedules[i]);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    int nw = std::min({n, 16, hw});
    if (ctx->batch_workers > 0) nw = std::min(n, ctx->batch_workers);
    std::atomic<int> next{0};
    std::mutex mu;
    ctx->batch_stats = gbd::Stats();
    int first_bad = n;
    std::string first_msg;
    auto record = [&](int i, int code, const std::string& msg) {
      results[i].status = code;
      std::lock_guard<std::mutex> g(mu);
      if (i < first_bad) {
        first_bad = i;
        first_msg = "problem " + std::to_string(i) + ": " + msg;
      }
    };
    auto worker = [&]() {
      gbd::set_host_threads(std::max(1, hw / nw));   // the workers share the host cores
      std::unique_ptr<gbd::Engine> eng;
      try {
        eng.reset(new gbd::Engine(ctx->device));
        eng->use_graphs = ctx->graphs;
        if (weights) eng->set_precond_weights(weights->data());
      } catch (const std::exception& ex) {
        // no engine: fail every problem this worker would have taken
        for (int j; (j = next.fetch_add(1)) < n;) record(order[j], GBD_ERR_CUDA, ex.what());
        return;
      }
      for (int j; (j = next.fetch_add(1)) < n;) {
        const int i = order[j];
        const gbd_problem* p = &problems[i];
        const gbd_schedule* s = &schedules[i];
        try {
          eng->prepare(p->n_orb, p->n_elec, p->two_sz, p->n_chol, p->h, p->chol, p->e_core, to_schedule(s));
          run_solve(*eng, p, s, &results[i]);
          std::lock_guard<std::mutex> g(mu);
          ctx->batch_stats.add(eng->stats);
        } catch (const gbd::Error& ex) {
          record(i, ex.code, ex.what());
        } catch (const std::bad_alloc&) {
          record(i, GBD_ERR_OOM, "host allocation failed");
        } catch (const std::exception& ex) {
          record(i, GBD_ERR_CUDA, ex.what());
        }
      }
    };
    std::vector<std::thread> pool;
    try {
      for (int w = 1; w < nw; ++w) pool.emplace_back(worker);
    } catch (const std::system_error&) {
      // fewer threads than asked for: the started ones and this one share the queue
    }
    worker();
    gbd::set_host_threads(0);   // this thread ran a worker too
    for (auto& t : pool) t.join();
    if (first_bad < n) return fail(ctx, results[first_bad].status, first_msg);
    return GBD_OK;
  });
}

int gbd_host_batch_costs(int32_t n, const gbd_problem* problems, const gbd_schedule* schedules, double* cost) {
  if (n < 0 || (n > 0 && (!problems || !schedules || !cost))) return GBD_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (schedules[i].n_sweeps < 1 || !schedules[i].bond_dim) return GBD_ERR_ARG;
    cost[i] = problem_cost(problems[i], schedules[i]);
  }
  return GBD_OK;
}

int gbd_host_partition(int32_t n, const double* cost, int32_t ranks, int32_t* owner, double* load) {
  if (n < 0 || ranks < 1 || (n > 0 && (!cost || !owner))) return GBD_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (!(cost[i] >= 0) || !std::isfinite(cost[i])) return GBD_ERR_ARG;
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<double> l(ranks, 0.0);
  for (int i : order) {
    int r = (int)(std::min_element(l.begin(), l.end()) - l.begin());   // first minimum: the lowest rank
    owner[i] = r;
    l[r] += cost[i];
  }
  if (load)
    for (int r = 0; r < ranks; ++r) load[r] = l[r];
  return GBD_OK;
}

int gbd_set_graphs(gbd_ctx* ctx, int32_t enable) {
  return guarded(ctx, [&]() {
    if (!ctx->eng) ctx->eng.reset(new gbd::Engine(ctx->device));
    ctx->eng->use_graphs = enable != 0;
    ctx->graphs = enable != 0;
    return GBD_OK;
  });
}

int gbd_set_tc_tile(gbd_ctx* ctx, int32_t ncap) {
  return guarded(ctx, [&]() {
    if (ncap != 0 && ncap != 64 && ncap != 128 && ncap != 256) return fail(ctx, GBD_ERR_ARG, "ncap not in {0,64,128,256}");
    if (!ctx->eng) ctx->eng.reset(new gbd::Engine(ctx->device));
    ctx->eng->tc_fixed_cap = ncap;
    return GBD_OK;
  });
}

int gbd_set_adaptive_bond_dim(gbd_ctx* ctx, double max_discarded, int32_t m_min) {
  return guarded(ctx, [&]() {
    if (!(max_discarded >= 0) || !std::isfinite(max_discarded) || m_min < 1)
      return fail(ctx, GBD_ERR_ARG, "max_discarded < 0 or m_min < 1");
    if (!ctx->eng) ctx->eng.reset(new gbd::Engine(ctx->device));
    ctx->eng->adapt_disc = max_discarded;
    ctx->eng->adapt_mmin = m_min;
    return GBD_OK;
  });
}

int gbd_set_tc_order(gbd_ctx* ctx, int32_t order) {
  return guarded(ctx, [&]() {
    if (order < 0 || order > 2) return fail(ctx, GBD_ERR_ARG, "order not in {0,1,2}");
    if (!ctx->eng) ctx->eng.reset(new gbd::Engine(ctx->device));
    ctx->eng->tc_order = order;
    return GBD_OK;
  });
}

int gbd_set_tc_sout_split(gbd_ctx* ctx, int32_t min_rows) {
  return guarded(ctx, [&]() {
    if (min_rows < 0) return fail(ctx, GBD_ERR_ARG, "min_rows < 0");
    if (!ctx->eng) ctx->eng.reset(new gbd::Engine(ctx->device));
    ctx->eng->tc_sout_min = min_rows;
    return GBD_OK;
  });
}

int gbd_set_tc_order_a(gbd_ctx* ctx, int32_t order) {
  return guarded(ctx, [&]() {
    if (order < 0 || order > 1) return fail(ctx, GBD_ERR_ARG, "order not in {0,1}");
    if (!ctx->eng) ctx->eng.reset(new gbd::Engine(ctx->device));
    ctx->eng->tc_order_a = order;
    return GBD_OK;
  });
}

int gbd_set_preconditioner(gbd_ctx* ctx, int32_t preconditioner) {
  return guarded(ctx, [&]() {
    if (!ctx->eng) return fail(ctx, GBD_ERR_STATE, "gbd_setup first");
    if (preconditioner < GBD_PRECOND_DIAG || preconditioner > GBD_PRECOND_PCG)
      return fail(ctx, GBD_ERR_ARG, "unknown preconditioner");
    if (preconditioner == GBD_PRECOND_LEARNED && !ctx->eng->mlp_loaded)
      return fail(ctx, GBD_ERR_STATE, "no preconditioner weights loaded");
    ctx->eng->sched.precond = preconditioner;
    return GBD_OK;
  });
}

int gbd_set_accurate_tier(gbd_ctx* ctx, int32_t prec) {
  return guarded(ctx, [&]() {
    if (prec != 3 && prec != 4) return fail(ctx, GBD_ERR_ARG, "accurate tier must be 3 (TF32x3) or 4 (BF16x3)");
    if (!ctx->eng) ctx->eng.reset(new gbd::Engine(ctx->device));
    ctx->eng->tier2 = prec == 3 ? 2 : 3;   // TcPrec kTF32x3 / kBF16x3
    return GBD_OK;
  });
}

int gbd_set_env_precision(gbd_ctx* ctx, int32_t prec) {
  return guarded(ctx, [&]() {
    if (prec != 0 && prec != 3 && prec != 4) return fail(ctx, GBD_ERR_ARG, "env precision must be 0, 3 or 4");
    if (!ctx->eng) ctx->eng.reset(new gbd::Engine(ctx->device));
    ctx->eng->env_prec = prec == 0 ? -1 : (prec == 3 ? gbd::kTF32x3 : gbd::kBF16x3);
    return GBD_OK;
  });
}

int gbd_set_env_conjugates(gbd_ctx* ctx, int32_t enable) {
  return guarded(ctx, [&]() {
    if (enable != 0 && enable != 1) return fail(ctx, GBD_ERR_ARG, "enable must be 0 or 1");
    if (!ctx->eng) ctx->eng.reset(new gbd::Engine(ctx->device));
    ctx->eng->env_conj = enable != 0;
    return GBD_OK;
  });
}

int gbd_env_conjugates(gbd_ctx* ctx, int32_t side, int32_t bond, int32_t* partner, int32_t* sign, int32_t cap,
                       int32_t* count) {
  return guarded(ctx, [&]() {
    if (!ctx->eng || ctx->eng->conj_l.empty()) return fail(ctx, GBD_ERR_STATE, "gbd_setup first");
    gbd::Engine& e = *ctx->eng;
    if (side != 0 && side != 1) return fail(ctx, GBD_ERR_ARG, "side must be 0 (left) or 1 (right)");
    if (bond < 0 || bond > e.n) return fail(ctx, GBD_ERR_ARG, "bond out of range");
    const auto& c = side == 0 ? e.conj_l[bond] : e.conj_r[bond];
    const auto& sg = side == 0 ? e.sign_l[bond] : e.sign_r[bond];
    if (count) *count = (int)c.size();
    if (partner || sign) {
      if (cap < (int)c.size()) return fail(ctx, GBD_ERR_ARG, "buffer too small");
      for (size_t i = 0; i < c.size(); ++i) {
        if (partner) partner[i] = c[i];
        if (sign) sign[i] = sg[i];
      }
    }
    return GBD_OK;
  });
}

int gbd_gemm_tc_selftest(gbd_ctx* ctx, int32_t M, int32_t N, int32_t K, int32_t nterms, int32_t flags, int32_t prec,
                         uint64_t seed, double* max_err, double* max_ref) {
  return guarded(ctx, [&]() {
    if (M < 1 || N < 1 || K < 1 || nterms < 1 || flags < 0 || flags > 3 || (prec != 3 && prec != 4) || !max_err ||
        !max_ref || (int64_t)M * N > (1 << 26) || (int64_t)K * std::max(M, N) * nterms > (1 << 27))
      return fail(ctx, GBD_ERR_ARG, "invalid self-test arguments");
    if (!ctx->eng) ctx->eng.reset(new gbd::Engine(ctx->device));
    ctx->eng->gemm_tc_selftest(M, N, K, nterms, flags, prec == 3 ? gbd::kTF32x3 : gbd::kBF16x3, seed, max_err,
                               max_ref);
    return GBD_OK;
  });
}

int gbd_set_tier_stop(gbd_ctx* ctx, double floor_mult, int32_t hard_stag) {
  return guarded(ctx, [&]() {
    if (!(floor_mult > 0) || !std::isfinite(floor_mult) || hard_stag < 0)
      return fail(ctx, GBD_ERR_ARG, "floor_mult must be positive and hard_stag >= 0");
    if (!ctx->eng) ctx->eng.reset(new gbd::Engine(ctx->device));
    ctx->eng->tier2_floor_mult = floor_mult;
    ctx->eng->hard_stag_iters = hard_stag;
    return GBD_OK;
  });
}

int gbd_set_tc_min_two_site(gbd_ctx* ctx, int64_t n) {
  return guarded(ctx, [&]() {
    if (n < 0) return fail(ctx, GBD_ERR_ARG, "n < 0");
    if (!ctx->eng) ctx->eng.reset(new gbd::Engine(ctx->device));
    ctx->eng->tc_min_two_site = n;
    return GBD_OK;
  });
}

int gbd_probe_step(gbd_ctx* ctx, int32_t k, int32_t precision, int32_t fp64_refine, double tol, double* theta,
                   double* e64, double* r64) {
  return guarded(ctx, [&]() {
    if (!ctx->eng) return fail(ctx, GBD_ERR_STATE, "gbd_setup first");
    if (precision < 0 || precision > 2 || fp64_refine < 0 || !(tol > 0) || !theta || !e64 || !r64)
      return fail(ctx, GBD_ERR_ARG, "bad probe arguments");
    ctx->eng->probe_step(k, precision, fp64_refine, tol, theta, e64, r64);
    return GBD_OK;
  });
}

int gbd_setup(gbd_ctx* ctx, const gbd_problem* p, const gbd_schedule* s) {
  return guarded(ctx, [&]() { return setup(ctx, p, s); });
}

int gbd_set_precision(gbd_ctx* ctx, int32_t precision, int32_t fp64_refine) {
  return guarded(ctx, [&]() {
    if (!ctx->eng) return fail(ctx, GBD_ERR_STATE, "gbd_setup first");
    if (precision < 0 || precision > 2 || fp64_refine < 0) return fail(ctx, GBD_ERR_ARG, "bad precision");
    ctx->eng->sched.precision = precision;
    ctx->eng->sched.refine = fp64_refine;
    return GBD_OK;
  });
}

int gbd_pcg_selftest(gbd_ctx* ctx, int32_t k, const double* x, const double* r, double theta, double* t,
                     int64_t* matvecs) {
  return guarded(ctx, [&]() {
    if (!x || !r || !t || !matvecs) return fail(ctx, GBD_ERR_ARG, "NULL argument");
    if (!ctx->eng || !ctx->eng->prepared) return fail(ctx, GBD_ERR_STATE, "no MPS installed");
    if (k < 0 || k + 1 >= ctx->eng->n) return fail(ctx, GBD_ERR_ARG, "centre outside the chain");
    ctx->eng->pcg_selftest(k, x, r, theta, t, matvecs);
    return GBD_OK;
  });
}

int gbd_save_state(gbd_ctx* ctx) {
  return guarded(ctx, [&]() {
    if (!ctx->eng || !ctx->eng->prepared) return fail(ctx, GBD_ERR_STATE, "no MPS to save");
    ctx->eng->save_state();
    return GBD_OK;
  });
}

int gbd_restore_state(gbd_ctx* ctx) {
  return guarded(ctx, [&]() {
    if (!ctx->eng || !ctx->eng->has_saved_state()) return fail(ctx, GBD_ERR_STATE, "no saved state");
    ctx->eng->restore_state();
    return GBD_OK;
  });
}

int gbd_set_sweep_schedule(gbd_ctx* ctx, int32_t sweep, int32_t M, double tol) {
  return guarded(ctx, [&]() {
    if (!ctx->eng) return fail(ctx, GBD_ERR_STATE, "no problem set up");
    gbd::Schedule& sc = ctx->eng->sched;
    if (sweep < 0 || sweep >= (int)sc.M.size()) return fail(ctx, GBD_ERR_ARG, "sweep outside the schedule");
    if (M < 1 || !(tol > 0) || !std::isfinite(tol)) return fail(ctx, GBD_ERR_ARG, "M < 1 or tol not positive");
    sc.M[sweep] = M;
    sc.tol[sweep] = tol;
    return GBD_OK;
  });
}

int gbd_init_state(gbd_ctx* ctx) {
  return guarded(ctx, [&]() {
    if (!ctx->eng) return fail(ctx, GBD_ERR_STATE, "gbd_setup first");
    ctx->eng->init_state();
    return GBD_OK;
  });
}

int gbd_run_sweep(gbd_ctx* ctx, int32_t sweep, double* energy) {
  return guarded(ctx, [&]() {
    if (!ctx->eng || !ctx->eng->prepared) return fail(ctx, GBD_ERR_STATE, "no state: gbd_init_state first");
    if (sweep < 0 || sweep >= (int)ctx->eng->sched.M.size()) return fail(ctx, GBD_ERR_ARG, "sweep index out of range");
    double e = ctx->eng->sweep(sweep);
    if (energy) *energy = e + ctx->eng->e_core;
    return GBD_OK;
  });
}

int gbd_final_energy(gbd_ctx* ctx, double* energy) {
  return guarded(ctx, [&]() {
    if (!ctx->eng || !ctx->eng->prepared) return fail(ctx, GBD_ERR_STATE, "no state");
    if (!energy) return fail(ctx, GBD_ERR_ARG, "energy is NULL");
    *energy = ctx->eng->final_energy() + ctx->eng->e_core;
    return GBD_OK;
  });
}

int gbd_get_bond(gbd_ctx* ctx, int32_t bond, int32_t* triples, int32_t cap, int32_t* count) {
  return guarded(ctx, [&]() {
    if (!ctx->eng || !ctx->eng->prepared) return fail(ctx, GBD_ERR_STATE, "no state");
    if (bond < 0 || bond > ctx->eng->n) return fail(ctx, GBD_ERR_ARG, "bond out of range");
    std::vector<int> v;
    ctx->eng->bond_sectors(bond, v);
    int nsec = (int)v.size() / 3;
    if (count) *count = nsec;
    if (triples) {
      if (cap < nsec) return fail(ctx, GBD_ERR_ARG, "triples buffer too small");
      std::memcpy(triples, v.data(), v.size() * sizeof(int));
    }
    return GBD_OK;
  });
}

int gbd_set_mps(gbd_ctx* ctx, const int32_t* n_sectors, const int32_t* sectors, const double* data, int32_t center) {
  return guarded(ctx, [&]() {
    if (!ctx->eng) return fail(ctx, GBD_ERR_STATE, "gbd_setup first");
    if (!n_sectors || !sectors || !data) return fail(ctx, GBD_ERR_ARG, "NULL MPS input");
    int n = ctx->eng->n;
    if (center < 0 || center > n - 2) return fail(ctx, GBD_ERR_ARG, "center out of range");
    ctx->eng->set_mps(n_sectors, sectors, data, center);
    return GBD_OK;
  });
}

int gbd_two_site_size(gbd_ctx* ctx, int32_t k, int64_t* size) {
  return guarded(ctx, [&]() {
    if (!ctx->eng || !ctx->eng->prepared) return fail(ctx, GBD_ERR_STATE, "no state");
    if (k < 0 || k > ctx->eng->n - 2) return fail(ctx, GBD_ERR_ARG, "k out of range");
    *size = ctx->eng->two_site_size(k);
    return GBD_OK;
  });
}

int gbd_apply_heff(gbd_ctx* ctx, int32_t k, const double* in, double* out, double* diag) {
  return guarded(ctx, [&]() {
    if (!ctx->eng || !ctx->eng->prepared) return fail(ctx, GBD_ERR_STATE, "no state");
    if (k < 0 || k > ctx->eng->n - 2) return fail(ctx, GBD_ERR_ARG, "k out of range");
    if (!in || !out) return fail(ctx, GBD_ERR_ARG, "NULL vector");
    ctx->eng->apply_heff(k, in, out, diag);
    return GBD_OK;
  });
}

int gbd_apply_heff_prec(gbd_ctx* ctx, int32_t k, int32_t prec, const double* in, double* out) {
  return guarded(ctx, [&]() {
    if (!ctx->eng || !ctx->eng->prepared) return fail(ctx, GBD_ERR_STATE, "no state");
    if (k < 0 || k > ctx->eng->n - 2) return fail(ctx, GBD_ERR_ARG, "k out of range");
    if (prec < 0 || prec > 4) return fail(ctx, GBD_ERR_ARG, "prec must be 0..4");
    if (!in || !out) return fail(ctx, GBD_ERR_ARG, "NULL vector");
    ctx->eng->apply_heff(k, in, out, nullptr, prec);
    return GBD_OK;
  });
}

int gbd_run_step(gbd_ctx* ctx, int32_t k, int32_t dir, int32_t M, double tol, double* energy, double* discarded,
                 double* kept, int32_t cap, int32_t* nkept) {
  return guarded(ctx, [&]() {
    if (!ctx->eng || !ctx->eng->prepared) return fail(ctx, GBD_ERR_STATE, "no state");
    if (k < 0 || k > ctx->eng->n - 2) return fail(ctx, GBD_ERR_ARG, "k out of range");
    if (dir != 0 && dir != 1) return fail(ctx, GBD_ERR_ARG, "dir must be 0 or 1");
    if (M < 1 || !(tol > 0)) return fail(ctx, GBD_ERR_ARG, "bad M or tol");
    std::vector<double> kw;
    double tau = 0;
    double e = ctx->eng->run_step(k, dir, M, tol, &tau, &kw);
    if (energy) *energy = e + ctx->eng->e_core;
    if (discarded) *discarded = tau;
    if (nkept) *nkept = (int)kw.size();
    if (kept) {
      if (cap < (int)kw.size()) return fail(ctx, GBD_ERR_ARG, "kept buffer too small");
      std::memcpy(kept, kw.data(), kw.size() * sizeof(double));
    }
    return GBD_OK;
  });
}

int gbd_rdms(gbd_ctx* ctx, double* rdm1, double* rdm2) {
  return guarded(ctx, [&]() {
    if (!ctx->eng || !ctx->eng->prepared) return fail(ctx, GBD_ERR_STATE, "no state");
    ctx->eng->rdms(rdm1, rdm2);
    return GBD_OK;
  });
}

int gbd_rdms_ci(gbd_ctx* ctx, double* rdm1, double* rdm2) {
  return guarded(ctx, [&]() {
    if (!ctx->eng || !ctx->eng->prepared) return fail(ctx, GBD_ERR_STATE, "no state");
    ctx->eng->rdms_ci(rdm1, rdm2);
    return GBD_OK;
  });
}

int gbd_orbital_rdms_ci(gbd_ctx* ctx, double* rho1, double* rho2) {
  return guarded(ctx, [&]() {
    if (!ctx->eng || !ctx->eng->prepared) return fail(ctx, GBD_ERR_STATE, "no state");
    ctx->eng->orbital_rdms_ci(rho1, rho2);
    return GBD_OK;
  });
}

int gbd_rdm3(gbd_ctx* ctx, double* rdm3) {
  return guarded(ctx, [&]() {
    if (!rdm3) return fail(ctx, GBD_ERR_ARG, "rdm3 is NULL");
    if (!ctx->eng || !ctx->eng->prepared) return fail(ctx, GBD_ERR_STATE, "no state");
    ctx->eng->rdm3(rdm3);
    return GBD_OK;
  });
}

int gbd_orbital_rdms(gbd_ctx* ctx, double* rho1, double* rho2) {
  return guarded(ctx, [&]() {
    if (!ctx->eng || !ctx->eng->prepared) return fail(ctx, GBD_ERR_STATE, "no state");
    ctx->eng->orbital_rdms(rho1, rho2);
    return GBD_OK;
  });
}

namespace {
// -tr rho ln rho from the eigenvalues above 1e-14 of the symmetrised rho
double entropy_of(int m, const double* rho) {
  std::vector<double> A((size_t)m * m), w(m), Z((size_t)m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) A[(size_t)i * m + j] = 0.5 * (rho[(size_t)i * m + j] + rho[(size_t)j * m + i]);
  if (gbd::sym_eig(m, A.data(), w.data(), Z.data()) != 0) throw gbd::Error(GBD_ERR_NOCONV, "entropy eigensolver failed");
  double s = 0;
  for (double x : w)
    if (x > 1e-14) s -= x * std::log(x);
  return s;
}

void entropies(gbd::Engine& e, double* s1, double* mi) {
  const int n = e.n;
  std::vector<double> r1((size_t)n * 16), r2((size_t)std::max(1, n * (n - 1) / 2) * 256);
  e.orbital_rdms(r1.data(), r2.data());
  std::vector<double> s(n);
  for (int i = 0; i < n; ++i) s[i] = entropy_of(4, r1.data() + (size_t)i * 16);
  if (s1) std::copy(s.begin(), s.end(), s1);
  if (mi) {
    for (int i = 0; i < n; ++i) mi[(size_t)i * n + i] = 0.0;
    for (int i = 0, pr = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j, ++pr) {
        const double v = std::max(0.0, s[i] + s[j] - entropy_of(16, r2.data() + (size_t)pr * 256));
        mi[(size_t)i * n + j] = mi[(size_t)j * n + i] = v;
      }
  }
}
}  // namespace

int gbd_orbital_entropies(gbd_ctx* ctx, double* s1, double* mi) {
  return guarded(ctx, [&]() {
    if (!ctx->eng || !ctx->eng->prepared) return fail(ctx, GBD_ERR_STATE, "no state");
    entropies(*ctx->eng, s1, mi);
    return GBD_OK;
  });
}

int gbd_mi_order(gbd_ctx* ctx, const gbd_problem* p, const gbd_schedule* s, int32_t* order, double* mi) {
  return guarded(ctx, [&]() {
    if (!order) return fail(ctx, GBD_ERR_ARG, "order is NULL");
    int rc = setup(ctx, p, s);
    if (rc != GBD_OK) return rc;
    gbd::Engine& e = *ctx->eng;
    if (s->preconditioner == GBD_PRECOND_LEARNED && !e.mlp_loaded)
      return fail(ctx, GBD_ERR_STATE, "learned preconditioner requested but no weights are loaded");
    std::vector<double> se(s->n_sweeps);
    gbd_result r{};
    r.sweep_energies = se.data();
    run_solve(e, p, s, &r);
    const int n = p->n_orb;
    std::vector<double> I((size_t)n * n);
    entropies(e, nullptr, I.data());
    if (mi) std::copy(I.begin(), I.end(), mi);
    rc = gbd_host_fiedler_order(n, I.data(), order);
    if (rc != GBD_OK) return fail(ctx, rc, "Fiedler order of the mutual information failed");
    return GBD_OK;
  });
}

int gbd_mpo_labels(gbd_ctx* ctx, int32_t bond, uint64_t* keys, int32_t cap, int32_t* count) {
  return guarded(ctx, [&]() {
    if (!ctx->eng) return fail(ctx, GBD_ERR_STATE, "gbd_setup first");
    if (bond < 0 || bond > ctx->eng->n) return fail(ctx, GBD_ERR_ARG, "bond out of range");
    auto v = ctx->eng->mpo_labels(bond);
    if (count) *count = (int)v.size();
    if (keys) {
      if (cap < (int)v.size()) return fail(ctx, GBD_ERR_ARG, "keys buffer too small");
      std::memcpy(keys, v.data(), v.size() * sizeof(uint64_t));
    }
    return GBD_OK;
  });
}

int gbd_env_block(gbd_ctx* ctx, int32_t side, int32_t bond, int32_t channel, int32_t sector, double* out,
                  int64_t cap, int32_t* rows, int32_t* cols) {
  return guarded(ctx, [&]() {
    if (!ctx->eng || !ctx->eng->prepared) return fail(ctx, GBD_ERR_STATE, "no state");
    if (bond < 0 || bond > ctx->eng->n) return fail(ctx, GBD_ERR_ARG, "bond out of range");
    if (channel < 0 || channel >= ctx->eng->mpo_bond_dim(bond)) return fail(ctx, GBD_ERR_ARG, "channel out of range");
    std::vector<int> sec;
    ctx->eng->bond_sectors(bond, sec);
    if (sector < 0 || sector >= (int)sec.size() / 3) return fail(ctx, GBD_ERR_ARG, "sector out of range");
    std::vector<double> v;
    int r = 0, c = 0;
    ctx->eng->env_block(side, bond, channel, sector, v, r, c);
    if (rows) *rows = r;
    if (cols) *cols = c;
    if (out) {
      if (cap < (int64_t)v.size()) return fail(ctx, GBD_ERR_ARG, "out buffer too small");
      std::memcpy(out, v.data(), v.size() * sizeof(double));
    }
    return GBD_OK;
  });
}

int gbd_multi_dot(gbd_ctx* ctx, const double* V, int64_t stride, int32_t k, const double* x, int64_t n, double* out) {
  return guarded(ctx, [&]() {
    if (!V || !x || !out) return fail(ctx, GBD_ERR_ARG, "NULL pointer");
    if (k < 1 || k > 32 || n < 0 || stride < n) return fail(ctx, GBD_ERR_ARG, "bad k, n or stride");
    if (!ctx->eng) ctx->eng.reset(new gbd::Engine(ctx->device));
    ctx->eng->multi_dot(V, stride, k, x, n, out);
    return GBD_OK;
  });
}

int gbd_train_precond(gbd_ctx* ctx, int32_t n_problems, const gbd_problem* problems, const gbd_schedule* schedules,
                      int32_t epochs, double lr, double* final_loss) {
  return guarded(ctx, [&]() {
    if (n_problems < 1 || !problems || !schedules || epochs < 1 || !(lr > 0)) return fail(ctx, GBD_ERR_ARG, "bad training arguments");
    for (int i = 0; i < n_problems; ++i) {
      gbd_schedule s = schedules[i];
      s.preconditioner = GBD_PRECOND_DIAG;
      int rc = setup(ctx, &problems[i], &s);
      if (rc != GBD_OK) return rc;
      gbd::Engine& e = *ctx->eng;
      e.init_state();
      e.recording = true;
      for (int k = 0; k < s.n_sweeps; ++k) e.sweep(k);
      e.recording = false;
    }
    double loss = ctx->eng->train_precond(epochs, lr, 1);
    if (final_loss) *final_loss = loss;
    return GBD_OK;
  });
}

int gbd_save_precond(gbd_ctx* ctx, const char* path) {
  return guarded(ctx, [&]() {
    if (!path) return fail(ctx, GBD_ERR_ARG, "NULL path");
    if (!ctx->eng) return fail(ctx, GBD_ERR_STATE, "no preconditioner weights");
    ctx->eng->save_precond(path);
    return GBD_OK;
  });
}

int gbd_load_precond(gbd_ctx* ctx, const char* path) {
  return guarded(ctx, [&]() {
    if (!path) return fail(ctx, GBD_ERR_ARG, "NULL path");
    if (!ctx->eng) ctx->eng.reset(new gbd::Engine(ctx->device));
    ctx->eng->load_precond(path);
    return GBD_OK;
  });
}

int gbd_set_precond_weights(gbd_ctx* ctx, const float* params) {
  return guarded(ctx, [&]() {
    if (!params) return fail(ctx, GBD_ERR_ARG, "NULL params");
    if (!ctx->eng) ctx->eng.reset(new gbd::Engine(ctx->device));
    ctx->eng->set_precond_weights(params);
    return GBD_OK;
  });
}

int gbd_mlp_loss_grad(gbd_ctx* ctx, const float* X, const float* y, const float* w, int64_t n, const float* params,
                      double lam, double* loss, double* grad) {
  return guarded(ctx, [&]() {
    if (!X || !y || !w || !params || !loss || !grad || n < 1 || !(lam >= 0))
      return fail(ctx, GBD_ERR_ARG, "bad arguments");
    if (!ctx->eng) ctx->eng.reset(new gbd::Engine(ctx->device));
    ctx->eng->mlp_loss_grad(X, y, w, n, params, lam, loss, grad);
    return GBD_OK;
  });
}

int gbd_mlp_precond(gbd_ctx* ctx, const double* r, const double* d, double theta, double iter, int64_t n, double* t) {
  return guarded(ctx, [&]() {
    if (!r || !d || !t || n < 1) return fail(ctx, GBD_ERR_ARG, "bad arguments");
    if (!ctx->eng) return fail(ctx, GBD_ERR_STATE, "no preconditioner weights");
    ctx->eng->mlp_apply(r, d, theta, iter, n, t);
    return GBD_OK;
  });
}

int gbd_davidson_counts(gbd_ctx* ctx, int64_t* iterations, int64_t* fallbacks, int64_t* samples) {
  return guarded(ctx, [&]() {
    if (!ctx->eng) return fail(ctx, GBD_ERR_STATE, "no engine");
    if (iterations) *iterations = ctx->eng->stats.davidson_iters;
    if (fallbacks) *fallbacks = ctx->eng->stats.precond_fallbacks;
    if (samples) *samples = ctx->eng->n_samples();
    return GBD_OK;
  });
}

static void copy_stats(const gbd::Stats& t, gbd_stats* s) {
  std::memset(s, 0, sizeof(*s));
  s->sigma_flops = t.sigma_flops;
  s->sigma_ms = t.sigma_ms;
  s->env_flops = t.env_flops;
  s->env_ms = t.env_ms;
  s->enlarge_ms = t.enl_ms;
  s->davidson_ms = t.davidson_ms;
  s->truncate_ms = t.trunc_ms;
  s->step_ms = t.step_ms;
  s->n_sigma = t.n_sigma;
  s->n_steps = t.n_steps;
  s->kernel_launches = t.launches;
  s->h2d_bytes = t.h2d;
  s->d2h_bytes = t.d2h;
  s->max_discarded_weight = t.max_discarded;
  s->sigma_flops_exec = t.sigma_flops_exec;
  s->tc_ms = t.tc_ms;
  s->tc_flops = t.tc_flops;
  s->n_sigma_tc = t.n_sigma_tc;
  for (int i = 0; i < 3; ++i) s->tier_iterations[i] = t.tier_iters[i];
  s->max_final_residual = t.max_final_residual;
  s->sum_final_residual = t.sum_final_residual;
  s->graph_launches = t.graph_launches;
  s->autotune_trials = t.autotune_trials;
  s->tc_gemm_ms = t.tc_gemm_ms;
  s->tc_bytes = t.tc_bytes;
  s->tc_build_ms = t.tc_build_ms;
  s->enlarge_host_ms = t.enl_host_ms;
  s->diag_ms = t.diag_ms;
  s->truncate_rho_ms = t.trunc_rho_ms;
  s->truncate_eig_ms = t.trunc_eig_ms;
  s->env_wall_ms = t.env_wall_ms;
  for (int i = 0; i < 5; ++i) s->tc_build_phase_ms[i] = t.tcb_ms[i];
  s->davidson_iterations = t.davidson_iters;
  s->inner_matvecs = t.inner_matvecs;
  s->n_solves = t.n_solves;
  s->n_solves_above_tol = t.n_above_tol;
  s->sweep_max_residual = t.sweep_max_residual;
  s->enlarge_dev_ms = t.enl_dev_ms;
  s->enlarge_bytes = t.enl_bytes;
  s->rdm_ms = t.rdm_ms;
  s->rdm_env_bytes = t.rdm_env_bytes;
  s->h2d_wait_ms = t.h2d_wait_ms;
  for (int i = 0; i < 2; ++i) {
    s->tc_stage_alg_bytes[i] = t.tc_alg_st[i];
    s->tc_stage_box_bytes[2 * i] = t.tc_box_st[i][0];
    s->tc_stage_box_bytes[2 * i + 1] = t.tc_box_st[i][1];
    s->tc_stage_dense_bytes[2 * i] = t.tc_dense_st[i][0];
    s->tc_stage_dense_bytes[2 * i + 1] = t.tc_dense_st[i][1];
    s->tc_gemm_ms_by_stage[i] = t.tc_gemm_ms_st[i];
  }
  for (int i = 0; i < 4; ++i) {
    s->tc_flops_by_type[i] = t.tc_flops_p[i];
    s->tc_gemm_ms_by_type[i] = t.tc_gemm_ms_p[i];
  }
}

int gbd_get_stats(const gbd_ctx* ctx, gbd_stats* s) {
  if (!ctx || !s) return GBD_ERR_ARG;
  std::memset(s, 0, sizeof(*s));
  if (ctx->eng) copy_stats(ctx->eng->stats, s);
  return GBD_OK;
}

int gbd_get_batch_stats(const gbd_ctx* ctx, gbd_stats* s) {
  if (!ctx || !s) return GBD_ERR_ARG;
  copy_stats(ctx->batch_stats, s);
  return GBD_OK;
}

int gbd_host_sym_eig(int32_t n, const double* A, double* w, double* Z) {
  if (n < 0 || (n > 0 && (!A || !w || !Z))) return GBD_ERR_ARG;
  try {
    return gbd::sym_eig(n, A, w, Z) == 0 ? GBD_OK : GBD_ERR_NOCONV;
  } catch (...) {
    return GBD_ERR_OOM;
  }
}

int gbd_host_initial_dims(int32_t n, int32_t n_alpha, int32_t n_beta, int32_t M, int32_t* n_sectors,
                          int32_t* triples, int32_t cap) {
  if (n < 1 || n > 32 || n_alpha < 0 || n_beta < 0 || n_alpha > n || n_beta > n || M < 1 || !n_sectors)
    return GBD_ERR_ARG;
  try {
    auto bonds = gbd::initial_bond_dims(n, n_alpha, n_beta, M);
    int pos = 0;
    for (int k = 0; k <= n; ++k) {
      n_sectors[k] = bonds[k].nsec();
      for (int j = 0; j < bonds[k].nsec(); ++j) {
        if (triples) {
          if (pos + 3 > 3 * cap) return GBD_ERR_ARG;
          triples[pos] = bonds[k].na[j];
          triples[pos + 1] = bonds[k].nb[j];
          triples[pos + 2] = bonds[k].dim[j];
        }
        pos += 3;
      }
    }
    return GBD_OK;
  } catch (...) {
    return GBD_ERR_ARG;
  }
}

int gbd_host_select(int32_t count, const double* lam, const int32_t* key, const int32_t* j, int32_t M,
                    double cutoff, double tie, double max_discarded, int32_t m_min, int32_t* kept_index,
                    int32_t* nkept, double* total) {
  if (count < 0 || (count > 0 && (!lam || !key || !j)) || M < 1 || !nkept) return GBD_ERR_ARG;
  if (!(max_discarded >= 0) || !std::isfinite(max_discarded) || m_min < 1) return GBD_ERR_ARG;
  std::vector<gbd::Weight> w;
  for (int i = 0; i < count; ++i) w.push_back({lam[i], key[i], i, j[i]});
  auto kw = gbd::select_states(w, M, cutoff, tie, total, max_discarded, m_min);
  *nkept = (int)kw.size();
  if (kept_index)
    for (size_t i = 0; i < kw.size(); ++i) kept_index[i] = kw[i].idx;
  return GBD_OK;
}

int gbd_host_mpo(int32_t n, const double* h, int32_t n_chol, const double* chol, int32_t k_switch,
                 int32_t* bond_dims, double* dense) {
  if (n < 1 || n > 32 || !h || (n_chol > 0 && !chol) || !bond_dims) return GBD_ERR_ARG;
  if (dense && n > 5) return GBD_ERR_ARG;
  try {
    std::vector<double> eri((size_t)n * n * n * n, 0.0);
    for (int Q = 0; Q < n_chol; ++Q)
      for (int pq = 0; pq < n * n; ++pq)
        for (int rs = 0; rs < n * n; ++rs)
          eri[(size_t)pq * n * n + rs] += chol[(size_t)Q * n * n + pq] * chol[(size_t)Q * n * n + rs];
    gbd::Mpo m;
    gbd::build_mpo(n, h, eri.data(), k_switch, m);
    for (int k = 0; k <= n; ++k) bond_dims[k] = (int)m.labels[k].size();
    if (dense) {
      // plain Kronecker contraction of the dressed tensors (site 0 most significant)
      std::vector<std::vector<double>> env(1, std::vector<double>(1, 1.0));
      int dim = 1;
      for (int i = 0; i < n; ++i) {
        int nd = dim * 4;
        std::vector<std::vector<double>> nx(m.labels[i + 1].size());
        for (const auto& e : m.W[i]) {
          if (env[e.a].empty()) continue;
          auto& t = nx[e.b];
          if (t.empty()) t.assign((size_t)nd * nd, 0.0);
          for (int r = 0; r < dim; ++r)
            for (int c = 0; c < dim; ++c) {
              double x = env[e.a][(size_t)r * dim + c];
              if (x == 0.0) continue;
              t[(size_t)(r * 4 + e.sout) * nd + c * 4 + e.sin] += x * e.v;
            }
        }
        env.swap(nx);
        dim = nd;
      }
      for (size_t i = 0; i < (size_t)dim * dim; ++i) dense[i] = env[0].empty() ? 0.0 : env[0][i];
    }
    return GBD_OK;
  } catch (...) {
    return GBD_ERR_ARG;
  }
}

int gbd_host_mpo_conjugates(int32_t n, const double* h, int32_t n_chol, const double* chol, int32_t k_switch,
                            int32_t side, int32_t bond, int32_t* partner, int32_t* sign, int32_t cap, int32_t* count) {
  if (n < 1 || n > 32 || !h || (n_chol > 0 && !chol) || (side != 0 && side != 1) || bond < 0 || bond > n)
    return GBD_ERR_ARG;
  try {
    std::vector<double> eri((size_t)n * n * n * n, 0.0);
    for (int Q = 0; Q < n_chol; ++Q)
      for (int pq = 0; pq < n * n; ++pq)
        for (int rs = 0; rs < n * n; ++rs)
          eri[(size_t)pq * n * n + rs] += chol[(size_t)Q * n * n + pq] * chol[(size_t)Q * n * n + rs];
    gbd::Mpo m;
    gbd::build_mpo(n, h, eri.data(), k_switch, m);
    std::vector<std::vector<int>> cl, sl, cr, sr;
    gbd::mpo_conjugates(m, cl, sl, cr, sr);
    const auto& c = side == 0 ? cl[bond] : cr[bond];
    const auto& sg = side == 0 ? sl[bond] : sr[bond];
    if (count) *count = (int)c.size();
    if (partner || sign) {
      if (cap < (int)c.size()) return GBD_ERR_ARG;
      for (size_t i = 0; i < c.size(); ++i) {
        if (partner) partner[i] = c[i];
        if (sign) sign[i] = sg[i];
      }
    }
    return GBD_OK;
  } catch (...) {
    return GBD_ERR_ARG;
  }
}

double gbd_mps_init_value(uint64_t seed, int32_t site, int32_t na, int32_t nb, int32_t s, int32_t row, int32_t col) {
  return gbd::mps_init_value(seed, site, na, nb, s, row, col);
}

}  // extern "C"

int gbd_correction_selftest(int32_t device, int32_t kind, int64_t n, const double* x, const double* sx,
                            const double* diag, double theta, double* r_out, double* t_out, double* rr) {
  using namespace gbd;
  if (!x || !sx || !diag || !r_out || !t_out || !rr || n < 1) return GBD_ERR_ARG;
  if (kind != GBD_PRECOND_DIAG && kind != GBD_PRECOND_OLSEN) return GBD_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return GBD_ERR_CUDA;
  const int nblk = reduction_blocks(n);
  const size_t vb = (size_t)n * sizeof(double);
  double* d = nullptr;
  const size_t total = 5 * (size_t)n + 2 * (size_t)nblk + 4;
  if (cudaMalloc(&d, total * sizeof(double)) != cudaSuccess) return GBD_ERR_OOM;
  double *dx = d, *dsx = d + n, *dd = d + 2 * n, *dr = d + 3 * n, *dt = d + 4 * n, *part = d + 5 * n,
         *sums = part + 2 * nblk;
  int rc = GBD_OK;
  if (cudaMemcpy(dx, x, vb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dsx, sx, vb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dd, diag, vb, cudaMemcpyHostToDevice) != cudaSuccess) {
    rc = GBD_ERR_CUDA;
  } else {
    launch_residual_precond(dx, dsx, dd, theta, n, dr, dt, part, nblk, sums + 2, 0);
    if (kind == GBD_PRECOND_OLSEN) launch_projected_precond(dr, dx, dd, theta, -1.0, n, dt, part, nblk, sums, 0);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(r_out, dr, vb, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(t_out, dt, vb, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(rr, sums + 2, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = GBD_ERR_CUDA;
  }
  cudaFree(d);
  return rc;
}

// Fiedler ordering of the orbitals from symmetric non-negative couplings W
// (n x n, diagonal ignored): the Laplacian D - W, the eigenvector f of its
// second-smallest eigenvalue, the orbitals in ascending f (equal values by
// index), the direction whose first orbital has the smaller index.
int gbd_host_fiedler_order(int32_t n, const double* W, int32_t* order) {
  if (n < 1 || !W || !order) return GBD_ERR_ARG;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double a = W[(size_t)i * n + j], b = W[(size_t)j * n + i];
      if (!std::isfinite(a) || (i != j && a < 0) || std::fabs(a - b) > 1e-12 * (1.0 + std::fabs(a)))
        return GBD_ERR_ARG;
    }
  for (int i = 0; i < n; ++i) order[i] = i;
  if (n <= 2) return GBD_OK;
  try {
    std::vector<double> L((size_t)n * n, 0.0), w(n), Z((size_t)n * n);
    for (int i = 0; i < n; ++i) {
      double d = 0;
      for (int j = 0; j < n; ++j)
        if (j != i) {
          L[(size_t)i * n + j] = -W[(size_t)i * n + j];
          d += W[(size_t)i * n + j];
        }
      L[(size_t)i * n + i] = d;
    }
    if (gbd::sym_eig(n, L.data(), w.data(), Z.data()) != 0) return GBD_ERR_NOCONV;
    const double tol = 1e-10 * std::max(1.0, std::fabs(w[n - 1]));
    if (w[1] - w[0] <= tol || w[2] - w[1] <= tol) return GBD_ERR_NOCONV;
    std::vector<int32_t> o(n);
    std::iota(o.begin(), o.end(), 0);
    std::stable_sort(o.begin(), o.end(), [&](int a, int b) { return Z[(size_t)a * n + 1] < Z[(size_t)b * n + 1]; });
    if (o[0] > o[n - 1]) std::reverse(o.begin(), o.end());
    std::copy(o.begin(), o.end(), order);
    return GBD_OK;
  } catch (...) {
    return GBD_ERR_ARG;
  }
}
