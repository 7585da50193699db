// Two-site DMRG sweep engine (host driver of the device kernels).
//
// Method (paper, Fig. 2 and Sec. "Cholesky decomposition for the
// wavefunction"): sites (k, k+1) are optimised against the left block and
// the right block; the two-site effective Hamiltonian is applied matrix-free
// through the MPO inside Davidson; the enlarged bond is decimated back to
// chi_k by the singular values of the two-site state, discarding weight
// tau = sum sigma^2 of the dropped states; the sweep runs left-to-right and
// back.  FP64 throughout in this path (Sec. "Computational details").
//
// GB300 formulation (ours).  Every tensor is blocked by the left-block
// particle numbers q = (N_alpha, N_beta).  With the MPO bond b between the
// two sites, H_eff = sum_b Lenl[b] (x) Renl[b], where
//   Lenl[b] = sum_a L_k[a] (x) W_k[a,b]        (enlarged left operator)
//   Renl[b] = sum_c W_{k+1}[b,c] (x) R_{k+2}[c] (enlarged right operator)
// are formed once per step, and each matvec is two grouped GEMM launches:
//   stage A  Y_b = psi Renl[b]^T      stage B  sigma = sum_b Lenl[b] Y_b.
// The environment update reuses Lenl (Renl): L_{k+1}[b] = U^T Lenl[b] U.
// The decimation diagonalises the per-sector reduced density matrix
// psi psi^T (or psi^T psi), whose eigenvalues are sigma^2.
#include "engine.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <mutex>
#include <memory>
#include <deque>
#include <condition_variable>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <numeric>
#include <thread>

#include "linalg_host.h"
#include "tc_gemm.h"

namespace gbd {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

void Bond::finalize() {
  std::vector<int> ord(na.size());
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](int x, int y) { return qkey(na[x], nb[x]) < qkey(na[y], nb[y]); });
  std::vector<int> a2, b2, d2;
  for (int i : ord) { a2.push_back(na[i]); b2.push_back(nb[i]); d2.push_back(dim[i]); }
  na = a2; nb = b2; dim = d2;
  off.assign(na.size() + 1, 0);
  idx.clear();
  for (size_t i = 0; i < na.size(); ++i) {
    off[i + 1] = off[i] + dim[i];
    idx.set(na[i], nb[i], (int)i);
  }
}

namespace {

constexpr uint64_t GOLDEN = 0x9E3779B97F4A7C15ull;
constexpr uint64_t SALT = 0x4D50535F494E4954ull;

uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  double r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return std::round(r);
}

thread_local int t_host_threads = 0;   // 0: min(hardware threads, 16)

// Persistent host worker pool shared by every engine in the process: a
// parallel_for call posts one job (a loop body and an index counter); the
// workers and the calling thread take indices until none is left, and the
// caller returns when every taken index has finished.  Several callers
// (batched engines) may post jobs at the same time.
class HostPool {
 public:
  static HostPool& get() {
    static HostPool pool;
    return pool;
  }
  int size() const { return (int)workers_.size(); }
  void run(int n, int width, const std::function<void(int)>& f) {
    auto job = std::make_shared<Job>();
    job->f = &f;
    job->n = n;
    job->slots = width - 1;   // workers that may join besides the caller
    {
      std::lock_guard<std::mutex> g(mu_);
      jobs_.push_back(job);
    }
    cv_.notify_all();
    work(*job);
    std::unique_lock<std::mutex> g(job->mu);
    job->cv.wait(g, [&]() { return job->done == job->n; });
  }

 private:
  struct Job {
    const std::function<void(int)>* f = nullptr;
    int n = 0;
    std::atomic<int> next{0}, slots{0};
    int done = 0;
    std::mutex mu;
    std::condition_variable cv;
  };
  HostPool() {
    const int nt = (int)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 16u) - 1;
    for (int t = 0; t < nt; ++t)
      workers_.emplace_back([this]() {
        for (;;) {
          std::shared_ptr<Job> job;
          {
            std::unique_lock<std::mutex> g(mu_);
            cv_.wait(g, [&]() { return stop_ || !jobs_.empty(); });
            if (stop_) return;
            job = jobs_.front();
            // a job leaves the queue once all its indices are taken or it
            // has no worker slots left
            if (job->next.load() >= job->n || --job->slots <= 0) jobs_.pop_front();
          }
          work(*job);
        }
      });
  }
  ~HostPool() {
    {
      std::lock_guard<std::mutex> g(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& w : workers_) w.join();
  }
  static void work(Job& job) {
    int finished = 0;
    for (int i = job.next++; i < job.n; i = job.next++) {
      (*job.f)(i);
      ++finished;
    }
    if (finished) {
      std::lock_guard<std::mutex> g(job.mu);
      job.done += finished;
      if (job.done == job.n) job.cv.notify_all();
    }
  }
  std::vector<std::thread> workers_;
  std::deque<std::shared_ptr<Job>> jobs_;
  std::mutex mu_;
  std::condition_variable cv_;
  bool stop_ = false;
};

void parallel_for(int n, const std::function<void(int)>& f) {
  int nt = (int)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 16u);
  if (t_host_threads > 0) nt = std::min(nt, t_host_threads);
  if (n < 2 || nt < 2) {
    for (int i = 0; i < n; ++i) f(i);
    return;
  }
  HostPool::get().run(n, std::min(nt, n), f);
}

}  // namespace

void set_host_threads(int n) { t_host_threads = n; }
void host_parallel_for(int n, const std::function<void(int)>& f) { parallel_for(n, f); }

// counter-based initial-MPS value (same published definition as the input
// generator: splitmix64 finalizer on a derived seed and an element key)
double mps_init_value(uint64_t seed, int site, int na, int nb, int s, int row, int col) {
  uint64_t base = mix64(seed ^ SALT);
  uint64_t key = ((((((uint64_t)site * 64 + na) * 64 + nb) * 4 + s) << 20 | (uint64_t)row) << 20) | (uint64_t)col;
  uint64_t z = mix64(base + (key + 1) * GOLDEN);
  return 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

// Initial bond dimensions (the paper leaves the initial state open): every
// sector allowed by the target particle numbers, with the exact dimension
// min(left multiplicity, right multiplicity); when the exact total T exceeds
// M, sector q gets min(d(q), max(1, floor(M d(q) / T))); then passes from
// the left (dim <= sum_s dim_{k-1}(q - s)) and from the right (dim <= sum_s
// dim_{k+1}(q + s)) repeat until nothing changes.
std::vector<Bond> initial_bond_dims(int n, int Na, int Nb, int M) {
  // initial bond dimensions: every allowed sector, scaled to M when the
  // exact total exceeds it, then made consistent from both sides
  std::vector<std::map<int, int64_t>> dims(n + 1);
  for (int k = 0; k <= n; ++k) {
    std::map<int, int64_t> ex;
    double T = 0;
    for (int a = 0; a <= std::min(k, Na); ++a)
      for (int b = 0; b <= std::min(k, Nb); ++b) {
        int ra = Na - a, rb = Nb - b;
        if (ra < 0 || rb < 0 || ra > n - k || rb > n - k) continue;
        double left = binom(k, a) * binom(k, b), right = binom(n - k, ra) * binom(n - k, rb);
        double d = std::min(left, right);
        if (d > 0) { ex[qkey(a, b)] = (int64_t)d; T += d; }
      }
    if (T <= M) dims[k] = ex;
    else {
      unsigned __int128 TT = 0;
      for (auto& kv : ex) TT += (unsigned __int128)kv.second;
      for (auto& kv : ex) {
        unsigned __int128 v = ((unsigned __int128)M * (unsigned __int128)kv.second) / TT;
        int64_t d = std::max<int64_t>(1, (int64_t)v);
        dims[k][kv.first] = std::min<int64_t>(kv.second, d);
      }
    }
  }
  bool changed = true;
  while (changed) {
    changed = false;
    for (int k = 1; k <= n; ++k)
      for (auto& kv : dims[k]) {
        int a = kv.first / 64, b = kv.first % 64;
        int64_t sup = 0;
        for (int s = 0; s < 4; ++s) {
          auto it = dims[k - 1].find(qkey(a - QA[s], b - QB[s]));
          if (a - QA[s] >= 0 && b - QB[s] >= 0 && it != dims[k - 1].end()) sup += it->second;
        }
        if (sup < kv.second) { kv.second = sup; changed = true; }
      }
    for (int k = n - 1; k >= 0; --k)
      for (auto& kv : dims[k]) {
        int a = kv.first / 64, b = kv.first % 64;
        int64_t sup = 0;
        for (int s = 0; s < 4; ++s) {
          auto it = dims[k + 1].find(qkey(a + QA[s], b + QB[s]));
          if (it != dims[k + 1].end()) sup += it->second;
        }
        if (sup < kv.second) { kv.second = sup; changed = true; }
      }
    for (int k = 0; k <= n; ++k)
      for (auto it = dims[k].begin(); it != dims[k].end();) {
        if (it->second == 0) { it = dims[k].erase(it); changed = true; }
        else ++it;
      }
  }
  std::vector<Bond> bonds(n + 1);
  for (int k = 0; k <= n; ++k) {
    for (auto& kv : dims[k]) {
      bonds[k].na.push_back(kv.first / 64);
      bonds[k].nb.push_back(kv.first % 64);
      bonds[k].dim.push_back((int)kv.second);
    }
    bonds[k].finalize();
  }
  return bonds;
}

// Decimation rule (the paper keeps chi_k states and discards tau = sum of
// the dropped sigma^2, Fig. 2): drop lambda = sigma^2 <= cutoff; order by
// lambda descending, equal values by (sector key, in-sector rank); keep
// min(M, count); if the last kept and the first dropped differ by <= tie,
// step back so that a near-degenerate cluster is never split at the cut
// (unless the cluster reaches the top, then keep min(M, count)).
// Per-bond adaptive bond dimension (a dynamically adapted bond dimension per
// bond, the paper's compression ingredient (ii)), when max_disc > 0: first
// the smallest m whose discarded weight (all but the first m, cut-off
// weights included) is <= max_disc, extended past a cluster it would split
// and raised to m_min; kept if below min(M, count), else the rule above.
std::vector<Weight> select_states(std::vector<Weight> w, int M, double cutoff, double tie, double* total,
                                  double max_disc, int m_min) {
  double tot = 0;
  std::vector<Weight> cand;
  for (auto& x : w) {
    tot += x.lam;
    if (x.lam > cutoff) cand.push_back(x);
  }
  if (total) *total = tot;
  std::stable_sort(cand.begin(), cand.end(), [](const Weight& a, const Weight& b) {
    if (a.lam != b.lam) return a.lam > b.lam;
    if (a.key != b.key) return a.key < b.key;
    return a.j < b.j;
  });
  const int cn = (int)cand.size();
  if (max_disc > 0.0) {
    int m = 0;
    double kept = 0.0;
    while (m < cn && tot - kept > max_disc) kept += cand[m++].lam;
    while (m > 0 && m < cn && cand[m - 1].lam - cand[m].lam <= tie) ++m;
    m = std::max(m, std::min(m_min, cn));
    if (m < std::min(M, cn)) {
      cand.resize(m);
      return cand;
    }
  }
  int nk = std::min<int>(M, (int)cand.size());
  if ((int)cand.size() > nk) {
    int j = nk;
    while (j > 0 && cand[j - 1].lam - cand[j].lam <= tie) --j;
    if (j > 0) nk = j;
  }
  cand.resize(nk);
  return cand;
}

// ------------------------------------------------------------------ basics
Engine::Engine(int dev) : device(dev) {
  CK(cudaSetDevice(device));
  CK(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device));
  CK(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
  CK(cudaEventCreate(&ev0));
  CK(cudaEventCreate(&ev1));
  CK(cudaEventCreate(&evg0));
  CK(cudaEventCreate(&evg1));
  CK(cudaEventCreate(&evgm));
  CK(cudaMallocHost(&tc_err_host, sizeof(int)));
  *tc_err_host = 0;
  pin_cap = (size_t)16 << 20;
  CK(cudaMallocHost(&pin_ring, pin_cap));
  cudaMemPool_t pool;
  CK(cudaDeviceGetDefaultMemPool(&pool, device));
  uint64_t thr = UINT64_MAX;
  CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
}

Engine::~Engine() {
  cudaSetDevice(device);
  if (tc_err_host) cudaFreeHost(tc_err_host);
  for (auto& e : Lenv) free_env(e);
  for (auto& e : Renv) free_env(e);
  for (auto& s : sites) free_site(s);
  free_snapshot();
  clear_states();
  if (psi) dfree(psi);
  if (d_env_err) dfree(d_env_err);
  cudaStreamSynchronize(stream);
  for (auto& u : pin_inflight) cudaEventDestroy(u.ev);
  for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
  for (auto& t : env_timers) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (cudaEvent_t e : timer_pool) cudaEventDestroy(e);
  if (pin_ring) cudaFreeHost(pin_ring);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (evg0) cudaEventDestroy(evg0);
  if (evg1) cudaEventDestroy(evg1);
  if (evgm) cudaEventDestroy(evgm);
  if (stream) cudaStreamDestroy(stream);
}

void Engine::dfree(void* p) {
  if (!p) return;
  allocs.erase((uintptr_t)p);
  if ((uintptr_t)p == chk_base) chk_size = 0;   // the cached allocation is gone
  CK(cudaFreeAsync(p, stream));
}

// Every block a plan touches must lie inside one live allocation; a planning
// error becomes a GBD_ERR_STATE instead of an out-of-bounds device access.
void Engine::check_range(const void* p, int64_t rows, int64_t cols, int64_t ld, const char* what) const {
  if (rows <= 0 || cols <= 0) return;
  if (rows > 1 && ld < cols) throw Error(-6, std::string("plan check: leading dimension too small for ") + what);
  uintptr_t a = (uintptr_t)p;
  uintptr_t end = a + (uintptr_t)(((rows - 1) * ld + cols) * (int64_t)sizeof(double));
  // consecutive checks mostly fall in the same allocation
  if (chk_size && a >= chk_base && end <= chk_base + chk_size) return;
  auto it = allocs.upper_bound(a);
  if (it == allocs.begin()) throw Error(-6, std::string("plan check: pointer outside allocations: ") + what);
  --it;
  if (a < it->first || end > it->first + it->second)
    throw Error(-6, std::string("plan check: block exceeds its allocation: ") + what);
  chk_base = it->first;
  chk_size = it->second;
}

bool Engine::in_allocation(const void* p, int64_t rows, int64_t cols, int64_t ld, AllocCache& c) const {
  if (rows <= 0 || cols <= 0) return true;
  if (rows > 1 && ld < cols) return false;
  const uintptr_t a = (uintptr_t)p;
  const uintptr_t end = a + (uintptr_t)(((rows - 1) * ld + cols) * (int64_t)sizeof(double));
  if (c.size && a >= c.base && end <= c.base + c.size) return true;
  auto it = allocs.upper_bound(a);
  if (it == allocs.begin()) return false;
  --it;
  if (a < it->first || end > it->first + it->second) return false;
  c.base = it->first;
  c.size = it->second;
  return true;
}

void Engine::check(const GemmPlan& p) const {
  for (const auto& o : p.outs) {
    check_range(o.C, o.M, o.N, o.ldc, "C");
    for (int t = o.t0; t < o.t1; ++t) {
      const GemmTerm& g = p.terms[t];
      if (g.K <= 0) continue;
      if (g.flags & 1) check_range(g.A, g.K, o.M, g.lda, "A^T");
      else check_range(g.A, o.M, g.K, g.lda, "A");
      if (g.flags & 2) check_range(g.B, o.N, g.K, g.ldb, "B^T");
      else check_range(g.B, g.K, o.N, g.ldb, "B");
    }
  }
}

void Engine::check(const AxpyPlan& p) const {
  for (const auto& o : p.outs) {
    check_range(o.dst, 1, o.len, o.len, "axpy dst");
    for (int t = o.t0; t < o.t1; ++t) check_range(p.terms[t].src, 1, o.len, o.len, "axpy src");
  }
}

void Engine::sync() {
  CK(cudaStreamSynchronize(stream));
  drain_timers();
}

void Engine::drain_timers() {
  if (env_tc_pending) {
    env_tc_pending = false;
    int flag = 0;
    CK(cudaMemcpy(&flag, d_env_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) throw Error(-5, "tensor-core environment update: a bounded device wait ran out");
  }
  for (auto& t : env_timers) {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, t.a, t.b));
    *t.acc += ms;
    timer_pool.push_back(t.a);
    timer_pool.push_back(t.b);
  }
  env_timers.clear();
}

cudaEvent_t Engine::pool_event() {
  if (!ev_pool.empty()) {
    cudaEvent_t e = ev_pool.back();
    ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return e;
}

void Engine::h2d(void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return;
  constexpr size_t kRingMax = (size_t)256 << 20;
  if (pin_ring && bytes > pin_cap / 4 && pin_cap < kRingMax) {
    // grow the ring (rare: a few times per engine at most): every staged
    // copy has to finish before the old ring is released
    size_t cap = pin_cap;
    while (bytes > cap / 4 && cap < kRingMax) cap *= 2;
    CK(cudaStreamSynchronize(stream));
    for (auto& u : pin_inflight) ev_pool.push_back(u.ev);
    pin_inflight.clear();
    CK(cudaFreeHost(pin_ring));
    pin_ring = nullptr;
    pin_cap = 0;
    pin_pos = 0;
    CK(cudaMallocHost(&pin_ring, cap));
    pin_cap = cap;
  }
  if (!pin_ring || bytes > pin_cap / 4) {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream));
    return;
  }
  const uint64_t n = (bytes + 255) & ~(uint64_t)255;
  uint64_t start = pin_pos;
  const uint64_t off = start % pin_cap;
  if (off + n > pin_cap) start += pin_cap - off;   // wrap: the region starts at ring offset 0
  // the ring bytes of [start, start + n) last held positions
  // [start - cap, start + n - cap): wait for the copies that read them
  while (!pin_inflight.empty() && pin_inflight.front().start + pin_cap < start + n) {
    if (cudaEventQuery(pin_inflight.front().ev) == cudaErrorNotReady) {
      const double tw = now_ms();
      CK(cudaEventSynchronize(pin_inflight.front().ev));
      stats.h2d_wait_ms += now_ms() - tw;
    }
    ev_pool.push_back(pin_inflight.front().ev);
    pin_inflight.pop_front();
  }
  uint8_t* slot = pin_ring + (start % pin_cap);
  std::memcpy(slot, src, bytes);
  CK(cudaMemcpyAsync(dst, slot, bytes, cudaMemcpyHostToDevice, stream));
  cudaEvent_t e = pool_event();
  CK(cudaEventRecord(e, stream));
  pin_inflight.push_back({start, start + n, e});
  pin_pos = start + n;
}

void Engine::upload(GemmPlan& p) {
  check(p);
  p.d_terms = dalloc<GemmTerm>(p.terms.size());
  p.d_outs = dalloc<GemmOut>(p.outs.size());
  // tiles: 32 x 32 outputs, or, where 32 x 32 tiles would leave more than
  // a quarter of their elements idle (sector blocks of a few tens) and the
  // summed K is short (environment updates, not the sigma's long term
  // lists, where register blocking pays), flat items of 256 elements with
  // one thread per element.  GB300's FP64 pipe is slow enough that the
  // unblocked loop keeps it busy, and both kernels run the same FMA
  // sequence per element.
  p.tiles.clear();
  p.flat.clear();
  for (int o = 0; o < (int)p.outs.size(); ++o) {
    const GemmOut& g = p.outs[o];
    const int64_t elems = (int64_t)g.M * g.N;
    const int64_t padded = (int64_t)((g.M + 31) / 32 * 32) * ((g.N + 31) / 32 * 32);
    int64_t ksum = 0;
    for (int t = g.t0; t < g.t1; ++t) ksum += p.terms[t].K;
    if (elems > 0 && 4 * elems < 3 * padded && ksum <= 1024) {
      for (int64_t e0 = 0; e0 < elems; e0 += 256) p.flat.push_back({o, -1, (int32_t)e0, 0});
      continue;
    }
    for (int tm = 0; tm * 32 < g.M; ++tm)
      for (int tn = 0; tn * 32 < g.N; ++tn) p.tiles.push_back({o, tm, tn, 0});
  }
  // longest term lists first for load balance
  std::stable_sort(p.tiles.begin(), p.tiles.end(), [&](const GemmTile& a, const GemmTile& b) {
    const GemmOut& x = p.outs[a.out];
    const GemmOut& y = p.outs[b.out];
    return (x.t1 - x.t0) > (y.t1 - y.t0);
  });
  std::stable_sort(p.flat.begin(), p.flat.end(), [&](const GemmTile& a, const GemmTile& b) {
    const GemmOut& x = p.outs[a.out];
    const GemmOut& y = p.outs[b.out];
    return (x.t1 - x.t0) > (y.t1 - y.t0);
  });
  p.d_tiles = dalloc<GemmTile>(std::max<size_t>(p.tiles.size(), 1));
  p.d_flat = dalloc<GemmTile>(std::max<size_t>(p.flat.size(), 1));
  h2d(p.d_flat, p.flat.data(), p.flat.size() * sizeof(GemmTile));
  h2d(p.d_terms, p.terms.data(), p.terms.size() * sizeof(GemmTerm));
  h2d(p.d_outs, p.outs.data(), p.outs.size() * sizeof(GemmOut));
  h2d(p.d_tiles, p.tiles.data(), p.tiles.size() * sizeof(GemmTile));
}

void Engine::release(GemmPlan& p) {
  dfree(p.d_terms);
  dfree(p.d_outs);
  dfree(p.d_tiles);
  dfree(p.d_flat);
  p.d_terms = nullptr;
  p.d_outs = nullptr;
  p.d_tiles = nullptr;
  p.d_flat = nullptr;
}

void Engine::upload(AxpyPlan& p) {
  check(p);
  p.cstart.resize(p.outs.size());
  p.nchunks = 0;
  p.bytes = 0;
  for (size_t o = 0; o < p.outs.size(); ++o) {
    p.cstart[o] = p.nchunks;
    p.nchunks += (p.outs[o].len + kAxpyChunk - 1) / kAxpyChunk;
    p.bytes += 8.0 * (p.outs[o].t1 - p.outs[o].t0 + 1) * (double)p.outs[o].len;
  }
  p.d_terms = dalloc<AxpyTerm>(p.terms.size());
  p.d_outs = dalloc<AxpyOut>(p.outs.size());
  p.d_cstart = dalloc<int64_t>(p.cstart.size());
  h2d(p.d_terms, p.terms.data(), p.terms.size() * sizeof(AxpyTerm));
  h2d(p.d_outs, p.outs.data(), p.outs.size() * sizeof(AxpyOut));
  h2d(p.d_cstart, p.cstart.data(), p.cstart.size() * sizeof(int64_t));
}

void Engine::release(AxpyPlan& p) {
  dfree(p.d_terms);
  dfree(p.d_outs);
  dfree(p.d_cstart);
  p.d_terms = nullptr;
  p.d_outs = nullptr;
  p.d_cstart = nullptr;
}

void Engine::run(GemmPlan& p) {
  if (p.tiles.empty() && p.flat.empty()) return;
  launch_gemm_f64(p, stream);
  stats.launches += (!p.tiles.empty()) + (!p.flat.empty());
  CK(cudaGetLastError());
}

void Engine::run(AxpyPlan& p) {
  if (p.outs.empty()) return;
  launch_axpy(p, stream);
  stats.launches++;
  CK(cudaGetLastError());
}

// ------------------------------------------------------------------ layout helpers
std::vector<std::pair<int, int>> Engine::bond_qs(const Bond& b) const {
  std::vector<std::pair<int, int>> q;
  for (int i = 0; i < b.nsec(); ++i) q.push_back({b.na[i], b.nb[i]});
  return q;
}

Space Engine::left_space(const Bond& bl, const std::vector<std::pair<int, int>>& Qs) const {
  Space sp;
  for (auto& Q : Qs) {
    std::array<int, 4> so, sq, sd;
    int tot = 0;
    for (int s = 0; s < 4; ++s) {
      int i = bl.find(Q.first - QA[s], Q.second - QB[s]);
      so[s] = i >= 0 ? tot : -1;
      sq[s] = i;
      sd[s] = i >= 0 ? bl.dim[i] : 0;
      tot += sd[s];
    }
    sp.idx.set(Q.first, Q.second, sp.n());
    sp.qa.push_back(Q.first);
    sp.qb.push_back(Q.second);
    sp.dim.push_back(tot);
    sp.soff.push_back(so);
    sp.ssec.push_back(sq);
    sp.sdim.push_back(sd);
  }
  return sp;
}

Space Engine::right_space(const Bond& br, const std::vector<std::pair<int, int>>& Qs) const {
  Space sp;
  for (auto& Q : Qs) {
    std::array<int, 4> so, sq, sd;
    int tot = 0;
    for (int s = 0; s < 4; ++s) {
      int i = br.find(Q.first + QA[s], Q.second + QB[s]);
      so[s] = i >= 0 ? tot : -1;
      sq[s] = i;
      sd[s] = i >= 0 ? br.dim[i] : 0;
      tot += sd[s];
    }
    sp.idx.set(Q.first, Q.second, sp.n());
    sp.qa.push_back(Q.first);
    sp.qb.push_back(Q.second);
    sp.dim.push_back(tot);
    sp.soff.push_back(so);
    sp.ssec.push_back(sq);
    sp.sdim.push_back(sd);
  }
  return sp;
}

// site i between bonds i and i+1.  FL: per sector Q of bond i+1, a
// (sum_s m_i(Q-s)) x m_{i+1}(Q) block.  FR: per sector q of bond i, a
// m_i(q) x (sum_s m_{i+1}(q+s)) block.
void Engine::layout_site(int i, int layout, Site& s) const {
  s.layout = layout;
  s.off.clear();
  int64_t tot = 0;
  if (layout == 0) {
    const Bond& br = bonds[i + 1];
    Space sp = left_space(bonds[i], bond_qs(br));
    for (int j = 0; j < br.nsec(); ++j) {
      s.off.push_back(tot);
      tot += (int64_t)sp.dim[j] * br.dim[j];
    }
  } else {
    const Bond& bl = bonds[i];
    Space sp = right_space(bonds[i + 1], bond_qs(bl));
    for (int j = 0; j < bl.nsec(); ++j) {
      s.off.push_back(tot);
      tot += (int64_t)bl.dim[j] * sp.dim[j];
    }
  }
  s.size = tot;
}

void Engine::free_site(Site& s) {
  if (s.d) dfree(s.d);
  s.d = nullptr;
  s.size = 0;
}

void Engine::free_env(Env& e) {
  if (e.d) dfree(e.d);
  e.d = nullptr;
  e.size = 0;
  e.valid = false;
}

void Engine::make_env(int bond, Env& e) {
  free_env(e);
  const Bond& b = bonds[bond];
  e.nch = (int)mpo.labels[bond].size();
  e.nsec = b.nsec();
  e.off.assign((size_t)e.nch * e.nsec, -1);
  e.rows.assign((size_t)e.nch * e.nsec, 0);
  e.cols.assign((size_t)e.nch * e.nsec, 0);
  int64_t tot = 0;
  for (int a = 0; a < e.nch; ++a)
    for (int q = 0; q < e.nsec; ++q) {
      int qo = b.find(b.na[q] + mpo.dA[bond][a], b.nb[q] + mpo.dB[bond][a]);
      if (qo < 0) continue;
      size_t id = (size_t)a * e.nsec + q;
      e.off[id] = tot;
      e.rows[id] = b.dim[qo];
      e.cols[id] = b.dim[q];
      tot += (int64_t)b.dim[qo] * b.dim[q];
    }
  e.size = tot;
  e.d = dalloc<double>(tot);
  CK(cudaMemsetAsync(e.d, 0, tot * sizeof(double), stream));
  e.valid = true;
}

// ------------------------------------------------------------------ enlarged operators
namespace {
// entries of one channel grouped into the 16 local matrix elements (so, si);
// rep[p] / ratio[p]: bucket p equals ratio * bucket rep (same channels), so
// its sub-blocks alias the combination formed for rep
struct Buckets {
  std::vector<std::pair<int, double>> lst[16];
  int rep[16];
  double ratio[16];
  void classify() {
    for (int p = 0; p < 16; ++p) {
      rep[p] = p;
      ratio[p] = 1.0;
      if (lst[p].empty()) continue;
      for (int q = 0; q < p; ++q) {
        if (rep[q] != q || lst[q].size() != lst[p].size()) continue;
        const double r = lst[p][0].second / lst[q][0].second;
        bool same = true;
        for (size_t i = 0; i < lst[p].size() && same; ++i)
          same = lst[p][i].first == lst[q][i].first && lst[p][i].second == r * lst[q][i].second;
        if (same) {
          rep[p] = q;
          ratio[p] = r;
          break;
        }
      }
    }
  }
};
}  // namespace

namespace {
// The share of one channel b of an enlarged operator, built by one host
// thread: sub-blocks with owned offsets and axpy outputs relative to the
// share; merge_parts concatenates the shares in b order (the serial layout).
struct EnlPart {
  std::vector<EnlSub> subs;
  std::vector<AxpyTerm> terms;
  std::vector<AxpyOut> outs;
  int64_t own = 0;
};
void merge_parts(std::vector<EnlPart>& parts, EnlOp& op, AxpyPlan& ax) {
  for (EnlPart& P : parts) {
    const int64_t ob = op.own_size;
    const int tb = (int)ax.terms.size();
    for (EnlSub s : P.subs) {
      if (s.own_off >= 0) s.own_off += ob;
      op.subs.push_back(s);
    }
    for (AxpyOut o : P.outs) {
      o.dst = (double*)((intptr_t)o.dst + ob);   // element offsets until finish_enl
      o.t0 += tb;
      o.t1 += tb;
      ax.outs.push_back(o);
    }
    ax.terms.insert(ax.terms.end(), P.terms.begin(), P.terms.end());
    op.own_size += P.own;
  }
}
}  // namespace

// Lenl[b] over E_L(Q) (Q in el), from L_k and W_k.  Sub-block (b, Qin, sin,
// sout) maps rows (q_l, sin) of E_L(Qin) to rows (q_l', sout) of E_L(Qout):
//   sum_a W_k[a,b](sout, sin) L_k[a](q_l' <- q_l).
// All channels a of one (b, sout, sin) bucket share delta_a, so a sector has
// either every block or none.  A single +-1 term aliases the environment
// block; other combinations are formed once and shared by proportional
// buckets (identity-like local operators give four of them).
void Engine::build_lenl(int k, const Env& Lk, const Space& el, EnlOp& op, AxpyPlan& ax) {
  const Bond& bk = bonds[k];
  const auto& W = mpo.W[k];
  op.subs.clear();
  op.own_size = 0;
  const int ns = bk.nsec();
  // runs of W_k entries with the same right channel b
  std::vector<std::pair<size_t, size_t>> runs;
  for (size_t e0 = 0; e0 < W.size();) {
    size_t e1 = e0;
    while (e1 < W.size() && W[e1].b == W[e0].b) ++e1;
    runs.push_back({e0, e1});
    e0 = e1;
  }
  std::vector<EnlPart> parts(runs.size());
  parallel_for((int)runs.size(), [&](int u) {
    EnlPart& P = parts[u];
    const size_t e0 = runs[u].first, e1 = runs[u].second;
    const int b = W[e0].b;
    if (env_derived(k + 1, b, true)) return;   // the transpose of its partner (append_conjugates)
    Buckets B;
    for (size_t e = e0; e < e1; ++e) B.lst[W[e].sout * 4 + W[e].sin].push_back({W[e].a, W[e].v});
    B.classify();
    std::vector<int64_t> combo(16 * (size_t)ns, -1);
    for (int p = 0; p < 16; ++p) {
      const auto& lst = B.lst[p];
      if (lst.empty()) continue;
      const int so = p / 4, si = p % 4;
      const int da = mpo.dA[k + 1][b] - (QA[so] - QA[si]);
      const int db = mpo.dB[k + 1][b] - (QB[so] - QB[si]);
      for (int il = 0; il < ns; ++il) {
        const int qin = el.find(bk.na[il] + QA[si], bk.nb[il] + QB[si]);
        if (qin < 0) continue;
        const int ilp = bk.find(bk.na[il] + da, bk.nb[il] + db);
        if (ilp < 0) continue;
        const int qout = el.find(bk.na[ilp] + QA[so], bk.nb[ilp] + QB[so]);
        if (qout < 0) continue;
        if (Lk.at(lst[0].first, il) < 0) continue;
        EnlSub sub{b, qin, si, qout, so, bk.dim[ilp], bk.dim[il], nullptr, -1, 1.0};
        if (lst.size() == 1) {
          sub.ptr = Lk.d + Lk.at(lst[0].first, il);
          sub.sign = lst[0].second;
        } else {
          const int r = B.rep[p];
          int64_t& off = combo[(size_t)r * ns + il];
          if (off < 0) {
            const int64_t len = (int64_t)sub.rows * sub.cols;
            off = P.own;
            AxpyOut o{(double*)(intptr_t)off, len, (int)P.terms.size(), 0};
            for (auto& t : B.lst[r]) P.terms.push_back({Lk.d + Lk.at(t.first, il), t.second});
            o.t1 = (int)P.terms.size();
            P.outs.push_back(o);
            P.own += len;
          }
          sub.own_off = off;
          sub.sign = B.ratio[p];
        }
        P.subs.push_back(sub);
      }
    }
  });
  merge_parts(parts, op, ax);
  append_conjugates(op, k + 1, true);
}

// Renl[b] over E_R(Q) (Q in er), from R_{i+1} and W_i (i = site).  Sub-block
// (b, Qin, sin, sout) maps columns (sin, q_r) of E_R(Qin) to (sout, q_r') of
// E_R(Qout):  sum_c W_i[b,c](sout, sin) R_{i+1}[c](q_r' <- q_r).
void Engine::build_renl(int i, const Env& R, const Space& er, EnlOp& op, AxpyPlan& ax) {
  const Bond& br = bonds[i + 1];
  const auto& W = mpo.W[i];
  op.subs.clear();
  op.own_size = 0;
  const int ns = br.nsec();
  // entries of W_i grouped by their left channel (called b here)
  std::vector<std::vector<const MpoEntry*>> bya(mpo.labels[i].size());
  for (const auto& e : W) bya[e.a].push_back(&e);
  std::vector<int> units;
  for (int b = 0; b < (int)bya.size(); ++b)
    if (!bya[b].empty()) units.push_back(b);
  std::vector<EnlPart> parts(units.size());
  parallel_for((int)units.size(), [&](int u) {
    EnlPart& P = parts[u];
    const int b = units[u];
    if (env_derived(i, b, false)) return;   // the transpose of its partner (append_conjugates)
    Buckets B;
    for (const MpoEntry* e : bya[b]) B.lst[e->sout * 4 + e->sin].push_back({e->b, e->v});
    B.classify();
    std::vector<int64_t> combo(16 * (size_t)ns, -1);
    for (int p = 0; p < 16; ++p) {
      const auto& lst = B.lst[p];
      if (lst.empty()) continue;
      const int so = p / 4, si = p % 4;
      const int dca = mpo.dA[i][b] + (QA[so] - QA[si]);
      const int dcb = mpo.dB[i][b] + (QB[so] - QB[si]);
      for (int ir = 0; ir < ns; ++ir) {
        const int qin = er.find(br.na[ir] - QA[si], br.nb[ir] - QB[si]);
        if (qin < 0) continue;
        const int irp = br.find(br.na[ir] + dca, br.nb[ir] + dcb);
        if (irp < 0) continue;
        const int qout = er.find(br.na[irp] - QA[so], br.nb[irp] - QB[so]);
        if (qout < 0) continue;
        if (R.at(lst[0].first, ir) < 0) continue;
        EnlSub sub{b, qin, si, qout, so, br.dim[irp], br.dim[ir], nullptr, -1, 1.0};
        if (lst.size() == 1) {
          sub.ptr = R.d + R.at(lst[0].first, ir);
          sub.sign = lst[0].second;
        } else {
          const int r = B.rep[p];
          int64_t& off = combo[(size_t)r * ns + ir];
          if (off < 0) {
            const int64_t len = (int64_t)sub.rows * sub.cols;
            off = P.own;
            AxpyOut o{(double*)(intptr_t)off, len, (int)P.terms.size(), 0};
            for (auto& t : B.lst[r]) P.terms.push_back({R.d + R.at(t.first, ir), t.second});
            o.t1 = (int)P.terms.size();
            P.outs.push_back(o);
            P.own += len;
          }
          sub.own_off = off;
          sub.sign = B.ratio[p];
        }
        P.subs.push_back(sub);
      }
    }
  });
  merge_parts(parts, op, ax);
  append_conjugates(op, i, false);
}

// A derived channel d of certified partner c (sign s): Enl[d] = s Enl[c]^T
// (Enl[b] = sum_a W[a,b] (x) Env[a] and the certification of W), so each
// sub-block (c; qin, sin -> qout, sout) gives (d; qout, sout -> qin, sin)
// reading the same memory transposed.  No combination is formed twice.
void Engine::append_conjugates(EnlOp& op, int bond, bool left) const {
  if (!env_conj) return;
  const auto& cj = left ? conj_l : conj_r;
  const auto& sg = left ? sign_l : sign_r;
  if (bond >= (int)cj.size()) return;
  const int nch = (int)cj[bond].size();
  std::vector<std::vector<size_t>> by((size_t)nch);
  const size_t n0 = op.subs.size();
  for (size_t i = 0; i < n0; ++i) by[op.subs[i].b].push_back(i);
  for (int d = 0; d < nch; ++d) {
    if (!env_derived(bond, d, left)) continue;
    for (size_t i : by[cj[bond][d]]) {
      const EnlSub s = op.subs[i];
      EnlSub t = s;
      t.b = d;
      t.qin = s.qout;
      t.sin = s.sout;
      t.qout = s.qin;
      t.sout = s.sin;
      t.rows = s.cols;
      t.cols = s.rows;
      t.sign = s.sign * sg[bond][d];
      t.trans = s.trans ^ 1;
      op.subs.push_back(t);
    }
  }
}

void Engine::finish_enl(EnlOp& op, AxpyPlan& ax) {
  op.own = dalloc<double>(op.own_size);
  for (auto& o : ax.outs) o.dst = op.own + (intptr_t)o.dst;
  for (auto& s : op.subs)
    if (s.own_off >= 0) s.ptr = op.own + s.own_off;
  upload(ax);
  if (!ax.outs.empty()) {
    EnvTimer t = timer_begin(&stats.enl_dev_ms);
    run(ax);
    timer_end(t);
    stats.enl_bytes += ax.bytes;
  }
  release(ax);
  ax.clear();
}

void Engine::free_enl(EnlOp& op) {
  if (op.own) dfree(op.own);
  op.own = nullptr;
  op.subs.clear();
}

// ------------------------------------------------------------------ environment updates
namespace {
// sub-block indices of an enlarged operator grouped by key b * nq + qin
// (counting sort, keys ascending, sub order kept within a key)
struct SubGroups {
  std::vector<int> start, idx;
  int nq = 0, nkeys = 0;
  SubGroups(const EnlOp& op, int nq_) : nq(nq_) {
    int nb = 0;
    for (const auto& s : op.subs) nb = std::max(nb, s.b + 1);
    nkeys = nb * nq;
    start.assign((size_t)nkeys + 1, 0);
    for (const auto& s : op.subs) start[(size_t)s.b * nq + s.qin + 1]++;
    for (int k = 0; k < nkeys; ++k) start[k + 1] += start[k];
    idx.resize(op.subs.size());
    std::vector<int> fill(start.begin(), start.end() - 1);
    for (size_t i = 0; i < op.subs.size(); ++i) idx[fill[(size_t)op.subs[i].b * nq + op.subs[i].qin]++] = (int)i;
  }
};
}  // namespace

// L_{k+1}[b](Qout <- Qin) = U_Qout^T (Lenl[b] U_Qin); U = A_k (fused-left).
void Engine::env_update_left(const EnlOp& lenl, const Space& el, const Site& A, const Bond& bnew, Env& out) {
  int bond = (int)(&bnew - &bonds[0]);
  make_env(bond, out);
  // T_b(Qin) blocks: rows E_L(Qout), cols m_new(Qin)
  const SubGroups groups(lenl, el.n());   // (b, qin) -> subs
  struct TB { int b, qin, qout, nin, nout; int64_t off; int key; };
  std::vector<TB> tbs;
  int64_t tsize = 0;
  for (int key = 0; key < groups.nkeys; ++key) {
    if (groups.start[key] == groups.start[key + 1]) continue;
    const int b = key / groups.nq, qin = key % groups.nq;
    if (env_derived(bond, b, true)) continue;   // filled by the transpose of its partner
    int jin = bnew.find(el.qa[qin], el.qb[qin]);
    if (jin < 0) continue;
    int qout = lenl.subs[groups.idx[groups.start[key]]].qout;
    int jout = bnew.find(el.qa[qout], el.qb[qout]);
    if (jout < 0) continue;
    tbs.push_back({b, qin, qout, jin, jout, tsize, key});
    tsize += (int64_t)el.dim[qout] * bnew.dim[jin];
  }
  double* T = dalloc<double>(tsize);
  GemmPlan p1, p2;
  for (auto& tb : tbs) {
    int nin = bnew.dim[tb.nin];
    const double* U_in = A.d + A.off[tb.nin];
    for (int so = 0; so < 4; ++so) {
      if (el.soff[tb.qout][so] < 0) continue;
      p1.add_out(T + tb.off + (int64_t)el.soff[tb.qout][so] * nin, nin, el.sdim[tb.qout][so], nin, 0);
      for (int gi = groups.start[tb.key]; gi < groups.start[tb.key + 1]; ++gi) {
        const EnlSub* s = &lenl.subs[groups.idx[gi]];
        if (s->sout != so) continue;
        if (s->trans) throw Error(-6, "environment update of a derived channel");
        p1.add_term(s->ptr, s->cols, U_in + (int64_t)el.soff[tb.qin][s->sin] * nin, nin, s->cols, 0, s->sign);
      }
    }
    int nout = bnew.dim[tb.nout];
    int64_t eo = out.at(tb.b, tb.nin);
    if (eo < 0) continue;
    p2.add_out(out.d + eo, nin, nout, nin, 0);
    p2.add_term(A.d + A.off[tb.nout], nout, T + tb.off, nin, el.dim[tb.qout], 1, 1.0);
  }
  const double th0 = now_ms();
  timed_env_launch(p1, p2);
  env_transposes(out, bond, true);
  stats.env_wall_ms += now_ms() - th0;
  stats.env_flops += p1.flops + p2.flops;
  dfree(T);
}

// a derived channel of an environment update: its certified Hermitian
// partner has a lower index, so its blocks are that partner's transposed
bool Engine::env_derived(int bond, int c, bool left) const {
  if (!env_conj) return false;
  const auto& cj = left ? conj_l : conj_r;
  if (bond >= (int)cj.size() || c >= (int)cj[bond].size()) return false;
  const int d = cj[bond][c];
  return d >= 0 && d < c;
}

// out[d](q' <- q) = sign out[c](q <- q')^T for every derived channel d of
// the bond (partner c, computed by the launch before), one tile list
void Engine::env_transposes(Env& out, int bond, bool left) {
  if (!env_conj) return;
  const auto& cj = left ? conj_l : conj_r;
  const auto& sg = left ? sign_l : sign_r;
  const Bond& bd = bonds[bond];
  std::vector<TransTask> tasks;
  std::vector<TransTile> tiles;
  for (int d = 0; d < out.nch; ++d) {
    if (!env_derived(bond, d, left)) continue;
    const int c = cj[bond][d];
    for (int q = 0; q < out.nsec; ++q) {
      const int64_t od = out.at(d, q);
      if (od < 0) continue;
      const int qo = bd.find(bd.na[q] + mpo.dA[bond][d], bd.nb[q] + mpo.dB[bond][d]);
      const int64_t oc = qo >= 0 ? out.at(c, qo) : -1;
      if (oc < 0) throw Error(-6, "conjugate channel block missing");
      const int rows = bd.dim[q], cols = bd.dim[qo];   // the partner's block (q <- q')
      const int t = (int)tasks.size();
      tasks.push_back({out.d + oc, out.d + od, rows, cols, (double)sg[bond][d]});
      for (int r0 = 0; r0 < rows; r0 += 32)
        for (int c0 = 0; c0 < cols; c0 += 32) tiles.push_back({t, r0, c0, 0});
    }
  }
  if (tiles.empty()) return;
  for (const TransTask& t : tasks) {
    check_range(t.src, t.rows, t.cols, t.cols, "transpose src");
    check_range(t.dst, t.cols, t.rows, t.rows, "transpose dst");
  }
  TransTask* d_tasks = dalloc<TransTask>(tasks.size());
  TransTile* d_tiles = dalloc<TransTile>(tiles.size());
  h2d(d_tasks, tasks.data(), tasks.size() * sizeof(TransTask));
  h2d(d_tiles, tiles.data(), tiles.size() * sizeof(TransTile));
  EnvTimer tm = timer_begin(&stats.env_ms);
  launch_block_transpose(d_tasks, d_tiles, (int)tiles.size(), stream);
  stats.launches++;
  CK(cudaGetLastError());
  timer_end(tm);
  dfree(d_tasks);
  dfree(d_tiles);
}

// a pair of timing events around device work on the engine stream; the
// time goes to *acc after the next stream synchronisation
Engine::EnvTimer Engine::timer_begin(double* acc) {
  EnvTimer t;
  t.acc = acc;
  for (cudaEvent_t* e : {&t.a, &t.b}) {
    if (!timer_pool.empty()) {
      *e = timer_pool.back();
      timer_pool.pop_back();
    } else {
      CK(cudaEventCreate(e));
    }
  }
  CK(cudaEventRecord(t.a, stream));
  return t;
}

void Engine::timer_end(EnvTimer t) {
  CK(cudaEventRecord(t.b, stream));
  env_timers.push_back(t);
}

// the two GEMM plans of an environment update (checked, uploaded, run and
// released), on the FP64 units or on the tensor cores
void Engine::timed_env_launch(GemmPlan& p1, GemmPlan& p2) {
  if (env_prec >= 0 && !force_fp64_env && sched.precision != 0) {
    check(p1);
    check(p2);
    EnvTimer t = timer_begin(&stats.env_ms);
    run_tc(p1, env_prec);
    run_tc(p2, env_prec);
    timer_end(t);
    env_tc_used = true;
    return;
  }
  upload(p1);
  upload(p2);
  EnvTimer t = timer_begin(&stats.env_ms);
  run(p1);
  run(p2);
  timer_end(t);
  release(p1);
  release(p2);
}

// R_{k+1}[b](Qout <- Qin) = B_Qout (Renl[b] B_Qin^T); B fused-right.
void Engine::env_update_right(const EnlOp& renl, const Space& er, const Site& B, const Bond& bnew, Env& out) {
  int bond = (int)(&bnew - &bonds[0]);
  make_env(bond, out);
  const SubGroups groups(renl, er.n());   // (b, qin) -> subs
  struct TB { int b, qin, qout, nin, nout; int64_t off; int key; };
  std::vector<TB> tbs;
  int64_t tsize = 0;
  for (int key = 0; key < groups.nkeys; ++key) {
    if (groups.start[key] == groups.start[key + 1]) continue;
    const int b = key / groups.nq, qin = key % groups.nq;
    if (env_derived(bond, b, false)) continue;   // filled by the transpose of its partner
    int jin = bnew.find(er.qa[qin], er.qb[qin]);
    if (jin < 0) continue;
    int qout = renl.subs[groups.idx[groups.start[key]]].qout;
    int jout = bnew.find(er.qa[qout], er.qb[qout]);
    if (jout < 0) continue;
    tbs.push_back({b, qin, qout, jin, jout, tsize, key});
    tsize += (int64_t)er.dim[qout] * bnew.dim[jin];
  }
  double* T = dalloc<double>(tsize);
  GemmPlan p1, p2;
  for (auto& tb : tbs) {
    int nin = bnew.dim[tb.nin];
    const double* B_in = B.d + B.off[tb.nin];   // nin x m_ER(qin)
    for (int so = 0; so < 4; ++so) {
      if (er.soff[tb.qout][so] < 0) continue;
      p1.add_out(T + tb.off + (int64_t)er.soff[tb.qout][so] * nin, nin, er.sdim[tb.qout][so], nin, 0);
      for (int gi = groups.start[tb.key]; gi < groups.start[tb.key + 1]; ++gi) {
        const EnlSub* s = &renl.subs[groups.idx[gi]];
        if (s->sout != so) continue;
        if (s->trans) throw Error(-6, "environment update of a derived channel");
        p1.add_term(s->ptr, s->cols, B_in + er.soff[tb.qin][s->sin], er.dim[tb.qin], s->cols, 2, s->sign);
      }
    }
    int nout = bnew.dim[tb.nout];
    int64_t eo = out.at(tb.b, tb.nin);
    if (eo < 0) continue;
    p2.add_out(out.d + eo, nin, nout, nin, 0);
    p2.add_term(B.d + B.off[tb.nout], er.dim[tb.qout], T + tb.off, nin, er.dim[tb.qout], 0, 1.0);
  }
  const double th0 = now_ms();
  timed_env_launch(p1, p2);
  env_transposes(out, bond, false);
  stats.env_wall_ms += now_ms() - th0;
  stats.env_flops += p1.flops + p2.flops;
  dfree(T);
}

// ------------------------------------------------------------------ two-site state
void Engine::setup_two_site(int k) {
  const Bond& bk = bonds[k];
  const Bond& bk2 = bonds[k + 2];
  std::vector<std::pair<int, int>> cand;
  for (int i = 0; i < bk.nsec(); ++i)
    for (int s = 0; s < 4; ++s) cand.push_back({bk.na[i] + QA[s], bk.nb[i] + QB[s]});
  std::sort(cand.begin(), cand.end(), [](auto& x, auto& y) { return qkey(x.first, x.second) < qkey(y.first, y.second); });
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  std::vector<std::pair<int, int>> Qs;
  for (auto& Q : cand) {
    bool r = false;
    for (int s = 0; s < 4; ++s)
      if (bk2.find(Q.first + QA[s], Q.second + QB[s]) >= 0) r = true;
    if (r) Qs.push_back(Q);
  }
  EL = left_space(bk, Qs);
  ER = right_space(bk2, Qs);
  psi_off.assign(Qs.size() + 1, 0);
  for (size_t i = 0; i < Qs.size(); ++i) psi_off[i + 1] = psi_off[i] + (int64_t)EL.dim[i] * ER.dim[i];
  psi_size = psi_off.back();
  if (psi) dfree(psi);
  psi = dalloc<double>(psi_size);
  cur_k = k;
}

// psi at (k, k+1) = sites[k] . sites[k+1] contracted over bond k+1.
void Engine::form_psi(int k, int) {
  const Site& X = sites[k];
  const Site& Y = sites[k + 1];
  const Bond& b1 = bonds[k + 1];
  GemmPlan p;
  for (int iq = 0; iq < EL.n(); ++iq) {
    int Qa = EL.qa[iq], Qb = EL.qb[iq];
    double* out = psi + psi_off[iq];
    int mEL = EL.dim[iq], mER = ER.dim[iq];
    if (X.layout == 0 && Y.layout == 1) {
      int j = b1.find(Qa, Qb);
      p.add_out(out, mER, mEL, mER, 0);
      if (j >= 0) p.add_term(X.d + X.off[j], b1.dim[j], Y.d + Y.off[j], mER, b1.dim[j], 0, 1.0);
    } else if (X.layout == 1 && Y.layout == 1) {
      // center X fused-right over (bond k, bond k+1), B = Y over (bond k+1, bond k+2)
      Space xr = right_space(b1, {});
      int j = b1.find(Qa, Qb);
      for (int s1 = 0; s1 < 4; ++s1) {
        if (EL.soff[iq][s1] < 0) continue;
        int iql = EL.ssec[iq][s1];
        int mql = EL.sdim[iq][s1];
        p.add_out(out + (int64_t)EL.soff[iq][s1] * mER, mER, mql, mER, 0);
        if (j < 0) continue;
        // column offset of (s1, Q) inside the fused-right block of q_l
        const Bond& bk = bonds[k];
        int coff = 0, xcols = 0;
        for (int s = 0; s < 4; ++s) {
          int jj = b1.find(bk.na[iql] + QA[s], bk.nb[iql] + QB[s]);
          if (s < s1 && jj >= 0) coff += b1.dim[jj];
          if (jj >= 0) xcols += b1.dim[jj];
        }
        p.add_term(X.d + X.off[iql] + coff, xcols, Y.d + Y.off[j], mER, b1.dim[j], 0, 1.0);
      }
      (void)xr;
    } else if (X.layout == 0 && Y.layout == 0) {
      // A = X fused-left over (bond k, bond k+1); center Y fused-left over (bond k+1, bond k+2)
      const Bond& bk2 = bonds[k + 2];
      for (int s2 = 0; s2 < 4; ++s2) {
        if (ER.soff[iq][s2] < 0) continue;
        int iqr = ER.ssec[iq][s2];
        int mqr = ER.sdim[iq][s2];
        p.add_out(out + ER.soff[iq][s2], mER, mEL, mqr, 0);
        int j = b1.find(Qa, Qb);
        if (j < 0) continue;
        int roff = 0;
        for (int s = 0; s < 4; ++s) {
          int jj = b1.find(bk2.na[iqr] - QA[s], bk2.nb[iqr] - QB[s]);
          if (s < s2 && jj >= 0) roff += b1.dim[jj];
        }
        p.add_term(X.d + X.off[j], b1.dim[j], Y.d + Y.off[iqr] + (int64_t)roff * mqr, mqr, b1.dim[j], 0, 1.0);
      }
    } else {
      throw Error(-6, "inconsistent site layouts for the two-site state");
    }
  }
  upload(p);
  run(p);
  release(p);
}

// ------------------------------------------------------------------ sigma
struct Engine::Sigma {
  EnlOp lenl, renl;
  double* Y = nullptr;
  double* in = nullptr;
  double* out = nullptr;
  GemmPlan A, B;
  GraphSeq graph;
};

void Engine::plan_sigma(const EnlOp& lenl, const EnlOp& renl, Sigma& sg) {
  // Y_b(Qin) exists when both operators have sub-blocks for (b, Qin)
  std::map<std::pair<int, int>, std::vector<const EnlSub*>> rby, lby;
  for (const auto& s : renl.subs) rby[{s.b, s.qin}].push_back(&s);
  for (const auto& s : lenl.subs) lby[{s.b, s.qin}].push_back(&s);
  std::map<std::pair<int, int>, int64_t> yoff;
  int64_t ysize = 0;
  std::vector<std::tuple<int, int, int>> ys;   // b, qin, qout
  for (auto& kv : rby) {
    if (!lby.count(kv.first)) continue;
    int qin = kv.first.second;
    int qout = kv.second[0]->qout;
    yoff[kv.first] = ysize;
    ys.push_back({kv.first.first, qin, qout});
    ysize += (int64_t)EL.dim[qin] * ER.dim[qout];
  }
  sg.Y = dalloc<double>(ysize);
  sg.in = dalloc<double>(psi_size);
  sg.out = dalloc<double>(psi_size);
  GemmPlan& A = sg.A;
  GemmPlan& B = sg.B;
  A.clear();
  B.clear();
  // stage A: Y_b(Qin)[:, cols (sout, q_r')] = sum psi(Qin)[:, cols (sin, q_r)] Rsub^T
  for (auto& y : ys) {
    int b = std::get<0>(y), qin = std::get<1>(y), qout = std::get<2>(y);
    double* Yb = sg.Y + yoff[{b, qin}];
    int ldy = ER.dim[qout];
    const auto& subs = rby[{b, qin}];
    for (int so = 0; so < 4; ++so) {
      if (ER.soff[qout][so] < 0) continue;
      A.add_out(Yb + ER.soff[qout][so], ldy, EL.dim[qin], ER.sdim[qout][so], 0);
      for (const EnlSub* s : subs) {
        if (s->sout != so) continue;
        if (s->trans)   // Rsub^T = sign * (the block at ptr), cols x rows
          A.add_term(sg.in + psi_off[qin] + ER.soff[qin][s->sin], ER.dim[qin], s->ptr, s->rows, s->cols, 0, s->sign);
        else
          A.add_term(sg.in + psi_off[qin] + ER.soff[qin][s->sin], ER.dim[qin], s->ptr, s->cols, s->cols, 2, s->sign);
      }
    }
  }
  // stage B: sigma(Qout)[rows (q_l', sout), :] = sum Lsub Y_b(Qin)[rows (q_l, sin), :]
  std::map<std::pair<int, int>, std::vector<const EnlSub*>> lout;
  for (const auto& s : lenl.subs) lout[{s.qout, s.sout}].push_back(&s);
  for (int q = 0; q < EL.n(); ++q)
    for (int so = 0; so < 4; ++so) {
      if (EL.soff[q][so] < 0) continue;
      int ld = ER.dim[q];
      B.add_out(sg.out + psi_off[q] + (int64_t)EL.soff[q][so] * ld, ld, EL.sdim[q][so], ld, 0);
      auto it = lout.find({q, so});
      if (it == lout.end()) continue;
      for (const EnlSub* s : it->second) {
        auto yo = yoff.find({s->b, s->qin});
        if (yo == yoff.end()) continue;
        B.add_term(s->ptr, s->trans ? s->rows : s->cols, sg.Y + yo->second + (int64_t)EL.soff[s->qin][s->sin] * ld, ld,
                   s->cols, s->trans ? 1 : 0, s->sign);
      }
    }
  upload(A);
  upload(B);
}

void Engine::sigma(Sigma& sg, const double* x, double* y) {
  settle();
  CK(cudaMemcpyAsync(sg.in, x, psi_size * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  CK(cudaEventRecord(ev0, stream));
  replay(sg.graph, [&]() {
    run(sg.A);
    run(sg.B);
  });
  CK(cudaEventRecord(ev1, stream));
  CK(cudaMemcpyAsync(y, sg.out, psi_size * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  sigma_pending = 1;
  stats.sigma_flops += sg.A.flops + sg.B.flops;
  stats.n_sigma++;
}

// diag(Q)[i,j] = sum_{b: delta_b = 0} Lenl[b](i,i) Renl[b](j,j)
void Engine::compute_diag(const EnlOp& lenl, const EnlOp& renl, double* diag) {
  int mid = cur_k + 1;
  std::vector<int> zc;   // channel -> column index
  std::vector<int> col(mpo.labels[mid].size(), -1);
  for (int b = 0; b < (int)mpo.labels[mid].size(); ++b)
    if (mpo.dA[mid][b] == 0 && mpo.dB[mid][b] == 0) {
      col[b] = (int)zc.size();
      zc.push_back(b);
    }
  int nz = (int)zc.size();
  std::vector<int64_t> dl_off(EL.n() + 1, 0), dr_off(EL.n() + 1, 0);
  for (int q = 0; q < EL.n(); ++q) {
    dl_off[q + 1] = dl_off[q] + (int64_t)EL.dim[q] * nz;
    dr_off[q + 1] = dr_off[q] + (int64_t)nz * ER.dim[q];
  }
  double* DL = dalloc<double>(dl_off.back());
  double* DR = dalloc<double>(dr_off.back());
  CK(cudaMemsetAsync(DL, 0, dl_off.back() * sizeof(double), stream));
  CK(cudaMemsetAsync(DR, 0, dr_off.back() * sizeof(double), stream));
  // gathers expressed as 1-wide GEMMs would be wasteful; use strided axpy:
  // each diagonal element is one 1x1 output of a GEMM with K=1 (A = element,
  // B = 1).  Cheaper: copy via the axpy kernel on strided views is not
  // supported, so gather on the device with tiny GEMMs of shape m x 1.
  GemmPlan g;
  static const double one = 1.0;
  double* d_one = dalloc<double>(1);
  h2d(d_one, &one, sizeof(double));
  for (const auto& s : lenl.subs) {
    if (s.qin != s.qout || s.sin != s.sout || col[s.b] < 0 || s.rows != s.cols) continue;
    // column vector of the diagonal: rows r -> DL(q)[soff + r, col]
    // express as M=rows, N=1, K=1 with A = diag elements (lda = cols+1), B = one
    g.add_out(DL + dl_off[s.qin] + (int64_t)EL.soff[s.qin][s.sin] * nz + col[s.b], nz, s.rows, 1, 0);
    g.add_term(s.ptr, s.cols + 1, d_one, 1, 1, 0, s.sign);
  }
  for (const auto& s : renl.subs) {
    if (s.qin != s.qout || s.sin != s.sout || col[s.b] < 0 || s.rows != s.cols) continue;
    // row vector: DR(q)[col, soff + r]: M=1, N=rows, K=1, A = one, B = diag (ldb = cols+1, transB)
    g.add_out(DR + dr_off[s.qin] + (int64_t)col[s.b] * ER.dim[s.qin] + ER.soff[s.qin][s.sin], 1, 1, s.rows, 0);
    g.add_term(d_one, 1, s.ptr, s.cols + 1, 1, 2, s.sign);
  }
  upload(g);
  run(g);
  release(g);
  GemmPlan p;
  for (int q = 0; q < EL.n(); ++q) {
    p.add_out(diag + psi_off[q], ER.dim[q], EL.dim[q], ER.dim[q], 0);
    if (nz > 0) p.add_term(DL + dl_off[q], nz, DR + dr_off[q], ER.dim[q], nz, 0, 1.0);
  }
  upload(p);
  run(p);
  release(p);
  dfree(DL);
  dfree(DR);
  dfree(d_one);
}

// Shift-and-invert inner PCG on the projected correction equation
// (I - x x^T)(H - theta)(I - x x^T) t = -r, t orthogonal to x, from t = 0
// with the projected diagonal preconditioner; a direction of non-positive
// curvature ends it (on the first direction the result is the
// preconditioned residual, i.e. the Olsen correction).  cg holds 4 psi_size
// work vectors, partial/nblk the reduction scratch, dsums 4 doubles.
void Engine::inner_pcg(const std::function<void(const double*, double*)>& op, const double* diag, const double* xr,
                       const double* rr_vec, double th, double* tout, double* cg, double* partial, int nblk,
                       double* dsums) {
  const int64_t n = psi_size;
  auto dot_host = [&](const double* a, const double* b) {
    launch_multi_dot(a, n, 1, b, n, dsums + 2, partial, nblk, stream);
    stats.launches += 2;
    double v;
    CK(cudaMemcpyAsync(&v, dsums + 2, sizeof(double), cudaMemcpyDeviceToHost, stream));
    sync();
    settle();
    stats.d2h += sizeof(double);
    return v;
  };
  double *res = cg, *z = cg + n, *p = cg + 2 * n, *ap = cg + 3 * n;
  launch_axpby(res, -1.0, rr_vec, 0.0, n, stream);
  const double xr0 = dot_host(xr, res);
  launch_axpby(res, -xr0, xr, 1.0, n, stream);
  CK(cudaMemsetAsync(tout, 0, n * sizeof(double), stream));
  launch_projected_precond(res, xr, diag, th, 1.0, n, z, partial, nblk, dsums, stream);
  CK(cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  stats.launches += 6;
  double rz = dot_host(res, z);
  const double nrhs = std::sqrt(std::max(dot_host(res, res), 0.0));
  for (int j = 0; j < pcg_steps; ++j) {
    op(p, ap);
    stats.inner_matvecs++;
    launch_axpby(ap, -th, p, 1.0, n, stream);
    const double xa = dot_host(xr, ap);
    launch_axpby(ap, -xa, xr, 1.0, n, stream);
    stats.launches += 2;
    const double pap = dot_host(p, ap);
    if (!(pap > 0.0)) {
      if (j == 0) CK(cudaMemcpyAsync(tout, z, n * sizeof(double), cudaMemcpyDeviceToDevice, stream));
      break;
    }
    const double alpha = rz / pap;
    launch_axpby(tout, alpha, p, 1.0, n, stream);
    launch_axpby(res, -alpha, ap, 1.0, n, stream);
    stats.launches += 2;
    if (std::sqrt(std::max(dot_host(res, res), 0.0)) < pcg_rel_tol * nrhs) break;
    launch_projected_precond(res, xr, diag, th, 1.0, n, z, partial, nblk, dsums, stream);
    const double rz1 = dot_host(res, z);
    launch_axpby(p, 1.0, z, rz1 / rz, n, stream);
    stats.launches += 4;
    rz = rz1;
  }
  if (pcg_steps == 0) CK(cudaMemcpyAsync(tout, z, n * sizeof(double), cudaMemcpyDeviceToDevice, stream));
}

// ------------------------------------------------------------------ Davidson
// Davidson (ground state) on the two-site state: Rayleigh-Ritz in FP64 on
// the host, vectors on the device; preconditioner t = -r / (diag - theta)
// with |diag - theta| clamped to 1e-8; two classical Gram-Schmidt passes;
// restart from the 4 lowest Ritz vectors when the space is full.
double Engine::davidson(const std::function<void(const double*, double*)>& op, const double* diag, double tol,
                        int max_iter, int max_space, double stag_rel) {
  // Two host synchronisations per iteration: the residual norm (convergence
  // test) and the new row of the projected matrix.  Gram-Schmidt
  // coefficients and the normalisation never leave the device.
  const int64_t n = psi_size;
  const int keep = 4;
  double* V = dalloc<double>((size_t)max_space * n);
  double* S = dalloc<double>((size_t)max_space * n);
  double* Vt = dalloc<double>((size_t)keep * n);
  double* St = dalloc<double>((size_t)keep * n);
  double* x = dalloc<double>(n);
  double* sx = dalloc<double>(n);
  double* r = dalloc<double>(n);
  double* t = dalloc<double>(n);
  int nblk = reduction_blocks(n);
  double* partial = dalloc<double>((size_t)nblk * (max_space + 2));
  double* dres = dalloc<double>(1);                 // ||r||^2
  double* dorth = dalloc<double>(max_space);        // Gram-Schmidt overlaps
  double* drow = dalloc<double>(max_space + 2);     // [V^T s_k, |t|^2]
  double* coef = dalloc<double>((size_t)max_space * keep + max_space);
  // Olsen / inner PCG: two sums, and the PCG vectors (residual, z, p, A p)
  const int pk = sched.precond;
  double* dsums = (pk == 2 || pk == 3) ? dalloc<double>(4) : nullptr;
  double* cg = pk == 3 ? dalloc<double>((size_t)4 * n) : nullptr;
  std::vector<double> Hs((size_t)max_space * max_space, 0.0), hd(max_space + 2);
  auto d2h = [&](double* host, const double* dev, int cnt) {
    CK(cudaMemcpyAsync(host, dev, cnt * sizeof(double), cudaMemcpyDeviceToHost, stream));
    sync();
    settle();
    stats.d2h += cnt * sizeof(double);
  };
  auto h2d = [&](double* dev, const double* host, int cnt) {
    this->h2d(dev, host, cnt * sizeof(double));
    stats.h2d += cnt * sizeof(double);
  };
  auto dots = [&](const double* base, int k, const double* vec, double* out_dev) {
    launch_multi_dot(base, n, k, vec, n, out_dev, partial, nblk, stream);
    stats.launches += 2;
  };
  // H_eff plus the deflation penalty w sum_j phi_j (phi_j . x)
  const int nphi = defl_phi ? (int)defl.size() : 0;
  double* dpen = nphi ? dalloc<double>(nphi) : nullptr;
  auto opp = [&](const double* a, double* b) {
    op(a, b);
    if (nphi) {
      dots(defl_phi, nphi, a, dpen);
      launch_lincomb(b, defl_phi, n, dpen, nphi, n, 1, stream, defl_w);
      stats.launches++;
    }
  };
  auto dot_host = [&](const double* a, const double* b) {
    dots(a, 1, b, dsums + 2);
    double v;
    d2h(&v, dsums + 2, 1);
    return v;
  };
  // v0 = psi / |psi|, s0 = H v0
  dots(psi, 1, psi, drow + max_space + 1);
  launch_normalize(psi, drow + max_space + 1, n, V, stream);
  stats.launches++;
  opp(V, S);
  dots(V, 1, S, drow);
  CK(cudaMemcpyAsync(hd.data(), drow, (max_space + 2) * sizeof(double), cudaMemcpyDeviceToHost, stream));
  sync();
  settle();
  if (!(hd[max_space + 1] > 0)) throw Error(-4, "two-site guess vector has zero norm");
  Hs[0] = hd[0];
  std::vector<double> rhist;
  int k = 1;
  double theta = hd[0];
  // learned preconditioner: RMS of (d - theta) from sums of d and d^2
  const bool learned = sched.precond == 1 && mlp_loaded;
  bool fallback = false;
  double sum_d = 0, sum_dd = 0;
  int* dbad = nullptr;
  if (learned || recording) {
    std::vector<double> hdiag(n);
    CK(cudaMemcpyAsync(hdiag.data(), diag, n * sizeof(double), cudaMemcpyDeviceToHost, stream));
    sync();
    for (double v : hdiag) {
      sum_d += v;
      sum_dd += v * v;
    }
    dbad = dalloc<int>(1);
    CK(cudaMemsetAsync(dbad, 0, sizeof(int), stream));
  }
  auto scalars = [&](double th, double rn, int it) {
    double var = (sum_dd - 2.0 * th * sum_d) / (double)n + th * th;
    return MlpScalars{th, rn + 1e-300, std::sqrt(std::max(var, 0.0)) + 1e-300, (double)it};
  };
  std::vector<double> w(max_space), Z((size_t)max_space * max_space), hk((size_t)max_space * max_space);
  for (int it = 0;; ++it) {
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) hk[(size_t)i * k + j] = 0.5 * (Hs[(size_t)i * max_space + j] + Hs[(size_t)j * max_space + i]);
    if (sym_eig(k, hk.data(), w.data(), Z.data()) != 0) throw Error(-4, "Rayleigh-Ritz eigensolver failed");
    theta = w[0];
    std::vector<double> c(k);
    for (int i = 0; i < k; ++i) c[i] = Z[(size_t)i * k + 0];
    h2d(coef, c.data(), k);
    launch_lincomb(x, V, n, coef, k, n, 0, stream);
    launch_lincomb(sx, S, n, coef, k, n, 0, stream);
    launch_residual_precond(x, sx, diag, theta, n, r, t, partial, nblk, dres, stream);
    stats.launches += 4;
    double rr;
    d2h(&rr, dres, 1);
    double rn = std::sqrt(std::max(rr, 0.0));
    stats.last_residual = rn;
    if (rn < tol || it >= max_iter) break;
    // reduced-precision operators have a residual floor near u |theta| (u =
    // the operator's relative error): below stag_rel * max(1, |theta|),
    // stop when three iterations have not reduced ||r|| by 30 %.  Above it
    // a plateau is ordinary Davidson behaviour (e.g. from a random start)
    // and the solve goes on, as the FP64 one does.
    rhist.push_back(rn);
    const double floor_here = stag_rel * std::max(1.0, std::fabs(theta));
    if (stag_rel > 0 && rhist.size() > 3 && rn > 0.7 * rhist[rhist.size() - 4] && rn < floor_here) break;
    // a reduced-precision tier that has not cut ||r|| by 30 % over
    // hard_stag_iters iterations stops at any level
    const size_t hs = (size_t)hard_stag_iters;
    if (stag_rel > 0 && hs > 0 && rhist.size() > hs && rn > 0.7 * rhist[rhist.size() - 1 - hs]) break;
    stats.davidson_iters++;
    if (recording) record_iteration(r, diag, x, scalars(theta, rn, it));
    if (learned && !fallback) {
      // back to the diagonal preconditioner when ||r|| has not dropped over
      // three iterations
      if (rhist.size() > 3 && rn >= rhist[rhist.size() - 4]) {
        fallback = true;
        stats.precond_fallbacks++;
      } else {
        launch_mlp_precond(r, diag, scalars(theta, rn, it), n, mlp_w16, t, dbad, stream);
        stats.launches++;
      }
    } else if (pk == 2) {
      launch_projected_precond(r, x, diag, theta, -1.0, n, t, partial, nblk, dsums, stream);   // Olsen
      stats.launches += 3;
    } else if (pk == 3) {
      inner_pcg(opp, diag, x, r, theta, t, cg, partial, nblk, dsums);
    }
    if (k == max_space) {
      int kk = std::min(keep, k);
      std::vector<double> cc((size_t)kk * k);
      for (int j = 0; j < kk; ++j)
        for (int i = 0; i < k; ++i) cc[(size_t)j * k + i] = Z[(size_t)i * k + j];
      h2d(coef, cc.data(), kk * k);
      for (int j = 0; j < kk; ++j) {
        launch_lincomb(Vt + (size_t)j * n, V, n, coef + (size_t)j * k, k, n, 0, stream);
        launch_lincomb(St + (size_t)j * n, S, n, coef + (size_t)j * k, k, n, 0, stream);
        stats.launches += 2;
      }
      CK(cudaMemcpyAsync(V, Vt, (size_t)kk * n * sizeof(double), cudaMemcpyDeviceToDevice, stream));
      CK(cudaMemcpyAsync(S, St, (size_t)kk * n * sizeof(double), cudaMemcpyDeviceToDevice, stream));
      std::fill(Hs.begin(), Hs.end(), 0.0);
      for (int j = 0; j < kk; ++j) Hs[(size_t)j * max_space + j] = w[j];
      k = kk;
    }
    // t <- t - V (V^T t), twice; v_k = t / |t|; s_k = H v_k
    for (int pass = 0; pass < 2; ++pass) {
      dots(V, k, t, dorth);
      launch_lincomb(t, V, n, dorth, k, n, 1, stream, -1.0);
      stats.launches++;
    }
    dots(t, 1, t, drow + max_space + 1);
    launch_normalize(t, drow + max_space + 1, n, V + (size_t)k * n, stream);
    stats.launches++;
    opp(V + (size_t)k * n, S + (size_t)k * n);
    dots(V, k + 1, S + (size_t)k * n, drow);
    CK(cudaMemcpyAsync(hd.data(), drow, (max_space + 2) * sizeof(double), cudaMemcpyDeviceToHost, stream));
    int hbad = 0;
    if (dbad) CK(cudaMemcpyAsync(&hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, stream));
    sync();
    settle();
    stats.d2h += (max_space + 2) * sizeof(double);
    if (hbad) {   // non-finite learned correction: drop it, use the diagonal from now on
      fallback = true;
      stats.precond_fallbacks++;
      CK(cudaMemsetAsync(dbad, 0, sizeof(int), stream));
      continue;
    }
    if (!(hd[max_space + 1] > 1e-28)) break;   // breakdown: t had no new direction
    for (int i = 0; i <= k; ++i) {
      Hs[(size_t)i * max_space + k] = hd[i];
      Hs[(size_t)k * max_space + i] = hd[i];
    }
    ++k;
  }
  // psi <- normalised Ritz vector
  dots(x, 1, x, drow + max_space + 1);
  launch_normalize(x, drow + max_space + 1, n, psi, stream);
  stats.launches++;
  if (recording) {
    sync();
    record_converged(psi);
  }
  if (dbad) dfree(dbad);
  for (void* p : {(void*)V, (void*)S, (void*)Vt, (void*)St, (void*)x, (void*)sx, (void*)r, (void*)t, (void*)partial,
                  (void*)dres, (void*)dorth, (void*)drow, (void*)coef})
    dfree(p);
  if (dsums) dfree(dsums);
  if (cg) dfree(cg);
  if (dpen) dfree(dpen);
  return theta;
}

// account the sigma build recorded by the last sigma()/tc_apply() once the
// stream has passed it
void Engine::settle() {
  if (!sigma_pending) return;
  CK(cudaEventSynchronize(ev1));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, ev0, ev1));
  stats.sigma_ms += ms;
  if (sigma_pending == 2) {
    stats.tc_ms += ms;
    float g = 0;
    CK(cudaEventElapsedTime(&g, evg0, evg1));
    float ga = 0;
    CK(cudaEventElapsedTime(&ga, evg0, evgm));
    stats.tc_gemm_ms_st[0] += ga;
    stats.tc_gemm_ms_st[1] += g - ga;
    stats.tc_gemm_ms += g;
    stats.tc_gemm_ms_p[stats.last_tc_prec] += g;
    if (*tc_err_host) throw Error(-5, "tensor-core sigma: a bounded device wait ran out");
  }
  sigma_pending = 0;
}

// ------------------------------------------------------------------ decimation
// Keep the M largest sigma^2 over all sectors (after dropping sigma^2 <=
// cutoff); equal values ordered by (sector, in-sector rank); a cluster of
// weights within `tie` of each other is never split at the cut.
void Engine::truncate(int k, int dir, int M, double* tau_out, std::vector<double>* kept_out) {
  const int nq = EL.n();
  std::vector<int64_t> roff(nq + 1, 0);
  std::vector<int> md(nq);
  for (int q = 0; q < nq; ++q) {
    md[q] = dir == 0 ? EL.dim[q] : ER.dim[q];
    roff[q + 1] = roff[q] + (int64_t)md[q] * md[q];
  }
  double tt0 = now_ms();
  double* rho = dalloc<double>(roff.back());
  GemmPlan p;
  for (int q = 0; q < nq; ++q) {
    const double* P = psi + psi_off[q];
    p.add_out(rho + roff[q], md[q], md[q], md[q], 0);
    if (dir == 0) p.add_term(P, ER.dim[q], P, ER.dim[q], ER.dim[q], 2, 1.0);
    else p.add_term(P, ER.dim[q], P, ER.dim[q], EL.dim[q], 1, 1.0);
  }
  upload(p);
  run(p);
  release(p);
  std::vector<double> h_rho(roff.back());
  CK(cudaMemcpyAsync(h_rho.data(), rho, roff.back() * sizeof(double), cudaMemcpyDeviceToHost, stream));
  sync();
  stats.d2h += roff.back() * sizeof(double);
  dfree(rho);
  double tt1 = now_ms();
  stats.trunc_rho_ms += tt1 - tt0;
  std::vector<std::vector<double>> ew(nq), ev(nq);
  std::atomic<int> fail(0);
  // largest sectors first, so that the longest eigensolve never starts last
  std::vector<int> byq(nq);
  std::iota(byq.begin(), byq.end(), 0);
  std::stable_sort(byq.begin(), byq.end(), [&](int a, int b) { return md[a] > md[b]; });
  parallel_for(nq, [&](int qi) {
    const int q = byq[qi];
    int m = md[q];
    ew[q].resize(m);
    ev[q].resize((size_t)m * m);
    if (sym_eig(m, h_rho.data() + roff[q], ew[q].data(), ev[q].data()) != 0) fail = 1;
  });
  if (fail) throw Error(-4, "density-matrix eigensolver failed");
  stats.trunc_eig_ms += now_ms() - tt1;
  std::vector<Weight> all;
  for (int q = 0; q < nq; ++q) {
    int m = md[q];
    for (int j = 0; j < m; ++j) all.push_back({ew[q][m - 1 - j], qkey(EL.qa[q], EL.qb[q]), q, j});
  }
  double total = 0, kept_sum = 0;
  std::vector<Weight> kw = select_states(all, M, sched.cutoff, sched.tie, &total, adapt_disc, adapt_mmin);
  std::vector<int> nkeep(nq, 0);
  for (auto& w : kw) {
    nkeep[w.idx]++;
    kept_sum += w.lam;
    if (kept_out) kept_out->push_back(w.lam);
  }
  double tau = total - kept_sum;
  if (tau_out) *tau_out = tau;
  stats.max_discarded = std::max(stats.max_discarded, tau);
  // new bond k+1
  Bond nb;
  std::vector<int> qmap;   // new sector -> two-site sector index
  for (int q = 0; q < nq; ++q)
    if (nkeep[q] > 0) {
      nb.na.push_back(EL.qa[q]);
      nb.nb.push_back(EL.qb[q]);
      nb.dim.push_back(nkeep[q]);
    }
  nb.finalize();
  for (int j = 0; j < nb.nsec(); ++j) qmap.push_back(EL.find(nb.na[j], nb.nb[j]));
  bonds[k + 1] = nb;
  // basis matrices
  Site U;
  int which = dir == 0 ? k : k + 1;
  free_site(sites[which]);
  layout_site(which, dir == 0 ? 0 : 1, U);
  std::vector<double> hU(U.size);
  for (int j = 0; j < nb.nsec(); ++j) {
    int q = qmap[j], m = md[q], nkq = nb.dim[j];
    double* dst = hU.data() + U.off[j];
    for (int c = 0; c < nkq; ++c)
      for (int i = 0; i < m; ++i) {
        double v = ev[q][(size_t)i * m + (m - 1 - c)];
        if (dir == 0) dst[(size_t)i * nkq + c] = v;   // U: m_EL x nk
        else dst[(size_t)c * m + i] = v;              // B = V^T: nk x m_ER
      }
  }
  U.d = dalloc<double>(U.size);
  h2d(U.d, hU.data(), U.size * sizeof(double));
  stats.h2d += U.size * sizeof(double);
  sites[which] = U;
  // center = U^T psi (L->R, site k+1 fused-right) or psi B^T (R->L, site k fused-left)
  int cw = dir == 0 ? k + 1 : k;
  free_site(sites[cw]);
  Site C;
  layout_site(cw, dir == 0 ? 1 : 0, C);
  C.d = dalloc<double>(C.size);
  GemmPlan pc;
  for (int j = 0; j < nb.nsec(); ++j) {
    int q = qmap[j], nkq = nb.dim[j];
    const double* P = psi + psi_off[q];
    if (dir == 0) {
      pc.add_out(C.d + C.off[j], ER.dim[q], nkq, ER.dim[q], 0);
      pc.add_term(U.d + U.off[j], nkq, P, ER.dim[q], EL.dim[q], 1, 1.0);
    } else {
      pc.add_out(C.d + C.off[j], nkq, EL.dim[q], nkq, 0);
      pc.add_term(P, ER.dim[q], U.d + U.off[j], ER.dim[q], ER.dim[q], 2, 1.0);
    }
  }
  upload(pc);
  run(pc);
  release(pc);
  sites[cw] = C;
}

// ------------------------------------------------------------------ one step
// Davidson of one step.  FP64 schedule: plain FP64 Davidson.  Reduced
// precision: tier 1 (BF16 or TF32 single pass) while the residual is large,
// tier 2 (TF32x3, split-K FP64 sums) to its floor, then at most `refine`
// FP64 iterations.  Each tier restarts from the previous tier's Ritz vector.
double Engine::solve_tiers(Sigma& sg, const double* diag, double tol, int precision, int refine, bool& planned) {
  double theta = 0;
  auto fp64op = [&](const double* x, double* y) {
    if (!planned) {
      plan_sigma(sg.lenl, sg.renl, sg);
      planned = true;
    }
    sigma(sg, x, y);
  };
  int64_t it0 = stats.davidson_iters;
  auto tier_done = [&](int t) {
    stats.tier_iters[t] += stats.davidson_iters - it0;
    it0 = stats.davidson_iters;
  };
  // a small two-site state (chain ends) costs more to plan and convert for
  // the tensor cores than its FP64 sigma takes: such steps stay FP64
  if (precision == 0 || psi_size < tc_min_two_site) {
    theta = davidson(fp64op, diag, tol, sched.max_iter, sched.max_space, 0.0);
    tier_done(2);
  } else {
    const int p1 = precision == 2 ? kBF16 : kTF32;
    const double floor1 = p1 == kBF16 ? 5e-2 : 1e-2;
    // measured relative sigma errors: BF16 2e-3, TF32 3e-4, TF32x3 2e-6, BF16x3 (see the
    // accuracy tests) of the same order
    const double u1 = p1 == kBF16 ? 2e-3 : 3e-4, u2 = tier2 == kBF16x3 ? 6e-6 : 3e-6;
    TcPlan* P = nullptr;
    stats.last_residual = 1e300;
    if (!skip_tier1) {
      P = tc_plan(sg.lenl, sg.renl, p1);
      theta = davidson([&](const double* x, double* y) { tc_apply(P, x, y); }, diag, std::max(tol, floor1),
                       sched.max_iter, sched.max_space, 10.0 * u1);
      tc_free(P);
      t1_iters_cur += stats.davidson_iters - it0;
      t1_steps_cur++;
      tier_done(0);
    }
    if (stats.last_residual >= tol) {
      P = tc_plan(sg.lenl, sg.renl, tier2);
      theta = davidson([&](const double* x, double* y) { tc_apply(P, x, y); }, diag, tol, sched.max_iter,
                       sched.max_space, tier2_floor_mult * u2);
      tc_free(P);
      tier_done(1);
    }
    if (refine > 0 && stats.last_residual >= tol) {
      theta = davidson(fp64op, diag, tol, refine, sched.max_space, 0.0);
      tier_done(2);
    }
  }
  stats.max_final_residual = std::max(stats.max_final_residual, stats.last_residual);
  stats.sum_final_residual += stats.last_residual;
  stats.sweep_max_residual = std::max(stats.sweep_max_residual, stats.last_residual);
  stats.n_solves++;
  if (stats.last_residual >= tol) stats.n_above_tol++;
  return theta;
}

void Engine::free_sigma(Sigma& sg, bool planned) {
  if (!planned) return;
  drop(sg.graph);
  release(sg.A);
  release(sg.B);
  dfree(sg.Y);
  dfree(sg.in);
  dfree(sg.out);
}

void Engine::probe_step(int k, int precision, int refine, double tol, double* theta, double* e64, double* r64) {
  if (k < 0 || k + 1 >= n || !Lenv[k].valid || !Renv[k + 2].valid)
    throw Error(-6, "probe_step needs valid environments at the centre k");
  setup_two_site(k);
  form_psi(k, 0);
  Sigma sg;
  AxpyPlan ax;
  build_lenl(k, Lenv[k], EL, sg.lenl, ax);
  finish_enl(sg.lenl, ax);
  build_renl(k + 1, Renv[k + 2], ER, sg.renl, ax);
  finish_enl(sg.renl, ax);
  double* diag = dalloc<double>(psi_size);
  compute_diag(sg.lenl, sg.renl, diag);
  bool planned = false;
  *theta = solve_tiers(sg, diag, tol, precision, refine, planned);
  if (!planned) {
    plan_sigma(sg.lenl, sg.renl, sg);
    planned = true;
  }
  double* y = dalloc<double>(psi_size);
  sigma(sg, psi, y);
  std::vector<double> hx(psi_size), hy(psi_size);
  CK(cudaMemcpyAsync(hx.data(), psi, psi_size * sizeof(double), cudaMemcpyDeviceToHost, stream));
  CK(cudaMemcpyAsync(hy.data(), y, psi_size * sizeof(double), cudaMemcpyDeviceToHost, stream));
  sync();
  settle();
  double xx = 0, xy = 0;
  for (int64_t i = 0; i < psi_size; ++i) {
    xx += hx[i] * hx[i];
    xy += hx[i] * hy[i];
  }
  const double e = xy / xx;
  double rr = 0;
  for (int64_t i = 0; i < psi_size; ++i) {
    const double d = hy[i] - e * hx[i];
    rr += d * d;
  }
  *e64 = e;
  *r64 = std::sqrt(rr / xx);
  dfree(y);
  dfree(diag);
  free_sigma(sg, planned);
  free_enl(sg.lenl);
  free_enl(sg.renl);
  sync();
}

void Engine::pcg_selftest(int k, const double* x_host, const double* r_host, double theta, double* t_host,
                          int64_t* matvecs) {
  if (k < 0 || k + 1 >= n || !Lenv[k].valid || !Renv[k + 2].valid)
    throw Error(-6, "pcg_selftest needs valid environments at the centre k");
  setup_two_site(k);
  Sigma sg;
  AxpyPlan ax;
  build_lenl(k, Lenv[k], EL, sg.lenl, ax);
  finish_enl(sg.lenl, ax);
  build_renl(k + 1, Renv[k + 2], ER, sg.renl, ax);
  finish_enl(sg.renl, ax);
  double* diag = dalloc<double>(psi_size);
  compute_diag(sg.lenl, sg.renl, diag);
  plan_sigma(sg.lenl, sg.renl, sg);
  const int64_t N = psi_size;
  double* x = dalloc<double>(N);
  double* r = dalloc<double>(N);
  double* t = dalloc<double>(N);
  double* cg = dalloc<double>((size_t)4 * N);
  const int nblk = reduction_blocks(N);
  double* partial = dalloc<double>((size_t)2 * nblk);
  double* dsums = dalloc<double>(4);
  // host vectors in the canonical two-site format <-> the fused layout
  const std::vector<CanonMap> maps = canonical_maps(k);
  std::vector<double> hx(N), hr(N), ht(N);
  to_fused(maps, x_host, hx.data());
  to_fused(maps, r_host, hr.data());
  CK(cudaMemcpyAsync(x, hx.data(), N * sizeof(double), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(r, hr.data(), N * sizeof(double), cudaMemcpyHostToDevice, stream));
  const int64_t m0 = stats.inner_matvecs;
  inner_pcg([&](const double* a, double* b) { sigma(sg, a, b); }, diag, x, r, theta, t, cg, partial, nblk, dsums);
  CK(cudaMemcpyAsync(ht.data(), t, N * sizeof(double), cudaMemcpyDeviceToHost, stream));
  sync();
  settle();
  from_fused(maps, ht.data(), t_host);
  *matvecs = stats.inner_matvecs - m0;
  for (void* q : {(void*)x, (void*)r, (void*)t, (void*)cg, (void*)partial, (void*)dsums, (void*)diag}) dfree(q);
  free_sigma(sg, true);
  free_enl(sg.lenl);
  free_enl(sg.renl);
  sync();
}

double Engine::step(int k, int dir, int M, double tol, double* tau, std::vector<double>* kept) {
  double t0 = now_ms();
  setup_two_site(k);
  form_psi(k, 0);
  Sigma sg;
  AxpyPlan ax;
  double te = now_ms();
  build_lenl(k, Lenv[k], EL, sg.lenl, ax);
  double th = now_ms() - te;
  finish_enl(sg.lenl, ax);
  double t1 = now_ms();
  build_renl(k + 1, Renv[k + 2], ER, sg.renl, ax);
  th += now_ms() - t1;
  finish_enl(sg.renl, ax);
  stats.enl_ms += now_ms() - te;
  stats.enl_host_ms += th;
  double tdg = now_ms();
  double* diag = dalloc<double>(psi_size);
  compute_diag(sg.lenl, sg.renl, diag);
  if (!defl.empty()) {
    // deflated states: their projections, and the diagonal of the penalty
    defl_phi = dalloc<double>((size_t)defl.size() * psi_size);
    deflation_vectors(k, defl_phi);
    launch_add_sq(diag, defl_phi, (int)defl.size(), psi_size, defl_w, stream);
  }
  stats.diag_ms += now_ms() - tdg;
  double td = now_ms();
  double theta = 0;
  bool planned = false;
  theta = solve_tiers(sg, diag, tol, sched.precision, sched.refine, planned);
  stats.davidson_ms += now_ms() - td;
  dfree(diag);
  if (defl_phi) {
    dfree(defl_phi);
    defl_phi = nullptr;
  }
  free_sigma(sg, planned);
  double tt = now_ms();
  truncate(k, dir, M, tau, kept);
  stats.trunc_ms += now_ms() - tt;
  // environment update on the side the sweep moves away from
  if (dir == 0) {
    Space el2 = EL;
    env_update_left(sg.lenl, el2, sites[k], bonds[k + 1], Lenv[k + 1]);
    Renv[k + 1].valid = false;
    for (int j = 0; j < (int)defl.size(); ++j) ov_update_left(j, k);
  } else {
    env_update_right(sg.renl, ER, sites[k + 1], bonds[k + 1], Renv[k + 1]);
    Lenv[k + 1].valid = false;
    for (int j = 0; j < (int)defl.size(); ++j) ov_update_right(j, k + 1);
  }
  free_enl(sg.lenl);
  free_enl(sg.renl);
  // no synchronisation: the next step's host planning overlaps these launches
  stats.n_steps++;
  stats.step_ms += now_ms() - t0;
  return theta;
}

// ------------------------------------------------------------------ initial MPS
void Engine::init_mps(uint64_t seed, int M) {
  bonds = initial_bond_dims(n, Na, Nb, M);
  // fused-right host tensors with counter-based entries
  std::vector<std::vector<double>> hs(n);
  std::vector<Site> lay(n);
  for (int i = 0; i < n; ++i) {
    layout_site(i, 1, lay[i]);
    hs[i].assign(lay[i].size, 0.0);
    const Bond& bl = bonds[i];
    const Bond& br = bonds[i + 1];
    for (int j = 0; j < bl.nsec(); ++j) {
      int cols = 0;
      int coff[4];
      for (int s = 0; s < 4; ++s) {
        int r = br.find(bl.na[j] + QA[s], bl.nb[j] + QB[s]);
        coff[s] = r >= 0 ? cols : -1;
        if (r >= 0) cols += br.dim[r];
      }
      for (int s = 0; s < 4; ++s) {
        if (coff[s] < 0) continue;
        int r = br.find(bl.na[j] + QA[s], bl.nb[j] + QB[s]);
        for (int row = 0; row < bl.dim[j]; ++row)
          for (int col = 0; col < br.dim[r]; ++col)
            hs[i][lay[i].off[j] + (int64_t)row * cols + coff[s] + col] =
                mps_init_value(seed, i, bl.na[j], bl.nb[j], s, row, col);
      }
    }
  }
  // right-canonicalise sites n-1 .. 1; absorb the triangular factor leftwards
  for (int i = n - 1; i >= 1; --i) {
    const Bond& bl = bonds[i];
    const Bond& bp = bonds[i - 1];
    for (int j = 0; j < bl.nsec(); ++j) {
      int m = bl.dim[j];
      int cols = (int)((j + 1 < bl.nsec() ? lay[i].off[j + 1] : lay[i].size) - lay[i].off[j]) / m;
      std::vector<double> Lo((size_t)m * m);
      if (row_orthonormalize(m, cols, hs[i].data() + lay[i].off[j], Lo.data()) != 0)
        throw Error(-4, "initial MPS is rank deficient");
      for (int jp = 0; jp < bp.nsec(); ++jp) {
        int coff = 0, pcols = 0, s_hit = -1, hit_off = 0;
        for (int s = 0; s < 4; ++s) {
          int r = bl.find(bp.na[jp] + QA[s], bp.nb[jp] + QB[s]);
          if (r < 0) continue;
          if (r == j) { s_hit = s; hit_off = coff; }
          coff += bl.dim[r];
        }
        pcols = coff;
        if (s_hit < 0) continue;
        int mp = bp.dim[jp];
        double* base = hs[i - 1].data() + lay[i - 1].off[jp];
        std::vector<double> tmp((size_t)mp * m);
        for (int rr = 0; rr < mp; ++rr)
          for (int c = 0; c < m; ++c) {
            double s = 0;
            for (int t = 0; t < m; ++t) s += base[(size_t)rr * pcols + hit_off + t] * Lo[(size_t)t * m + c];
            tmp[(size_t)rr * m + c] = s;
          }
        for (int rr = 0; rr < mp; ++rr)
          for (int c = 0; c < m; ++c) base[(size_t)rr * pcols + hit_off + c] = tmp[(size_t)rr * m + c];
      }
    }
  }
  double nrm = 0;
  for (double v : hs[0]) nrm += v * v;
  nrm = std::sqrt(nrm);
  for (double& v : hs[0]) v /= nrm;
  for (auto& s : sites) free_site(s);
  sites.assign(n, Site());
  for (int i = 0; i < n; ++i) {
    sites[i] = lay[i];
    sites[i].d = dalloc<double>(lay[i].size);
    CK(cudaMemcpyAsync(sites[i].d, hs[i].data(), lay[i].size * sizeof(double), cudaMemcpyHostToDevice, stream));
    stats.h2d += lay[i].size * sizeof(double);
  }
  sync();
}

void Engine::build_right_envs(int from_k) {
  // R_n = 1 on channel H; R_i = B_i Renl_i B_i^T for i = n-1 .. from_k;
  // environments built outside the sweep steps are FP64
  const bool f0 = force_fp64_env;
  force_fp64_env = true;
  struct Restore { bool& f; bool v; ~Restore() { f = v; } } restore{force_fp64_env, f0};
  env_tc_used = false;
  for (auto& e : Renv) free_env(e);
  Renv.assign(n + 1, Env());
  make_env(n, Renv[n]);
  {
    double one = 1.0;
    int64_t o = Renv[n].at(mpo.ham_channel[n], 0);
    CK(cudaMemcpyAsync(Renv[n].d + o, &one, sizeof(double), cudaMemcpyHostToDevice, stream));
    sync();
  }
  for (int i = n - 1; i >= from_k; --i) {
    Space er = right_space(bonds[i + 1], bond_qs(bonds[i]));
    EnlOp op;
    AxpyPlan ax;
    build_renl(i, Renv[i + 1], er, op, ax);
    finish_enl(op, ax);
    env_update_right(op, er, sites[i], bonds[i], Renv[i]);
    free_enl(op);
  }
}

void Engine::build_left_envs(int to_k) {
  const bool f0 = force_fp64_env;
  force_fp64_env = true;
  struct Restore { bool& f; bool v; ~Restore() { f = v; } } restore{force_fp64_env, f0};
  for (auto& e : Lenv) free_env(e);
  Lenv.assign(n + 1, Env());
  make_env(0, Lenv[0]);
  double one = 1.0;
  int64_t o = Lenv[0].at(mpo.ident_channel[0], 0);
  CK(cudaMemcpyAsync(Lenv[0].d + o, &one, sizeof(double), cudaMemcpyHostToDevice, stream));
  sync();
  for (int i = 0; i < to_k; ++i) {
    Space el = left_space(bonds[i], bond_qs(bonds[i + 1]));
    EnlOp op;
    AxpyPlan ax;
    build_lenl(i, Lenv[i], el, op, ax);
    finish_enl(op, ax);
    env_update_left(op, el, sites[i], bonds[i + 1], Lenv[i + 1]);
    free_enl(op);
  }
}

// ------------------------------------------------------------------ public driver
void Engine::prepare(int n_, int n_elec, int two_sz, int n_chol, const double* h_, const double* chol,
                     double e_core_, const Schedule& sch) {
  CK(cudaSetDevice(device));
  n = n_;
  Na = (n_elec + two_sz) / 2;
  Nb = (n_elec - two_sz) / 2;
  e_core = e_core_;
  sched = sch;
  h.assign(h_, h_ + (size_t)n * n);
  eri.assign((size_t)n * n * n * n, 0.0);
  for (int Q = 0; Q < n_chol; ++Q) {
    const double* L = chol + (size_t)Q * n * n;
    for (int pq = 0; pq < n * n; ++pq) {
      double v = L[pq];
      if (v == 0.0) continue;
      double* row = eri.data() + (size_t)pq * n * n;
      for (int rs = 0; rs < n * n; ++rs) row[rs] += v * L[rs];
    }
  }
  build_mpo(n, h.data(), eri.data(), n / 2, mpo);
  mpo_conjugates(mpo, conj_l, sign_l, conj_r, sign_r);
  clear_states();   // deflated states and a saved MPS belong to the previous problem
  free_snapshot();
  stats = Stats();
  sweep_E.clear();
  prepared = false;
  t1_iters_cur = t1_steps_cur = t1_steps_prev = 0;
  t1_iters_prev = -1;
  skip_tier1 = false;
}

void Engine::free_snapshot() {
  for (auto& st : snap_sites) free_site(st);
  snap_sites.clear();
  snap_bonds.clear();
}

void Engine::save_state() {
  if (!prepared || (int)sites.size() != n) throw Error(-6, "save_state before an MPS exists");
  free_snapshot();
  snap_bonds = bonds;
  for (const Site& st : sites) {
    Site c = st;
    c.d = dalloc<double>(st.size);
    CK(cudaMemcpyAsync(c.d, st.d, st.size * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    snap_sites.push_back(c);
  }
  sync();
}

void Engine::restore_state() {
  if (snap_sites.empty()) throw Error(-6, "restore_state without a saved state");
  for (auto& st : sites) free_site(st);
  sites.assign(n, Site());
  bonds = snap_bonds;
  for (int i = 0; i < n; ++i) {
    Site c = snap_sites[i];
    c.d = dalloc<double>(c.size);
    CK(cudaMemcpyAsync(c.d, snap_sites[i].d, c.size * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    sites[i] = c;
  }
  build_right_envs(2);
  build_left_envs(0);
  sync();
}

void Engine::init_state() {
  init_mps(sched.seed, sched.M.empty() ? 1 : sched.M[0]);
  build_right_envs(2);
  build_left_envs(0);
  prepared = true;
}

double Engine::sweep(int s) {
  if (!prepared) throw Error(-6, "sweep before prepare");
  int M = sched.M[s];
  double tol = sched.tol[s];
  double e = 0;
  if (t1_steps_cur > 0) {   // the last sweep that ran tier 1 decides
    t1_iters_prev = t1_iters_cur;
    t1_steps_prev = t1_steps_cur;
  }
  t1_iters_cur = t1_steps_cur = 0;
  skip_tier1 = s > 0 && t1_steps_prev > 0 && t1_iters_prev < 2 * t1_steps_prev;
  stats.sweep_max_residual = 0;
  for (int k = 0; k <= n - 2; ++k) e = step(k, 0, M, tol, nullptr, nullptr);
  for (int k = n - 2; k >= 0; --k) e = step(k, 1, M, tol, nullptr, nullptr);
  sync();   // every launch of the sweep done and timed
  sweep_E.push_back(e);
  return e;
}

// <psi|H|psi> / <psi|psi> at bond (0,1) of the current MPS, with FP64
// environments (right environments updated on the tensor cores are rebuilt)
double Engine::final_energy() {
  if (env_tc_used) build_right_envs(2);
  setup_two_site(0);
  form_psi(0, 0);
  Sigma sg;
  AxpyPlan ax;
  build_lenl(0, Lenv[0], EL, sg.lenl, ax);
  finish_enl(sg.lenl, ax);
  build_renl(1, Renv[2], ER, sg.renl, ax);
  finish_enl(sg.renl, ax);
  plan_sigma(sg.lenl, sg.renl, sg);
  double* y = dalloc<double>(psi_size);
  sigma(sg, psi, y);
  int nblk = reduction_blocks(psi_size);
  double* partial = dalloc<double>(nblk * 2);
  double* dots = dalloc<double>(2);
  double hv[2];
  launch_multi_dot(psi, psi_size, 1, y, psi_size, dots, partial, nblk, stream);
  launch_multi_dot(psi, psi_size, 1, psi, psi_size, dots + 1, partial + nblk, nblk, stream);
  CK(cudaMemcpyAsync(hv, dots, 2 * sizeof(double), cudaMemcpyDeviceToHost, stream));
  sync();
  release(sg.A);
  release(sg.B);
  for (void* p : {(void*)sg.Y, (void*)sg.in, (void*)sg.out, (void*)y, (void*)partial, (void*)dots}) dfree(p);
  free_enl(sg.lenl);
  free_enl(sg.renl);
  return hv[0] / hv[1];
}

// ------------------------------------------------------------------ test hooks
void Engine::bond_sectors(int bond, std::vector<int>& out) const {
  out.clear();
  const Bond& b = bonds[bond];
  for (int i = 0; i < b.nsec(); ++i) {
    out.push_back(b.na[i]);
    out.push_back(b.nb[i]);
    out.push_back(b.dim[i]);
  }
}

std::vector<uint64_t> Engine::mpo_labels(int bond) const {
  std::vector<uint64_t> v;
  for (auto& l : mpo.labels[bond]) v.push_back(l.key());
  return v;
}

// canonical block order per site i: for q_l in bond i (sorted), s = 0..3,
// q_r = q_l + s in bond i+1: a m_i(q_l) x m_{i+1}(q_r) row-major block
void Engine::set_mps(const int* nsec, const int* sectors, const double* data, int center) {
  bonds.assign(n + 1, Bond());
  int pos = 0;
  for (int k = 0; k <= n; ++k) {
    for (int j = 0; j < nsec[k]; ++j) {
      bonds[k].na.push_back(sectors[pos++]);
      bonds[k].nb.push_back(sectors[pos++]);
      bonds[k].dim.push_back(sectors[pos++]);
    }
    bonds[k].finalize();
  }
  for (auto& s : sites) free_site(s);
  sites.assign(n, Site());
  int64_t dpos = 0;
  for (int i = 0; i < n; ++i) {
    int layout = i < center ? 0 : 1;
    Site s;
    layout_site(i, layout, s);
    std::vector<double> hs(s.size, 0.0);
    const Bond& bl = bonds[i];
    const Bond& br = bonds[i + 1];
    for (int j = 0; j < bl.nsec(); ++j)
      for (int st = 0; st < 4; ++st) {
        int r = br.find(bl.na[j] + QA[st], bl.nb[j] + QB[st]);
        if (r < 0) continue;
        int ml = bl.dim[j], mr = br.dim[r];
        if (layout == 0) {
          // FL block of sector r: rows concat_s (q_r - s); our rows start at soff(st)
          int roff = 0, rows = 0;
          for (int s2 = 0; s2 < 4; ++s2) {
            int jj = bl.find(br.na[r] - QA[s2], br.nb[r] - QB[s2]);
            if (jj < 0) continue;
            if (s2 < st) roff += bl.dim[jj];
            rows += bl.dim[jj];
          }
          double* dst = hs.data() + s.off[r] + (int64_t)roff * mr;
          for (int a = 0; a < ml; ++a)
            for (int c = 0; c < mr; ++c) dst[(size_t)a * mr + c] = data[dpos + (int64_t)a * mr + c];
        } else {
          int coff = 0, cols = 0;
          for (int s2 = 0; s2 < 4; ++s2) {
            int rr = br.find(bl.na[j] + QA[s2], bl.nb[j] + QB[s2]);
            if (rr < 0) continue;
            if (s2 < st) coff += br.dim[rr];
            cols += br.dim[rr];
          }
          double* dst = hs.data() + s.off[j] + coff;
          for (int a = 0; a < ml; ++a)
            for (int c = 0; c < mr; ++c) dst[(size_t)a * cols + c] = data[dpos + (int64_t)a * mr + c];
        }
        dpos += (int64_t)ml * mr;
      }
    s.d = dalloc<double>(s.size);
    CK(cudaMemcpyAsync(s.d, hs.data(), s.size * sizeof(double), cudaMemcpyHostToDevice, stream));
    sync();
    sites[i] = s;
  }
  build_right_envs(center + 2);
  build_left_envs(center);
  prepared = true;
}

int64_t Engine::two_site_size(int k) {
  setup_two_site(k);
  return psi_size;
}

// psi in the canonical two-site order: for q_l in bond k (sorted), s1, s2 with
// q_r = q_l + s1 + s2 in bond k+2: a m_k(q_l) x m_{k+2}(q_r) block
// blocks of the canonical two-site vector format (q_l, s1, s2 with q_r =
// q_l + s1 + s2) in the engine's fused layout of the current step
std::vector<Engine::CanonMap> Engine::canonical_maps(int k) const {
  const Bond& bk = bonds[k];
  const Bond& bk2 = bonds[k + 2];
  std::vector<CanonMap> maps;
  int64_t pos = 0;
  for (int j = 0; j < bk.nsec(); ++j)
    for (int s1 = 0; s1 < 4; ++s1)
      for (int s2 = 0; s2 < 4; ++s2) {
        int r = bk2.find(bk.na[j] + QA[s1] + QA[s2], bk.nb[j] + QB[s1] + QB[s2]);
        if (r < 0) continue;
        int q = EL.find(bk.na[j] + QA[s1], bk.nb[j] + QB[s1]);
        int ml = bk.dim[j], mr = bk2.dim[r];
        int ld = ER.dim[q];
        maps.push_back({pos, psi_off[q] + (int64_t)EL.soff[q][s1] * ld + ER.soff[q][s2], ml, mr, ld});
        pos += (int64_t)ml * mr;
      }
  return maps;
}

void Engine::to_fused(const std::vector<CanonMap>& maps, const double* in, double* out) const {
  std::fill(out, out + psi_size, 0.0);
  for (auto& m : maps)
    for (int a = 0; a < m.rows; ++a)
      for (int c = 0; c < m.cols; ++c) out[m.dst + (int64_t)a * m.ld + c] = in[m.src + (int64_t)a * m.cols + c];
}

void Engine::from_fused(const std::vector<CanonMap>& maps, const double* in, double* out) const {
  for (auto& m : maps)
    for (int a = 0; a < m.rows; ++a)
      for (int c = 0; c < m.cols; ++c) out[m.src + (int64_t)a * m.cols + c] = in[m.dst + (int64_t)a * m.ld + c];
}

void Engine::apply_heff(int k, const double* in, double* out, double* diag_out, int prec) {
  setup_two_site(k);
  const std::vector<CanonMap> maps = canonical_maps(k);
  std::vector<double> hp(psi_size, 0.0);
  to_fused(maps, in, hp.data());
  CK(cudaMemcpyAsync(psi, hp.data(), psi_size * sizeof(double), cudaMemcpyHostToDevice, stream));
  Sigma sg;
  AxpyPlan ax;
  build_lenl(k, Lenv[k], EL, sg.lenl, ax);
  finish_enl(sg.lenl, ax);
  build_renl(k + 1, Renv[k + 2], ER, sg.renl, ax);
  finish_enl(sg.renl, ax);
  double* y = dalloc<double>(psi_size);
  if (prec == 0) {
    plan_sigma(sg.lenl, sg.renl, sg);
    sigma(sg, psi, y);
  } else {
    TcPlan* P = tc_plan(sg.lenl, sg.renl, prec == 1 ? kTF32 : prec == 2 ? kBF16 : prec == 3 ? kTF32x3 : kBF16x3);
    tc_apply(P, psi, y);
    tc_free(P);
  }
  std::vector<double> hy(psi_size);
  CK(cudaMemcpyAsync(hy.data(), y, psi_size * sizeof(double), cudaMemcpyDeviceToHost, stream));
  sync();
  settle();   // the stats include this build when the call returns
  from_fused(maps, hy.data(), out);
  if (diag_out) {
    compute_diag(sg.lenl, sg.renl, y);
    CK(cudaMemcpyAsync(hy.data(), y, psi_size * sizeof(double), cudaMemcpyDeviceToHost, stream));
    sync();
    from_fused(maps, hy.data(), diag_out);
  }
  if (prec == 0) {
    release(sg.A);
    release(sg.B);
    for (void* p : {(void*)sg.Y, (void*)sg.in, (void*)sg.out}) dfree(p);
  }
  dfree(y);
  free_enl(sg.lenl);
  free_enl(sg.renl);
  sync();
}

void Engine::multi_dot(const double* V, int64_t stride, int k, const double* x, int64_t n, double* out_host) {
  int nblk = reduction_blocks(n);
  double* partial = dalloc<double>((size_t)nblk * k);
  double* dots = dalloc<double>(k);
  launch_multi_dot(V, stride, k, x, n, dots, partial, nblk, stream);
  stats.launches += 2;
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out_host, dots, k * sizeof(double), cudaMemcpyDeviceToHost, stream));
  sync();
  dfree(partial);
  dfree(dots);
}

double Engine::run_step(int k, int dir, int M, double tol, double* tau, std::vector<double>* kept) {
  const double e = step(k, dir, M, tol, tau, kept);
  sync();
  return e;
}

void Engine::env_block(int side, int bond, int ch, int sec, std::vector<double>& out, int& rows, int& cols) {
  const Env& e = side == 0 ? Lenv[bond] : Renv[bond];
  if (!e.valid) throw Error(-6, "environment not built at this bond");
  int64_t o = e.at(ch, sec);
  if (o < 0) { rows = cols = 0; out.clear(); return; }
  rows = e.rows[(size_t)ch * e.nsec + sec];
  cols = e.cols[(size_t)ch * e.nsec + sec];
  out.resize((size_t)rows * cols);
  CK(cudaMemcpyAsync(out.data(), e.d + o, out.size() * sizeof(double), cudaMemcpyDeviceToHost, stream));
  sync();
}

}  // namespace gbd
