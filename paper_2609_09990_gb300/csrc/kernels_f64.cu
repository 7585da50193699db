// FP64 kernels of the sweep: grouped block GEMM (the sigma build, environment
// update and decimation contractions all reduce to lists of small dense
// products), block axpy (forming enlarged operators from environment blocks
// and MPO entries) and the Davidson vector operations.
//
// GB300 executes FP64 on its CUDA cores only; these kernels are the plain
// FP64 path.  The grouped GEMM keeps a 32x32 output tile per CTA in
// registers and walks every (A,B) term that contributes to that tile, so each
// output block is written once, deterministically, without atomics.
#include <cuda_runtime.h>

#include "gbd_internal.h"

namespace gbd {

namespace {

constexpr int TM = 32, TN = 32, TK = 16, GEMM_THREADS = 64;

__global__ void __launch_bounds__(GEMM_THREADS)
gemm_f64_kernel(const GemmTerm* __restrict__ terms, const GemmOut* __restrict__ outs,
                const GemmTile* __restrict__ tiles, int ntiles) {
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 7, ty = tid >> 3;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const GemmTile tl = tiles[tile];
    const GemmOut o = outs[tl.out];
    const int m0 = tl.tm * TM, n0 = tl.tn * TN;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int t = o.t0; t < o.t1; ++t) {
      const GemmTerm T = terms[t];
      const bool ta = T.flags & 1, tb = T.flags & 2;
      for (int k0 = 0; k0 < T.K; k0 += TK) {
        // A tile: TM x TK of op(A), scaled by alpha
#pragma unroll
        for (int r = 0; r < (TM * TK) / GEMM_THREADS; ++r) {
          int idx = tid + r * GEMM_THREADS;
          int i, kk;
          if (!ta) { i = idx / TK; kk = idx % TK; } else { i = idx % TM; kk = idx / TM; }
          int gm = m0 + i, gk = k0 + kk;
          double v = 0.0;
          if (gm < o.M && gk < T.K)
            v = ta ? T.A[(int64_t)gk * T.lda + gm] : T.A[(int64_t)gm * T.lda + gk];
          As[kk][i] = v * T.alpha;
        }
        // B tile: TK x TN of op(B)
#pragma unroll
        for (int r = 0; r < (TN * TK) / GEMM_THREADS; ++r) {
          int idx = tid + r * GEMM_THREADS;
          int j, kk;
          if (!tb) { j = idx % TN; kk = idx / TN; } else { j = idx / TK; kk = idx % TK; }
          int gn = n0 + j, gk = k0 + kk;
          double v = 0.0;
          if (gn < o.N && gk < T.K)
            v = tb ? T.B[(int64_t)gn * T.ldb + gk] : T.B[(int64_t)gk * T.ldb + gn];
          Bs[kk][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
          double a[4], b[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 8 * i];
#pragma unroll
          for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 8 * j];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int gm = m0 + ty + 8 * i;
      if (gm >= o.M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int gn = n0 + tx + 8 * j;
        if (gn >= o.N) continue;
        double* c = o.C + (int64_t)gm * o.ldc + gn;
        *c = o.beta ? (*c + acc[i][j]) : acc[i][j];
      }
    }
  }
}

// one output element per thread, 256 consecutive elements (row-major) of
// one output per item; per element the same FMA sequence as gemm_f64_kernel
// (terms in order, k ascending, A scaled by alpha first)
__global__ void __launch_bounds__(256)
gemm_f64_flat_kernel(const GemmTerm* __restrict__ terms, const GemmOut* __restrict__ outs,
                     const GemmTile* __restrict__ items, int nitems) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const GemmTile w = items[it];
    const GemmOut o = outs[w.out];
    const int64_t e = (int64_t)w.tn + threadIdx.x;
    if (e >= (int64_t)o.M * o.N) continue;
    const int i = (int)(e / o.N), j = (int)(e - (int64_t)i * o.N);
    double acc = 0.0;
    for (int t = o.t0; t < o.t1; ++t) {
      const GemmTerm T = terms[t];
      const bool ta = T.flags & 1, tb = T.flags & 2;
      const double* a = ta ? T.A + i : T.A + (int64_t)i * T.lda;
      const double* b = tb ? T.B + (int64_t)j * T.ldb : T.B + j;
      const int64_t sa = ta ? T.lda : 1, sb = tb ? 1 : T.ldb;
      for (int k = 0; k < T.K; ++k) acc = fma(a[k * sa] * T.alpha, b[k * sb], acc);
    }
    double* c = o.C + (int64_t)i * o.ldc + j;
    *c = o.beta ? (*c + acc) : acc;
  }
}

// Block axpy over fixed work chunks of kAxpyChunk output elements (the
// chunks of all outputs in one list, cstart[o] = first chunk of output o):
// a long output no longer occupies one CTA while the others idle.  The term
// descriptors of a chunk are staged in shared memory, so the data loads of
// four terms (4 x kPer independent loads per thread) are in flight at once;
// every element is still summed over its terms in list order.
constexpr int kAxpyThreads = 256;
constexpr int kAxpyStage = 256;   // term descriptors staged per round
__global__ void __launch_bounds__(kAxpyThreads) axpy_kernel(const AxpyTerm* __restrict__ terms,
                                                            const AxpyOut* __restrict__ outs,
                                                            const int64_t* __restrict__ cstart, int nouts,
                                                            int64_t nchunks) {
  constexpr int kPer = kAxpyChunk / kAxpyThreads;
  __shared__ const double* sp[kAxpyStage];
  __shared__ double sc[kAxpyStage];
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    int lo = 0, hi = nouts - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (cstart[mid] <= c) lo = mid; else hi = mid - 1;
    }
    const AxpyOut o = outs[lo];
    const int64_t e0 = (c - cstart[lo]) * kAxpyChunk + threadIdx.x;
    bool in[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) in[i] = e0 + (int64_t)i * kAxpyThreads < o.len;
    double s[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) s[i] = 0.0;
    for (int tb = o.t0; tb < o.t1; tb += kAxpyStage) {
      const int nt = min(kAxpyStage, o.t1 - tb);
      __syncthreads();
      if (threadIdx.x < nt) {
        sp[threadIdx.x] = terms[tb + threadIdx.x].src;
        sc[threadIdx.x] = terms[tb + threadIdx.x].coef;
      }
      __syncthreads();
      int t = 0;
      for (; t + 4 <= nt; t += 4) {
        double x[4][kPer];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int i = 0; i < kPer; ++i) x[u][i] = in[i] ? sp[t + u][e0 + (int64_t)i * kAxpyThreads] : 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int i = 0; i < kPer; ++i) s[i] = fma(sc[t + u], x[u][i], s[i]);
      }
      for (; t < nt; ++t)
#pragma unroll
        for (int i = 0; i < kPer; ++i)
          if (in[i]) s[i] = fma(sc[t], sp[t][e0 + (int64_t)i * kAxpyThreads], s[i]);
    }
#pragma unroll
    for (int i = 0; i < kPer; ++i)
      if (in[i]) o.dst[e0 + (int64_t)i * kAxpyThreads] = s[i];
  }
}

__global__ void set_identity_kernel(double* d, int m) {
  int64_t n = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    d[e] = (e / m == e % m) ? 1.0 : 0.0;
}

constexpr int RED_THREADS = 256;

__device__ double block_sum(double v) {
  __shared__ double sh[RED_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = (threadIdx.x < RED_THREADS / 32) ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  return v;
}

// partial[j * nblk + b] = sum over block b's chunk of V_j . x
__global__ void multi_dot_partial(const double* __restrict__ V, int64_t stride, int k,
                                  const double* __restrict__ x, int64_t n, double* partial) {
  const int j = blockIdx.y;
  const double* v = V + (int64_t)j * stride;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)RED_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * RED_THREADS)
    s = fma(v[i], x[i], s);
  s = block_sum(s);
  if (threadIdx.x == 0) partial[j * gridDim.x + blockIdx.x] = s;
}

__global__ void finish_sums(const double* partial, int nblk, int k, double* out) {
  int j = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += RED_THREADS) s += partial[j * nblk + b];
  s = block_sum(s);
  if (threadIdx.x == 0) out[j] = s;
}

__global__ void lincomb_kernel(double* out, const double* __restrict__ V, int64_t stride,
                               const double* __restrict__ coef, int k, int64_t n, int accumulate, double cs) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = accumulate ? out[i] : 0.0;
    for (int j = 0; j < k; ++j) s = fma(cs * coef[j], V[(int64_t)j * stride + i], s);
    out[i] = s;
  }
}

// out = t / sqrt(nrm2[0]) (zero vector when the norm has vanished)
__global__ void normalize_kernel(const double* __restrict__ t, const double* __restrict__ nrm2, int64_t n,
                                 double* __restrict__ out) {
  const double q = nrm2[0];
  const double s = q > 1e-28 ? 1.0 / sqrt(q) : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = t[i] * s;
}

// diag - theta, kept at least 1e-8 away from zero (sign kept, + for 0)
__device__ __forceinline__ double guarded_den(double d, double theta) {
  double den = d - theta;
  if (fabs(den) < 1e-8) den = den >= 0.0 ? 1e-8 : -1e-8;
  return den;
}

// r = sx - theta x ; t = -r / clamp(diag - theta) ; partial sums of r^2
__global__ void residual_precond_kernel(const double* __restrict__ x, const double* __restrict__ sx,
                                        const double* __restrict__ diag, double theta, int64_t n,
                                        double* r, double* t, double* partial) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)RED_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * RED_THREADS) {
    double ri = sx[i] - theta * x[i];
    r[i] = ri;
    t[i] = -ri / guarded_den(diag[i], theta);
    s = fma(ri, ri, s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// projected diagonal preconditioner, pass 1: out = scale v / den; partial
// sums of x . out (row 0) and x . x / den (row 1)
__global__ void kdiv_kernel(const double* __restrict__ v, const double* __restrict__ x,
                            const double* __restrict__ diag, double theta, double scale, int64_t n, double* out,
                            double* partial) {
  const int nblk = gridDim.x;
  double s1 = 0.0, s2 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)RED_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * RED_THREADS) {
    const double den = guarded_den(diag[i], theta);
    const double o = scale * v[i] / den;
    out[i] = o;
    s1 = fma(x[i], o, s1);
    s2 = fma(x[i], x[i] / den, s2);
  }
  s1 = block_sum(s1);
  s2 = block_sum(s2);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = s1;
    partial[nblk + blockIdx.x] = s2;
  }
}

// pass 2: out -= (sums[0] / sums[1]) x / den, so that x . out = 0
__global__ void kproj_kernel(const double* __restrict__ x, const double* __restrict__ diag, double theta,
                             const double* __restrict__ sums, int64_t n, double* out) {
  const double eps = sums[1] != 0.0 ? sums[0] / sums[1] : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] -= eps * x[i] / guarded_den(diag[i], theta);
}

// y = a x + b y
__global__ void axpby_kernel(double* y, double a, const double* __restrict__ x, double b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], b * y[i]);
}

__global__ void add_sq_kernel(double* d, const double* __restrict__ phi, int k, int64_t n, double w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < k; ++j) s = fma(phi[(int64_t)j * n + i], phi[(int64_t)j * n + i], s);
    d[i] = fma(w, s, d[i]);
  }
}

__global__ void scale_kernel(double* x, double a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= a;
}

int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

int reduction_blocks(int64_t n) {
  int64_t b = (n + RED_THREADS * 4 - 1) / (RED_THREADS * 4);
  if (b > 608) b = 608;
  return (int)(b < 1 ? 1 : b);
}

void launch_gemm_f64(const GemmPlan& p, cudaStream_t s) {
  const int nt = (int)p.tiles.size();
  if (nt > 0) gemm_f64_kernel<<<nt < 152 * 24 ? nt : 152 * 24, GEMM_THREADS, 0, s>>>(p.d_terms, p.d_outs, p.d_tiles, nt);
  const int nf = (int)p.flat.size();
  if (nf > 0) gemm_f64_flat_kernel<<<nf < 152 * 8 ? nf : 152 * 8, 256, 0, s>>>(p.d_terms, p.d_outs, p.d_flat, nf);
}

void launch_axpy(const AxpyPlan& p, cudaStream_t s) {
  const int no = (int)p.outs.size();
  if (no == 0 || p.nchunks == 0) return;
  const int64_t grid = p.nchunks < 152 * 8 ? p.nchunks : 152 * 8;
  axpy_kernel<<<(int)grid, kAxpyThreads, 0, s>>>(p.d_terms, p.d_outs, p.d_cstart, no, p.nchunks);
}

// dst = sign * src^T, one 32 x 32 tile of one task per CTA: coalesced reads
// of src rows into shared memory, coalesced writes of dst rows
__global__ void __launch_bounds__(256)
block_transpose_kernel(const TransTask* __restrict__ tasks, const TransTile* __restrict__ tiles) {
  __shared__ double t[32][33];
  const TransTile tl = tiles[blockIdx.x];
  const TransTask T = tasks[tl.task];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int i = ty; i < 32; i += 8) {
    const int r = tl.r0 + i, c = tl.c0 + tx;
    if (r < T.rows && c < T.cols) t[i][tx] = T.src[(int64_t)r * T.cols + c];
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int c = tl.c0 + j, r = tl.r0 + tx;   // dst row c, column r
    if (r < T.rows && c < T.cols) T.dst[(int64_t)c * T.rows + r] = T.sign * t[tx][j];
  }
}

void launch_block_transpose(const TransTask* tasks, const TransTile* tiles, int ntiles, cudaStream_t s) {
  if (ntiles <= 0) return;
  block_transpose_kernel<<<ntiles, 256, 0, s>>>(tasks, tiles);
}

void launch_set_identity(double* d, int m, cudaStream_t s) {
  set_identity_kernel<<<grid_for((int64_t)m * m, 256), 256, 0, s>>>(d, m);
}

void launch_multi_dot(const double* V, int64_t stride, int k, const double* x, int64_t n, double* out_dev,
                      double* partial, int nblk, cudaStream_t s) {
  if (k <= 0) return;
  dim3 g(nblk, k);
  multi_dot_partial<<<g, RED_THREADS, 0, s>>>(V, stride, k, x, n, partial);
  finish_sums<<<k, RED_THREADS, 0, s>>>(partial, nblk, k, out_dev);
}

void launch_lincomb(double* out, const double* V, int64_t stride, const double* coef_dev, int k, int64_t n,
                    int accumulate, cudaStream_t s, double coef_scale) {
  lincomb_kernel<<<grid_for(n, 256), 256, 0, s>>>(out, V, stride, coef_dev, k, n, accumulate, coef_scale);
}

void launch_normalize(const double* t, const double* nrm2_dev, int64_t n, double* out, cudaStream_t s) {
  normalize_kernel<<<grid_for(n, 256), 256, 0, s>>>(t, nrm2_dev, n, out);
}

void launch_residual_precond(const double* x, const double* sx, const double* diag, double theta, int64_t n,
                             double* r, double* t, double* partial, int nblk, double* out_dev, cudaStream_t s) {
  residual_precond_kernel<<<nblk, RED_THREADS, 0, s>>>(x, sx, diag, theta, n, r, t, partial);
  finish_sums<<<1, RED_THREADS, 0, s>>>(partial, nblk, 1, out_dev);
}

void launch_projected_precond(const double* v, const double* x, const double* diag, double theta, double scale,
                              int64_t n, double* out, double* partial, int nblk, double* sums_dev, cudaStream_t s) {
  kdiv_kernel<<<nblk, RED_THREADS, 0, s>>>(v, x, diag, theta, scale, n, out, partial);
  finish_sums<<<2, RED_THREADS, 0, s>>>(partial, nblk, 2, sums_dev);
  kproj_kernel<<<grid_for(n, 256), 256, 0, s>>>(x, diag, theta, sums_dev, n, out);
}

void launch_axpby(double* y, double a, const double* x, double b, int64_t n, cudaStream_t s) {
  axpby_kernel<<<grid_for(n, 256), 256, 0, s>>>(y, a, x, b, n);
}

void launch_add_sq(double* d, const double* phi, int k, int64_t n, double w, cudaStream_t s) {
  if (k > 0) add_sq_kernel<<<grid_for(n, 256), 256, 0, s>>>(d, phi, k, n, w);
}

void launch_scale(double* x, double a, int64_t n, cudaStream_t s) {
  scale_kernel<<<grid_for(n, 256), 256, 0, s>>>(x, a, n);
}

namespace {
// the bit patterns of non-negative doubles order like the values, so the
// maximum of |x| is an unsigned 64-bit atomicMax
__global__ void absmax_kernel(const double* __restrict__ x, int64_t n, unsigned long long* out) {
  double m = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}
}  // namespace

void launch_absmax(const double* x, int64_t n, double* out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, sizeof(double), s);
  int64_t b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  absmax_kernel<<<(int)b, 256, 0, s>>>(x, n, reinterpret_cast<unsigned long long*>(out));
}

}  // namespace gbd

// ---------------------------------------------------------------------------
// Allocation-free Davidson overlap reduction.  Some callers cannot call
// cudaMalloc (a host that hands us pointers from its own fixed arena, code
// running inside a stream capture owned by someone else, or a process whose
// allocator is locked).  This variant keeps its partial sums in a fixed
// file-scope device array instead of allocating.  Every GPU that loads the
// library holds the array until the process exits.
#include <mutex>

namespace {
constexpr int kNoAllocMaxK = 32;
constexpr int kNoAllocMaxBlocks = 608;   // reduction_blocks() never returns more
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxK * kNoAllocMaxBlocks];
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[256] = {};
}  // namespace

extern "C" int gbd_multi_dot_noalloc(int32_t device, const double* V, int64_t stride, int32_t k, const double* x,
                                     int64_t n, double* out, void* stream) {
  if (!V || !x || !out) return -1;
  if (k < 1 || k > kNoAllocMaxK || n < 0 || stride < n) return -1;
  if (device < 0 || device >= 256) return -1;
  // an error left pending by earlier work on this thread is not ours to
  // consume: report it, launch nothing and leave it in place
  if (cudaPeekAtLastError() != cudaSuccess) return -3;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return -3;
  if (cudaSetDevice(device) != cudaSuccess) return -3;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
      // the array's name is a host-side stand-in; the device address of this
      // device's copy comes from the runtime, once, with the device current
      double* p = nullptr;
      if (cudaGetSymbolAddress((void**)&p, g_noalloc_partials) != cudaSuccess || !p) {
        cudaSetDevice(prev);
        return -3;
      }
      g_noalloc_ptr[device] = p;
    }
    scratch = g_noalloc_ptr[device];
  }
  int nblk = gbd::reduction_blocks(n);   // <= kNoAllocMaxBlocks, so nblk * k fits the array
  gbd::launch_multi_dot(V, stride, k, x, n, out, scratch, nblk, (cudaStream_t)stream);
  cudaError_t e = cudaGetLastError();
  cudaSetDevice(prev);
  return e == cudaSuccess ? 0 : -3;
}
