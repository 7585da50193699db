// tcgen05 + TMA grouped GEMM for the reduced-precision sigma build (sm_103a).
//
// Persistent, warp-specialised CTA of 6 warps (one per SM):
//   warp 0   TMA producer: one thread streams the A and B boxes of every
//            K chunk of every term of the CTA's tiles into a ring of
//            shared-memory stages (128B-swizzled, mbarrier complete_tx);
//   warp 1   owns TMEM (512 columns = two 128x256 FP32 accumulators) and one
//            thread issues tcgen05.mma (M = 128, N = n_mma, K step 16 for
//            BF16 / 8 for TF32) and tcgen05.commit;
//   warps 2-5 epilogue: tcgen05.ld of the accumulator rows they may access
//            (TMEM lane quarter = warp id % 4), conversion, global stores.
// Two accumulators let the epilogue of tile i overlap the MMAs of tile i+1.
// TF32x3 and BF16x3 (accurate tiers) split every operand into hi + lo of
// that type and issue hi*hi + hi*lo + lo*hi into the same accumulator.
// Every mbarrier wait is bounded: on timeout the kernel raises *err, all
// roles stop issuing, and TMEM is released before the CTA exits.
#include <mutex>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "tc_gemm.h"

namespace gbd {

namespace {

constexpr int kThreads = 192;
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr int kStageA = 128 * 128;          // bytes of one A box (128 rows x 128 B)
constexpr int kSmemBudget = 232448;         // dynamic shared memory per CTA
constexpr int kMaxStages = 8;

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; false (and *err raised) when the limit runs out or another
// role already failed
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* err) {
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    if (mbar_try(b, parity)) return true;
    if ((it & 1023u) == 1023u && *(volatile int*)err) return false;
  }
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(saddr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), SM100 descriptor version 1
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                 // LBO (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;       // SBO
  d |= (uint64_t)1 << 46;                 // version
  d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__global__ void __launch_bounds__(kThreads, 1) tc_gemm_kernel(const __grid_constant__ TcMaps maps,
                                                             const TcLaunch L) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const bool x3 = L.prec == kTF32x3 || L.prec == kBF16x3;
  const bool bf = L.prec == kBF16 || L.prec == kBF16x3;
  // B boxes of this launch are at most L.ncap rows; the ring holds as many
  // stages as fit (tc_stages)
  const int bstage = L.ncap * 128;
  const int stages = L.stages;
  const int stage_bytes = (kStageA + bstage) * (x3 ? 2 : 1);
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(base + stages * stage_bytes);
  uint64_t* empty = full + stages;
  uint64_t* tfull = empty + stages;     // [2]
  uint64_t* tempty = tfull + 2;         // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tempty + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kc = bf ? kTcKChunk16 : kTcKChunk32;     // K elements per stage
  const int kstep = bf ? 16 : 8;                      // K per MMA

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(saddr(tslot)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    int stage = 0;
    uint32_t ph = 0;
    bool ok = true;
    // descriptors are software-pipelined: the next tile's and the next
    // term's loads are in flight while the current ones are issued
    TcTile Tn;
    if (blockIdx.x < L.ntiles) Tn = L.tiles[blockIdx.x];
    for (int tile = blockIdx.x; tile < L.ntiles && ok; tile += gridDim.x) {
      const TcTile T = Tn;
      if (tile + (int)gridDim.x < L.ntiles) Tn = L.tiles[tile + gridDim.x];
      const int bbytes = (16 << T.bsel) * 128;
      const uint32_t tx = (uint32_t)(kStageA + bbytes) * (x3 ? 2 : 1);
      TcTerm tmn;
      if (T.t1 > T.t0) tmn = L.terms[T.t0];
      for (int t = T.t0; t < T.t1 && ok; ++t) {
        const TcTerm tm = tmn;
        if (t + 1 < T.t1) tmn = L.terms[t + 1];
        for (int k0 = 0; k0 < tm.k; k0 += kc) {
          if (!mbar_wait(&empty[stage], ph ^ 1, L.err)) { ok = false; break; }
          uint8_t* sa = base + stage * stage_bytes;
          uint8_t* sb = sa + kStageA;
          // K-blocked operands step down by ays / bys rows per box,
          // the others step right by one box
          const int kb = k0 / kc;
          const int xa = tm.ax + (tm.ays ? 0 : k0), ya = tm.ay + T.m0 + kb * tm.ays;
          const int xb = tm.bx + (tm.bys ? 0 : k0), yb = tm.by + T.n0 + kb * tm.bys;
          mbar_expect_tx(&full[stage], tx);
          tma_load_2d(sa, &maps.a[0], xa, ya, &full[stage]);
          tma_load_2d(sb, &maps.b[0][T.bsel], xb, yb, &full[stage]);
          if (x3) {
            uint8_t* sa2 = sb + bstage;
            tma_load_2d(sa2, &maps.a[1], xa, ya, &full[stage]);
            tma_load_2d(sa2 + kStageA, &maps.b[1][T.bsel], xb, yb, &full[stage]);
          }
          if (++stage == stages) { stage = 0; ph ^= 1; }
        }
      }
    }
    // a chunk armed but never consumed (error path): let its copies land
    // before the CTA can exit
    if (!ok || *(volatile int*)L.err) {
      for (int s = 0; s < stages; ++s)
        for (uint32_t it = 0; it < (1u << 20) && !mbar_try(&full[s], ph); ++it) {
        }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    int stage = 0;
    uint32_t ph = 0;
    int acc_i = 0;
    bool ok = true;
    const uint32_t fmt = bf ? 1u : 2u;
    TcTile Tn;
    if (blockIdx.x < L.ntiles) Tn = L.tiles[blockIdx.x];
    for (int tile = blockIdx.x; tile < L.ntiles && ok; tile += gridDim.x, ++acc_i) {
      const TcTile T = Tn;
      if (tile + (int)gridDim.x < L.ntiles) Tn = L.tiles[tile + gridDim.x];
      TcTerm tmn;
      if (T.t1 > T.t0) tmn = L.terms[T.t0];
      const int a = acc_i & 1;
      const uint32_t aph = (acc_i >> 1) & 1;
      if (!mbar_wait(&tempty[a], aph ^ 1, L.err)) { ok = false; break; }
      tc_fence_after();
      const uint32_t dt = tmem + (uint32_t)(a * 256);
      uint32_t first = 1;
      for (int t = T.t0; t < T.t1 && ok; ++t) {
        const TcTerm tm = tmn;
        if (t + 1 < T.t1) tmn = L.terms[t + 1];
        const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(tm.neg & 1) << 13) |
                               ((uint32_t)(T.n_mma >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
        for (int k0 = 0; k0 < tm.k; k0 += kc) {
          if (!mbar_wait(&full[stage], ph, L.err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = saddr(base + stage * stage_bytes);
          const uint32_t sb = sa + kStageA;
          const int nk = min(kc, tm.k - k0) / kstep;
          for (int kk = 0; kk < nk; ++kk) {
            const uint64_t ad = smem_desc(sa + kk * 32), bd = smem_desc(sb + kk * 32);
            if (bf) {
              mma_bf16(dt, ad, bd, idesc, first ? 0u : 1u);
              if (x3) {
                const uint32_t sa2 = sb + bstage, sb2 = sa2 + kStageA;
                mma_bf16(dt, ad, smem_desc(sb2 + kk * 32), idesc, 1u);                 // hi * lo
                mma_bf16(dt, smem_desc(sa2 + kk * 32), bd, idesc, 1u);                 // lo * hi
              }
            } else {
              mma_tf32(dt, ad, bd, idesc, first ? 0u : 1u);
              if (x3) {
                const uint32_t sa2 = sb + bstage, sb2 = sa2 + kStageA;
                mma_tf32(dt, ad, smem_desc(sb2 + kk * 32), idesc, 1u);                 // hi * lo
                mma_tf32(dt, smem_desc(sa2 + kk * 32), bd, idesc, 1u);                 // lo * hi
              }
            }
            first = 0;
          }
          mma_commit(&empty[stage]);
          if (++stage == stages) { stage = 0; ph ^= 1; }
        }
      }
      mma_commit(&tfull[a]);
    }
  } else if (warp >= 2) {
    // ---------------- epilogue: TMEM -> registers -> global
    const int q = warp & 3;              // TMEM lane quarter this warp may read
    const int row = q * 32 + lane;       // accumulator row (A row within the tile)
    int acc_i = 0;
    for (int tile = blockIdx.x; tile < L.ntiles; tile += gridDim.x, ++acc_i) {
      // descriptor and output row are loaded before the accumulator wait
      const TcTile T = L.tiles[tile];
      const bool has = T.t1 > T.t0;
      const bool live = row < T.m_valid;
      int pcol = 0;
      TcYRow yr{};
      if (T.mode == kTcYT && live) {
        int r = T.m0 + row, s = 0;
        for (int u = 1; u < 4; ++u)
          if (r >= T.rbreak[u]) s = u;
        pcol = T.rpad[s] + (r - T.rbreak[s]);
      } else if (T.mode == kTcYTblk && live) {
        const int64_t r = T.out + row;
        yr = L.yrows[L.ymem[r]];
        yr.base += (r - yr.first) * (int64_t)kc;
      }
      const int a = acc_i & 1;
      const uint32_t aph = (acc_i >> 1) & 1;
      if (!mbar_wait(&tfull[a], aph, L.err)) break;
      tc_fence_after();
      for (int c0 = 0; c0 < T.n_mma; c0 += 16) {
        float v[16];
        if (has) {
          tmem_ld16(tmem + (uint32_t)(a * 256 + c0) + ((uint32_t)(q * 32) << 16), v);
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = 0.f;
        }
        if (!live) continue;
        if (T.mode == kTcYTblk) {
          // 16 contiguous output columns: section s, K offset k, block k / kc
          if (c0 >= T.n_valid) continue;
          const int c = T.n0 + c0;
          int s = 0;
          for (int u = 1; u < 4; ++u)
            if (c >= T.rbreak[u]) s = u;
          if (yr.koff[s] < 0) continue;
          const int k = yr.koff[s] + (c - T.rbreak[s]);
          const int64_t idx = yr.base + (int64_t)(k / kc) * yr.stride + (k % kc);
          if (bf) {
            uint32_t w[8], wl[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              __nv_bfloat162 p2 = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
              w[i] = *reinterpret_cast<uint32_t*>(&p2);
              __nv_bfloat162 l2 = __floats2bfloat162_rn(v[2 * i] - __low2float(p2), v[2 * i + 1] - __high2float(p2));
              wl[i] = *reinterpret_cast<uint32_t*>(&l2);
            }
            uint4* d = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(L.yt_hi) + idx);
            d[0] = make_uint4(w[0], w[1], w[2], w[3]);
            d[1] = make_uint4(w[4], w[5], w[6], w[7]);
            if (x3) {
              uint4* dl = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(L.yt_lo) + idx);
              dl[0] = make_uint4(wl[0], wl[1], wl[2], wl[3]);
              dl[1] = make_uint4(wl[4], wl[5], wl[6], wl[7]);
            }
          } else {
            float h[16], l[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              h[i] = to_tf32(v[i]);
              l[i] = to_tf32(v[i] - h[i]);
            }
            float4* dh = reinterpret_cast<float4*>(reinterpret_cast<float*>(L.yt_hi) + idx);
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) dh[q4] = make_float4(h[4 * q4], h[4 * q4 + 1], h[4 * q4 + 2], h[4 * q4 + 3]);
            if (x3) {
              float4* dl = reinterpret_cast<float4*>(reinterpret_cast<float*>(L.yt_lo) + idx);
#pragma unroll
              for (int q4 = 0; q4 < 4; ++q4)
                dl[q4] = make_float4(l[4 * q4], l[4 * q4 + 1], l[4 * q4 + 2], l[4 * q4 + 3]);
            }
          }
          continue;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int j = c0 + i;
          if (j >= T.n_valid) break;
          if (T.mode == kTcSigma) {
            double* o = L.f64 + T.out + (int64_t)j * T.ld + T.m0 + row;
            *o = T.beta ? (*o + (double)v[i]) : (double)v[i];
          } else if (T.mode == kTcPart) {
            L.part[T.out + (int64_t)j * 128 + row] = v[i];
          } else {
            const int64_t idx = (T.out + j) * (int64_t)T.ld + pcol;
            if (bf) {
              const __nv_bfloat16 hb = __float2bfloat16_rn(v[i]);
              reinterpret_cast<__nv_bfloat16*>(L.yt_hi)[idx] = hb;
              if (x3) reinterpret_cast<__nv_bfloat16*>(L.yt_lo)[idx] = __float2bfloat16_rn(v[i] - __bfloat162float(hb));
            } else {
              const float hi = to_tf32(v[i]);
              reinterpret_cast<float*>(L.yt_hi)[idx] = hi;
              if (x3) reinterpret_cast<float*>(L.yt_lo)[idx] = to_tf32(v[i] - hi);
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&tempty[a]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

// ---------------------------------------------------------------- bounded waits
// The failure path of every mbarrier wait above, on its own: one thread
// waits (with the same bounded helper) on a barrier that is completed only
// when `arrive` is set.  Without the arrival the wait runs out, raises
// *err and the kernel returns; nothing hangs and no memory is touched
// outside the barrier and the flag.
__global__ void bounded_wait_probe_kernel(int arrive, int* err, int* waited_ok) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (arrive) mbar_arrive(&bar);
    *waited_ok = mbar_wait(&bar, 0, err) ? 1 : 0;
  }
}

// ---------------------------------------------------------------- split-K sum
// one thread per output element; the slots are summed in FP64 with eight
// interleaved partial sums combined in a fixed order (deterministic).  The
// eight loads of a round are independent, so a long slot list is not a
// chain of dependent memory latencies.
__global__ void tc_reduce_kernel(const TcRed* __restrict__ tasks, int ntasks, int64_t total,
                                 const float* __restrict__ part, double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tasks[mid].e0 <= e) lo = mid; else hi = mid - 1;
    }
    const TcRed R = tasks[lo];
    const int loc = (int)(e - R.e0);
    const int j = loc / R.m_valid, i = loc - j * R.m_valid;
    const int64_t ss = (int64_t)128 * R.n_stride;
    const float* p = part + R.slot0 + (int64_t)j * 128 + i;
    double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int s = 0;
    for (; s + 8 <= R.nslot; s += 8) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = p[(s + u) * ss];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] += (double)v[u];
    }
    for (int u = 0; s < R.nslot; ++s, ++u) a[u] += (double)p[s * ss];
    out[R.out + (int64_t)j * R.ld + R.m0 + i] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
  }
}

// ---------------------------------------------------------------- conversions
__device__ __forceinline__ void store_conv(double x, int prec, void* hi, void* lo, int64_t idx) {
  if (prec == kBF16 || prec == kBF16x3) {
    const __nv_bfloat16 h = __double2bfloat16(x);
    reinterpret_cast<__nv_bfloat16*>(hi)[idx] = h;
    if (prec == kBF16x3) reinterpret_cast<__nv_bfloat16*>(lo)[idx] = __double2bfloat16(x - (double)__bfloat162float(h));
  } else {
    const float h = to_tf32((float)x);
    reinterpret_cast<float*>(hi)[idx] = h;
    if (prec == kTF32x3) reinterpret_cast<float*>(lo)[idx] = to_tf32((float)(x - (double)h));
  }
}

__global__ void tc_convert_kernel(const TcConv* __restrict__ tasks, int ntasks, int prec, void* hi, void* lo,
                                  int64_t pitch) {
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const TcConv c = tasks[t];
    const int64_t n = (int64_t)c.rows * c.cols;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
      // transposed sources are walked along their rows (consecutive r), so
      // that the reads stay coalesced
      const int r = c.trans ? (int)(e % c.rows) : (int)(e / c.cols);
      const int col = c.trans ? (int)(e / c.rows) : (int)(e % c.cols);
      const int64_t dst = c.kstride > 0
                              ? ((int64_t)c.r0 + (int64_t)((c.c0 + col) / pitch) * c.kstride + r) * pitch +
                                    (c.c0 + col) % pitch
                              : (int64_t)(c.r0 + r) * pitch + c.c0 + col;
      const double x = c.trans ? c.src[(int64_t)col * c.ld_src + r] : c.src[(int64_t)r * c.ld_src + col];
      store_conv(c.scale * x, prec, hi, lo, dst);
    }
  }
}

__global__ void tc_convert_psi_kernel(const double* __restrict__ psi, const TcPsiSector* __restrict__ sec, int nsec,
                                      int64_t total, int prec, void* hi, void* lo, int64_t pitch) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int lo_i = 0, hi_i = nsec - 1;
    while (lo_i < hi_i) {
      const int mid = (lo_i + hi_i + 1) >> 1;
      if (sec[mid].src_off <= e) lo_i = mid; else hi_i = mid - 1;
    }
    const TcPsiSector S = sec[lo_i];
    const int r = (int)((e - S.src_off) / S.cols);
    const int c = (int)((e - S.src_off) % S.cols);
    int s = 0, t = 0;
    for (int u = 1; u < 4; ++u) {
      if (c >= S.cbreak[u]) s = u;
      if (r >= S.rbreak[u]) t = u;
    }
    const int64_t prow = S.r0 + S.rpad[t] + (r - S.rbreak[t]);
    store_conv(psi[e], prec, hi, lo, prow * pitch + S.cpad[s] + (c - S.cbreak[s]));
  }
}

}  // namespace

void launch_tc_reduce(const TcRed* tasks, int ntasks, int64_t total, const float* part, double* out,
                      cudaStream_t s) {
  if (ntasks <= 0 || total <= 0) return;
  int64_t b = (total + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  tc_reduce_kernel<<<(int)b, 256, 0, s>>>(tasks, ntasks, total, part, out);
}

bool bounded_wait_probe(int arrive, int* err_dev, int* ok_dev, cudaStream_t s) {
  bounded_wait_probe_kernel<<<1, 32, 0, s>>>(arrive, err_dev, ok_dev);
  return cudaGetLastError() == cudaSuccess;
}

int tc_stages(int prec, int ncap) {
  const int stage_bytes = (kStageA + ncap * 128) * (prec == kTF32x3 || prec == kBF16x3 ? 2 : 1);
  int s = (kSmemBudget - 1024 - 256) / stage_bytes;
  return s < kMaxStages ? s : kMaxStages;
}

int tc_smem_bytes(int prec, int ncap) {
  const int stages = tc_stages(prec, ncap);
  const int stage_bytes = (kStageA + ncap * 128) * (prec == kTF32x3 || prec == kBF16x3 ? 2 : 1);
  return 1024 + stages * stage_bytes + (2 * stages + 4) * 8 + 16;
}

bool launch_tc_gemm(const TcMaps& maps, const TcLaunch& L, int num_sms, cudaStream_t s) {
  if (L.ncap != 64 && L.ncap != 128 && L.ncap != 256) return false;
  if (L.stages != tc_stages(L.prec, L.ncap)) return false;
  if (L.ntiles <= 0) return true;
  const int smem = tc_smem_bytes(L.prec, L.ncap);
  static std::once_flag attr_once;   // engines on several host threads share the kernel
  std::call_once(attr_once, []() {
    cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget);
  });
  const int grid = L.ntiles < num_sms ? L.ntiles : num_sms;
  tc_gemm_kernel<<<grid, kThreads, smem, s>>>(maps, L);
  return true;
}

void launch_tc_convert(const TcConv* tasks, int ntasks, int prec, void* hi, void* lo, int64_t pitch,
                       cudaStream_t s) {
  if (ntasks <= 0) return;
  tc_convert_kernel<<<ntasks < 152 * 16 ? ntasks : 152 * 16, 256, 0, s>>>(tasks, ntasks, prec, hi, lo, pitch);
}

void launch_tc_convert_psi(const double* psi, const TcPsiSector* sec, int nsec, int64_t total, int prec, void* hi,
                           void* lo, int64_t pitch, cudaStream_t s) {
  if (total <= 0) return;
  int64_t b = (total + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  tc_convert_psi_kernel<<<(int)b, 256, 0, s>>>(psi, sec, nsec, total, prec, hi, lo, pitch);
}

// tensor maps: 2D, inner dimension = pitch (K), box = 128 bytes x box_rows,
// 128-byte swizzle, zero fill outside the panel
bool tc_encode_panel(CUtensorMap* m, int elem_bytes, const void* base, uint64_t pitch, uint64_t rows,
                     uint32_t box_rows) {
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return false;
    fn = reinterpret_cast<EncodeFn>(p);
  }
  const CUtensorMapDataType dt = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  cuuint64_t dims[2] = {pitch, rows < 1 ? 1 : rows};
  cuuint64_t strides[1] = {pitch * (cuuint64_t)elem_bytes};
  cuuint32_t box[2] = {(cuuint32_t)(128 / elem_bytes), box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace gbd
