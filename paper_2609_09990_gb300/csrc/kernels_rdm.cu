// Kernels of the RDM pass (once per solve, FP64): scatter of the MPS
// amplitudes into the determinant basis, and D[pq] = E_pq C for a chunk of
// alpha strings.  The contractions themselves (prefix/suffix products and
// the Gram matrix D D^T) reuse the grouped block GEMM.
#include <cuda_runtime.h>

#include "gbd_internal.h"

namespace gbd {

namespace {

// C[(aP[i] + aS[j]) * Nb + bP[i] + bS[j]] = sign * A[i * nsuf + j]
__global__ void scatter_ci_kernel(const double* __restrict__ A, int npref, int nsuf, const int* __restrict__ aP,
                                  const int* __restrict__ bP, const signed char* __restrict__ sP,
                                  const int* __restrict__ aS, const int* __restrict__ bS,
                                  const signed char* __restrict__ sS, double sector_sign, int64_t Nb,
                                  double* __restrict__ C) {
  int64_t total = (int64_t)npref * nsuf;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / nsuf), j = (int)(e % nsuf);
    int64_t Ia = aP[i] + aS[j], Ib = bP[i] + bS[j];
    C[Ia * Nb + Ib] = sector_sign * sP[i] * sS[j] * A[e];
  }
}

// D[pq][(ja - ja0) * Nb + ib] = sA * C[Ia, ib] + sB * C[ja, Ib] with
// (Ia, sA) = excA[ja][pq], (Ib, sB) = excB[ib][pq]; entries are
// (source + 1) * sign, 0 when E_pq has no source string.
__global__ void apply_e_chunk_kernel(const double* __restrict__ C, int64_t Nb, const int* __restrict__ excA,
                                     const int* __restrict__ excB, int n2, int ja0, int cs,
                                     double* __restrict__ D) {
  int64_t per = (int64_t)cs * Nb;
  int64_t total = per * n2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int pq = (int)(e / per);
    int64_t r = e % per;
    int ja = ja0 + (int)(r / Nb);
    int64_t ib = r % Nb;
    double v = 0.0;
    int ea = excA[(int64_t)ja * n2 + pq];
    if (ea) {
      int64_t src = (ea > 0 ? ea : -ea) - 1;
      v += (ea > 0 ? 1.0 : -1.0) * C[src * Nb + ib];
    }
    int eb = excB[ib * n2 + pq];
    if (eb) {
      int64_t src = (eb > 0 ? eb : -eb) - 1;
      v += (eb > 0 ? 1.0 : -1.0) * C[(int64_t)ja * Nb + src];
    }
    D[e] = v;
  }
}

// out[v][ja * Nb + ib] = sA * V[v][Ia, ib] + sB * V[v][ja, Ib] for the one
// excitation E_rs (rs fixed) applied to nv vectors V[v] of the determinant
// length Na * Nb; (Ia, sA) = excA[ja][rs], (Ib, sB) = excB[ib][rs].
__global__ void apply_e_vecs_kernel(const double* __restrict__ V, int nv, int64_t Na, int64_t Nb,
                                    const int* __restrict__ excA, const int* __restrict__ excB, int n2, int rs,
                                    double* __restrict__ out) {
  const int64_t per = Na * Nb;
  const int64_t total = per * nv;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = e / per, r = e % per;
    const int64_t ja = r / Nb, ib = r % Nb;
    const double* Vv = V + v * per;
    double x = 0.0;
    const int ea = excA[ja * n2 + rs];
    if (ea) x += (ea > 0 ? 1.0 : -1.0) * Vv[(int64_t)((ea > 0 ? ea : -ea) - 1) * Nb + ib];
    const int eb = excB[ib * n2 + rs];
    if (eb) x += (eb > 0 ? 1.0 : -1.0) * Vv[ja * Nb + ((eb > 0 ? eb : -eb) - 1)];
    out[e] = x;
  }
}

// Two-orbital reduced density matrices.  For pair (i<j) and determinant D =
// (alpha bits A, beta bits B) the local state of the pair is
// x = a_i + 2 b_i + 4 (a_j + 2 b_j) (modes i alpha, i beta, j alpha, j beta),
// and c_x(R) = s_D C(D) with R the rest of D and s_D the parity of moving
// the local modes to the front in that order (the other modes keep their
// alpha-first order).  rho_ij[x', x] = sum_R c_x'(R) c_x(R).  One thread
// takes the group of determinants sharing R (at most 2 alpha x 2 beta local
// variants) through its representative (a local electron on i rather than
// j) and adds the group's products to the 26 distinct symmetric slots of
// the block-diagonal rho_ij; blocks reduce them in a fixed order into
// partial[pair][block][26].
__device__ __forceinline__ int colex_addr(uint32_t bits, const int* __restrict__ binom, int n) {
  int addr = 0, pos = 0;
  for (int o = 0; o < n; ++o)
    if (bits >> o & 1u) addr += binom[o * 33 + (++pos)];
  return addr;
}

__device__ __forceinline__ int local_parity(uint32_t A, uint32_t B, int i, int j, int NaTot) {
  const int ai = A >> i & 1, aj = A >> j & 1, bi = B >> i & 1, bj = B >> j & 1;
  const uint32_t mi = (1u << i) - 1u, mj = (1u << j) - 1u;
  const int nonloc_a = NaTot - ai - aj;
  int p = 0;
  if (ai) p += __popc(A & mi);
  if (aj) p += __popc(A & mj) - ai;
  if (bi) p += nonloc_a + __popc(B & mi);
  if (bj) p += nonloc_a + __popc(B & mj) - bi;
  p += aj * bi;
  return p & 1;
}

__global__ void pair_rdm_kernel(const double* __restrict__ C, int64_t NaS, int64_t NbS, const uint32_t* __restrict__ strA,
                                const uint32_t* __restrict__ strB, const int* __restrict__ binom, int n, int NaTot,
                                const int* __restrict__ pairs, double* __restrict__ partial) {
  const int pr = blockIdx.y;
  const int i = pairs[2 * pr], j = pairs[2 * pr + 1];
  const uint32_t bit_i = 1u << i, bit_j = 1u << j;
  double acc[26];
#pragma unroll
  for (int t = 0; t < 26; ++t) acc[t] = 0.0;
  const int64_t ndet = NaS * NbS;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ndet; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t Ia = e / NbS, Ib = e % NbS;
    const uint32_t A = strA[Ia], B = strB[Ib];
    const int ai = A >> i & 1, aj = A >> j & 1, bi = B >> i & 1, bj = B >> j & 1;
    if ((aj && !ai) || (bj && !bi)) continue;   // not the group's representative
    const int na = ai + aj, nb = bi + bj;
    // alpha variants (bits, address), beta variants
    uint32_t Av[2] = {A, A ^ bit_i ^ bit_j}, Bv[2] = {B, B ^ bit_i ^ bit_j};
    const int nav = na == 1 ? 2 : 1, nbv = nb == 1 ? 2 : 1;
    int64_t Iav[2] = {Ia, 0}, Ibv[2] = {Ib, 0};
    if (nav == 2) Iav[1] = colex_addr(Av[1], binom, n);
    if (nbv == 2) Ibv[1] = colex_addr(Bv[1], binom, n);
    double c[4];
    int k = 0;
    for (int u = 0; u < nav; ++u)
      for (int v = 0; v < nbv; ++v, ++k) {
        const double amp = C[Iav[u] * NbS + Ibv[v]];
        c[k] = local_parity(Av[u], Bv[v], i, j, NaTot) ? -amp : amp;
      }
    // slot layout: sector (na, nb) -> base; within a sector of d variants
    // the upper triangle (k <= l) in row-major order
    const int d = nav * nbv;
    int base;
    if (d == 1) base = (na / 2) * 2 + (nb / 2);           // (0,0) 0, (0,2) 1, (2,0) 2, (2,2) 3
    else if (d == 2) base = 4 + 3 * (na == 1 ? (nb / 2) : 2 + na / 2);   // (1,0) 4, (1,2) 7, (0,1) 10, (2,1) 13
    else base = 16;                                        // (1,1): 10 slots
    int t = base;
    for (int a2 = 0; a2 < d; ++a2)
      for (int b2 = a2; b2 < d; ++b2, ++t) {
        // unrolled register indexing: the compiler resolves t only at run time,
        // so accumulate through a small switch over the 26 slots
#pragma unroll
        for (int q = 0; q < 26; ++q)
          if (q == t) acc[q] += c[a2] * c[b2];
      }
  }
  // block reduction in a fixed order: warp shuffles, then warps in order
  __shared__ double sh[26][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 26; ++q) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 26) {
    double v = 0.0;
    const int nw = blockDim.x >> 5;
    for (int w = 0; w < nw; ++w) v += sh[threadIdx.x][w];
    partial[((int64_t)pr * gridDim.x + blockIdx.x) * 26 + threadIdx.x] = v;
  }
}

int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

void launch_scatter_ci(const double* A, int npref, int nsuf, const int* aP, const int* bP, const signed char* sP,
                       const int* aS, const int* bS, const signed char* sS, double sector_sign, int64_t Nb,
                       double* C, cudaStream_t s) {
  scatter_ci_kernel<<<grid_for((int64_t)npref * nsuf), 256, 0, s>>>(A, npref, nsuf, aP, bP, sP, aS, bS, sS,
                                                                     sector_sign, Nb, C);
}

void launch_apply_e_vecs(const double* V, int nv, int64_t Na, int64_t Nb, const int* excA, const int* excB, int n2,
                         int rs, double* out, cudaStream_t s) {
  apply_e_vecs_kernel<<<grid_for(Na * Nb * nv), 256, 0, s>>>(V, nv, Na, Nb, excA, excB, n2, rs, out);
}

int pair_rdm_blocks(int64_t ndet) {
  int64_t b = (ndet + 255) / 256;
  if (b > 152 * 2) b = 152 * 2;
  return (int)(b < 1 ? 1 : b);
}

void launch_pair_rdm(const double* C, int64_t NaS, int64_t NbS, const uint32_t* strA, const uint32_t* strB,
                     const int* binom, int n, int NaTot, const int* pairs, int npairs, double* partial,
                     cudaStream_t s) {
  dim3 g(pair_rdm_blocks(NaS * NbS), npairs);
  pair_rdm_kernel<<<g, 256, 0, s>>>(C, NaS, NbS, strA, strB, binom, n, NaTot, pairs, partial);
}

void launch_apply_e_chunk(const double* C, int64_t Nb, const int* excA, const int* excB, int n2, int ja0, int cs,
                          double* D, cudaStream_t s) {
  apply_e_chunk_kernel<<<grid_for((int64_t)cs * Nb * n2), 256, 0, s>>>(C, Nb, excA, excB, n2, ja0, cs, D);
}

}  // namespace gbd
