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

void launch_apply_e_chunk(const double* C, int64_t Nb, const int* excA, const int* excB, int n2, int ja0, int cs,
                          double* D, cudaStream_t s) {
  apply_e_chunk_kernel<<<grid_for((int64_t)cs * Nb * n2), 256, 0, s>>>(C, Nb, excA, excB, n2, ja0, cs, D);
}

}  // namespace gbd
