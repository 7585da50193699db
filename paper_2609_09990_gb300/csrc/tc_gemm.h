// Tensor-core grouped GEMM (tcgen05 + TMA) used by the reduced-precision
// sigma build.
//
// Operands live in "panels": row-major 2D buffers with a fixed row pitch
// (a multiple of 64 elements) holding many sub-blocks, each sub-block's K
// range starting at a column that is a multiple of 16 and zero-padded to a
// multiple of the MMA K step.  One TMA tensor map per panel (and per B box
// height) then serves every block product of a launch.
//
// A work tile is 128 rows of A (M) by n_mma (<= 256, multiple of 16) rows
// of B (N); it accumulates C += sign * A_t B_t^T over its terms t in TMEM
// (FP32) and is written by one of two epilogues:
//   kTcYT    : C^T into a panel (BF16, TF32, or TF32 hi/lo), row j of the
//              output is panel row out + j, output column = the padded
//              position of tile row m0 + i (rmap: 4 breaks + 4 pads),
//   kTcSigma : C^T into FP64, out[j * ld + m0 + i] (= or +=).
#pragma once

#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

namespace gbd {

enum TcPrec { kBF16 = 0, kTF32 = 1, kTF32x3 = 2 };
enum TcMode { kTcYT = 0, kTcSigma = 1 };

struct TcTerm {
  int32_t ax, ay;   // A box origin: column (K) and row (before adding the tile's m0)
  int32_t by;       // B sub-block first row (K starts at column 0)
  int32_t k;        // K, a multiple of the MMA K step (16 BF16, 8 TF32)
  int32_t neg;      // 1: subtract the product
  int32_t pad;
};

struct TcTile {
  int32_t t0, t1;
  int32_t m0, m_valid;
  int32_t n_mma, n_valid;
  int32_t bsel;          // B box height index: 16 << bsel rows
  int32_t mode, beta, ld;
  int64_t out;           // output element offset (panel row for kTcYT)
  int32_t rbreak[4], rpad[4];
};

struct TcMaps {
  CUtensorMap a[2];      // [hi, lo]
  CUtensorMap b[2][5];   // [hi, lo][box height 16, 32, 64, 128, 256]
};

struct TcLaunch {
  const TcTile* tiles;
  const TcTerm* terms;
  int ntiles;
  int prec;
  void* yt_hi;           // kTcYT outputs (uint16 BF16 or float TF32)
  void* yt_lo;           // TF32x3 low part
  double* f64;           // kTcSigma output
  int* err;              // device flag: 1 = a bounded wait ran out
};

constexpr int kTcKChunk16 = 64;   // BF16 elements per 128-byte TMA box row
constexpr int kTcKChunk32 = 32;   // TF32 elements per 128-byte TMA box row

// encode the tensor maps of one panel (pitch in elements)
bool tc_encode_panel(CUtensorMap* m, int prec_elem_bytes, const void* base, uint64_t pitch, uint64_t rows,
                     uint32_t box_rows);
void launch_tc_gemm(const TcMaps& maps, const TcLaunch& L, int num_sms, cudaStream_t s);

// conversion of FP64 blocks into panels: rows x cols block at src (ld_src)
// written at panel row r0, column c0 (pitch); lo != nullptr for TF32x3
struct TcConv {
  const double* src;
  double scale;          // multiplies every element (the sub-block's coefficient)
  int32_t rows, cols, ld_src;
  int32_t r0, c0;
};
void launch_tc_convert(const TcConv* tasks, int ntasks, int prec, void* hi, void* lo, int64_t pitch,
                       cudaStream_t s);
// psi (fused FP64 layout) -> panel with padded column sub-ranges
struct TcPsiSector {
  int64_t src_off;       // offset of the sector block in psi
  int32_t rows, cols;    // m_EL, m_ER
  int32_t r0;            // panel row of its first row
  int32_t cbreak[4], cpad[4];
};
void launch_tc_convert_psi(const double* psi, const TcPsiSector* sec, int nsec, int64_t total, int prec, void* hi,
                           void* lo, int64_t pitch, cudaStream_t s);

}  // namespace gbd
