// Tensor-core grouped GEMM (tcgen05 + TMA) used by the reduced-precision
// sigma build.
//
// Operands live in "panels": row-major 2D buffers with a fixed row pitch
// (a multiple of 64 elements) holding many sub-blocks, each sub-block's K
// range starting at a column that is a multiple of 16 and zero-padded to a
// multiple of the MMA K step.  One TMA tensor map per panel (and per B box
// height) then serves every block product of a launch.  A K-blocked panel
// has a pitch of one 128-byte box row: its K range is cut into blocks of W
// columns stacked vertically, so a term walks down it (TcTerm::ays/bys)
// and every box is dense.
//
// A work tile is 128 rows of A (M) by n_mma (<= 256, multiple of 16) rows
// of B (N) starting at A row ay + m0 and B row by + n0 of each term, so that
// all tiles of one output block share one term list; it accumulates
// C += sign * A_t B_t^T over its terms t in TMEM
// (FP32) and is written by one of four epilogues:
//   kTcYT    : C^T into a panel (BF16, TF32, or TF32 hi/lo), row j of the
//              output is panel row out + j, output column = the padded
//              position of tile row m0 + i (rmap: 4 breaks + 4 pads),
//   kTcYTblk : C into a K-blocked panel (pitch = one box row, W elements;
//              element (m, k) of a block at ((k / W) * rows + m) * W + k % W):
//              tile row r = out + i belongs to run yrows[ymem[r]] (a run of
//              consecutive rows: position of its first row in block 0, the
//              block stride, and for each of the 4 column sections of B the
//              K offset where that section goes, or -1 to drop it);
//              sections start at rbreak[s] (tile columns n0 + j).
//              Every 16-column chunk lies in one section and one block, so
//              it is stored with vector stores,
//   kTcSigma : C^T into FP64, out[j * ld + m0 + i] (= or +=),
//   kTcPart  : C^T into an FP32 partial slot, part[out + j * 128 + i]; the
//              partial slots of one output tile (split K) are summed in FP64
//              by tc_reduce in a fixed order.
#pragma once

#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

namespace gbd {

enum TcPrec { kBF16 = 0, kTF32 = 1, kTF32x3 = 2, kBF16x3 = 3 };
enum TcMode { kTcYT = 0, kTcSigma = 1, kTcPart = 2, kTcYTblk = 4 };

struct TcTerm {
  int32_t ax, ay;   // A box origin: column (K) and row (before adding the tile's m0)
  int32_t by;       // B sub-block first row (before adding the tile's n0)
  int32_t k;        // K, a multiple of the MMA K step (16 BF16, 8 TF32)
  int32_t neg;      // 1: subtract the product
  int32_t bx;       // B box first column (K origin)
  int32_t ays, bys; // > 0: K-blocked operand, each K box is ays (bys) rows further
                    // down at the same column; 0: the next K box is the next columns
};

// a run of consecutive output rows of kTcYTblk tiles (row first + i goes
// to element base + i * W, W = elements per box row)
struct TcYRow {
  int64_t base;      // element offset of (first row, k = 0)
  int32_t stride;    // elements from one K block to the next
  int32_t koff[4];   // K offset of column section s, -1: not stored
  int32_t first;     // tile-row index (out + i) of the run's first row
};

struct TcTile {
  int32_t t0, t1;
  int32_t m0, m_valid;
  int32_t n_mma, n_valid;
  int32_t bsel;          // B box height index: 16 << bsel rows
  int32_t mode, beta, ld;
  int64_t out;           // output element offset (panel row for kTcYT, first yrows entry for kTcYTblk)
  int32_t rbreak[4], rpad[4];
  int32_t n0;            // offset of the tile's first B row (kTcYTblk: also its first output column)
  int32_t unused;
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
  float* part;           // kTcPart output slots
  const TcYRow* yrows;   // kTcYTblk output row runs
  const int32_t* ymem;   // kTcYTblk: run of every output row
  int ncap;              // largest n_mma of the launch's tiles: 64, 128 or 256
  int stages;            // = tc_stages(prec, ncap)
};
// shared-memory pipeline depth for B boxes of at most ncap rows
int tc_stages(int prec, int ncap);
// one bounded mbarrier wait (the helper every role of tc_gemm_kernel uses);
// without `arrive` it runs out and raises *err_dev
bool bounded_wait_probe(int arrive, int* err_dev, int* ok_dev, cudaStream_t s);

// out[j * ld + m0 + i] = sum over the nslot consecutive partial slots
// starting at float offset slot0 (slot s at slot0 + s * 128 * n_stride)
// (e0: first element of the task in the flattened list of all tasks'
// m_valid x n_valid elements; total = sum of those counts)
struct TcRed {
  int64_t out, slot0, e0;
  int32_t ld, m0, m_valid, n_valid, n_stride, nslot;
};
void launch_tc_reduce(const TcRed* tasks, int ntasks, int64_t total, const float* part, double* out,
                      cudaStream_t s);

constexpr int kTcKChunk16 = 64;   // BF16 elements per 128-byte TMA box row
constexpr int kTcKChunk32 = 32;   // TF32 elements per 128-byte TMA box row

// encode the tensor maps of one panel (pitch in elements)
bool tc_encode_panel(CUtensorMap* m, int prec_elem_bytes, const void* base, uint64_t pitch, uint64_t rows,
                     uint32_t box_rows);
// false (nothing launched) when ncap/stages are not a valid pair
bool launch_tc_gemm(const TcMaps& maps, const TcLaunch& L, int num_sms, cudaStream_t s);

// conversion of FP64 blocks into panels: rows x cols block at src (ld_src)
// written at panel row r0, column c0 (pitch); lo != nullptr for the split
// (x3) types.  kstride > 0: K-blocked panel, column c0 + j goes to row
// r0 + ((c0 + j) / pitch) * kstride, column (c0 + j) % pitch.
struct TcConv {
  const double* src;
  double scale;          // multiplies every element (the sub-block's coefficient)
  int32_t rows, cols, ld_src;
  int32_t r0, c0;
  int32_t kstride;
  int32_t trans;         // 1: element (r, c) of the block is src[c * ld_src + r]
};
void launch_tc_convert(const TcConv* tasks, int ntasks, int prec, void* hi, void* lo, int64_t pitch,
                       cudaStream_t s);
// psi (fused FP64 layout) -> panel with padded column sub-ranges
struct TcPsiSector {
  int64_t src_off;       // offset of the sector block in psi
  int32_t rows, cols;    // m_EL, m_ER
  int32_t r0;            // panel row of its first (padded) row
  int32_t cbreak[4], cpad[4];
  int32_t rbreak[4], rpad[4];   // rows: E_L s-sections, each starting at a multiple of 16
};
void launch_tc_convert_psi(const double* psi, const TcPsiSector* sec, int nsec, int64_t total, int prec, void* hi,
                           void* lo, int64_t pitch, cudaStream_t s);

}  // namespace gbd
