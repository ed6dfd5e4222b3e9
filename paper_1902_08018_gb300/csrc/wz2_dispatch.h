// wz2_dispatch.h -- host-side entry points of the WZ2 kernels, one translation
// unit per rate (wz2_r<rate>.cu) so that the instantiations build in parallel.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "wz2_batch.h"

namespace whff {

// Polls of a bounded device-side wait (tensor-core kernels) before it gives up
// and records WHFF_ETIMEOUT: about a second of try_wait.
constexpr uint32_t kWaitPolls = 1u << 22;

struct Wz2Step {
  const uint8_t* stream;
  int64_t M, N, BM, BN;
  const float* x;
  int64_t ldx;
  bool x_vec_ok;
  int64_t L;       // blocks per warp range
  int maxseg;      // most ranges sharing one band
  double* ws;
  double* y;
  int64_t ldy;
  double* state;
  double decay;
  int64_t ctas;    // grid size (persistent)
  int unroll;      // blocks in flight per lane: 2, 4 or 8 (R = 1), 2 otherwise
  bool lift;
  int R;           // 1, 2, 4 or 8
  bool red32;      // fold lanes with the FP32 pair butterfly (short bands)
  bool groups8;    // four 8-lane groups per warp, one band each (short bands)
  float* xt;       // lift: scratch for (2G)^T x, 4 BN floats per right-hand side (8 columns)
  bool staged;     // R = 1: stream each warp's range through shared memory by bulk copies
  int* status;     // device status word (bounded waits of the staged kernel)
};

// Bytes a handle's device stream allocation carries past the stream, so that
// 16-byte-rounded bulk copies of the last blocks stay inside it.
constexpr int kStreamPad = 256;


struct Wz2Batch {
  const dev::BatchEntry* entries;  // device table
  const int64_t* row_begin;        // device prefix of rows
  int nentries;
  int64_t total_blocks, total_rows, L;
  int64_t ctas;
  bool any_shared;                 // some band is split between warp ranges
  bool lift;
  int R;
};

// A batch of one scaled format (BF16, FP16, FP8, FP32): same tables, units
// are 16-byte column chunks (BN of them per band), stream = the payload.
int scaled_batched_launch(int fmt, const Wz2Batch& b, cudaStream_t st);

// state step of a batch (rate independent; defined in the rate-16 unit)
int wz2_batched_state_launch(const dev::BatchState* table, const int64_t* row_begin, int n, int64_t total_rows,
                             cudaStream_t st);

struct ScaledStep {
  int fmt;  // 2 BF16, 3 FP16, 4 FP8 E4M3
  const uint8_t* payload;
  const float* scales;
  int64_t M, N, ld, TN;
  const float* x;
  int64_t ldx;
  bool x_vec_ok;
  int64_t L;
  int maxseg;
  double* ws;
  double* y;
  int64_t ldy;
  double* state;
  double decay;
  int64_t ctas;
  int R;
  bool red32;
  bool groups8;  // four 8-lane groups per warp, one band each (short bands)
};
int scaled_launch(const ScaledStep& a, cudaStream_t st);  // scaled.cu

// Tensor-core pass of up to 32 right-hand sides over a WZ2 matrix (mma.cu).
struct MmaStep {
  int rate;
  bool lift;
  const uint8_t* stream;
  int64_t M, N, BM, BN;
  const float* x;
  int64_t ldx;
  int R;           // 1..32 (padded to 16 or 32 inside)
  int64_t L;       // (tile, stage) items per CTA: tile = 32 bands, stage = 16 blocks
  int ctas;        // persistent grid, ceil(items / L)
  int maxseg;      // most CTAs sharing one tile
  double* ws;      // tiles x maxseg x R x 128 FP64 partials
  uint8_t* btiles; // B operand pieces of every 16-block stage (built per pass)
  double* y;
  int64_t ldy;
  double* state;
  double decay;
  int* status;
  uint32_t spin;   // polls of an in-loop mbarrier wait before it gives up (kWaitPolls)
};
int mma_launch(const MmaStep& a, cudaStream_t st);

// The tensor-core passes of a batch that share one width class (NR 16 or 32),
// in one persistent launch (mma.cu).  members / passes: device tables.
struct MmaBatchStep {
  int rate;
  bool lift;
  int nr;
  const dev::MmaMember* members;
  const dev::MmaPass* passes;
  int nmem;
  int64_t total, L;  // items of all members, items per CTA
  int ctas;
  int64_t bt_threads, fin_threads;
  int* status;
  uint32_t spin;
};
int mma_batch_launch(const MmaBatchStep& a, cudaStream_t st);
int mma_max_members();  // most members of one batched launch
// resident CTAs per SM of the tensor-core kernel at this rate for R <= nr (0 on error)
int mma_occupancy(int rate, bool lift, int nr);
int scaled_occupancy(int fmt, bool groups8);  // resident CTAs per SM of the R = 1 kernel

// Tensor-core pass of up to 32 right-hand sides over a BF16 / FP16 / FP8
// matrix (scaled_mma.cu): items (tile of 128 rows, stage of 64 columns).
struct ScaledMmaStep {
  int fmt;
  const uint8_t* payload;
  const float* scales;
  int64_t M, N, ld, TN;
  const float* x;
  int64_t ldx;
  int R;           // 1..32 (padded to 16 or 32 inside)
  int64_t L;       // items per CTA
  int ctas;
  int maxseg;      // most CTAs sharing one tile
  double* ws;      // tiles x maxseg x R x 128 FP64 partials
  uint8_t* btiles; // B operand pieces of every stage (built per pass)
  double* y;
  int64_t ldy;
  double* state;
  double decay;
  int* status;
  uint32_t spin;
  const void* tmap;  // BF16 / FP16: CUtensorMap of the whole stored matrix (A tiles by TMA), or null
  int64_t row0;      // first row of this pass within that matrix (row views)
  int* colexp;       // FP16 with tmap: 32 ints of scratch for the per-column exponents of x
};
int scaled_mma_launch(const ScaledMmaStep& a, cudaStream_t st);
// Host: encode the TMA map of a BF16 or FP16 (fmt 3) payload (M x ld
// elements, row-major, box 64 x 128, 128-byte swizzle) into out (a
// CUtensorMap, 128 bytes, 64-byte aligned); 0 on success.
int scaled_tma_map(void* out, const void* payload, int64_t M, int64_t ld, int fmt);
// resident CTAs per SM for R <= 32 (0 on error); tma: the TMA-fed BF16 kernel
int scaled_mma_occupancy(int fmt, bool tma);

// Fixed-accuracy (WZ3) pass: (2G)^T x, then persistent warp ranges of L runs
// over the pass's bands in band-major order, then (maxseg > 1) the segment
// epilogue for bands shared by several ranges.  band0 is the first band of a
// row view within the matrix (its index is the matrix's).
struct Wz3Step {
  const uint64_t* index;  // the matrix's run index (BM_total x RB)
  const uint8_t* area;    // the block area
  int64_t band0;
  int64_t M, N, BM, BN, RB;
  const float* x;
  int64_t ldx;
  float* xt;  // scratch: (2G)^T x, 4 BN floats per right-hand side
  int R;      // 1 or 8
  int64_t L;      // runs per warp range
  int maxseg;     // most ranges sharing one band
  int64_t ctas;   // grid size
  double* ws;     // BM x maxseg x R x 4 segment partials when maxseg > 1
  double* y;
  int64_t ldy;
  double* state;
  double decay;
};
int wz3_launch(const Wz3Step& a, cudaStream_t st);
int wz3_occupancy(int R);  // resident CTAs per SM of the R-column kernel (0 on error)
int wz3_decompress(const uint64_t* index, const uint8_t* area, int64_t M, int64_t N, double* out, int64_t ldo,
                   cudaStream_t st);

template <int RATE>
int wz2_launch(const Wz2Step& a, cudaStream_t st);
template <int RATE>
int wz2_batched_launch(const Wz2Batch& b, cudaStream_t st);
template <int RATE>
int wz2_decompress(const uint8_t* stream, int64_t M, int64_t N, int64_t BN, int64_t nblocks, double* out,
                   int64_t ldo, bool lift, cudaStream_t st);
// resident CTAs per SM of the R = 1 kernel for the given unroll (0 on error)
template <int RATE>
int wz2_occupancy(bool lift, int unroll);
// resident CTAs per SM of the staged R = 1 kernel (0 on error)
template <int RATE>
int wz2_stream_occupancy(bool lift);

}  // namespace whff
