// wz2_batch.h -- one entry of a batched WZ2 launch (shared by the kernels and
// the host code that fills the device table).
#pragma once
#include <cstdint>

namespace whff {
namespace dev {

// One matrix of a batch: its compressed stream, vectors and place in the
// concatenated band-major block order of the whole batch.
struct BatchEntry {
  const uint8_t* stream;
  const float* x;
  double* y;
  double* state;
  double* ws;             // segment partials of this entry's shared bands
  int64_t M, N, BM, BN;
  int64_t ldx, ldy;
  int64_t block_begin;    // first global block index of this entry
  int maxseg;
  double decay;
  const float* scales;    // scaled formats: the tile scales (stream = the payload)
  int64_t ld, TN;         // scaled formats: payload row length, 128-column tiles per row
};

// The carried state of one batched matrix, applied after all its column
// groups: for r = 0..R-1 in order, s <- decay*s + y[:, r].
struct BatchState {
  double* state;
  const double* y;
  int64_t ldy, M;
  int R;
  double decay;
};

// One matrix of a tensor-core launch: a pass of up to NR columns over its
// (tile of 32 bands, stage of 16 blocks) items, which occupy
// [item_begin, item_begin + tiles * S) of the launch's item sequence.
struct MmaMember {
  const uint8_t* stream;  // compressed stream (WZ2 blocks, band-major)
  const uint8_t* btiles;  // the pass's B tiles, one per stage
  double* ws;             // FP64 segment partials: tiles x maxseg x R x 128
  int64_t BM, BN;         // block grid
  int64_t item_begin;
  int S, tiles, R, maxseg;  // stages per tile, tiles, columns of the pass, segments per tile
};

// The vectors of one tensor-core pass (rewritten every step): B tiles are
// built from x, the finish writes y.  bt_begin / fin_begin: the member's first
// thread in the launch-wide B-tile and finish grids.
struct MmaPass {
  const float* x;
  double* y;
  uint8_t* btiles;
  const double* ws;
  int64_t ldx, ldy, N, M;
  int64_t item_begin, bt_begin, fin_begin;
  int S, tiles, R, maxseg;
};

}  // namespace dev
}  // namespace whff
