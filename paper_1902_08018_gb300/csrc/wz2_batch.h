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

}  // namespace dev
}  // namespace whff
