// WZ2 kernels at rate 16 (bits per value): instantiation unit.
#include "wz2_dispatch.cuh"
WHFF_INSTANTIATE_WZ2(16)

int whff::wz2_batched_state_launch(const whff::dev::BatchState* table, const int64_t* row_begin, int n,
                                   int64_t total_rows, cudaStream_t st) {
  whff::dev::wz2_batched_state<<<(unsigned)((total_rows + 255) / 256), 256, 0, st>>>(table, row_begin, n, total_rows);
  return 0;
}
