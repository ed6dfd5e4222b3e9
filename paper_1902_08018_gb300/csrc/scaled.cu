// Scaled-format GEMV launches (BF16, FP16, FP8 E4M3, FP32): instantiation unit.
#include "scaled_kernels.cuh"
#include "whff_blob.h"
#include "wz2_dispatch.h"

namespace whff {

template <int FMT, int R>
static void scaled_one(const ScaledStep& a, cudaStream_t st) {
  if (a.groups8)
    dev::scaled_range_kernel<FMT, R, 8><<<(unsigned)a.ctas, dev::kWarpsPerCta * 32, 0, st>>>(
        a.payload, a.scales, a.M, a.N, a.ld, a.TN, a.x, a.ldx, a.x_vec_ok, a.L, a.maxseg, a.ws, a.y, a.ldy, a.state,
        a.decay, a.red32);
  else
    dev::scaled_range_kernel<FMT, R, 32><<<(unsigned)a.ctas, dev::kWarpsPerCta * 32, 0, st>>>(
        a.payload, a.scales, a.M, a.N, a.ld, a.TN, a.x, a.ldx, a.x_vec_ok, a.L, a.maxseg, a.ws, a.y, a.ldy, a.state,
        a.decay, a.red32);
}

template <int FMT>
static int scaled_fmt(const ScaledStep& a, cudaStream_t st) {
  switch (a.R) {
    case 1: scaled_one<FMT, 1>(a, st); break;
    case 2: scaled_one<FMT, 2>(a, st); break;
    case 4: scaled_one<FMT, 4>(a, st); break;
    case 8: scaled_one<FMT, 8>(a, st); break;
    default: return -1;
  }
  return 0;
}

int scaled_launch(const ScaledStep& a, cudaStream_t st) {
  int e;
  switch (a.fmt) {
    case 2: e = scaled_fmt<2>(a, st); break;
    case 3: e = scaled_fmt<3>(a, st); break;
    case 4: e = scaled_fmt<4>(a, st); break;
    case 7: e = scaled_fmt<7>(a, st); break;
    default: return -1;
  }
  if (e) return e;
  if (a.maxseg > 1) {  // shared bands: the chunks of a band are the "blocks" of the segment epilogue
    const int V = scaled_vec(a.fmt);
    dev::wz2_segment_epilogue<<<(unsigned)((dev::segment_epilogue_threads(a.M, a.ld / V, a.L) + 255) / 256), 256, 0, st>>>(a.ws, a.M, a.ld / V, a.L, a.maxseg,
                                                                            a.R, a.y, a.ldy, a.state, a.decay);
  }
  return 0;
}

template <int FMT>
static int scaled_batched_fmt(const Wz2Batch& b, cudaStream_t st) {
  const unsigned grid = (unsigned)b.ctas, threads = dev::kWarpsPerCta * 32;
  switch (b.R) {
    case 1: dev::scaled_batched_kernel<FMT, 1><<<grid, threads, 0, st>>>(b.entries, b.nentries, b.total_blocks, b.L); break;
    case 2: dev::scaled_batched_kernel<FMT, 2><<<grid, threads, 0, st>>>(b.entries, b.nentries, b.total_blocks, b.L); break;
    case 4: dev::scaled_batched_kernel<FMT, 4><<<grid, threads, 0, st>>>(b.entries, b.nentries, b.total_blocks, b.L); break;
    case 8: dev::scaled_batched_kernel<FMT, 8><<<grid, threads, 0, st>>>(b.entries, b.nentries, b.total_blocks, b.L); break;
    default: return -1;
  }
  return 0;
}

int scaled_batched_launch(int fmt, const Wz2Batch& b, cudaStream_t st) {
  int e;
  switch (fmt) {
    case 2: e = scaled_batched_fmt<2>(b, st); break;
    case 3: e = scaled_batched_fmt<3>(b, st); break;
    case 4: e = scaled_batched_fmt<4>(b, st); break;
    case 7: e = scaled_batched_fmt<7>(b, st); break;
    default: return -1;
  }
  if (e) return e;
  if (b.any_shared)
    dev::wz2_batched_epilogue<<<(unsigned)((b.total_rows + 255) / 256), 256, 0, st>>>(b.entries, b.row_begin,
                                                                                     b.nentries, b.total_rows, b.L,
                                                                                     b.R);
  return 0;
}

template <int FMT>
static cudaError_t scaled_occ(int* occ, bool groups8, int threads) {
  if (groups8) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, dev::scaled_range_kernel<FMT, 1, 8>, threads, 0);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, dev::scaled_range_kernel<FMT, 1, 32>, threads, 0);
}

int scaled_occupancy(int fmt, bool groups8) {
  int occ = 0;
  cudaError_t e = cudaErrorInvalidValue;
  const int threads = dev::kWarpsPerCta * 32;
  if (fmt == 2) e = scaled_occ<2>(&occ, groups8, threads);
  if (fmt == 3) e = scaled_occ<3>(&occ, groups8, threads);
  if (fmt == 4) e = scaled_occ<4>(&occ, groups8, threads);
  if (fmt == 7) e = scaled_occ<7>(&occ, groups8, threads);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ;
}

}  // namespace whff
