// wz2_dispatch.cuh -- definitions behind wz2_dispatch.h; included once per
// rate by wz2_r<rate>.cu, which instantiates them for that rate.
#pragma once
#include "wz2_dispatch.h"
#include "wz2_kernels.cuh"
#include "wz2_stream.cuh"

namespace whff {

template <int RATE, bool LIFT, int R, int U, int GL = 32>
static void wz2_launch_one(const Wz2Step& a, cudaStream_t st) {
  dev::wz2_gemv_entry<RATE, LIFT, R, U, GL>()<<<(unsigned)a.ctas, dev::kWarpsPerCta * 32, 0, st>>>(
      a.stream, a.M, a.N, a.BM, a.BN, a.x, a.ldx, a.x_vec_ok, a.L, a.maxseg, a.ws, a.y, a.ldy, a.state, a.decay,
      a.red32);
}

template <int RATE, bool LIFT>
static int wz2_stream_smem_attr() {
  static int done = 0;  // once per instantiation and process (the attribute is per function)
  if (!done) {
    if (cudaFuncSetAttribute(dev::wz2_stream_kernel<RATE, LIFT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             dev::Wz2Stream<RATE>::kSmemBytes) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    done = 1;
  }
  return 0;
}

template <int RATE, bool LIFT>
static int wz2_launch_lift(const Wz2Step& a, cudaStream_t st) {
  if (a.staged && a.R == 1 && !a.groups8) {
    if (wz2_stream_smem_attr<RATE, LIFT>()) return -1;
    dev::wz2_stream_kernel<RATE, LIFT><<<(unsigned)a.ctas, dev::kWarpsPerCta * 32, dev::Wz2Stream<RATE>::kSmemBytes,
                                         st>>>(a.stream, a.M, a.N, a.BM, a.BN, a.x, a.ldx, a.x_vec_ok, a.L, a.maxseg,
                                               a.ws, a.y, a.ldy, a.state, a.decay, a.red32, a.status);
  } else if (a.groups8) {  // short bands: four 8-lane groups per warp, two blocks in flight per lane
    switch (a.R) {
      case 1: wz2_launch_one<RATE, LIFT, 1, 2, 8>(a, st); break;
      case 2: wz2_launch_one<RATE, LIFT, 2, 2, 8>(a, st); break;
      case 4: wz2_launch_one<RATE, LIFT, 4, 2, 8>(a, st); break;
      case 8: wz2_launch_one<RATE, LIFT, 8, 2, 8>(a, st); break;
      default: return -1;
    }
  } else switch (a.R) {
    case 1:
      if (a.unroll == 8) wz2_launch_one<RATE, LIFT, 1, 8>(a, st);
      else if (a.unroll == 4) wz2_launch_one<RATE, LIFT, 1, 4>(a, st);
      else wz2_launch_one<RATE, LIFT, 1, 2>(a, st);
      break;
    case 2: wz2_launch_one<RATE, LIFT, 2, 2>(a, st); break;
    case 4: wz2_launch_one<RATE, LIFT, 4, 2>(a, st); break;
    case 8: wz2_launch_one<RATE, LIFT, 8, 2>(a, st); break;
    default: return -1;
  }
  if (a.maxseg > 1)
    dev::wz2_segment_epilogue<<<(unsigned)((dev::segment_epilogue_threads(a.M, a.BN, a.L) + 255) / 256), 256, 0, st>>>(a.ws, a.M, a.BN, a.L, a.maxseg, a.R,
                                                                            a.y, a.ldy, a.state, a.decay);
  return 0;
}

template <int RATE>
int wz2_launch(const Wz2Step& a, cudaStream_t st) {
  if (!a.lift) return wz2_launch_lift<RATE, false>(a, st);
  // the lift: transform x once per pass, then the kernels read (2G)^T x as their x
  const int64_t ldt = 4 * a.BN, n = (int64_t)a.R * a.BN;
  dev::wz2_xt_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a.x, a.ldx, a.N, a.R, a.BN, a.xt, ldt);
  Wz2Step b = a;
  b.x = a.xt;
  b.ldx = ldt;
  b.N = ldt;
  b.x_vec_ok = true;
  return wz2_launch_lift<RATE, true>(b, st);
}

template <int RATE, bool LIFT, int R>
static void wz2_batched_one(const Wz2Batch& b, cudaStream_t st) {
  constexpr int U = 2;
  dev::wz2_batched_kernel<RATE, LIFT, R, U><<<(unsigned)b.ctas, dev::kWarpsPerCta * 32, 0, st>>>(
      b.entries, b.nentries, b.total_blocks, b.L);
}

template <int RATE>
int wz2_batched_launch(const Wz2Batch& b, cudaStream_t st) {
#define WZ2B(LF, RR) \
  if (b.lift == LF && b.R == RR) wz2_batched_one<RATE, LF, RR>(b, st);
  WZ2B(true, 1) WZ2B(true, 2) WZ2B(true, 4) WZ2B(true, 8)
  WZ2B(false, 1) WZ2B(false, 2) WZ2B(false, 4) WZ2B(false, 8)
#undef WZ2B
  if (b.R != 1 && b.R != 2 && b.R != 4 && b.R != 8) return -1;
  if (b.any_shared)
    dev::wz2_batched_epilogue<<<(unsigned)((b.total_rows + 255) / 256), 256, 0, st>>>(b.entries, b.row_begin,
                                                                                     b.nentries, b.total_rows, b.L,
                                                                                     b.R);
  return 0;
}

template <int RATE>
int wz2_decompress(const uint8_t* stream, int64_t M, int64_t N, int64_t BN, int64_t nblocks, double* out,
                   int64_t ldo, bool lift, cudaStream_t st) {
  const unsigned grid = (unsigned)((nblocks + 255) / 256);
  if (lift)
    dev::wz2_decompress_kernel<RATE, true><<<grid, 256, 0, st>>>(stream, M, N, BN, nblocks, out, ldo);
  else
    dev::wz2_decompress_kernel<RATE, false><<<grid, 256, 0, st>>>(stream, M, N, BN, nblocks, out, ldo);
  return 0;
}

template <int RATE, bool LIFT>
static cudaError_t wz2_occ_lift(int* occ, int unroll, int threads) {
  if (unroll == 8)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, dev::wz2_gemv_entry<RATE, LIFT, 1, 8, 32>(), threads, 0);
  if (unroll == 4)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, dev::wz2_gemv_entry<RATE, LIFT, 1, 4, 32>(), threads, 0);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, dev::wz2_gemv_entry<RATE, LIFT, 1, 2, 32>(), threads, 0);
}

template <int RATE>
int wz2_stream_occupancy(bool lift) {
  int occ = 0;
  const int threads = dev::kWarpsPerCta * 32;
  const int smem = dev::Wz2Stream<RATE>::kSmemBytes;
  cudaError_t e;
  if (lift) {
    e = wz2_stream_smem_attr<RATE, true>() ? cudaErrorInvalidValue
                                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                                &occ, dev::wz2_stream_kernel<RATE, true>, threads, smem);
  } else {
    e = wz2_stream_smem_attr<RATE, false>() ? cudaErrorInvalidValue
                                           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                                 &occ, dev::wz2_stream_kernel<RATE, false>, threads, smem);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ;
}

template <int RATE>
int wz2_occupancy(bool lift, int unroll) {
  int occ = 0;
  const int threads = dev::kWarpsPerCta * 32;
  const cudaError_t e = lift ? wz2_occ_lift<RATE, true>(&occ, unroll, threads)
                             : wz2_occ_lift<RATE, false>(&occ, unroll, threads);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ;
}

}  // namespace whff

#define WHFF_INSTANTIATE_WZ2(RATE)                                                                            \
  template int whff::wz2_launch<RATE>(const whff::Wz2Step&, cudaStream_t);                                    \
  template int whff::wz2_batched_launch<RATE>(const whff::Wz2Batch&, cudaStream_t);                           \
  template int whff::wz2_decompress<RATE>(const uint8_t*, int64_t, int64_t, int64_t, int64_t, double*, int64_t, \
                                          bool, cudaStream_t);                                                \
  template int whff::wz2_occupancy<RATE>(bool, int);                                                         \
  template int whff::wz2_stream_occupancy<RATE>(bool);
