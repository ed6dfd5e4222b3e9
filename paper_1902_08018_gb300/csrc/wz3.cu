// Fixed-accuracy (WZ3) launches: instantiation unit.
#include "wz2_dispatch.h"
#include "wz3_kernels.cuh"

namespace whff {

int wz3_launch(const Wz3Step& a, cudaStream_t st) {
  if (a.R != 1 && a.R != 8) return -1;
  // (2G)^T x once per pass, 4 BN floats per right-hand side
  const int64_t ldt = 4 * a.BN, n = (int64_t)a.R * a.BN;
  dev::wz2_xt_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a.x, a.ldx, a.N, a.R, a.BN, a.xt, ldt);
  const uint64_t* index = a.index + a.band0 * a.RB;  // the view's first band
  const unsigned grid = (unsigned)a.ctas, threads = dev::kWarpsPerCta * 32;
  if (a.R == 1)
    dev::wz3_gemv_kernel<1><<<grid, threads, 0, st>>>(index, a.area, a.M, a.BM, (int)a.BN, (int)a.RB, a.xt, ldt, a.L,
                                                      a.maxseg, a.ws, a.y, a.ldy, a.state, a.decay);
  else
    dev::wz3_gemv_kernel<8><<<grid, threads, 0, st>>>(index, a.area, a.M, a.BM, (int)a.BN, (int)a.RB, a.xt, ldt, a.L,
                                                      a.maxseg, a.ws, a.y, a.ldy, a.state, a.decay);
  if (a.maxseg > 1)  // units per band: runs
    dev::wz2_segment_epilogue<<<(unsigned)((dev::segment_epilogue_threads(a.M, a.RB, a.L) + 255) / 256), 256, 0, st>>>(a.ws, a.M, a.RB, a.L, a.maxseg, a.R,
                                                                            a.y, a.ldy, a.state, a.decay);
  return 0;
}

int wz3_occupancy(int R) {
  int occ = 0;
  const int threads = dev::kWarpsPerCta * 32;
  const cudaError_t e = R == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dev::wz3_gemv_kernel<1>, threads, 0)
                               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dev::wz3_gemv_kernel<8>, threads, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ;
}

int wz3_decompress(const uint64_t* index, const uint8_t* area, int64_t M, int64_t N, double* out, int64_t ldo,
                   cudaStream_t st) {
  const int64_t BM = (M + 3) / 4, BN = (N + 3) / 4, RB = (BN + 31) / 32, nb = BM * BN;
  dev::wz3_decompress_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(index, area, M, N, BN, RB, nb, out, ldo);
  return 0;
}

}  // namespace whff
