// Tensor-core (tcgen05) passes for the scaled formats: instantiation unit.
#include <algorithm>

#include "scaled_mma.cuh"
#include "wz2_dispatch.h"

namespace whff {

template <int FMT, int NR>
static int scaled_mma_one(const ScaledMmaStep& a, cudaStream_t st) {
  using S = dev::ScaledMmaSmem<FMT, NR>;
  auto kern = dev::scaled_mma_kernel<FMT, NR>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
          cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  const int nstages = (int)((a.N + 63) / 64);
  const int tiles = (int)((a.M + 127) / 128);
  const dev::MmaPass pass{a.x, a.y, a.btiles, a.ws, a.ldx, a.ldy, a.N, a.M, 0, 0, 0, nstages, tiles, a.R, a.maxseg};
  const int64_t bthreads = (int64_t)nstages * dev::kMmaStageBlocks * NR;
  dev::wz2_mma_btiles<false, NR><<<(unsigned)((bthreads + 255) / 256), 256, 0, st>>>(pass, nullptr, 1, bthreads);
  kern<<<(unsigned)a.ctas, dev::kMmaThreads, S::kBytes, st>>>(a.payload, a.scales, a.M, a.ld, a.TN, a.btiles, a.ws,
                                                              nstages, a.R, a.maxseg, (int64_t)tiles * nstages, a.L,
                                                              a.status, a.spin);
  const int64_t fin = (int64_t)tiles * a.R * 128;
  dev::scaled_mma_finish<<<(unsigned)((fin + 255) / 256), 256, 0, st>>>(a.ws, a.M, nstages, a.R, a.maxseg, tiles, a.L,
                                                                       a.y, a.ldy);
  if (a.state)
    dev::wz2_mma_state<<<(unsigned)((a.M + 255) / 256), 256, 0, st>>>(a.y, a.ldy, a.R, a.M, a.state, a.decay);
  return 0;
}

template <int FMT>
static int scaled_mma_fmt(const ScaledMmaStep& a, cudaStream_t st) {
  return a.R <= 16 ? scaled_mma_one<FMT, 16>(a, st) : scaled_mma_one<FMT, 32>(a, st);
}

int scaled_mma_launch(const ScaledMmaStep& a, cudaStream_t st) {
  if (a.R < 1 || a.R > 32 || a.ctas < 1 || a.L < 1) return -1;
  switch (a.fmt) {
    case 2: return scaled_mma_fmt<2>(a, st);
    case 3: return scaled_mma_fmt<3>(a, st);
    case 4: return scaled_mma_fmt<4>(a, st);
    default: return -1;
  }
}

// Resident CTAs per SM from the kernel's registers, shared memory and TMEM
// columns (as for the fixed-allocation tensor-core kernel).
template <int FMT, int NR>
static int scaled_mma_occ_one() {
  using S = dev::ScaledMmaSmem<FMT, NR>;
  auto kern = dev::scaled_mma_kernel<FMT, NR>;
  cudaFuncAttributes fa;
  int dev = 0, smem_sm = 0, regs_sm = 0, reserved = 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
          cudaSuccess ||
      cudaFuncGetAttributes(&fa, kern) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int warps = dev::kMmaThreads / 32;
  const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
  const int by_regs = regs_sm / (regs_warp * warps);
  const int by_smem = smem_sm / (S::kBytes + (int)fa.sharedSizeBytes + reserved);
  const int by_tmem = 512 / (int)dev::mma_tmem_cols<NR>();
  return std::min(std::min(by_regs, by_smem), by_tmem);
}

int scaled_mma_occupancy(int fmt) {
  switch (fmt) {
    case 2: return std::min(scaled_mma_occ_one<2, 16>(), scaled_mma_occ_one<2, 32>());
    case 3: return std::min(scaled_mma_occ_one<3, 16>(), scaled_mma_occ_one<3, 32>());
    case 4: return std::min(scaled_mma_occ_one<4, 16>(), scaled_mma_occ_one<4, 32>());
    default: return 0;
  }
}

}  // namespace whff
