// Tensor-core (tcgen05) launches for many right-hand sides: instantiation unit.
#include <algorithm>

#include "mma_kernels.cuh"
#include "wz2_dispatch.h"

namespace whff {

template <int RATE, bool LIFT, int NR>
static int mma_one(const MmaStep& a, cudaStream_t st) {
  using S = dev::MmaSmem<RATE, NR>;
  auto kern = dev::wz2_mma_kernel<RATE, LIFT, NR>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
          cudaSuccess)
    return -1;
  const int64_t nstages = (a.BN + dev::kMmaStageBlocks - 1) / dev::kMmaStageBlocks;
  const int64_t tiles = (a.BM + dev::kMmaBands - 1) / dev::kMmaBands;
  const int64_t bthreads = nstages * dev::kMmaStageBlocks * NR;
  dev::wz2_mma_btiles<LIFT, NR><<<(unsigned)((bthreads + 255) / 256), 256, 0, st>>>(a.x, a.ldx, a.N, a.R, nstages,
                                                                                   a.btiles);
  kern<<<(unsigned)a.ctas, dev::kMmaThreads, S::kBytes, st>>>(a.stream, a.BM, a.BN, a.btiles, a.R, nstages,
                                                             tiles * nstages, a.L, a.maxseg, a.ws, a.status);
  const int64_t fin_threads = tiles * a.R * 32;
  dev::wz2_mma_finish<LIFT><<<(unsigned)((fin_threads + 255) / 256), 256, 0, st>>>(a.ws, nstages, a.L, a.maxseg, a.R,
                                                                                  a.M, a.y, a.ldy);
  if (a.state)
    dev::wz2_mma_state<<<(unsigned)((a.M + 255) / 256), 256, 0, st>>>(a.y, a.ldy, a.R, a.M, a.state, a.decay);
  return 0;
}

template <int RATE>
static int mma_rate(const MmaStep& a, cudaStream_t st) {
  const int nr = a.R <= 16 ? 16 : 32;
  if (a.lift) return nr == 16 ? mma_one<RATE, true, 16>(a, st) : mma_one<RATE, true, 32>(a, st);
  return nr == 16 ? mma_one<RATE, false, 16>(a, st) : mma_one<RATE, false, 32>(a, st);
}

int mma_launch(const MmaStep& a, cudaStream_t st) {
  if (a.R < 1 || a.R > 32 || a.ctas < 1 || a.L < 1) return -1;
  switch (a.rate) {
    case 8: return mma_rate<8>(a, st);
    case 12: return mma_rate<12>(a, st);
    case 16: return mma_rate<16>(a, st);
    case 20: return mma_rate<20>(a, st);
    case 24: return mma_rate<24>(a, st);
    default: return -1;
  }
}

// Resident CTAs per SM from the kernel's registers, shared memory and TMEM
// columns (the occupancy API under-reports this kernel); a persistent grid
// sized from a value that is too high is still correct, only slower.
template <int RATE, bool LIFT, int NR>
static int mma_occ_one() {
  using S = dev::MmaSmem<RATE, NR>;
  auto kern = dev::wz2_mma_kernel<RATE, LIFT, NR>;
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
  const int by_tmem = 512 / (4 * NR);
  return std::min(std::min(by_regs, by_smem), by_tmem);
}

template <int RATE>
static int mma_occ_rate(bool lift, int nr) {
  if (lift) return nr <= 16 ? mma_occ_one<RATE, true, 16>() : mma_occ_one<RATE, true, 32>();
  return nr <= 16 ? mma_occ_one<RATE, false, 16>() : mma_occ_one<RATE, false, 32>();
}

int mma_occupancy(int rate, bool lift, int nr) {
  switch (rate) {
    case 8: return mma_occ_rate<8>(lift, nr);
    case 12: return mma_occ_rate<12>(lift, nr);
    case 16: return mma_occ_rate<16>(lift, nr);
    case 20: return mma_occ_rate<20>(lift, nr);
    case 24: return mma_occ_rate<24>(lift, nr);
    default: return 0;
  }
}

}  // namespace whff
