// Tensor-core (tcgen05) launches for many right-hand sides: instantiation unit.
#include "mma_kernels.cuh"
#include "wz2_dispatch.h"

namespace whff {

template <int RATE, bool LIFT, int NR>
static int mma_one(const MmaStep& a, cudaStream_t st) {
  using S = dev::MmaSmem<NR>;
  auto kern = dev::wz2_mma_kernel<RATE, LIFT, NR>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes) != cudaSuccess) return -1;
  const int64_t nstages = (a.BN + dev::kMmaStageBlocks - 1) / dev::kMmaStageBlocks;
  const int64_t bthreads = nstages * dev::kMmaStageBlocks * NR;
  dev::wz2_mma_btiles<LIFT, NR><<<(unsigned)((bthreads + 255) / 256), 256, 0, st>>>(a.x, a.ldx, a.N, a.R, nstages,
                                                                                   a.btiles);
  dim3 grid((unsigned)((a.BM + dev::kMmaBands - 1) / dev::kMmaBands), (unsigned)a.ksplit);
  kern<<<grid, dev::kMmaThreads, S::kBytes, st>>>(a.stream, a.BM, a.BN, a.btiles, a.R, a.jchunk, a.ws, a.Mpad,
                                                 a.status);
  dev::wz2_mma_finish<LIFT><<<(unsigned)((a.BM + 127) / 128), 128, 0, st>>>(a.ws, a.ksplit, a.R, a.Mpad, a.M, a.y,
                                                                           a.ldy, a.state, a.decay);
  return 0;
}

template <int RATE>
static int mma_rate(const MmaStep& a, cudaStream_t st) {
  const int nr = a.R <= 16 ? 16 : 32;
  if (a.lift) return nr == 16 ? mma_one<RATE, true, 16>(a, st) : mma_one<RATE, true, 32>(a, st);
  return nr == 16 ? mma_one<RATE, false, 16>(a, st) : mma_one<RATE, false, 32>(a, st);
}

int mma_launch(const MmaStep& a, cudaStream_t st) {
  if (a.R < 1 || a.R > 32) return -1;
  switch (a.rate) {
    case 8: return mma_rate<8>(a, st);
    case 12: return mma_rate<12>(a, st);
    case 16: return mma_rate<16>(a, st);
    case 20: return mma_rate<20>(a, st);
    case 24: return mma_rate<24>(a, st);
    default: return -1;
  }
}

}  // namespace whff
