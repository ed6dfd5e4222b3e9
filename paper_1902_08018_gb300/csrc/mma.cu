// Tensor-core (tcgen05) launches for many right-hand sides: instantiation unit.
#include <algorithm>

#include "mma_kernels.cuh"
#include "wz2_dispatch.h"

namespace whff {

constexpr int kMaxMembers = 64;  // members of one batched tensor-core launch (their table sits in smem)

template <int RATE, bool LIFT, int NR, bool TABLE>
static int mma_set_smem(int bytes) {
  auto kern = dev::wz2_mma_kernel<RATE, LIFT, NR, TABLE>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
          cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return 0;
}

template <int RATE, bool LIFT, int NR>
static int mma_one(const MmaStep& a, cudaStream_t st) {
  using S = dev::MmaSmem<RATE, NR>;
  const int smem = S::kBytes;
  if (mma_set_smem<RATE, LIFT, NR, false>(smem)) return -1;
  const int nstages = (int)((a.BN + dev::kMmaStageBlocks - 1) / dev::kMmaStageBlocks);
  const int tiles = (int)((a.BM + dev::kMmaBands - 1) / dev::kMmaBands);
  const dev::MmaMember mem{a.stream, a.btiles, a.ws, a.BM, a.BN, 0, nstages, tiles, a.R, a.maxseg};
  const dev::MmaPass pass{a.x, a.y, a.btiles, a.ws, a.ldx, a.ldy, a.N, a.M, 0, 0, 0, nstages, tiles, a.R, a.maxseg};
  const int64_t bthreads = (int64_t)nstages * dev::kMmaStageBlocks * NR;
  dev::wz2_mma_btiles<LIFT, NR><<<(unsigned)((bthreads + 255) / 256), 256, 0, st>>>(pass, nullptr, 1, bthreads);
  dev::wz2_mma_kernel<RATE, LIFT, NR, false><<<(unsigned)a.ctas, dev::kMmaThreads, smem, st>>>(
      mem, nullptr, 1, (int64_t)tiles * nstages, a.L, a.status, a.spin);
  const int64_t fin_threads = (int64_t)tiles * a.R * 32;
  dev::wz2_mma_finish<LIFT><<<(unsigned)((fin_threads + 255) / 256), 256, 0, st>>>(pass, nullptr, 1, fin_threads,
                                                                                  a.L);
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

// A batch's passes of one width class in one persistent launch: B tiles of
// every pass, the tensor-core kernel over the concatenated item sequence,
// every pass's finish (the states are the caller's).
template <int RATE, bool LIFT, int NR>
static int mma_batch_one(const MmaBatchStep& a, cudaStream_t st) {
  using S = dev::MmaSmem<RATE, NR>;
  const int smem = S::kBytes + a.nmem * (int)sizeof(dev::MmaMember);
  if (mma_set_smem<RATE, LIFT, NR, true>(smem)) return -1;
  const dev::MmaMember m0{};
  const dev::MmaPass p0{};
  dev::wz2_mma_btiles<LIFT, NR><<<(unsigned)((a.bt_threads + 255) / 256), 256, 0, st>>>(p0, a.passes, a.nmem,
                                                                                       a.bt_threads);
  dev::wz2_mma_kernel<RATE, LIFT, NR, true><<<(unsigned)a.ctas, dev::kMmaThreads, smem, st>>>(m0, a.members, a.nmem,
                                                                                            a.total, a.L, a.status,
                                                                                            a.spin);
  dev::wz2_mma_finish<LIFT><<<(unsigned)((a.fin_threads + 255) / 256), 256, 0, st>>>(p0, a.passes, a.nmem,
                                                                                    a.fin_threads, a.L);
  return 0;
}

template <int RATE>
static int mma_batch_rate(const MmaBatchStep& a, cudaStream_t st) {
  if (a.lift) return a.nr == 16 ? mma_batch_one<RATE, true, 16>(a, st) : mma_batch_one<RATE, true, 32>(a, st);
  return a.nr == 16 ? mma_batch_one<RATE, false, 16>(a, st) : mma_batch_one<RATE, false, 32>(a, st);
}

int mma_batch_launch(const MmaBatchStep& a, cudaStream_t st) {
  if ((a.nr != 16 && a.nr != 32) || a.nmem < 1 || a.nmem > kMaxMembers || a.ctas < 1 || a.L < 1) return -1;
  switch (a.rate) {
    case 8: return mma_batch_rate<8>(a, st);
    case 12: return mma_batch_rate<12>(a, st);
    case 16: return mma_batch_rate<16>(a, st);
    case 20: return mma_batch_rate<20>(a, st);
    case 24: return mma_batch_rate<24>(a, st);
    default: return -1;
  }
}

int mma_max_members() { return kMaxMembers; }

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
  auto kern = dev::wz2_mma_kernel<RATE, LIFT, NR, true>;  // the larger of the two (registers, table)
  const int smem = S::kBytes + kMaxMembers * (int)sizeof(dev::MmaMember);
  cudaFuncAttributes fa;
  int dev = 0, smem_sm = 0, regs_sm = 0, reserved = 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
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
  const int by_smem = smem_sm / (smem + (int)fa.sharedSizeBytes + reserved);
  const int by_tmem = 512 / (int)dev::mma_tmem_cols<NR>();
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
