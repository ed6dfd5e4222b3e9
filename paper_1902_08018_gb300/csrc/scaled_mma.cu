// Tensor-core (tcgen05) passes for the scaled formats: instantiation unit.
#include <algorithm>

#include <cudaTypedefs.h>

#include "scaled_mma.cuh"
#include "scaled_mma_tma.cuh"
#include "wz2_dispatch.h"

namespace whff {

// The TMA-fed kernel (BF16, or FP16 with F16): its shared-memory attribute,
// set once per width and type.
template <int NR, bool F16>
static int scaled_tma_attr() {
  static int done = 0;
  if (!done) {
    auto kern = dev::scaled_mma_tma_kernel<NR, F16>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dev::TmaSmem<NR>::kBytes) !=
            cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
            cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    done = 1;
  }
  return 0;
}

template <int FMT, int NR>
static int scaled_mma_one(const ScaledMmaStep& a, cudaStream_t st) {
  using S = dev::ScaledMmaSmem<FMT, NR>;
  auto kern = dev::scaled_mma_kernel<FMT, NR>;
  constexpr bool kF16 = FMT == 3;
  const bool tma = (FMT == 2 || FMT == 3) && a.tmap != nullptr;
  if (tma ? scaled_tma_attr<NR, kF16>() != 0
          : (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes) != cudaSuccess ||
             cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  cudaSharedmemCarveoutMaxShared) != cudaSuccess)) {
    cudaGetLastError();
    return -1;
  }
  const int nstages = (int)((a.N + 63) / 64);
  const int tiles = (int)((a.M + 127) / 128);
  const dev::MmaPass pass{a.x, a.y, a.btiles, a.ws, a.ldx, a.ldy, a.N, a.M, 0, 0, 0, nstages, tiles, a.R, a.maxseg};
  const int64_t bthreads = (int64_t)nstages * dev::kMmaStageBlocks * NR;
  const bool f16_pieces = tma && kF16;  // FP16 A by TMA: FP16 B pieces of x scaled per column
  if (f16_pieces) {
    dev::f16_colexp_kernel<<<(unsigned)NR, 256, 0, st>>>(a.x, a.ldx, a.N, a.R, a.colexp);
    dev::f16_mma_btiles<NR><<<(unsigned)((bthreads + 255) / 256), 256, 0, st>>>(pass, a.colexp, bthreads);
  } else {
    dev::wz2_mma_btiles<false, NR><<<(unsigned)((bthreads + 255) / 256), 256, 0, st>>>(pass, nullptr, 1, bthreads);
  }
  if (tma) {
    dev::scaled_mma_tma_kernel<NR, kF16><<<(unsigned)a.ctas, dev::kTmaThreads, dev::TmaSmem<NR>::kBytes, st>>>(
        *static_cast<const CUtensorMap*>(a.tmap), a.row0, a.scales, a.TN, a.btiles, a.ws, nstages, a.R, a.maxseg,
        (int64_t)tiles * nstages, a.L, a.status, a.spin);
  } else {
    kern<<<(unsigned)a.ctas, dev::kMmaThreads, S::kBytes, st>>>(a.payload, a.scales, a.M, a.ld, a.TN, a.btiles,
                                                                a.ws, nstages, a.R, a.maxseg,
                                                                (int64_t)tiles * nstages, a.L, a.status, a.spin);
  }
  const int64_t fin = (int64_t)tiles * a.R * 128;
  dev::scaled_mma_finish<<<(unsigned)((fin + 255) / 256), 256, 0, st>>>(a.ws, a.M, nstages, a.R, a.maxseg, tiles, a.L,
                                                                       a.y, a.ldy, f16_pieces ? a.colexp : nullptr);
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

// Resident CTAs per SM of the TMA-fed kernel, from its registers, shared
// memory and TMEM columns (the occupancy API reported one CTA where two fit).
template <int NR, bool F16>
static int scaled_tma_occ_one() {
  auto kern = dev::scaled_mma_tma_kernel<NR, F16>;
  cudaFuncAttributes fa;
  int dev = 0, smem_sm = 0, regs_sm = 0, reserved = 0;
  if (scaled_tma_attr<NR, F16>() || cudaFuncGetAttributes(&fa, kern) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int warps = dev::kTmaThreads / 32;
  const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
  const int by_regs = regs_sm / (regs_warp * warps);
  const int by_smem = smem_sm / (dev::TmaSmem<NR>::kBytes + (int)fa.sharedSizeBytes + reserved);
  const int by_tmem = 512 / (int)dev::mma_tmem_cols<NR>();
  return std::min(std::min(by_regs, by_smem), by_tmem);
}

int scaled_mma_occupancy(int fmt, bool tma) {
  switch (fmt) {
    case 2:
      return tma ? std::min(scaled_tma_occ_one<16, false>(), scaled_tma_occ_one<32, false>())
                 : std::min(scaled_mma_occ_one<2, 16>(), scaled_mma_occ_one<2, 32>());
    case 3:
      return tma ? std::min(scaled_tma_occ_one<16, true>(), scaled_tma_occ_one<32, true>())
                 : std::min(scaled_mma_occ_one<3, 16>(), scaled_mma_occ_one<3, 32>());
    case 4: return std::min(scaled_mma_occ_one<4, 16>(), scaled_mma_occ_one<4, 32>());
    default: return 0;
  }
}

}  // namespace whff

namespace whff {

int scaled_tma_map(void* out, const void* payload, int64_t M, int64_t ld, int fmt) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return -1;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)M};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};  // bytes between rows (a multiple of 16: ld % 16 == 0)
  const cuuint32_t box[2] = {64, 128};                  // 128 bytes x 128 rows: one stage
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(static_cast<CUtensorMap*>(out),
                            fmt == 3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                            const_cast<void*>(payload), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}

}  // namespace whff
