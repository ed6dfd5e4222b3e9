// whff_noalloc.cu -- a control step that allocates nothing.
//
// Some callers cannot call cudaMalloc: a controller whose memory is fixed at
// start-up (certified real-time code that forbids allocation after
// initialisation), code running inside a process that owns a private memory
// pool, or an application that must keep allocation out of its timed loop.
// They hand in the compressed stream, x, y and the state in memory they
// already own; the only extra memory this step needs -- the FP64 split-K
// partial sums of wide matrices -- lives in the file-scope device array below.
//
// The array is a static __device__ object: every GPU that loads this library
// holds its kNoallocScratchBytes until the process exits.  All calls share it
// and it keeps the last call's contents; each call writes every partial it
// later reads, so nothing has to start at zero.  Calls whose kernels overlap
// on the GPU (two streams, or two host threads) race on the array: serialise
// them.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "gemv_kernels.cuh"
#include "whff.h"
#include "whff_blob.h"

namespace whff {
void set_error(const std::string& msg);  // whff_runtime.cu
}

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)WHFF_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) double g_noalloc_scratch[kNoallocScratchBytes / sizeof(double)];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};  // device address of the array, per device
int g_sm_count[kMaxDevices] = {};

// Once per device, with that device current: the device address of the
// array (the host-side symbol is only a stand-in, not a device address).
// The address is cached for the process; it does not survive cudaDeviceReset.
int device_setup(int dev, double** scratch, int* sms) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      whff::set_error(std::string("whff_step_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      return WHFF_ECUDA;
    }
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
      whff::set_error(std::string("whff_step_noalloc: cudaDeviceGetAttribute failed: ") + cudaGetErrorString(e));
      return WHFF_ECUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
    g_sm_count[dev] = n;
  }
  *scratch = g_scratch_addr[dev];
  *sms = g_sm_count[dev];
  return WHFF_OK;
}

template <int NW32, int R>
void launch(const uint8_t* s, int64_t M, int64_t N, int64_t BM, int64_t BN, const float* x, int64_t ldx, bool vec,
            int ksplit, int64_t chunk, double* ws, double* y, int64_t ldy, double* state, double decay,
            cudaStream_t st) {
  dim3 grid((unsigned)((BM + whff::dev::kWarpsPerCta - 1) / whff::dev::kWarpsPerCta), (unsigned)ksplit);
  whff::dev::wz1_gemv_kernel<NW32, R><<<grid, whff::dev::kWarpsPerCta * 32, 0, st>>>(
      s, M, N, BM, BN, x, ldx, vec, ksplit, chunk, ws, y, ldy, state, decay);
}

template <int NW32>
int launch_rhs(int R, const uint8_t* s, int64_t M, int64_t N, int64_t BM, int64_t BN, const float* x, int64_t ldx,
               bool vec, int ksplit, int64_t chunk, double* ws, double* y, int64_t ldy, double* state, double decay,
               cudaStream_t st) {
  switch (R) {
    case 1: launch<NW32, 1>(s, M, N, BM, BN, x, ldx, vec, ksplit, chunk, ws, y, ldy, state, decay, st); break;
    case 2: launch<NW32, 2>(s, M, N, BM, BN, x, ldx, vec, ksplit, chunk, ws, y, ldy, state, decay, st); break;
    case 4: launch<NW32, 4>(s, M, N, BM, BN, x, ldx, vec, ksplit, chunk, ws, y, ldy, state, decay, st); break;
    case 8: launch<NW32, 8>(s, M, N, BM, BN, x, ldx, vec, ksplit, chunk, ws, y, ldy, state, decay, st); break;
    default: return WHFF_EINVAL;
  }
  return WHFF_OK;
}

}  // namespace

extern "C" int whff_step_noalloc(const void* stream_dev, int rate, int64_t M, int64_t N, const float* x, int R,
                                 int64_t ldx, double* y, int64_t ldy, double* state, double decay, void* stream) {
  using whff::set_error;
  if (!stream_dev || !x || !y || !whff::shape_ok(M, N) || ldx < N || ldy < M) {
    set_error("whff_step_noalloc: null pointer, empty or oversized shape, or leading dimension too small");
    return WHFF_EINVAL;
  }
  if (rate != 8 && rate != 12 && rate != 16) {
    set_error("whff_step_noalloc: rate must be 8, 12 or 16");
    return WHFF_EINVAL;
  }
  if (R != 1 && R != 2 && R != 4 && R != 8) {
    set_error("whff_step_noalloc: R must be 1, 2, 4 or 8");
    return WHFF_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(stream_dev) % (rate == 12 ? 8 : 16) != 0) {
    set_error("whff_step_noalloc: the compressed stream must be 16-byte aligned (8 for rate 12)");
    return WHFF_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    set_error("whff_step_noalloc: no usable CUDA device");
    return WHFF_ECUDA;
  }
  double* scratch = nullptr;
  int sms = 0;
  int e = device_setup(dev, &scratch, &sms);
  if (e) return e;

  // same split rule as the handle path: enough 4-row bands x splits to fill the GPU
  const int64_t BM = (M + 3) / 4, BN = (N + 3) / 4, Mpad = 4 * BM;
  const int64_t target_warps = (int64_t)sms * 48;
  int64_t ks = (target_warps + BM - 1) / BM;
  ks = std::max<int64_t>(1, std::min<int64_t>(ks, BN / 32));
  ks = std::min<int64_t>(ks, 256);
  const int64_t chunk = (BN + ks - 1) / ks;
  const int ksplit = (int)((BN + chunk - 1) / chunk);
  if (ksplit > 1) {
    const size_t need = (size_t)ksplit * (size_t)R * (size_t)Mpad * sizeof(double);
    if (need > kNoallocScratchBytes) {
      set_error("whff_step_noalloc: split-K partials need " + std::to_string(need) +
                " bytes, more than the static scratch of " + std::to_string(kNoallocScratchBytes) + " bytes");
      return WHFF_EINVAL;
    }
  }
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const bool vec = (reinterpret_cast<uintptr_t>(x) % 16 == 0) && (ldx % 4 == 0);
  const auto* s = static_cast<const uint8_t*>(stream_dev);
  switch (rate) {
    case 8: e = launch_rhs<4>(R, s, M, N, BM, BN, x, ldx, vec, ksplit, chunk, scratch, y, ldy, state, decay, st); break;
    case 12: e = launch_rhs<6>(R, s, M, N, BM, BN, x, ldx, vec, ksplit, chunk, scratch, y, ldy, state, decay, st); break;
    default: e = launch_rhs<8>(R, s, M, N, BM, BN, x, ldx, vec, ksplit, chunk, scratch, y, ldy, state, decay, st); break;
  }
  if (e) return e;
  if (ksplit > 1) {
    whff::dev::splitk_epilogue_kernel<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(scratch, ksplit, R, Mpad, M, y,
                                                                                   ldy, state, decay);
  }
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    set_error(std::string("whff_step_noalloc: launch failed: ") + cudaGetErrorString(ce));
    return WHFF_ECUDA;
  }
  return WHFF_OK;
}
