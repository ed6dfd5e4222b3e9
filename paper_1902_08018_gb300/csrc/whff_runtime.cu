// whff_runtime.cu -- device runtime of the library: resident handles, the
// step launch (fused decode + GEMV, FP64 epilogue), decompression, errors.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gemv_kernels.cuh"
#include "wz2_dispatch.h"
#include "whff.h"
#include "whff_blob.h"

namespace whff {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

#define WHFF_CUDA_TRY(expr)                                                                     \
  do {                                                                                          \
    cudaError_t e_ = (expr);                                                                    \
    if (e_ != cudaSuccess) {                                                                    \
      set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));                            \
      return WHFF_ECUDA;                                                                        \
    }                                                                                           \
  } while (0)

}  // namespace whff

struct whff_handle {
  whff::BlobInfo info;
  int device = 0;
  int sm_count = 0;
  int max_rhs = 32;
  uint8_t* d_stream = nullptr;  // the blob's stream, 256-byte aligned (device address)
  uint8_t* h_stream = nullptr;  // host-resident handles: the pinned, mapped host copy behind d_stream
  double* d_ws = nullptr;       // split-K partials: ksplit x max_rhs x Mpad
  size_t ws_bytes = 0;
  int* d_status = nullptr;      // device-side error word
  float* d_x = nullptr;         // staging for whff_step_host
  double* d_y = nullptr;
  int64_t BM = 0, BN = 0;       // WZ1 block grid
  int64_t Mpad = 0;             // rows rounded up to 4
  int ksplit = 1;
  int64_t chunk = 0;            // J blocks (WZ1) or columns (scaled) per split
  int ctas_per_sm = 4;          // resident CTAs per SM of the persistent kernels
  bool red32 = false;           // WZ2 / scaled: fold lanes in FP32 pairs (short bands) instead of FP64
  bool groups8 = false;         // WZ2: four 8-lane groups per warp, one band each (short bands)
  int unroll = 2;               // WZ2: blocks in flight per lane (R = 1 kernel)
  bool bulk = false;            // WZ2, R = 1: blocks staged through shared memory by bulk copies
  int64_t range_ctas = 0;       // WZ2: CTAs of the range-partitioned persistent grid
  int64_t range_len = 0;        // WZ2: blocks per warp range
  int maxseg = 1;               // WZ2: most ranges sharing one band (1 = none shared)
  int ws_rhs = 8;               // right-hand sides the workspace is sized for
  double* d_ws_mma = nullptr;   // WZ2 tensor-core passes: tiles x maxseg x 32 x 128 partials
  uint8_t* d_btiles = nullptr;  // WZ2 tensor-core passes: B operand pieces per stage
  size_t btile_bytes = 0;       // their size; kColexpBytes of FP16 column exponents follow
  float* d_xt = nullptr;        // WZ2 lift: (2G)^T x of a CUDA-core pass, 4 BN floats x 8 columns
  size_t ws_mma_bytes = 0;
  int64_t mma_L = 0;            // (tile, stage) items per CTA of the persistent tensor-core grid
  int mma_ctas = 0;
  int mma_maxseg = 1;
  int mma_min_rhs = 4;          // passes of at least this many columns use tcgen05 (whff_set_crossover, whff_tune)
  int mma_occ = 0;              // resident tensor-core CTAs per SM
  size_t ws_mma_cap = 0;        // bytes of d_ws_mma
  const float* d_scales = nullptr;  // scaled formats: the tile scales after the payload
  int64_t slice_rows = 0;       // > 0: whff_step runs as consecutive slits of this many rows
  alignas(64) unsigned char tmap[128] = {};  // BF16: TMA map of the stored matrix (tensor-core passes)
  bool has_tmap = false;
  int64_t tma_row0 = 0;         // first row of a row view within the map's matrix
  const uint64_t* wz3_index = nullptr;  // fixed accuracy: the run index and the block area (device)
  const uint8_t* wz3_area = nullptr;
  int64_t wz3_RB = 0;           // runs per band
  int64_t band0 = 0;            // fixed accuracy: first band of a row view
  uint32_t wait_polls = whff::kWaitPolls;  // in-loop bounded waits of the tensor-core kernels
  cudaStream_t create_stream = nullptr;
};

namespace whff {
namespace {

constexpr int kMaxRhsKernel = 8;  // right-hand sides handled per kernel pass

constexpr size_t kColexpBytes = 256;  // 32 column exponents of an FP16 tensor-core pass, padded

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// A handle's kernels run on the device it was created on: a call made while
// another device is current would launch there against this device's memory.
int check_device(const whff_handle* h, const char* fn) {
  int d = -1;
  if (cudaGetDevice(&d) != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string(fn) + ": no current CUDA device");
    return WHFF_ECUDA;
  }
  if (d != h->device) {
    set_error(std::string(fn) + ": the current CUDA device is not the one the matrix was made resident on");
    return WHFF_EINVAL;
  }
  return WHFF_OK;
}

// WZ1: split-K so that the grid holds enough warps for the GPU: each warp owns
// one 4-row band; when bands are few (wide matrices), split the columns.
// WZ2, WZ3 and the scaled formats: split the band-major unit order into one
// contiguous range per resident warp (exact balance); bands that straddle
// ranges get segments.
// Units of a band that the persistent ranges count: runs of 32 blocks for the
// fixed-accuracy format, blocks (WZ2) or 16-byte chunks (scaled) otherwise.
int64_t band_units(const whff_handle* h) { return is_wz3(h->info.fmt) ? ceil_div(h->BN, 32) : h->BN; }

void choose_ranges(whff_handle* h) {
  if (!is_blocked(h->info.fmt) && !is_wz3(h->info.fmt)) {  // scaled: units are 16-byte chunks of a 4-row band
    h->BM = ceil_div(h->info.M, 4);
    h->BN = scaled_ld(h->info.N) / scaled_vec(h->info.fmt);
  }
  const int64_t U = band_units(h);
  const int64_t total = h->BM * U;
  const int64_t warps_cap = (int64_t)h->sm_count * h->ctas_per_sm * dev::kWarpsPerCta;
  const int64_t min_units = is_wz3(h->info.fmt) ? 2 : 64;  // >= 64 blocks (2 runs of 32) per warp
  int64_t warps = std::min<int64_t>(warps_cap, std::max<int64_t>(1, (total + min_units - 1) / min_units));
  warps = (warps + dev::kWarpsPerCta - 1) / dev::kWarpsPerCta * dev::kWarpsPerCta;
  h->range_ctas = warps / dev::kWarpsPerCta;
  h->range_len = (total + warps - 1) / warps;
  int maxseg = 1;
  for (int64_t I = 0; I < h->BM; ++I) {
    const int64_t lo = (I * U) / h->range_len, hi = ((I + 1) * U - 1) / h->range_len;
    maxseg = (int)std::max<int64_t>(maxseg, hi - lo + 1);
  }
  h->maxseg = maxseg;
  h->ksplit = 1;
  h->chunk = U;
}

void choose_split(whff_handle* h) {
  if (h->info.fmt != WHFF_FMT_ZFP) {  // WZ2, WZ3 and scaled formats: persistent warp ranges
    choose_ranges(h);
    return;
  }
  const int64_t bands = h->Mpad / 4;
  const int64_t target_warps = (int64_t)h->sm_count * 48;  // ~3/4 of 64 resident warps per SM
  int64_t ks = (target_warps + bands - 1) / bands;
  if (is_blocked(h->info.fmt)) {
    // at least 32 blocks (one per lane) per split
    ks = std::max<int64_t>(1, std::min<int64_t>(ks, h->BN / 32));
    h->ksplit = (int)std::min<int64_t>(ks, 256);
    h->chunk = (h->BN + h->ksplit - 1) / h->ksplit;
  } else {
    const int V = scaled_vec(h->info.fmt);
    const int64_t ld = scaled_ld(h->info.N);
    const int64_t unit = 32 * V;  // columns per warp iteration
    const int64_t units = (ld + unit - 1) / unit;
    ks = std::max<int64_t>(1, std::min<int64_t>(ks, units));
    h->ksplit = (int)std::min<int64_t>(ks, 256);
    h->chunk = ((units + h->ksplit - 1) / h->ksplit) * unit;
    h->ksplit = (int)((ld + h->chunk - 1) / h->chunk);
  }
}

// Persistent tensor-core grid: `ctas` CTAs at most over the items (tile of
// 128 rows = 32 bands, stage of 64 columns = 16 blocks), equal contiguous ranges.
void plan_mma(whff_handle* h, int64_t ctas) {
  const int64_t tiles = ceil_div(h->info.M, 128), stages = ceil_div(h->info.N, 64), items = tiles * stages;
  h->mma_L = ceil_div(items, std::max<int64_t>(1, ctas));
  h->mma_ctas = (int)ceil_div(items, h->mma_L);
  h->mma_maxseg = 1;
  for (int64_t tl = 0; tl < tiles; ++tl)
    h->mma_maxseg = std::max<int>(h->mma_maxseg,
                                  (int)(((tl + 1) * stages - 1) / h->mma_L - (tl * stages) / h->mma_L + 1));
}

size_t mma_ws_need(const whff_handle* h, int R) {
  return (size_t)ceil_div(h->info.M, 128) * (size_t)h->mma_maxseg * (size_t)R * 128 * 8;
}

// The lift's transformed x: 4 BN floats per right-hand side of a pass (up to 8).
size_t xt_bytes(const whff_handle* h) {
  return (size_t)4 * h->BN * std::min(h->max_rhs, kMaxRhsKernel) * sizeof(float);
}

// Workspace bytes a CUDA-core pass of the plan needs.
size_t ws_need(const whff_handle* h) {
  if (h->info.fmt == WHFF_FMT_ZFP)
    return h->ksplit > 1 ? (size_t)h->ksplit * (size_t)h->ws_rhs * (size_t)h->Mpad * 8 : 0;
  return h->maxseg > 1 ? (size_t)h->BM * (size_t)h->maxseg * (size_t)h->ws_rhs * 4 * 8 : 0;
}

template <int NW32>
int launch_wz1_nw(const whff_handle* h, const float* x, int R, int64_t ldx, bool vec, double* y, int64_t ldy,
                  double* state, double decay, cudaStream_t st) {
  dim3 grid((unsigned)((h->BM + dev::kWarpsPerCta - 1) / dev::kWarpsPerCta), (unsigned)h->ksplit);
  dim3 block(dev::kWarpsPerCta * 32);
  const uint8_t* s = h->d_stream;
  const auto& b = h->info;
#define WZ1_CASE(RR)                                                                                      \
  case RR:                                                                                                \
    dev::wz1_gemv_kernel<NW32, RR><<<grid, block, 0, st>>>(s, b.M, b.N, h->BM, h->BN, x, ldx, vec,      \
                                                           h->ksplit, h->chunk, h->d_ws, y, ldy, state,   \
                                                           decay);                                        \
    break;
  switch (R) {
    WZ1_CASE(1)
    WZ1_CASE(2)
    WZ1_CASE(4)
    WZ1_CASE(8)
    default:
      return WHFF_EINVAL;
  }
#undef WZ1_CASE
  return WHFF_OK;
}

int launch_wz1(const whff_handle* h, const float* x, int R, int64_t ldx, bool vec, double* y, int64_t ldy,
               double* state, double decay, cudaStream_t st) {
  switch (h->info.rate) {
    case 8:
      return launch_wz1_nw<4>(h, x, R, ldx, vec, y, ldy, state, decay, st);
    case 12:
      return launch_wz1_nw<6>(h, x, R, ldx, vec, y, ldy, state, decay, st);
    case 16:
      return launch_wz1_nw<8>(h, x, R, ldx, vec, y, ldy, state, decay, st);
    default:
      set_error("whff_step: the fused kernel is built for rates 8, 12 and 16");
      return WHFF_EINVAL;
  }
}

int launch_wz2(const whff_handle* h, const float* x, int R, int64_t ldx, bool vec, double* y, int64_t ldy,
               double* state, double decay, cudaStream_t st) {
  // the staged kernel needs a padded device stream aligned for its bulk copies
  const bool staged = h->bulk && R == 1 && !h->groups8 && !h->h_stream &&
                      reinterpret_cast<uintptr_t>(h->d_stream) % (h->info.rate % 8 == 0 ? 16 : 8) == 0;
  Wz2Step a{h->d_stream, h->info.M, h->info.N, h->BM, h->BN, x, ldx, vec, h->range_len, h->maxseg, h->d_ws,
            y, ldy, state, decay, h->range_ctas, R == 1 ? h->unroll : 2, h->info.fmt == WHFF_FMT_FIXED_LIFT, R,
            h->red32, h->groups8, h->d_xt, staged, h->d_status};
  int e;
  switch (h->info.rate) {
    case 8: e = wz2_launch<8>(a, st); break;
    case 12: e = wz2_launch<12>(a, st); break;
    case 16: e = wz2_launch<16>(a, st); break;
    case 20: e = wz2_launch<20>(a, st); break;
    case 24: e = wz2_launch<24>(a, st); break;
    default: e = -1;
  }
  if (e) {
    set_error("whff_step: WZ2 rates are 8..24 in steps of 4 and R 1, 2, 4 or 8 per pass");
    return WHFF_EINVAL;
  }
  return WHFF_OK;
}

int wz2_occ(int rate, bool lift, int unroll) {
  switch (rate) {
    case 8: return wz2_occupancy<8>(lift, unroll);
    case 12: return wz2_occupancy<12>(lift, unroll);
    case 16: return wz2_occupancy<16>(lift, unroll);
    case 20: return wz2_occupancy<20>(lift, unroll);
    case 24: return wz2_occupancy<24>(lift, unroll);
    default: return 0;
  }
}

int wz2_stream_occ(int rate, bool lift) {
  switch (rate) {
    case 8: return wz2_stream_occupancy<8>(lift);
    case 12: return wz2_stream_occupancy<12>(lift);
    case 16: return wz2_stream_occupancy<16>(lift);
    case 20: return wz2_stream_occupancy<20>(lift);
    case 24: return wz2_stream_occupancy<24>(lift);
    default: return 0;
  }
}

int launch_scaled(const whff_handle* h, const float* x, int R, int64_t ldx, bool vec, double* y, int64_t ldy,
                  double* state, double decay, cudaStream_t st) {
  const auto& b = h->info;
  const int64_t ld = scaled_ld(b.N);
  ScaledStep a{b.fmt, h->d_stream, h->d_scales, b.M, b.N, ld, ceil_div(b.N, kScaleTile), x, ldx, vec,
               h->range_len, h->maxseg, h->d_ws, y, ldy, state, decay, h->range_ctas, R, h->red32, h->groups8};
  if (scaled_launch(a, st)) {
    set_error("whff_step: scaled formats take R 1, 2, 4 or 8 per pass");
    return WHFF_EINVAL;
  }
  return WHFF_OK;
}

int launch_pass(const whff_handle* h, const float* x, int R, int64_t ldx, double* y, int64_t ldy, double* state,
                double decay, cudaStream_t st) {
  const bool vec = (reinterpret_cast<uintptr_t>(x) % 16 == 0) && (ldx % 4 == 0);
  int e;
  switch (h->info.fmt) {
    case WHFF_FMT_ZFP:
      e = launch_wz1(h, x, R, ldx, vec, y, ldy, state, decay, st);
      break;
    case WHFF_FMT_FIXED_LIFT:
    case WHFF_FMT_FIXED_BFP:
      e = launch_wz2(h, x, R, ldx, vec, y, ldy, state, decay, st);
      break;
    case WHFF_FMT_BF16:
    case WHFF_FMT_FP16:
    case WHFF_FMT_FP8E4M3:
    case WHFF_FMT_FP32:
      e = launch_scaled(h, x, R, ldx, vec, y, ldy, state, decay, st);
      break;
    case WHFF_FMT_FIXED_ACC: {
      Wz3Step a{h->wz3_index, h->wz3_area, h->band0, h->info.M, h->info.N, h->BM, h->BN, h->wz3_RB, x, ldx,
                h->d_xt, R, h->range_len, h->maxseg, h->range_ctas, h->d_ws, y, ldy, state, decay};
      e = wz3_launch(a, st) ? WHFF_EINVAL : WHFF_OK;
      if (e) set_error("whff_step: fixed-accuracy passes take 1 or 8 right-hand sides");
      break;
    }
    default:
      e = WHFF_EINVAL;
  }
  if (e) return e;
  if (h->ksplit > 1 && h->info.fmt == WHFF_FMT_ZFP) {
    const int threads = 256;
    dev::splitk_epilogue_kernel<<<(unsigned)((h->info.M + threads - 1) / threads), threads, 0, st>>>(
        h->d_ws, h->ksplit, R, h->Mpad, h->info.M, y, ldy, state, decay);
  }
  WHFF_CUDA_TRY(cudaGetLastError());
  return WHFF_OK;
}

}  // namespace
}  // namespace whff

using namespace whff;

namespace whff {
namespace dev {
// The achievable-read probe: each thread keeps four 16-byte streaming loads in
// flight and folds them into one XOR word; a warp folds its lanes, lane 0 adds
// its word to the result with one atomic.
static __global__ void __launch_bounds__(256) read_probe_kernel(const uint4* __restrict__ p, int64_t n16,
                                                                uint32_t* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  for (; i + 3 * stride < n16; i += 4 * stride) {
    const uint4 a = __ldcs(p + i), b = __ldcs(p + i + stride), c = __ldcs(p + i + 2 * stride),
                d = __ldcs(p + i + 3 * stride);
    acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
  }
  for (; i < n16; i += stride) {
    const uint4 a = __ldcs(p + i);
    acc ^= a.x ^ a.y ^ a.z ^ a.w;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) acc ^= __shfl_xor_sync(0xFFFFFFFFu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicXor(out, acc);
}
}  // namespace dev
}  // namespace whff

extern "C" int whff_read_probe(const void* buf, size_t bytes, uint32_t* d_xor, void* stream) {
  if (!buf || !d_xor || bytes % 16 || reinterpret_cast<uintptr_t>(buf) % 16) {
    set_error("whff_read_probe: null pointer, or buffer not 16-byte aligned / sized");
    return WHFF_EINVAL;
  }
  int dev = 0, sms = 0;
  WHFF_CUDA_TRY(cudaGetDevice(&dev));
  WHFF_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t n16 = (int64_t)(bytes / 16);
  if (n16 == 0) return WHFF_OK;
  const int64_t ctas = std::min<int64_t>((int64_t)sms * 8, (n16 + 255) / 256);  // 8 CTAs of 256 threads per SM
  dev::read_probe_kernel<<<(unsigned)ctas, 256, 0, as_stream(stream)>>>(static_cast<const uint4*>(buf), n16, d_xor);
  WHFF_CUDA_TRY(cudaGetLastError());
  return WHFF_OK;
}

extern "C" const char* whff_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* whff_version(void) { return "whff 0.1 sm_103a"; }

extern "C" int whff_create(const void* blob, size_t len, int max_rhs, void* stream, whff_handle** out) {
  return whff_create_ex(blob, len, max_rhs, 0u, stream, out);
}

namespace whff {
namespace {
// The runs of a fixed-accuracy stream (host copy) lie back to back in
// band-major order from the start of the block area, each of width at most 31
// (a run of width 0 stores 8 zero bytes per block): the kernels then read only
// the stream.
int wz3_check_index(const uint8_t* stream, uint64_t sbytes, int64_t BM, int64_t BN) {
  const int64_t RB = ceil_div(BN, 32);
  const uint64_t head = 8 + 8 * (uint64_t)(BM * RB);
  if (sbytes < head) return WHFF_EFORMAT;
  const uint64_t area = sbytes - head;
  uint64_t next = 0;  // where the next run must start
  for (int64_t I = 0; I < BM; ++I)
    for (int64_t r = 0; r < RB; ++r) {
      uint64_t e;
      std::memcpy(&e, stream + 8 + 8 * (uint64_t)(I * RB + r), 8);
      const int W = (int)(e >> 56);
      const uint64_t off = e & 0x00FFFFFFFFFFFFFFull;
      const uint64_t nb = (uint64_t)(std::min<int64_t>(BN, 32 * r + 32) - 32 * r);
      const uint64_t bytes = nb * (uint64_t)(8 * ((13 + 16 * W + 63) / 64));
      if (W > 31 || off != next || bytes > area - off) return WHFF_EFORMAT;
      next = off + bytes;
    }
  return WHFF_OK;
}

// A handle for the matrix `info` describes.  src (host memory, info.stream_bytes)
// is uploaded on `stream`; with src == nullptr the device stream is allocated and
// left for the caller to fill (the slots of a field pipeline).
int create_impl(const BlobInfo& info, const uint8_t* src, int max_rhs, unsigned flags, void* stream,
                whff_handle** out);
}  // namespace
}  // namespace whff

extern "C" int whff_create_ex(const void* blob, size_t len, int max_rhs, unsigned flags, void* stream,
                              whff_handle** out) {
  if (!out || (flags & ~(unsigned)WHFF_CREATE_HOST_RESIDENT)) {
    set_error("whff_create: null output handle or unknown flag");
    return WHFF_EINVAL;
  }
  *out = nullptr;
  BlobInfo info;
  int e = read_header((const uint8_t*)blob, len, &info, true);
  if (e) {
    set_error("whff_create: blob header, size or CRC check failed");
    return e;
  }
  return create_impl(info, (const uint8_t*)blob + kHeaderBytes, max_rhs, flags, stream, out);
}

namespace whff {
namespace {
int create_impl(const BlobInfo& info, const uint8_t* src, int max_rhs, unsigned flags, void* stream,
                whff_handle** out) {
  if (max_rhs <= 0) max_rhs = 32;
  if (max_rhs > 1024) {
    set_error("whff_create: max_rhs > 1024");
    return WHFF_EINVAL;
  }
  auto* h = new whff_handle;
  h->info = info;
  h->max_rhs = max_rhs;
  h->create_stream = as_stream(stream);
  auto fail = [&](int code) {
    whff_destroy(h);
    return code;
  };
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    set_error("whff_create: no usable CUDA device");
    return fail(WHFF_ECUDA);
  }
  h->Mpad = 4 * ceil_div(info.M, 4);
  if (info.fmt == WHFF_FMT_FIXED_LIFT || info.fmt == WHFF_FMT_FIXED_BFP) {
    const int occ = wz2_occ(info.rate, info.fmt == WHFF_FMT_FIXED_LIFT, h->unroll);
    h->ctas_per_sm = occ > 0 ? occ : 4;
  } else if (is_wz3(info.fmt)) {
    const int occ = wz3_occupancy(1);
    h->ctas_per_sm = occ > 0 ? occ : 4;
  } else if (!is_blocked(info.fmt)) {  // the kernel the fold default below picks
    const int occ = scaled_occupancy(info.fmt, scaled_ld(info.N) / scaled_vec(info.fmt) < 256);
    h->ctas_per_sm = occ > 0 ? occ : 4;
  }
  if (is_blocked(info.fmt) || is_wz3(info.fmt)) {
    h->BM = ceil_div(info.M, 4);
    h->BN = ceil_div(info.N, 4);
  }
  if (is_wz3(info.fmt)) {  // the run index must stay inside the stream: checked once, here
    const int e = src ? wz3_check_index(src, info.stream_bytes, h->BM, h->BN) : WHFF_EFORMAT;
    if (e) {
      set_error("whff_create: fixed-accuracy run index out of range (width above 31 or run past the stream)");
      return fail(e);
    }
  }
  choose_split(h);
  // short bands (tall matrices) fold their lanes in FP32 pairs, long ones in
  // FP64; very short ones give each band a group of 8 lanes.  BN counts a
  // band's lane work units: 4-column blocks (WZ2) or 16-byte chunks (scaled).
  h->red32 = info.fmt != WHFF_FMT_ZFP && h->BN < 4096;
  h->groups8 = info.fmt != WHFF_FMT_ZFP && h->BN < 256;
  const cudaStream_t st = as_stream(stream);
  if (flags & WHFF_CREATE_HOST_RESIDENT) {  // pinned host memory, read by the kernels over the CPU link
    void* dp = nullptr;
    if (cudaHostAlloc(reinterpret_cast<void**>(&h->h_stream), info.stream_bytes + kStreamPad, cudaHostAllocMapped) !=
            cudaSuccess ||
        cudaHostGetDevicePointer(&dp, h->h_stream, 0) != cudaSuccess) {
      cudaGetLastError();
      set_error("whff_create: pinned mapped host allocation of the compressed stream failed");
      return fail(WHFF_ENOMEM);
    }
    h->d_stream = static_cast<uint8_t*>(dp);
    if (src) std::memcpy(h->h_stream, src, info.stream_bytes);
  } else if (cudaMalloc(&h->d_stream, info.stream_bytes + kStreamPad) != cudaSuccess) {
    cudaGetLastError();
    set_error("whff_create: cudaMalloc of the compressed stream failed");
    return fail(WHFF_ENOMEM);
  }
  h->ws_bytes = h->ksplit > 1 ? (size_t)h->ksplit * (size_t)std::min(max_rhs, kMaxRhsKernel) * (size_t)h->Mpad * 8 : 0;
  if (h->maxseg > 1)
    h->ws_bytes = (size_t)h->BM * (size_t)h->maxseg * (size_t)std::min(max_rhs, kMaxRhsKernel) * 4 * 8;
  h->ws_rhs = std::min(max_rhs, kMaxRhsKernel);
  const bool wz2 = info.fmt == WHFF_FMT_FIXED_LIFT || info.fmt == WHFF_FMT_FIXED_BFP;
  const bool scaled16 = info.fmt == WHFF_FMT_BF16 || info.fmt == WHFF_FMT_FP16 || info.fmt == WHFF_FMT_FP8E4M3;
  if ((wz2 || scaled16) && max_rhs >= 2) {
    // tensor-core passes: a persistent grid (all resident CTAs) over the items
    // (tile of 128 rows, stage of 64 columns), equal contiguous ranges per CTA
    const bool lift = info.fmt == WHFF_FMT_FIXED_LIFT;
    // BF16 in device memory: the TMA-fed kernel (its map is encoded below)
    const bool tma = (info.fmt == WHFF_FMT_BF16 || info.fmt == WHFF_FMT_FP16) && !(flags & WHFF_CREATE_HOST_RESIDENT);
    const int occ = wz2 ? std::min(mma_occupancy(info.rate, lift, 16), mma_occupancy(info.rate, lift, 32))
                        : scaled_mma_occupancy(info.fmt, tma);
    if (occ < 1) {
      set_error("whff_create: the tensor-core kernel cannot be resident");
      return fail(WHFF_ECUDA);
    }
    h->mma_occ = occ;
    plan_mma(h, (int64_t)h->sm_count * occ);
    h->ws_mma_cap = mma_ws_need(h, std::min(max_rhs, 32));
    h->ws_mma_bytes = h->ws_mma_cap;
    const size_t btile_bytes = (size_t)ceil_div(info.N, 64) * 3 * 4 * 32 * 16 * 2;  // stages x pieces x ksteps x NR<=32 tile
    h->btile_bytes = btile_bytes;
    h->ws_mma_bytes += btile_bytes + kColexpBytes;  // FP16 passes: per-column exponents of x after the tiles
    if (cudaMalloc(&h->d_ws_mma, h->ws_mma_bytes - btile_bytes - kColexpBytes) != cudaSuccess ||
        cudaMalloc(&h->d_btiles, btile_bytes + kColexpBytes) != cudaSuccess) {
      cudaGetLastError();
      set_error("whff_create: cudaMalloc of the tensor-core workspace failed");
      return fail(WHFF_ENOMEM);
    }
  }
  if (((info.fmt == WHFF_FMT_FIXED_LIFT || is_wz3(info.fmt)) && cudaMalloc(&h->d_xt, xt_bytes(h)) != cudaSuccess) ||
      (h->ws_bytes && cudaMalloc(&h->d_ws, h->ws_bytes) != cudaSuccess) ||
      cudaMalloc(&h->d_status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->d_x, (size_t)info.N * (size_t)max_rhs * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&h->d_y, (size_t)info.M * (size_t)max_rhs * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    set_error("whff_create: cudaMalloc of the workspace failed");
    return fail(WHFF_ENOMEM);
  }
  if (cudaMemsetAsync(h->d_status, 0, sizeof(int), st) != cudaSuccess ||
      (!h->h_stream && src &&
       cudaMemcpyAsync(h->d_stream, src, info.stream_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    set_error(std::string("whff_create: upload failed: ") + cudaGetErrorString(cudaGetLastError()));
    return fail(WHFF_ECUDA);
  }
  if (is_wz3(info.fmt)) {
    h->wz3_RB = ceil_div(h->BN, 32);
    h->wz3_index = reinterpret_cast<const uint64_t*>(h->d_stream + 8);
    h->wz3_area = h->d_stream + 8 + 8 * (uint64_t)(h->BM * h->wz3_RB);
  } else if (!is_blocked(info.fmt)) {
    h->d_scales = reinterpret_cast<const float*>(h->d_stream + (uint64_t)info.M * (uint64_t)scaled_ld(info.N) *
                                                                   (uint64_t)elem_bytes(info.fmt));
  }
  // BF16 and FP16 tensor-core passes take their A tiles by TMA from device
  // memory (if the map cannot be encoded the register-fed kernel runs instead:
  // the same results for BF16, the same accuracy bar for FP16)
  if ((info.fmt == WHFF_FMT_BF16 || info.fmt == WHFF_FMT_FP16) && h->d_ws_mma && !h->h_stream)
    h->has_tmap = scaled_tma_map(h->tmap, h->d_stream, info.M, scaled_ld(info.N), info.fmt) == 0;
  *out = h;
  return WHFF_OK;
}
}  // namespace
}  // namespace whff

extern "C" int whff_info(const whff_handle* h, int* fmt, int* rate, int64_t* M, int64_t* N, size_t* device_bytes) {
  if (!h) {
    set_error("whff_info: null handle");
    return WHFF_EINVAL;
  }
  if (fmt) *fmt = h->info.fmt;
  if (rate) *rate = h->info.rate;
  if (M) *M = h->info.M;
  if (N) *N = h->info.N;
  if (device_bytes)
    *device_bytes = (h->h_stream ? 0 : h->info.stream_bytes) + h->ws_bytes + h->ws_mma_bytes + sizeof(int) +
                    (size_t)h->info.N * h->max_rhs * 4 + (size_t)h->info.M * h->max_rhs * 8 +
                    (h->d_xt ? xt_bytes(h) : 0);
  return WHFF_OK;
}

namespace whff {
namespace {
int launch_mma(const whff_handle* h, const float* x, int R, int64_t ldx, double* y, int64_t ldy, double* state,
               double decay, cudaStream_t st) {
  int e;
  if (is_blocked(h->info.fmt)) {
    MmaStep a{h->info.rate, h->info.fmt == WHFF_FMT_FIXED_LIFT, h->d_stream, h->info.M, h->info.N, h->BM, h->BN,
              x, ldx, R, h->mma_L, h->mma_ctas, h->mma_maxseg, h->d_ws_mma, h->d_btiles, y, ldy, state, decay,
              h->d_status, h->wait_polls};
    e = mma_launch(a, st);
  } else {
    ScaledMmaStep a{h->info.fmt, h->d_stream, h->d_scales, h->info.M, h->info.N, scaled_ld(h->info.N),
                    ceil_div(h->info.N, kScaleTile), x, ldx, R, h->mma_L, h->mma_ctas, h->mma_maxseg,
                    h->d_ws_mma, h->d_btiles, y, ldy, state, decay, h->d_status, h->wait_polls,
                    h->has_tmap ? h->tmap : nullptr, h->tma_row0,
                    reinterpret_cast<int*>(h->d_btiles + h->btile_bytes)};
    e = scaled_mma_launch(a, st);
  }
  if (e) {
    set_error("whff_step: tensor-core pass failed to launch");
    return WHFF_ECUDA;
  }
  WHFF_CUDA_TRY(cudaGetLastError());
  return WHFF_OK;
}
}  // namespace
}  // namespace whff

extern "C" int whff_plan(const whff_handle* h, int* ksplit, int* launches) {
  if (!h) {
    set_error("whff_plan: null handle");
    return WHFF_EINVAL;
  }
  if (ksplit) *ksplit = h->ksplit;
  if (launches)
    *launches = ((h->ksplit > 1 || h->maxseg > 1) ? 2 : 1) +
                (h->info.fmt == WHFF_FMT_FIXED_LIFT || is_wz3(h->info.fmt) ? 1 : 0);
  return WHFF_OK;
}

namespace whff {
namespace {
// The passes of one step on a handle or on a row view of it: up to 32
// columns per tensor-core pass, else 8, 4, 2, 1 per CUDA-core pass; the state
// update is applied pass by pass, which keeps the column order r = 0..R-1.
int step_passes(const whff_handle* h, const float* x, int R, int64_t ldx, double* y, int64_t ldy, double* state,
                double decay, cudaStream_t st) {
  int r0 = 0;
  while (r0 < R) {
    const int left = R - r0;
    int e;
    if (h->d_ws_mma && left >= h->mma_min_rhs) {  // dense contraction: tcgen05, up to 32 columns per pass
      const int pass = left < 32 ? left : 32;
      e = launch_mma(h, x + (int64_t)r0 * ldx, pass, ldx, y + (int64_t)r0 * ldy, ldy, state, decay, st);
      r0 += pass;
    } else {
      const int pass = left >= 8 ? 8 : is_wz3(h->info.fmt) ? 1 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
      e = launch_pass(h, x + (int64_t)r0 * ldx, pass, ldx, y + (int64_t)r0 * ldy, ldy, state, decay, st);
      r0 += pass;
    }
    if (e) return e;
  }
  return WHFF_OK;
}
}  // namespace
}  // namespace whff

namespace whff {
namespace {
// Rows [row0, row0 + nrows) of the matrix (row0 aligned to the format's band or
// scale tile): a view with the handle's buffers and its own launch plan,
// shrunk until its partials fit the handle's workspaces.
int step_view(const whff_handle* h, int64_t row0, int64_t nrows, const float* x, int R, int64_t ldx, double* y,
              int64_t ldy, double* state, double decay, cudaStream_t st) {
  const int fmt = h->info.fmt;
  whff_handle v = *h;
  v.info.M = nrows;
  v.Mpad = ceil_div(nrows, 4) * 4;
  if (is_blocked(fmt)) {
    v.BM = ceil_div(nrows, 4);
    v.d_stream = h->d_stream + (uint64_t)(row0 / 4) * (uint64_t)h->BN * (uint64_t)(2 * h->info.rate);
  } else if (is_wz3(fmt)) {  // the same index and blocks, from band row0 / 4 on
    v.BM = ceil_div(nrows, 4);
    v.band0 = h->band0 + row0 / 4;
  } else {
    v.d_stream = h->d_stream + (uint64_t)row0 * (uint64_t)scaled_ld(h->info.N) * (uint64_t)elem_bytes(fmt);
    v.d_scales = h->d_scales + (row0 / kScaleTile) * ceil_div(h->info.N, kScaleTile);
    v.tma_row0 = h->tma_row0 + row0;
  }
  choose_split(&v);
  for (int c = v.ctas_per_sm; ws_need(&v) > h->ws_bytes;) {  // fewer warps: longer ranges, fewer segments
    if (fmt == WHFF_FMT_ZFP) {
      v.ksplit = (int)std::max<size_t>(1, h->ws_bytes / ((size_t)v.ws_rhs * (size_t)v.Mpad * 8));
      v.chunk = ceil_div(v.BN, v.ksplit);
      v.ksplit = (int)ceil_div(v.BN, v.chunk);
      if (v.ksplit > 1 && ws_need(&v) > h->ws_bytes) v.ksplit = 1, v.chunk = v.BN;
      break;
    }
    if (c == 1) {  // ranges of whole bands: no band is shared, so no partials at all
      const int64_t U = band_units(&v);
      v.range_len = ceil_div(v.range_len, U) * U;
      v.range_ctas = ceil_div(ceil_div(v.BM * U, v.range_len), dev::kWarpsPerCta);
      v.maxseg = 1;
      break;
    }
    v.ctas_per_sm = --c;
    choose_ranges(&v);
  }
  if (h->d_ws_mma) {
    int64_t ctas = (int64_t)h->sm_count * h->mma_occ;
    for (plan_mma(&v, ctas); mma_ws_need(&v, std::min(R, 32)) > h->ws_mma_cap && ctas > 1;
         plan_mma(&v, ctas = ctas * 3 / 4)) {
    }
    if (mma_ws_need(&v, std::min(R, 32)) > h->ws_mma_cap) v.mma_min_rhs = 33;  // CUDA cores only
  }
  return step_passes(&v, x, R, ldx, y, ldy, state, decay, st);
}
}  // namespace
}  // namespace whff

extern "C" int whff_step(whff_handle* h, const float* x, int R, int64_t ldx, double* y, int64_t ldy, double* state,
                         double decay, void* stream) {
  if (!h || !x || !y || R <= 0 || R > h->max_rhs || ldx < h->info.N || ldy < h->info.M) {
    set_error("whff_step: null pointer, R out of [1, max_rhs], or leading dimension too small");
    return WHFF_EINVAL;
  }
  if (const int de = check_device(h, "whff_step")) return de;
  const cudaStream_t st = as_stream(stream);
  const int64_t M = h->info.M, slice = h->slice_rows;
  if (slice <= 0 || slice >= M) return step_passes(h, x, R, ldx, y, ldy, state, decay, st);
  for (int64_t r0 = 0; r0 < M; r0 += slice) {  // time slices: one launch sequence per slit
    const int e = step_view(h, r0, std::min(slice, M - r0), x, R, ldx, y + r0, ldy, state ? state + r0 : nullptr,
                            decay, st);
    if (e) return e;
  }
  return WHFF_OK;
}

// A slit (Sec. 2.1, divide and conquer: C_slit is a block of rows of the
// resident C_field): rows [row0, row0 + nrows) of the matrix, which are one
// contiguous byte range of its stream, so nothing is copied.
extern "C" int whff_step_rows(whff_handle* h, int64_t row0, int64_t nrows, const float* x, int R, int64_t ldx,
                              double* y, int64_t ldy, double* state, double decay, void* stream) {
  if (!h || !x || !y || R <= 0 || R > h->max_rhs || ldx < h->info.N || row0 < 0 || nrows <= 0 ||
      nrows > h->info.M - row0 || ldy < nrows) {
    set_error("whff_step_rows: null pointer, R out of [1, max_rhs], rows outside the matrix, or ld too small");
    return WHFF_EINVAL;
  }
  if (row0 % row_align(h->info.fmt)) {
    set_error("whff_step_rows: row0 must be a multiple of 4 (block formats) or 128 (scaled formats)");
    return WHFF_EINVAL;
  }
  if (const int de = check_device(h, "whff_step_rows")) return de;
  return step_view(h, row0, nrows, x, R, ldx, y, ldy, state, decay, as_stream(stream));
}

extern "C" int whff_get_slice_rows(const whff_handle* h, int64_t* rows) {
  if (!h || !rows) {
    set_error("whff_get_slice_rows: null argument");
    return WHFF_EINVAL;
  }
  *rows = h->slice_rows;
  return WHFF_OK;
}

extern "C" int whff_set_slice_rows(whff_handle* h, int64_t rows) {
  if (!h || rows < 0 || rows % row_align(h->info.fmt)) {
    set_error("whff_set_slice_rows: rows >= 0, a multiple of 4 (block formats) or 128 (scaled formats)");
    return WHFF_EINVAL;
  }
  h->slice_rows = rows;
  return WHFF_OK;
}

extern "C" int whff_step_host(whff_handle* h, const float* x_host, int R, int64_t ldx, double* y_host, int64_t ldy,
                              double* state, double decay, void* stream) {
  if (!h || !x_host || !y_host || R <= 0 || R > h->max_rhs || ldx < h->info.N || ldy < h->info.M) {
    set_error("whff_step_host: null pointer, R out of [1, max_rhs], or leading dimension too small");
    return WHFF_EINVAL;
  }
  if (const int de = check_device(h, "whff_step_host")) return de;
  const cudaStream_t st = as_stream(stream);
  const int64_t N = h->info.N, M = h->info.M;
  WHFF_CUDA_TRY(cudaMemcpy2DAsync(h->d_x, N * sizeof(float), x_host, ldx * sizeof(float), N * sizeof(float), R,
                                  cudaMemcpyHostToDevice, st));
  int e = whff_step(h, h->d_x, R, N, h->d_y, M, state, decay, stream);
  if (e) return e;
  WHFF_CUDA_TRY(cudaMemcpy2DAsync(y_host, ldy * sizeof(double), h->d_y, M * sizeof(double), M * sizeof(double), R,
                                  cudaMemcpyDeviceToHost, st));
  return WHFF_OK;
}

// ------------------------------------------------------------- CUDA graphs
struct whff_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  float* d_x = nullptr;   // graph-owned staging (host variant)
  double* d_y = nullptr;
  // slit graphs (whff_graph_create_rows): what a re-capture for another slit needs
  whff_handle* h = nullptr;
  int64_t row0 = -1, nrows = 0;
  const float* x = nullptr;
  int R = 0;
  int64_t ldx = 0, ldy = 0;
  double* y = nullptr;  // field-sized: the slit writes rows [row0, row0 + nrows)
  double* state = nullptr;
  double decay = 0.0;
  cudaStream_t cap = nullptr;  // private capture stream for the updates
};

namespace {

// Capture fn() on `stream` (or a temporary stream when it is the legacy one).
template <class F>
int capture_graph(void* stream, whff_graph* g, F&& fn) {
  cudaStream_t st = as_stream(stream);
  cudaStream_t tmp = nullptr;
  if (!st) {
    if (cudaStreamCreateWithFlags(&tmp, cudaStreamNonBlocking) != cudaSuccess) {
      set_error("whff_graph_create: cannot create a capture stream");
      return WHFF_ECUDA;
    }
    st = tmp;
  }
  int e = WHFF_OK;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    set_error(std::string("whff_graph_create: begin capture: ") + cudaGetErrorString(cudaGetLastError()));
    e = WHFF_ECUDA;
  } else {
    e = fn(st);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (e == WHFF_OK && ce != cudaSuccess) {
      set_error(std::string("whff_graph_create: end capture: ") + cudaGetErrorString(ce));
      e = WHFF_ECUDA;
    }
    g->graph = graph;
    if (e == WHFF_OK && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
      set_error(std::string("whff_graph_create: instantiate: ") + cudaGetErrorString(cudaGetLastError()));
      e = WHFF_ECUDA;
    }
  }
  if (tmp) cudaStreamDestroy(tmp);
  return e;
}

}  // namespace

extern "C" void whff_graph_destroy(whff_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->cap) cudaStreamDestroy(g->cap);
  cudaFree(g->d_x);
  cudaFree(g->d_y);
  cudaGetLastError();
  delete g;
}

extern "C" int whff_graph_create(whff_handle* h, const float* x, int R, int64_t ldx, double* y, int64_t ldy,
                                 double* state, double decay, void* stream, whff_graph** out) {
  if (!out || !h) {
    set_error("whff_graph_create: null argument");
    return WHFF_EINVAL;
  }
  *out = nullptr;
  auto* g = new whff_graph;
  int e = capture_graph(stream, g, [&](cudaStream_t st) {
    return whff_step(h, x, R, ldx, y, ldy, state, decay, reinterpret_cast<void*>(st));
  });
  if (e) {
    whff_graph_destroy(g);
    return e;
  }
  *out = g;
  return WHFF_OK;
}

extern "C" int whff_graph_create_host(whff_handle* h, const float* x_host, int R, int64_t ldx, double* y_host,
                                      int64_t ldy, double* state, double decay, void* stream, whff_graph** out) {
  if (!out || !h || !x_host || !y_host || R <= 0 || R > h->max_rhs || ldx < h->info.N || ldy < h->info.M) {
    set_error("whff_graph_create_host: invalid argument");
    return WHFF_EINVAL;
  }
  if (const int de = check_device(h, "whff_graph_create_host")) return de;
  *out = nullptr;
  auto* g = new whff_graph;
  const int64_t N = h->info.N, M = h->info.M;
  if (cudaMalloc(&g->d_x, (size_t)N * R * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&g->d_y, (size_t)M * R * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    whff_graph_destroy(g);
    set_error("whff_graph_create_host: cudaMalloc failed");
    return WHFF_ENOMEM;
  }
  int e = capture_graph(stream, g, [&](cudaStream_t st) {
    if (cudaMemcpy2DAsync(g->d_x, N * sizeof(float), x_host, ldx * sizeof(float), N * sizeof(float), R,
                          cudaMemcpyHostToDevice, st) != cudaSuccess) {
      set_error("whff_graph_create_host: H2D copy node");
      return WHFF_ECUDA;
    }
    int e2 = whff_step(h, g->d_x, R, N, g->d_y, M, state, decay, reinterpret_cast<void*>(st));
    if (e2) return e2;
    if (cudaMemcpy2DAsync(y_host, ldy * sizeof(double), g->d_y, M * sizeof(double), M * sizeof(double), R,
                          cudaMemcpyDeviceToHost, st) != cudaSuccess) {
      set_error("whff_graph_create_host: D2H copy node");
      return WHFF_ECUDA;
    }
    return WHFF_OK;
  });
  if (e) {
    whff_graph_destroy(g);
    return e;
  }
  *out = g;
  return WHFF_OK;
}

namespace {
int check_slit(const whff_handle* h, int64_t row0, int64_t nrows, const char* who) {
  if (row0 < 0 || nrows <= 0 || nrows > h->info.M - row0 || row0 % row_align(h->info.fmt)) {
    set_error(std::string(who) + ": rows outside the matrix, or row0 not a multiple of 4 (block formats) / 128 "
                                 "(scaled formats)");
    return WHFF_EINVAL;
  }
  return WHFF_OK;
}

// The slit step of g (rows [row0, row0 + g->nrows) of handle h) captured into a fresh graph.
int capture_slit(whff_graph* g, whff_handle* h, int64_t row0, cudaGraph_t* out) {
  *out = nullptr;
  if (cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    set_error(std::string("whff_graph: begin capture: ") + cudaGetErrorString(cudaGetLastError()));
    return WHFF_ECUDA;
  }
  int e = step_view(h, row0, g->nrows, g->x, g->R, g->ldx, g->y + row0, g->ldy, g->state ? g->state + row0 : nullptr,
                    g->decay, g->cap);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(g->cap, &graph);
  if (e == WHFF_OK && ce != cudaSuccess) {
    set_error(std::string("whff_graph: end capture: ") + cudaGetErrorString(ce));
    e = WHFF_ECUDA;
  }
  if (e) {
    if (graph) cudaGraphDestroy(graph);
    return e;
  }
  *out = graph;
  return WHFF_OK;
}
}  // namespace

extern "C" int whff_graph_create_rows(whff_handle* h, int64_t row0, int64_t nrows, const float* x, int R, int64_t ldx,
                                      double* y, int64_t ldy, double* state, double decay, void* stream,
                                      whff_graph** out) {
  (void)stream;
  if (!out || !h || !x || !y || R <= 0 || R > h->max_rhs || ldx < h->info.N || ldy < h->info.M) {
    set_error("whff_graph_create_rows: null argument, R out of [1, max_rhs], or leading dimension too small");
    return WHFF_EINVAL;
  }
  if (const int de = check_device(h, "whff_graph_create_rows")) return de;
  *out = nullptr;
  int e = check_slit(h, row0, nrows, "whff_graph_create_rows");
  if (e) return e;
  auto* g = new whff_graph;
  g->h = h;
  g->nrows = nrows;
  g->x = x;
  g->R = R;
  g->ldx = ldx;
  g->y = y;
  g->ldy = ldy;
  g->state = state;
  g->decay = decay;
  if (cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete g;
    set_error("whff_graph_create_rows: cannot create a capture stream");
    return WHFF_ECUDA;
  }
  if ((e = capture_slit(g, h, row0, &g->graph)) != WHFF_OK) {
    whff_graph_destroy(g);
    return e;
  }
  if (cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) {
    set_error(std::string("whff_graph_create_rows: instantiate: ") + cudaGetErrorString(cudaGetLastError()));
    whff_graph_destroy(g);
    return WHFF_ECUDA;
  }
  g->row0 = row0;
  *out = g;
  return WHFF_OK;
}

extern "C" int whff_graph_set_rows(whff_graph* g, whff_handle* h, int64_t row0) {
  if (!g || !g->cap) {
    set_error("whff_graph_set_rows: not a slit graph (whff_graph_create_rows)");
    return WHFF_EINVAL;
  }
  if (!h) h = g->h;
  if (const int de = check_device(h, "whff_graph_set_rows")) return de;
  if (h != g->h && (h->info.fmt != g->h->info.fmt || h->info.rate != g->h->info.rate || h->info.M != g->h->info.M ||
                    h->info.N != g->h->info.N || h->max_rhs < g->R)) {
    set_error("whff_graph_set_rows: the new handle differs in format, rate, shape or max_rhs");
    return WHFF_EINVAL;
  }
  int e = check_slit(h, row0, g->nrows, "whff_graph_set_rows");
  if (e) return e;
  if (h == g->h && row0 == g->row0) return WHFF_OK;
  cudaGraph_t graph = nullptr;
  if ((e = capture_slit(g, h, row0, &graph)) != WHFF_OK) return e;
  // same plan (it depends on the slit height and the handle's launch shape, not on
  // row0), so the same nodes: only kernel arguments change
  cudaGraphExecUpdateResultInfo info;
  if (cudaGraphExecUpdate(g->exec, graph, &info) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(graph);
    set_error("whff_graph_set_rows: the slit's launch sequence differs from the captured one (was the handle's "
              "launch shape or crossover changed?)");
    return WHFF_EINVAL;
  }
  cudaGraphDestroy(g->graph);
  g->graph = graph;
  g->h = h;
  g->row0 = row0;
  return WHFF_OK;
}

extern "C" int whff_graph_launch(whff_graph* g, void* stream) {
  if (!g || !g->exec) {
    set_error("whff_graph_launch: null graph");
    return WHFF_EINVAL;
  }
  WHFF_CUDA_TRY(cudaGraphLaunch(g->exec, as_stream(stream)));
  return WHFF_OK;
}

extern "C" int whff_decompress(whff_handle* h, double* out, int64_t ldo, void* stream) {
  if (!h || !out || ldo < h->info.N) {
    set_error("whff_decompress: null pointer or ldo < N");
    return WHFF_EINVAL;
  }
  if (const int de = check_device(h, "whff_decompress")) return de;
  const cudaStream_t st = as_stream(stream);
  const auto& b = h->info;
  const int threads = 256;
  if (b.fmt == WHFF_FMT_ZFP) {
    const int64_t nb = h->BM * h->BN;
    const unsigned grid = (unsigned)((nb + threads - 1) / threads);
#define DZ(R_)                                                                                          \
  case R_:                                                                                              \
    dev::wz1_decompress_kernel<R_ / 2><<<grid, threads, 0, st>>>(h->d_stream, b.M, b.N, h->BN, nb, out, ldo); \
    break;
    switch (b.rate) {
      DZ(4) DZ(8) DZ(12) DZ(16) DZ(20) DZ(24) DZ(28) DZ(32) DZ(36) DZ(40) DZ(44) DZ(48) DZ(52) DZ(56) DZ(60) DZ(64)
      default:
        set_error("whff_decompress: unsupported rate");
        return WHFF_EINVAL;
    }
#undef DZ
  } else if (is_wz3(b.fmt)) {
    wz3_decompress(h->wz3_index, h->wz3_area, b.M, b.N, out, ldo, st);
  } else if (is_blocked(b.fmt)) {
    const int64_t nb = h->BM * h->BN;
    const bool lift = b.fmt == WHFF_FMT_FIXED_LIFT;
    int e;
    switch (b.rate) {
      case 8: e = wz2_decompress<8>(h->d_stream, b.M, b.N, h->BN, nb, out, ldo, lift, st); break;
      case 12: e = wz2_decompress<12>(h->d_stream, b.M, b.N, h->BN, nb, out, ldo, lift, st); break;
      case 16: e = wz2_decompress<16>(h->d_stream, b.M, b.N, h->BN, nb, out, ldo, lift, st); break;
      case 20: e = wz2_decompress<20>(h->d_stream, b.M, b.N, h->BN, nb, out, ldo, lift, st); break;
      case 24: e = wz2_decompress<24>(h->d_stream, b.M, b.N, h->BN, nb, out, ldo, lift, st); break;
      default: e = -1;
    }
    if (e) {
      set_error("whff_decompress: unsupported WZ2 rate");
      return WHFF_EINVAL;
    }
  } else {
    const int64_t ld = scaled_ld(b.N), TN = ceil_div(b.N, kScaleTile);
    const float* scales = h->d_scales;
    const int V = scaled_vec(b.fmt);
    const int64_t work = b.M * (ld / V);
    const unsigned grid = (unsigned)((work + threads - 1) / threads);
    if (b.fmt == WHFF_FMT_BF16)
      dev::scaled_decompress_kernel<2><<<grid, threads, 0, st>>>(h->d_stream, scales, b.M, b.N, ld, TN, out, ldo);
    else if (b.fmt == WHFF_FMT_FP16)
      dev::scaled_decompress_kernel<3><<<grid, threads, 0, st>>>(h->d_stream, scales, b.M, b.N, ld, TN, out, ldo);
    else if (b.fmt == WHFF_FMT_FP8E4M3)
      dev::scaled_decompress_kernel<4><<<grid, threads, 0, st>>>(h->d_stream, scales, b.M, b.N, ld, TN, out, ldo);
    else
      dev::scaled_decompress_kernel<7><<<grid, threads, 0, st>>>(h->d_stream, scales, b.M, b.N, ld, TN, out, ldo);
  }
  WHFF_CUDA_TRY(cudaGetLastError());
  return WHFF_OK;
}

extern "C" int whff_sync_status(whff_handle* h, void* stream) {
  if (!h) {
    set_error("whff_sync_status: null handle");
    return WHFF_EINVAL;
  }
  const cudaStream_t st = as_stream(stream);
  int status = 0;
  WHFF_CUDA_TRY(cudaMemcpyAsync(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  WHFF_CUDA_TRY(cudaMemsetAsync(h->d_status, 0, sizeof(int), st));
  WHFF_CUDA_TRY(cudaStreamSynchronize(st));
  if (status) set_error("device status word reported an error");
  return status;
}

extern "C" void whff_destroy(whff_handle* h) {
  if (!h) return;
  // stream-ordered: outstanding work on the creation stream finishes first
  if (h->create_stream) cudaStreamSynchronize(h->create_stream);
  if (h->h_stream)
    cudaFreeHost(h->h_stream);
  else
    cudaFree(h->d_stream);
  cudaFree(h->d_ws);
  cudaFree(h->d_ws_mma);
  cudaFree(h->d_btiles);
  cudaFree(h->d_xt);
  cudaFree(h->d_status);
  cudaFree(h->d_x);
  cudaFree(h->d_y);
  cudaGetLastError();
  delete h;
}

// ------------------------------------------------------------------ tuning
namespace {

int apply_config(whff_handle* h, int unroll, int ctas_per_sm, int fold) {
  h->unroll = unroll;
  h->ctas_per_sm = ctas_per_sm;
  h->red32 = (fold & WHFF_FOLD_FP32_PAIRS) != 0;
  h->groups8 = (fold & WHFF_FOLD_LANE_GROUPS) != 0;
  h->bulk = (fold & WHFF_CONFIG_BULK) != 0;
  choose_ranges(h);
  const size_t need = h->maxseg > 1 ? (size_t)h->BM * (size_t)h->maxseg * (size_t)h->ws_rhs * 4 * 8 : 0;
  if (need > h->ws_bytes) {
    cudaFree(h->d_ws);
    h->d_ws = nullptr;
    if (cudaMalloc(&h->d_ws, need) != cudaSuccess) {
      cudaGetLastError();
      h->ws_bytes = 0;
      set_error("whff_set_config: workspace allocation failed");
      return WHFF_ENOMEM;
    }
    h->ws_bytes = need;
  }
  return WHFF_OK;
}

bool is_wz2(const whff_handle* h) {
  return h->info.fmt == WHFF_FMT_FIXED_LIFT || h->info.fmt == WHFF_FMT_FIXED_BFP;
}

}  // namespace

extern "C" int whff_get_config(const whff_handle* h, int* unroll, int* ctas_per_sm, int* fold) {
  if (!h) {
    set_error("whff_get_config: null handle");
    return WHFF_EINVAL;
  }
  if (unroll) *unroll = h->unroll;
  if (ctas_per_sm) *ctas_per_sm = h->ctas_per_sm;
  if (fold)
    *fold = (h->red32 ? WHFF_FOLD_FP32_PAIRS : 0) | (h->groups8 ? WHFF_FOLD_LANE_GROUPS : 0) |
            (h->bulk ? WHFF_CONFIG_BULK : 0);
  return WHFF_OK;
}

extern "C" int whff_set_config(whff_handle* h, int unroll, int ctas_per_sm, int fold) {
  if (!h || !is_wz2(h) || (unroll != 2 && unroll != 4 && unroll != 8) || ctas_per_sm < 1 || fold < 0 || fold > 7 ||
      (unroll != 2 && (fold & WHFF_FOLD_LANE_GROUPS)) ||
      ((fold & WHFF_CONFIG_BULK) && (fold & WHFF_FOLD_LANE_GROUPS))) {
    set_error("whff_set_config: WZ2 handles only; unroll 2, 4 or 8 (2 with lane groups); ctas_per_sm >= 1; "
              "flags 0..7, bulk staging not with lane groups");
    return WHFF_EINVAL;
  }
  const bool lift = h->info.fmt == WHFF_FMT_FIXED_LIFT;
  const int occ = (fold & WHFF_CONFIG_BULK) ? wz2_stream_occ(h->info.rate, lift) : wz2_occ(h->info.rate, lift, unroll);
  if (occ <= 0 || ctas_per_sm > occ) {
    set_error("whff_set_config: more CTAs per SM than can be resident");
    return WHFF_EINVAL;
  }
  return apply_config(h, unroll, ctas_per_sm, fold);
}

extern "C" int whff_set_wait_limit(whff_handle* h, int64_t polls) {
  if (!h || polls > (int64_t)0x7FFFFFFF) {
    set_error("whff_set_wait_limit: null handle or polls above 2^31 - 1");
    return WHFF_EINVAL;
  }
  h->wait_polls = polls < 0 ? kWaitPolls : (uint32_t)polls;
  return WHFF_OK;
}

extern "C" int whff_get_crossover(const whff_handle* h, int* min_rhs) {
  if (!h || !min_rhs) {
    set_error("whff_get_crossover: null argument");
    return WHFF_EINVAL;
  }
  *min_rhs = h->d_ws_mma ? h->mma_min_rhs : 33;
  return WHFF_OK;
}

extern "C" int whff_set_crossover(whff_handle* h, int min_rhs) {
  if (!h || min_rhs < 2 || min_rhs > 33 || (!h->d_ws_mma && min_rhs != 33)) {
    set_error("whff_set_crossover: WZ2 handles created with max_rhs >= 2; min_rhs in [2, 33]");
    return WHFF_EINVAL;
  }
  h->mma_min_rhs = min_rhs;
  return WHFF_OK;
}

// Time every (unroll, CTAs per SM, lane fold) candidate on this matrix with
// R = 1 and keep the fastest.  Uses the handle's own staging buffers (x = 0).
extern "C" int whff_tune(whff_handle* h, int iters, void* stream, double* best_ms) {
  if (!h || !is_wz2(h) || iters < 1) {
    set_error("whff_tune: WZ2 handles only, iters >= 1");
    return WHFF_EINVAL;
  }
  if (const int de = check_device(h, "whff_tune")) return de;
  const cudaStream_t st = as_stream(stream);
  WHFF_CUDA_TRY(cudaMemsetAsync(h->d_x, 0, (size_t)h->info.N * 4, st));
  cudaEvent_t e0, e1;
  WHFF_CUDA_TRY(cudaEventCreate(&e0));
  WHFF_CUDA_TRY(cudaEventCreate(&e1));
  const int orig_u = h->unroll, orig_c = h->ctas_per_sm;
  const int orig_f = (h->red32 ? WHFF_FOLD_FP32_PAIRS : 0) | (h->groups8 ? WHFF_FOLD_LANE_GROUPS : 0) |
                     (h->bulk ? WHFF_CONFIG_BULK : 0);
  double best = 1e30;
  int bu = orig_u, bc = orig_c, bf = orig_f;
  int err = WHFF_OK;
  const bool lift = h->info.fmt == WHFF_FMT_FIXED_LIFT;
  // candidates: the top three CTA counts per SM x (unroll 2 with each of the four
  // folds, unroll 4 and 8 with the two whole-warp folds, and -- on device-resident
  // streams -- the bulk-staged kernel with the two whole-warp folds)
  const int ncand = h->h_stream ? 24 : 30;
  for (int cand = 0; cand < ncand && err == WHFF_OK; ++cand) {
    const int u = cand < 12 ? 2 : cand < 18 ? 4 : cand < 24 ? 8 : 2;
    const int f = (cand & 1) | (cand < 12 && (cand & 2) ? WHFF_FOLD_LANE_GROUPS : 0) | (cand >= 24 ? WHFF_CONFIG_BULK : 0);
    const int c = (cand >= 24 ? wz2_stream_occ(h->info.rate, lift) : wz2_occ(h->info.rate, lift, u)) -
                  (cand < 12 ? cand / 4 : cand < 18 ? (cand - 12) / 2 : cand < 24 ? (cand - 18) / 2 : (cand - 24) / 2);
    if (c < 1) continue;
    if ((err = apply_config(h, u, c, f)) != WHFF_OK) break;
    if ((err = whff_step(h, h->d_x, 1, h->info.N, h->d_y, h->info.M, nullptr, 0.0, stream)) != WHFF_OK) break;
    cudaEventRecord(e0, st);
    for (int k = 0; k < iters && err == WHFF_OK; ++k)
      err = whff_step(h, h->d_x, 1, h->info.N, h->d_y, h->info.M, nullptr, 0.0, stream);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) err = WHFF_ECUDA;
    if (err) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms / iters < best) {
      best = ms / iters;
      bu = u;
      bc = c;
      bf = f;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err) {
    apply_config(h, orig_u, orig_c, orig_f);
    return err;
  }
  if (best_ms) *best_ms = best;
  if ((err = apply_config(h, bu, bc, bf)) != WHFF_OK) return err;
  // the engine crossover: the fewest columns from which one tensor-core pass is
  // no slower than the CUDA-core passes (it only grows with R on the CUDA cores)
  if (h->d_ws_mma && h->max_rhs >= 2) {
    WHFF_CUDA_TRY(cudaMemsetAsync(h->d_x, 0, (size_t)h->info.N * 4 * std::min(h->max_rhs, 8), st));
    WHFF_CUDA_TRY(cudaEventCreate(&e0));
    WHFF_CUDA_TRY(cudaEventCreate(&e1));
    auto time_r = [&](int R, int cross, double* ms) {
      h->mma_min_rhs = cross;
      int e = whff_step(h, h->d_x, R, h->info.N, h->d_y, h->info.M, nullptr, 0.0, stream);
      cudaEventRecord(e0, st);
      for (int k = 0; k < iters && e == WHFF_OK; ++k)
        e = whff_step(h, h->d_x, R, h->info.N, h->d_y, h->info.M, nullptr, 0.0, stream);
      cudaEventRecord(e1, st);
      if (e == WHFF_OK && cudaEventSynchronize(e1) != cudaSuccess) e = WHFF_ECUDA;
      float f = 0.f;
      cudaEventElapsedTime(&f, e0, e1);
      *ms = f;
      return e;
    };
    int cross = 9;  // from 9 columns on the tensor cores always win
    for (int R = 2; R <= std::min(h->max_rhs, 8) && err == WHFF_OK; ++R) {
      double cc = 0, tc = 0;
      if ((err = time_r(R, 33, &cc)) != WHFF_OK || (err = time_r(R, 2, &tc)) != WHFF_OK) break;
      if (tc <= cc) {
        cross = R;
        break;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->mma_min_rhs = cross;
  }
  return err;
}

// ------------------------------------------------------------------ batches
struct whff_batch {
  struct Group {
    int R = 1;
    std::vector<int> members;          // (handle index, column offset) pairs flattened below
    std::vector<int> col0;
    std::vector<dev::BatchEntry> host;  // filled per step
    dev::BatchEntry* d_entries = nullptr;
    int64_t* d_row_begin = nullptr;
    std::vector<double*> ws;
    int64_t total_blocks = 0, total_rows = 0, L = 1, ctas = 1;
    bool any_shared = false;
  };
  std::vector<whff_handle*> hs;
  int rate = 0;
  bool lift = true;
  int scaled_fmt = 0;              // a batch of one scaled format (0: WZ2)
  std::vector<int> own_passes;     // scaled matrices stepped by their own tensor-core passes
  std::vector<Group> groups;
  dev::BatchEntry* pinned = nullptr;   // staging for the table uploads
  size_t pinned_entries = 0;
  dev::BatchState* state_pinned = nullptr;
  dev::BatchState* d_state = nullptr;
  int64_t* d_state_rows = nullptr;
  int64_t state_rows = 0;
  std::vector<int> R;
  cudaEvent_t copied = nullptr;        // the last step's table copies have been read
  // Matrices with R at or above their crossover: their passes of up to 32
  // columns, grouped by width class (16 or 32 TMEM columns), each group one
  // persistent tensor-core launch over the concatenated items of its passes.
  struct MmaGroup {
    int nr = 32;
    std::vector<int> of, col0;                 // handle index and first column of each pass
    std::vector<dev::MmaMember> members;       // static, on the device in d_members
    std::vector<dev::MmaPass> passes;          // vectors rewritten per step
    dev::MmaMember* d_members = nullptr;
    dev::MmaPass* d_passes = nullptr;
    dev::MmaPass* pinned = nullptr;
    double* ws = nullptr;
    uint8_t* btiles = nullptr;
    int64_t total = 0, L = 1, bt_threads = 0, fin_threads = 0;
    int ctas = 1;
  };
  std::vector<MmaGroup> mma_groups;
};

extern "C" void whff_batch_destroy(whff_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  for (auto& g : b->groups) {
    cudaFree(g.d_entries);
    cudaFree(g.d_row_begin);
    for (double* w : g.ws) cudaFree(w);
  }
  if (b->copied) cudaEventDestroy(b->copied);
  for (auto& g : b->mma_groups) {
    cudaFree(g.d_members);
    cudaFree(g.d_passes);
    cudaFreeHost(g.pinned);
    cudaFree(g.ws);
    cudaFree(g.btiles);
  }
  cudaFreeHost(b->pinned);
  cudaFreeHost(b->state_pinned);
  cudaFree(b->d_state);
  cudaFree(b->d_state_rows);
  cudaGetLastError();
  delete b;
}

// Plan one persistent launch per right-hand-side class (1, 2, 4, 8) over
// count resident matrices of one WZ2 format and rate; R[i] may be any
// positive count, taken in column groups of 8, 4, 2, 1 (a matrix with 32
// right-hand sides enters the R = 8 launch four times).
extern "C" int whff_batch_create(whff_handle* const* hs, const int* R, int count, whff_batch** out) {
  if (!hs || !R || !out || count < 1) {
    set_error("whff_batch_create: bad argument");
    return WHFF_EINVAL;
  }
  *out = nullptr;
  auto* b = new whff_batch;
  b->hs.assign(hs, hs + count);
  const auto scaled = [](const whff_handle* h) {
    const int f = h->info.fmt;
    return f == WHFF_FMT_BF16 || f == WHFF_FMT_FP16 || f == WHFF_FMT_FP8E4M3 || f == WHFF_FMT_FP32;
  };
  if (!hs[0]) {
    whff_batch_destroy(b);
    set_error("whff_batch_create: null handle");
    return WHFF_EINVAL;
  }
  b->rate = hs[0]->info.rate;
  b->lift = hs[0]->info.fmt == WHFF_FMT_FIXED_LIFT;
  b->scaled_fmt = scaled(hs[0]) ? hs[0]->info.fmt : 0;
  for (int i = 0; i < count; ++i) {
    // R[i] <= max_rhs: a matrix stepped by its own passes uses its handle's workspaces
    const bool ok = hs[i] && R[i] >= 1 && R[i] <= hs[i]->max_rhs && hs[i]->device == hs[0]->device &&
                    (b->scaled_fmt ? hs[i]->info.fmt == b->scaled_fmt
                                   : is_wz2(hs[i]) && hs[i]->info.rate == b->rate &&
                                         (hs[i]->info.fmt == WHFF_FMT_FIXED_LIFT) == b->lift);
    if (!ok) {
      whff_batch_destroy(b);
      set_error("whff_batch_create: all matrices must be resident WZ2 of one format and rate, or of one scaled "
                "format on one device; 1 <= R[i] <= the handle's max_rhs");
      return WHFF_EINVAL;
    }
  }
  const int classes[4] = {8, 4, 2, 1};
  for (int cls : classes) {
    whff_batch::Group g;
    g.R = cls;
    for (int i = 0; i < count; ++i) {
      if (R[i] >= hs[i]->mma_min_rhs && hs[i]->d_ws_mma) continue;  // tensor-core passes instead
      int c = 0, left = R[i];
      for (int k : classes) {  // decompose R[i] into 8s, then one 4, 2, 1
        while (left >= k && (k == 8 || left < 2 * k)) {
          if (k == cls) {
            g.members.push_back(i);
            g.col0.push_back(c);
          }
          c += k;
          left -= k;
        }
      }
    }
    if (!g.members.empty()) b->groups.push_back(g);
  }
  const whff_handle* h0 = hs[0];
  for (auto& g : b->groups) {
    const int n = (int)g.members.size();
    g.host.resize(n);
    int64_t blocks = 0, rows = 0;
    std::vector<int64_t> row_begin(n);
    for (int k = 0; k < n; ++k) {
      const whff_handle* h = hs[g.members[k]];
      g.host[k].block_begin = blocks;
      row_begin[k] = rows;
      blocks += h->BM * h->BN;
      rows += h->info.M;
    }
    g.total_blocks = blocks;
    g.total_rows = rows;
    const int occ = b->scaled_fmt ? scaled_occupancy(b->scaled_fmt, false) : wz2_occ(b->rate, b->lift, g.R == 1 ? 2 : 1);
    const int64_t warps_cap = (int64_t)h0->sm_count * std::max(occ, 1) * dev::kWarpsPerCta;
    int64_t warps = std::min<int64_t>(warps_cap, std::max<int64_t>(1, (blocks + 63) / 64));
    warps = (warps + dev::kWarpsPerCta - 1) / dev::kWarpsPerCta * dev::kWarpsPerCta;
    g.ctas = warps / dev::kWarpsPerCta;
    g.L = (blocks + warps - 1) / warps;
    for (int k = 0; k < n; ++k) {
      const whff_handle* h = hs[g.members[k]];
      int maxseg = 1;
      for (int64_t I = 0; I < h->BM; ++I) {
        const int64_t first = g.host[k].block_begin + I * h->BN;
        maxseg = (int)std::max<int64_t>(maxseg, (first + h->BN - 1) / g.L - first / g.L + 1);
      }
      g.host[k].maxseg = maxseg;
      double* w = nullptr;
      if (maxseg > 1) {
        g.any_shared = true;
        if (cudaMalloc(&w, (size_t)h->BM * maxseg * g.R * 4 * 8) != cudaSuccess) {
          cudaGetLastError();
          whff_batch_destroy(b);
          set_error("whff_batch_create: workspace allocation failed");
          return WHFF_ENOMEM;
        }
      }
      g.ws.push_back(w);
    }
    if (cudaMalloc(&g.d_entries, sizeof(dev::BatchEntry) * n) != cudaSuccess ||
        cudaMalloc(&g.d_row_begin, sizeof(int64_t) * n) != cudaSuccess ||
        cudaMemcpy(g.d_row_begin, row_begin.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      whff_batch_destroy(b);
      set_error("whff_batch_create: table allocation failed");
      return WHFF_ENOMEM;
    }
    b->pinned_entries += n;
  }
  b->R.assign(R, R + count);
  if (b->scaled_fmt) {  // scaled matrices at or above their crossover take their own tensor-core passes
    for (int i = 0; i < count; ++i)
      if (R[i] >= hs[i]->mma_min_rhs && hs[i]->d_ws_mma) b->own_passes.push_back(i);
  }
  // tensor-core passes: one group per width class and per kMaxMembers passes
  for (int nr : {16, 32}) {
    if (b->scaled_fmt) break;
    whff_batch::MmaGroup g;
    g.nr = nr;
    auto close = [&]() {
      if (!g.of.empty()) b->mma_groups.push_back(g);
      g = whff_batch::MmaGroup();
      g.nr = nr;
    };
    for (int i = 0; i < count; ++i) {
      if (!(R[i] >= hs[i]->mma_min_rhs && hs[i]->d_ws_mma)) continue;
      for (int c = 0; c < R[i]; c += 32) {
        const int rp = std::min(32, R[i] - c);
        if ((rp <= 16 ? 16 : 32) != nr) continue;
        if ((int)g.of.size() == mma_max_members()) close();
        g.of.push_back(i);
        g.col0.push_back(c);
      }
    }
    close();
  }
  for (auto& g : b->mma_groups) {
    const int n = (int)g.of.size();
    const size_t kB = (size_t)3 * 4 * g.nr * 16 * 2;  // B tile bytes per stage
    int64_t items = 0, bt = 0, fin = 0;
    size_t ws_words = 0, bt_bytes = 0;
    g.members.resize(n);
    g.passes.resize(n);
    for (int k = 0; k < n; ++k) {
      const whff_handle* h = hs[g.of[k]];
      const int rp = std::min(32, R[g.of[k]] - g.col0[k]);
      dev::MmaMember& m = g.members[k];
      m.stream = h->d_stream;
      m.BM = h->BM;
      m.BN = h->BN;
      m.S = (int)ceil_div(h->BN, 16);
      m.tiles = (int)ceil_div(h->BM, 32);
      m.R = rp;
      m.item_begin = items;
      items += (int64_t)m.tiles * m.S;
    }
    g.total = items;
    g.L = ceil_div(items, (int64_t)h0->sm_count * std::max(1, h0->mma_occ));
    g.ctas = (int)ceil_div(items, g.L);
    std::vector<size_t> ws_off(n), bt_off(n);
    for (int k = 0; k < n; ++k) {
      dev::MmaMember& m = g.members[k];
      m.maxseg = 1;
      for (int64_t tl = 0; tl < m.tiles; ++tl) {
        const int64_t first = m.item_begin + tl * m.S;
        m.maxseg = std::max<int>(m.maxseg, (int)((first + m.S - 1) / g.L - first / g.L + 1));
      }
      ws_off[k] = ws_words;
      ws_words += (size_t)m.tiles * m.maxseg * m.R * 128;
      bt_off[k] = bt_bytes;
      bt_bytes += (size_t)m.S * kB;
      dev::MmaPass& ps = g.passes[k];
      ps = dev::MmaPass{};
      ps.N = hs[g.of[k]]->info.N;
      ps.M = hs[g.of[k]]->info.M;
      ps.item_begin = m.item_begin;
      ps.bt_begin = bt;
      ps.fin_begin = fin;
      ps.S = m.S;
      ps.tiles = m.tiles;
      ps.R = m.R;
      ps.maxseg = m.maxseg;
      bt += (int64_t)m.S * 16 * g.nr;
      fin += (int64_t)m.tiles * m.R * 32;
    }
    g.bt_threads = bt;
    g.fin_threads = fin;
    if (cudaMalloc(&g.ws, ws_words * 8) != cudaSuccess || cudaMalloc(&g.btiles, bt_bytes) != cudaSuccess ||
        cudaMalloc(&g.d_members, sizeof(dev::MmaMember) * n) != cudaSuccess ||
        cudaMalloc(&g.d_passes, sizeof(dev::MmaPass) * n) != cudaSuccess ||
        cudaMallocHost(&g.pinned, sizeof(dev::MmaPass) * n) != cudaSuccess) {
      cudaGetLastError();
      whff_batch_destroy(b);
      set_error("whff_batch_create: tensor-core workspace allocation failed");
      return WHFF_ENOMEM;
    }
    for (int k = 0; k < n; ++k) {
      g.members[k].ws = g.ws + ws_off[k];
      g.members[k].btiles = g.btiles + bt_off[k];
      g.passes[k].ws = g.members[k].ws;
      g.passes[k].btiles = g.btiles + bt_off[k];
    }
    if (cudaMemcpy(g.d_members, g.members.data(), sizeof(dev::MmaMember) * n, cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      cudaGetLastError();
      whff_batch_destroy(b);
      set_error("whff_batch_create: tensor-core table upload failed");
      return WHFF_ECUDA;
    }
  }
  std::vector<int64_t> srows(count);
  for (int i = 0; i < count; ++i) {
    srows[i] = b->state_rows;
    b->state_rows += hs[i]->info.M;
  }
  if (cudaMallocHost(&b->state_pinned, sizeof(dev::BatchState) * count) != cudaSuccess ||
      cudaMalloc(&b->d_state, sizeof(dev::BatchState) * count) != cudaSuccess ||
      cudaMalloc(&b->d_state_rows, sizeof(int64_t) * count) != cudaSuccess ||
      cudaMemcpy(b->d_state_rows, srows.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    whff_batch_destroy(b);
    set_error("whff_batch_create: state table allocation failed");
    return WHFF_ENOMEM;
  }
  if (cudaEventCreateWithFlags(&b->copied, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost(&b->pinned, sizeof(dev::BatchEntry) * b->pinned_entries) != cudaSuccess) {
    cudaGetLastError();
    whff_batch_destroy(b);
    set_error("whff_batch_create: pinned staging allocation failed");
    return WHFF_ENOMEM;
  }
  *out = b;
  return WHFF_OK;
}

// One step of every matrix of the batch: x[i] (N_i x R_i, ldx[i]), y[i]
// (M_i x R_i, ldy[i]) and state[i] (M_i or NULL) are device pointers; the
// state update keeps the column order r = 0..R_i-1 (the column groups of a
// matrix run in order: R = 8 launches first, then 4, 2, 1).
extern "C" int whff_batch_step(whff_batch* b, const float* const* x, const int64_t* ldx, double* const* y,
                               const int64_t* ldy, double* const* state, double decay, void* stream) {
  if (!b || !x || !ldx || !y || !ldy) {
    set_error("whff_batch_step: bad argument");
    return WHFF_EINVAL;
  }
  if (const int de = check_device(b->hs[0], "whff_batch_step")) return de;
  const cudaStream_t st = as_stream(stream);
  // the pinned tables are reused: wait until the previous step's copies ran
  WHFF_CUDA_TRY(cudaEventSynchronize(b->copied));
  // matrices with many right-hand sides: one persistent tensor-core launch per width class
  // (their states are applied with everyone else's by the batch's state pass at the end)
  for (auto& g : b->mma_groups) {
    const int n = (int)g.of.size();
    for (int k = 0; k < n; ++k) {
      const int i = g.of[k];
      dev::MmaPass ps = g.passes[k];
      ps.x = x[i] + (int64_t)g.col0[k] * ldx[i];
      ps.y = y[i] + (int64_t)g.col0[k] * ldy[i];
      ps.ldx = ldx[i];
      ps.ldy = ldy[i];
      g.pinned[k] = ps;
    }
    WHFF_CUDA_TRY(cudaMemcpyAsync(g.d_passes, g.pinned, sizeof(dev::MmaPass) * n, cudaMemcpyHostToDevice, st));
    const whff_handle* h0 = b->hs[g.of[0]];
    MmaBatchStep a{b->rate, b->lift, g.nr, g.d_members, g.d_passes, n, g.total, g.L, g.ctas, g.bt_threads,
                   g.fin_threads, h0->d_status, h0->wait_polls};
    if (mma_batch_launch(a, st)) {
      set_error("whff_batch_step: tensor-core launch failed");
      return WHFF_ECUDA;
    }
  }
  for (int i : b->own_passes) {  // scaled matrices with many columns: their own passes, state applied below
    const int e = step_passes(b->hs[i], x[i], b->R[i], ldx[i], y[i], ldy[i], nullptr, decay, st);
    if (e) return e;
  }
  size_t off = 0;
  for (auto& g : b->groups) {
    const int n = (int)g.members.size();
    for (int k = 0; k < n; ++k) {
      const int i = g.members[k];
      const whff_handle* h = b->hs[i];
      dev::BatchEntry& e = g.host[k];
      e.stream = h->d_stream;
      e.x = x[i] + (int64_t)g.col0[k] * ldx[i];
      e.y = y[i] + (int64_t)g.col0[k] * ldy[i];
      e.state = nullptr;  // the state is applied once per matrix after all groups
      e.ws = g.ws[k];
      e.M = h->info.M;
      e.N = h->info.N;
      e.BM = h->BM;
      e.BN = h->BN;
      e.ldx = ldx[i];
      e.ldy = ldy[i];
      e.decay = decay;
      if (b->scaled_fmt) {
        e.scales = h->d_scales;
        e.ld = scaled_ld(h->info.N);
        e.TN = ceil_div(h->info.N, kScaleTile);
      }
      b->pinned[off + k] = e;
    }
    WHFF_CUDA_TRY(cudaMemcpyAsync(g.d_entries, b->pinned + off, sizeof(dev::BatchEntry) * n,
                                  cudaMemcpyHostToDevice, st));
    Wz2Batch a{g.d_entries, g.d_row_begin, n, g.total_blocks, g.total_rows, g.L, g.ctas, g.any_shared, b->lift, g.R};
    int e;
    if (b->scaled_fmt) e = scaled_batched_launch(b->scaled_fmt, a, st);
    else switch (b->rate) {
      case 8: e = wz2_batched_launch<8>(a, st); break;
      case 12: e = wz2_batched_launch<12>(a, st); break;
      case 16: e = wz2_batched_launch<16>(a, st); break;
      case 20: e = wz2_batched_launch<20>(a, st); break;
      case 24: e = wz2_batched_launch<24>(a, st); break;
      default: e = -1;
    }
    if (e) {
      set_error("whff_batch_step: launch failed");
      return WHFF_EINVAL;
    }
    off += n;
  }
  if (state) {
    const int count = (int)b->hs.size();
    for (int i = 0; i < count; ++i)
      b->state_pinned[i] = dev::BatchState{state[i], y[i], ldy[i], b->hs[i]->info.M, b->R[i], decay};
    WHFF_CUDA_TRY(cudaMemcpyAsync(b->d_state, b->state_pinned, sizeof(dev::BatchState) * count,
                                  cudaMemcpyHostToDevice, st));
    wz2_batched_state_launch(b->d_state, b->d_state_rows, count, b->state_rows, st);
  }
  WHFF_CUDA_TRY(cudaEventRecord(b->copied, st));
  WHFF_CUDA_TRY(cudaGetLastError());
  return WHFF_OK;
}

// ------------------------------------------------------------ field pipeline
// Sec. 4.3 (Fig. compression_cost, Table comp_metrics): the compressed C_field of
// the next exposure field crosses the host link while the GPU runs the slit steps
// of the current one.  nbuf resident slots, each a full handle (device stream,
// workspaces, launch plan) whose stream is rewritten by whff_fields_load; two
// events per slot order the copy stream against the compute stream.
struct whff_fields {
  BlobInfo info;
  bool verify = false;
  std::vector<whff_handle*> slots;
  std::vector<cudaEvent_t> loaded, released;
};

extern "C" void whff_fields_destroy(whff_fields* f) {
  if (!f) return;
  for (cudaEvent_t e : f->loaded)
    if (e) cudaEventSynchronize(e);
  for (cudaEvent_t e : f->released)
    if (e) cudaEventSynchronize(e);
  for (whff_handle* h : f->slots) whff_destroy(h);
  for (cudaEvent_t e : f->loaded)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : f->released)
    if (e) cudaEventDestroy(e);
  cudaGetLastError();
  delete f;
}

extern "C" int whff_fields_create(int fmt, int rate, int64_t M, int64_t N, int nbuf, int max_rhs, unsigned flags,
                                  void* stream, whff_fields** out) {
  if (!out || nbuf < 1 || nbuf > 16 || (flags & ~(unsigned)WHFF_FIELDS_VERIFY_CRC)) {
    set_error("whff_fields_create: null output, nbuf outside 1..16 or unknown flag");
    return WHFF_EINVAL;
  }
  *out = nullptr;
  BlobInfo info;
  info.fmt = fmt;
  info.rate = is_blocked(fmt) ? rate : 8 * elem_bytes(fmt);
  info.M = M;
  info.N = N;
  info.stream_bytes = stream_size(fmt, info.rate, M, N);
  if (!info.stream_bytes) {
    set_error("whff_fields_create: invalid format, rate or shape");
    return WHFF_EINVAL;
  }
  auto* f = new whff_fields;
  f->info = info;
  f->verify = (flags & WHFF_FIELDS_VERIFY_CRC) != 0;
  for (int k = 0; k < nbuf; ++k) {
    whff_handle* h = nullptr;
    int e = create_impl(info, nullptr, max_rhs, 0u, stream, &h);
    if (e) {
      whff_fields_destroy(f);
      return e;
    }
    f->slots.push_back(h);
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreateWithFlags(&a, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (a) cudaEventDestroy(a);
      whff_fields_destroy(f);
      set_error("whff_fields_create: event creation failed");
      return WHFF_ECUDA;
    }
    f->loaded.push_back(a);
    f->released.push_back(b);
  }
  *out = f;
  return WHFF_OK;
}

extern "C" int whff_fields_load(whff_fields* f, int slot, const void* blob, size_t len, void* copy_stream) {
  if (!f || slot < 0 || slot >= (int)f->slots.size() || !blob) {
    set_error("whff_fields_load: null argument or slot out of range");
    return WHFF_EINVAL;
  }
  BlobInfo b;
  int e = read_header(static_cast<const uint8_t*>(blob), len, &b, f->verify);
  if (e) {
    set_error("whff_fields_load: blob header, size or CRC check failed");
    return e;
  }
  if (b.fmt != f->info.fmt || b.rate != f->info.rate || b.M != f->info.M || b.N != f->info.N) {
    set_error("whff_fields_load: the blob's format, rate or shape differs from the pipeline's");
    return WHFF_EINVAL;
  }
  const cudaStream_t cs = as_stream(copy_stream);
  whff_handle* h = f->slots[slot];
  // the slot's previous field is no longer read once its release event has passed
  WHFF_CUDA_TRY(cudaStreamWaitEvent(cs, f->released[slot], 0));
  WHFF_CUDA_TRY(cudaMemcpyAsync(h->d_stream, static_cast<const uint8_t*>(blob) + kHeaderBytes, b.stream_bytes,
                                cudaMemcpyHostToDevice, cs));
  WHFF_CUDA_TRY(cudaEventRecord(f->loaded[slot], cs));
  h->info.crc_stream = b.crc_stream;
  return WHFF_OK;
}

extern "C" int whff_fields_acquire(whff_fields* f, int slot, void* compute_stream, whff_handle** h) {
  if (!f || slot < 0 || slot >= (int)f->slots.size() || !h) {
    set_error("whff_fields_acquire: null argument or slot out of range");
    return WHFF_EINVAL;
  }
  WHFF_CUDA_TRY(cudaStreamWaitEvent(as_stream(compute_stream), f->loaded[slot], 0));
  *h = f->slots[slot];
  return WHFF_OK;
}

extern "C" int whff_fields_release(whff_fields* f, int slot, void* compute_stream) {
  if (!f || slot < 0 || slot >= (int)f->slots.size()) {
    set_error("whff_fields_release: null argument or slot out of range");
    return WHFF_EINVAL;
  }
  WHFF_CUDA_TRY(cudaEventRecord(f->released[slot], as_stream(compute_stream)));
  return WHFF_OK;
}
