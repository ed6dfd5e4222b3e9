// whff_runtime.cu -- device runtime of the library: resident handles, the
// step launch (fused decode + GEMV, FP64 epilogue), decompression, errors.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>

#include "gemv_kernels.cuh"
#include "wz2_kernels.cuh"
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
  uint8_t* d_stream = nullptr;  // the blob's stream, 256-byte aligned
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
  int64_t range_ctas = 0;       // WZ2: CTAs of the range-partitioned persistent grid
  int64_t range_len = 0;        // WZ2: blocks per warp range
  int maxseg = 1;               // WZ2: most ranges sharing one band (1 = none shared)
  cudaStream_t create_stream = nullptr;
};

namespace whff {
namespace {

constexpr int kMaxRhsKernel = 8;  // right-hand sides handled per kernel pass

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Split-K so that the grid holds enough warps for the GPU: each warp owns one
// 4-row band; when bands are few (wide matrices), split the columns.
// WZ2: split the band-major block order into one contiguous range per
// resident warp (exact balance); bands that straddle ranges get segments.
void choose_ranges(whff_handle* h) {
  const int64_t total = h->BM * h->BN;
  const int64_t warps_cap = (int64_t)h->sm_count * h->ctas_per_sm * dev::kWarpsPerCta;
  int64_t warps = std::min<int64_t>(warps_cap, std::max<int64_t>(1, (total + 63) / 64));  // >= 64 blocks each
  warps = (warps + dev::kWarpsPerCta - 1) / dev::kWarpsPerCta * dev::kWarpsPerCta;
  h->range_ctas = warps / dev::kWarpsPerCta;
  h->range_len = (total + warps - 1) / warps;
  int maxseg = 1;
  for (int64_t I = 0; I < h->BM; ++I) {
    const int64_t lo = (I * h->BN) / h->range_len, hi = ((I + 1) * h->BN - 1) / h->range_len;
    maxseg = (int)std::max<int64_t>(maxseg, hi - lo + 1);
  }
  h->maxseg = maxseg;
  h->ksplit = 1;
  h->chunk = h->BN;
}

void choose_split(whff_handle* h) {
  if (h->info.fmt == WHFF_FMT_FIXED_LIFT || h->info.fmt == WHFF_FMT_FIXED_BFP) {
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
    const int V = h->info.fmt == WHFF_FMT_FP8E4M3 ? 16 : 8;
    const int64_t ld = scaled_ld(h->info.N);
    const int64_t unit = 32 * V;  // columns per warp iteration
    const int64_t units = (ld + unit - 1) / unit;
    ks = std::max<int64_t>(1, std::min<int64_t>(ks, units));
    h->ksplit = (int)std::min<int64_t>(ks, 256);
    h->chunk = ((units + h->ksplit - 1) / h->ksplit) * unit;
    h->ksplit = (int)((ld + h->chunk - 1) / h->chunk);
  }
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

template <int RATE, bool LIFT>
int launch_wz2_rate(const whff_handle* h, const float* x, int R, int64_t ldx, bool vec, double* y, int64_t ldy,
                    double* state, double decay, cudaStream_t st) {
  // persistent: one wave of CTAs; warp g owns blocks [g*L, (g+1)*L) of the band-major order
  dim3 grid((unsigned)h->range_ctas);
  dim3 block(dev::kWarpsPerCta * 32);
  const uint8_t* s = h->d_stream;
  const auto& b = h->info;
#define WZ2_CASE(RR)                                                                                      \
  case RR:                                                                                                \
    dev::wz2_gemv_kernel<RATE, LIFT, RR><<<grid, block, 0, st>>>(s, b.M, b.N, h->BM, h->BN, x, ldx, vec, \
                                                                 h->range_len, h->maxseg, h->d_ws, y,     \
                                                                 ldy, state, decay);                      \
    break;
  switch (R) {
    WZ2_CASE(1)
    WZ2_CASE(2)
    WZ2_CASE(4)
    WZ2_CASE(8)
    default:
      return WHFF_EINVAL;
  }
#undef WZ2_CASE
  if (h->maxseg > 1) {
    dev::wz2_segment_epilogue<<<(unsigned)((b.M + 255) / 256), 256, 0, st>>>(h->d_ws, b.M, h->BN, h->range_len,
                                                                            h->maxseg, R, y, ldy, state, decay);
  }
  return WHFF_OK;
}

template <bool LIFT>
int launch_wz2(const whff_handle* h, const float* x, int R, int64_t ldx, bool vec, double* y, int64_t ldy,
               double* state, double decay, cudaStream_t st) {
  switch (h->info.rate) {
    case 8:
      return launch_wz2_rate<8, LIFT>(h, x, R, ldx, vec, y, ldy, state, decay, st);
    case 12:
      return launch_wz2_rate<12, LIFT>(h, x, R, ldx, vec, y, ldy, state, decay, st);
    case 16:
      return launch_wz2_rate<16, LIFT>(h, x, R, ldx, vec, y, ldy, state, decay, st);
    case 20:
      return launch_wz2_rate<20, LIFT>(h, x, R, ldx, vec, y, ldy, state, decay, st);
    case 24:
      return launch_wz2_rate<24, LIFT>(h, x, R, ldx, vec, y, ldy, state, decay, st);
    default:
      set_error("whff_step: WZ2 rates are 8..24 in steps of 4");
      return WHFF_EINVAL;
  }
}

template <int FMT>
int launch_scaled_fmt(const whff_handle* h, const float* x, int R, int64_t ldx, bool vec, double* y, int64_t ldy,
                      double* state, double decay, cudaStream_t st) {
  const auto& b = h->info;
  const int64_t ld = scaled_ld(b.N);
  const int64_t TN = ceil_div(b.N, kScaleTile);
  const uint8_t* payload = h->d_stream;
  const float* scales =
      reinterpret_cast<const float*>(h->d_stream + (uint64_t)b.M * (uint64_t)ld * (uint64_t)elem_bytes(FMT));
  dim3 grid((unsigned)((h->Mpad / 4 + dev::kWarpsPerCta - 1) / dev::kWarpsPerCta), (unsigned)h->ksplit);
  dim3 block(dev::kWarpsPerCta * 32);
#define SC_CASE(RR)                                                                                         \
  case RR:                                                                                                  \
    dev::scaled_gemv_kernel<FMT, RR><<<grid, block, 0, st>>>(payload, scales, b.M, b.N, ld, TN, x, ldx, vec, \
                                                             h->ksplit, h->chunk, h->d_ws, y, ldy, state,    \
                                                             decay);                                        \
    break;
  switch (R) {
    SC_CASE(1)
    SC_CASE(2)
    SC_CASE(4)
    SC_CASE(8)
    default:
      return WHFF_EINVAL;
  }
#undef SC_CASE
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
      e = launch_wz2<true>(h, x, R, ldx, vec, y, ldy, state, decay, st);
      break;
    case WHFF_FMT_FIXED_BFP:
      e = launch_wz2<false>(h, x, R, ldx, vec, y, ldy, state, decay, st);
      break;
    case WHFF_FMT_BF16:
      e = launch_scaled_fmt<2>(h, x, R, ldx, vec, y, ldy, state, decay, st);
      break;
    case WHFF_FMT_FP16:
      e = launch_scaled_fmt<3>(h, x, R, ldx, vec, y, ldy, state, decay, st);
      break;
    case WHFF_FMT_FP8E4M3:
      e = launch_scaled_fmt<4>(h, x, R, ldx, vec, y, ldy, state, decay, st);
      break;
    default:
      e = WHFF_EINVAL;
  }
  if (e) return e;
  if (h->ksplit > 1 && h->info.fmt != WHFF_FMT_FIXED_LIFT && h->info.fmt != WHFF_FMT_FIXED_BFP) {
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

extern "C" const char* whff_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* whff_version(void) { return "whff 0.1 sm_103a"; }

extern "C" int whff_create(const void* blob, size_t len, int max_rhs, void* stream, whff_handle** out) {
  if (!out) {
    set_error("whff_create: null output handle");
    return WHFF_EINVAL;
  }
  *out = nullptr;
  BlobInfo info;
  int e = read_header((const uint8_t*)blob, len, &info, true);
  if (e) {
    set_error("whff_create: blob header, size or CRC check failed");
    return e;
  }
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
    // resident CTAs per SM of the persistent kernel (same for every R <= 8 within 1)
    int occ = 0;
    const bool lift = info.fmt == WHFF_FMT_FIXED_LIFT;
    cudaError_t oe = cudaErrorInvalidValue;
#define OCC(RT)                                                                                              \
  case RT:                                                                                                   \
    oe = lift ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dev::wz2_gemv_kernel<RT, true, 1>,     \
                                                              dev::kWarpsPerCta * 32, 0)                    \
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dev::wz2_gemv_kernel<RT, false, 1>,    \
                                                              dev::kWarpsPerCta * 32, 0);                   \
    break;
    switch (info.rate) {
      OCC(8) OCC(12) OCC(16) OCC(20) OCC(24)
      default: break;
    }
#undef OCC
    if (oe != cudaSuccess || occ <= 0) {
      cudaGetLastError();
      occ = 4;
    }
    h->ctas_per_sm = occ;
  }
  if (is_blocked(info.fmt)) {
    h->BM = ceil_div(info.M, 4);
    h->BN = ceil_div(info.N, 4);
  }
  choose_split(h);
  const cudaStream_t st = as_stream(stream);
  if (cudaMalloc(&h->d_stream, info.stream_bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("whff_create: cudaMalloc of the compressed stream failed");
    return fail(WHFF_ENOMEM);
  }
  h->ws_bytes = h->ksplit > 1 ? (size_t)h->ksplit * (size_t)std::min(max_rhs, kMaxRhsKernel) * (size_t)h->Mpad * 8 : 0;
  if (h->maxseg > 1)
    h->ws_bytes = (size_t)h->BM * (size_t)h->maxseg * (size_t)std::min(max_rhs, kMaxRhsKernel) * 4 * 8;
  if ((h->ws_bytes && cudaMalloc(&h->d_ws, h->ws_bytes) != cudaSuccess) ||
      cudaMalloc(&h->d_status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->d_x, (size_t)info.N * (size_t)max_rhs * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&h->d_y, (size_t)info.M * (size_t)max_rhs * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    set_error("whff_create: cudaMalloc of the workspace failed");
    return fail(WHFF_ENOMEM);
  }
  if (cudaMemsetAsync(h->d_status, 0, sizeof(int), st) != cudaSuccess ||
      cudaMemcpyAsync(h->d_stream, (const uint8_t*)blob + kHeaderBytes, info.stream_bytes, cudaMemcpyHostToDevice,
                      st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    set_error(std::string("whff_create: upload failed: ") + cudaGetErrorString(cudaGetLastError()));
    return fail(WHFF_ECUDA);
  }
  *out = h;
  return WHFF_OK;
}

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
    *device_bytes = h->info.stream_bytes + h->ws_bytes + sizeof(int) + (size_t)h->info.N * h->max_rhs * 4 +
                    (size_t)h->info.M * h->max_rhs * 8;
  return WHFF_OK;
}

extern "C" int whff_plan(const whff_handle* h, int* ksplit, int* launches) {
  if (!h) {
    set_error("whff_plan: null handle");
    return WHFF_EINVAL;
  }
  if (ksplit) *ksplit = h->ksplit;
  if (launches) *launches = (h->ksplit > 1 || h->maxseg > 1) ? 2 : 1;
  return WHFF_OK;
}

extern "C" int whff_step(whff_handle* h, const float* x, int R, int64_t ldx, double* y, int64_t ldy, double* state,
                         double decay, void* stream) {
  if (!h || !x || !y || R <= 0 || R > h->max_rhs || ldx < h->info.N || ldy < h->info.M) {
    set_error("whff_step: null pointer, R out of [1, max_rhs], or leading dimension too small");
    return WHFF_EINVAL;
  }
  const cudaStream_t st = as_stream(stream);
  // right-hand sides go through the kernel in passes of 8, 4, 2, 1; the state
  // update is applied pass by pass, which keeps the column order r = 0..R-1
  int r0 = 0;
  while (r0 < R) {
    const int left = R - r0;
    const int pass = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
    int e = launch_pass(h, x + (int64_t)r0 * ldx, pass, ldx, y + (int64_t)r0 * ldy, ldy, state, decay, st);
    if (e) return e;
    r0 += pass;
  }
  return WHFF_OK;
}

extern "C" int whff_step_host(whff_handle* h, const float* x_host, int R, int64_t ldx, double* y_host, int64_t ldy,
                              double* state, double decay, void* stream) {
  if (!h || !x_host || !y_host || R <= 0 || R > h->max_rhs || ldx < h->info.N || ldy < h->info.M) {
    set_error("whff_step_host: null pointer, R out of [1, max_rhs], or leading dimension too small");
    return WHFF_EINVAL;
  }
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
  } else if (is_blocked(b.fmt)) {
    const int64_t nb = h->BM * h->BN;
    const unsigned grid = (unsigned)((nb + threads - 1) / threads);
    const bool lift = b.fmt == WHFF_FMT_FIXED_LIFT;
#define D2(R_)                                                                                                  \
  case R_:                                                                                                      \
    if (lift)                                                                                                   \
      dev::wz2_decompress_kernel<R_, true><<<grid, threads, 0, st>>>(h->d_stream, b.M, b.N, h->BN, nb, out, ldo); \
    else                                                                                                        \
      dev::wz2_decompress_kernel<R_, false><<<grid, threads, 0, st>>>(h->d_stream, b.M, b.N, h->BN, nb, out, ldo); \
    break;
    switch (b.rate) {
      D2(8) D2(12) D2(16) D2(20) D2(24)
      default:
        set_error("whff_decompress: unsupported WZ2 rate");
        return WHFF_EINVAL;
    }
#undef D2
  } else {
    const int64_t ld = scaled_ld(b.N), TN = ceil_div(b.N, kScaleTile);
    const float* scales =
        reinterpret_cast<const float*>(h->d_stream + (uint64_t)b.M * (uint64_t)ld * (uint64_t)elem_bytes(b.fmt));
    const int V = b.fmt == WHFF_FMT_FP8E4M3 ? 16 : 8;
    const int64_t work = b.M * (ld / V);
    const unsigned grid = (unsigned)((work + threads - 1) / threads);
    if (b.fmt == WHFF_FMT_BF16)
      dev::scaled_decompress_kernel<2><<<grid, threads, 0, st>>>(h->d_stream, scales, b.M, b.N, ld, TN, out, ldo);
    else if (b.fmt == WHFF_FMT_FP16)
      dev::scaled_decompress_kernel<3><<<grid, threads, 0, st>>>(h->d_stream, scales, b.M, b.N, ld, TN, out, ldo);
    else
      dev::scaled_decompress_kernel<4><<<grid, threads, 0, st>>>(h->d_stream, scales, b.M, b.N, ld, TN, out, ldo);
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
  cudaFree(h->d_stream);
  cudaFree(h->d_ws);
  cudaFree(h->d_status);
  cudaFree(h->d_x);
  cudaFree(h->d_y);
  cudaGetLastError();
  delete h;
}
