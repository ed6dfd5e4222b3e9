// gemv_kernels.cuh -- the fused decode + GEMV kernels of the control step and
// their FP64 epilogue (Sec. 4.4: FP32 products, FP64 reduction; Sec. 2.1:
// carried state), plus the decode-only kernels (Sec. 5.2).
//
// Work split (WZ1): one warp owns one 4-row band of A (one block row) over a
// column range; lanes take consecutive 4x4 blocks, so a warp streams one
// contiguous run of the compressed stream per iteration.  (The fixed-
// allocation and scaled formats use the persistent range schedule of
// wz2_kernels.cuh / scaled_kernels.cuh.)  Each lane keeps compensated FP32 sums
// (TwoSum: hi + lo) per row and right-hand side; the warp folds them in FP64
// with shuffles.  With one column range per band the warp finishes y and the
// state itself; with several (split-K, for wide matrices whose few rows
// cannot fill the GPU -- the cuBLAS failure mode of Sec. 5.1) the FP64
// partials go to a workspace and a second kernel sums them in split order.
#pragma once
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <cstdint>

#include "wz1_decode.cuh"

namespace whff {
namespace dev {

constexpr int kWarpsPerCta = 8;

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float p) {
  const float s = hi + p;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (p - bp);
  hi = s;
  lo += err;
}

// Sum over aligned groups of GL lanes (GL = 32: the warp); every lane of a
// group ends with its group's sum.  All 32 lanes must execute it.
template <int GL = 32>
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = GL / 2; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of the 32 lanes' compensated (hi, lo) pairs, in a fixed butterfly:
// each level adds the partner's hi with TwoSum (its error is exact whatever
// the operand order) and the partner's lo plainly, so every lane ends with
// the same pair, good to about 2^-48.  FP32 work only: on GB300 the FP64
// pipe is a small fraction of the FP32 one, and only the result is widened.
// It pays where bands are short (tall matrices: many band sums per block
// streamed); on long bands the FP64 butterfly above is a little faster, so
// the choice is a per-matrix setting (see whff_set_config).
template <int GL = 32>
__device__ __forceinline__ double warp_sum_pair(float hi, float lo) {
#pragma unroll
  for (int o = GL / 2; o; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    const float s = hi + h2;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (h2 - bp);
    hi = s;
    lo = (lo + l2) + e;
  }
  return (double)hi + (double)lo;
}

// Fold a lane's (hi, lo) sums for 4 rows x R columns and write either the
// final y (+ state) or the split-K partial.  Deterministic: fixed shuffle tree.
template <int R>
__device__ __forceinline__ void finish_band(const float (&hi)[4][R], const float (&lo)[4][R], int lane, int64_t row0,
                                            int64_t M, int split, int ksplit, int64_t Mpad, double* __restrict__ ws,
                                            double* __restrict__ y, int64_t ldy, double* __restrict__ state,
                                            double decay) {
  double tot[4][R];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int r = 0; r < R; ++r) tot[i][r] = warp_sum((double)hi[i][r] + (double)lo[i][r]);
  // lane (i*R + r) writes value (i, r)
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (lane != i * R + r) continue;
      const int64_t row = row0 + i;
      if (ksplit > 1) {
        ws[((int64_t)split * R + r) * Mpad + row] = tot[i][r];
      } else if (row < M) {
        y[(int64_t)r * ldy + row] = tot[i][r];
      }
    }
  if (ksplit == 1 && state != nullptr && lane < 4) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (lane != i) continue;
      const int64_t row = row0 + i;
      if (row < M) {
        double s = state[row];
#pragma unroll
        for (int r = 0; r < R; ++r) s = decay * s + tot[i][r];
        state[row] = s;
      }
    }
  }
}

// x[4J .. 4J+3] of column r, zero beyond N.
__device__ __forceinline__ float4 load_x4(const float* __restrict__ x, int64_t ldx, int r, int64_t c0, int64_t N,
                                          bool vec_ok) {
  const float* p = x + (int64_t)r * ldx + c0;
  if (vec_ok && c0 + 3 < N) return __ldg(reinterpret_cast<const float4*>(p));
  float4 v;
  v.x = c0 < N ? __ldg(p) : 0.f;
  v.y = c0 + 1 < N ? __ldg(p + 1) : 0.f;
  v.z = c0 + 2 < N ? __ldg(p + 2) : 0.f;
  v.w = c0 + 3 < N ? __ldg(p + 3) : 0.f;
  return v;
}

// --------------------------------------------------------------- WZ1 GEMV
template <int NW32, int R>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
    wz1_gemv_kernel(const uint8_t* __restrict__ stream, int64_t M, int64_t N, int64_t BM, int64_t BN,
                    const float* __restrict__ x, int64_t ldx, bool x_vec_ok, int ksplit, int64_t jchunk,
                    double* __restrict__ ws, double* __restrict__ y, int64_t ldy, double* __restrict__ state,
                    double decay) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t I = (int64_t)blockIdx.x * kWarpsPerCta + warp;
  if (I >= BM) return;  // whole warp
  const int split = blockIdx.y;
  const int64_t J0 = (int64_t)split * jchunk;
  const int64_t J1 = min(BN, J0 + jchunk);

  float hi[4][R], lo[4][R];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int r = 0; r < R; ++r) hi[i][r] = lo[i][r] = 0.f;

  __shared__ uint32_t planes[kPlaneWords];  // the decoder's plane words, a column per thread
  uint32_t* Ps = planes + threadIdx.x;
  const int64_t rowblk = I * BN;
  for (int64_t J = J0 + lane; J < J1; J += 32) {
    uint32_t w[NW32 + 2];
    load_block<NW32>(stream, rowblk + J, w);
    int32_t q[16];
    int emax;
    const bool nz = decode_block<NW32>(w, Ps, q, emax);
    if (!nz) continue;
    const float scale = __int_as_float((emax - 26 + 127) << 23);  // 2^(emax-26), a normal float
    float a[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = __int2float_rn(q[i]);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float4 xv = load_x4(x, ldx, r, 4 * J, N, x_vec_ok);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float p = a[4 * i] * xv.x;
        p = fmaf(a[4 * i + 1], xv.y, p);
        p = fmaf(a[4 * i + 2], xv.z, p);
        p = fmaf(a[4 * i + 3], xv.w, p);
        two_sum_acc(hi[i][r], lo[i][r], p * scale);
      }
    }
  }
  finish_band<R>(hi, lo, lane, 4 * I, M, split, ksplit, 4 * BM, ws, y, ldy, state, decay);
}

// ------------------------------------------------------- scaled-format GEMV
// Element decode: FMT 2 = BF16, 3 = FP16, 4 = FP8 E4M3.  A lane reads 16
// bytes: V = 8 (16-bit) or 16 (8-bit) consecutive elements of one row.
template <int FMT>
struct ScaledTraits;
template <>
struct ScaledTraits<2> {
  static constexpr int V = 8;
  __device__ static __forceinline__ void decode(uint4 raw, float (&f)[8]) {
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      f[2 * i] = __uint_as_float(w[i] << 16);
      f[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
    }
  }
};
template <>
struct ScaledTraits<3> {
  static constexpr int V = 8;
  __device__ static __forceinline__ void decode(uint4 raw, float (&f)[8]) {
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __half2_raw hr;
      hr.x = (unsigned short)(w[i] & 0xFFFF);
      hr.y = (unsigned short)(w[i] >> 16);
      const float2 v = __half22float2(__half2(hr));
      f[2 * i] = v.x;
      f[2 * i + 1] = v.y;
    }
  }
};
template <>
struct ScaledTraits<4> {
  static constexpr int V = 16;
  __device__ static __forceinline__ void decode(uint4 raw, float (&f)[16]) {
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[i] & 0xFFFF), __NV_E4M3);
      const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[i] >> 16), __NV_E4M3);
      const float2 a = __half22float2(__half2(lo));
      const float2 b = __half22float2(__half2(hi));
      f[4 * i] = a.x;
      f[4 * i + 1] = a.y;
      f[4 * i + 2] = b.x;
      f[4 * i + 3] = b.y;
    }
  }
};

// FP32 storage (the uncompressed comparison): four values per 16 bytes.
template <>
struct ScaledTraits<7> {
  static constexpr int V = 4;
  __device__ static __forceinline__ void decode(uint4 raw, float (&f)[4]) {
    f[0] = __uint_as_float(raw.x);
    f[1] = __uint_as_float(raw.y);
    f[2] = __uint_as_float(raw.z);
    f[3] = __uint_as_float(raw.w);
  }
};

// bytes per element of a scaled format
template <int FMT>
__host__ __device__ constexpr int scaled_elem_bytes() {
  return FMT == 4 ? 1 : FMT == 7 ? 4 : 2;
}

// --------------------------------------------------- split-K epilogue (FP64)
static __global__ void splitk_epilogue_kernel(const double* __restrict__ ws, int ksplit, int R, int64_t Mpad, int64_t M,
                                       double* __restrict__ y, int64_t ldy, double* __restrict__ state,
                                       double decay) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= M) return;
  double s = state ? state[row] : 0.0;
  for (int r = 0; r < R; ++r) {
    double t = 0.0;
    for (int k = 0; k < ksplit; ++k) t += ws[((int64_t)k * R + r) * Mpad + row];
    y[(int64_t)r * ldy + row] = t;
    s = decay * s + t;
  }
  if (state) state[row] = s;
}

// ------------------------------------------------------------- decode only
template <int NW32>
__global__ void wz1_decompress_kernel(const uint8_t* __restrict__ stream, int64_t M, int64_t N, int64_t BN,
                                      int64_t nblocks, double* __restrict__ out, int64_t ldo) {
  __shared__ uint32_t planes[kPlaneWords];  // the decoder's plane words, a column per thread
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblocks) return;
  const int64_t I = b / BN, J = b - (b / BN) * BN;
  uint32_t w[NW32 + 2];
  load_block<NW32>(stream, b, w);
  int32_t q[16];
  int emax;
  const bool nz = decode_block<NW32>(w, planes + threadIdx.x, q, emax);
  const double scale = nz ? ldexp(1.0, emax - 26) : 0.0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t row = 4 * I + r;
    if (row >= M) break;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t col = 4 * J + c;
      if (col < N) out[row * ldo + col] = (double)__int2float_rn(q[4 * r + c]) * scale;
    }
  }
}

template <int FMT>
__global__ void scaled_decompress_kernel(const uint8_t* __restrict__ payload, const float* __restrict__ scales,
                                         int64_t M, int64_t N, int64_t ld, int64_t TN, double* __restrict__ out,
                                         int64_t ldo) {
  using T = ScaledTraits<FMT>;
  constexpr int V = T::V;
  constexpr int EB = scaled_elem_bytes<FMT>();
  const int64_t chunks_per_row = ld / V;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= M * chunks_per_row) return;
  const int64_t row = t / chunks_per_row, c = (t - row * chunks_per_row) * V;
  const uint4 raw = __ldcs(reinterpret_cast<const uint4*>(payload + ((uint64_t)row * ld + c) * EB));
  float f[V];
  T::decode(raw, f);
  const double s = (double)__ldg(scales + (row / 128) * TN + c / 128);
#pragma unroll
  for (int v = 0; v < V; ++v)
    if (c + v < N) out[row * ldo + c + v] = s * (double)f[v];
}

}  // namespace dev
}  // namespace whff
