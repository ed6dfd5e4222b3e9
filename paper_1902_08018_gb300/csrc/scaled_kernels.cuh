// scaled_kernels.cuh -- GEMV on the scaled element formats (BF16, FP16, FP8
// E4M3 with one FP32 scale per 128 x 128 tile): the precision layer.
//
// Same schedule as the fixed-allocation kernels: the warps of a persistent
// grid split the band-major sequence of 16-byte column chunks of all 4-row
// bands into equal contiguous ranges; a lane keeps two chunks (4 rows each) in
// flight; each group of 4 products enters a TwoSum accumulator together with
// the exact rounding error of its product with the tile scale.  FP32 storage
// (FMT 7, unit scales) follows the paper's mixed precision instead (Sec. 4.4):
// every product is rounded to FP32 on its own and enters the TwoSum alone.
#pragma once
#include <cstdint>

#include "gemv_kernels.cuh"
#include "wz2_kernels.cuh"

namespace whff {
namespace dev {

template <int FMT, int R>
__device__ __forceinline__ void scaled_chunk(const uint8_t* __restrict__ payload, const float* __restrict__ scales,
                                             int64_t M, int64_t N, int64_t ld, int64_t TN, int64_t row0, int64_t c,
                                             const uint4 (&raw)[4], const float* __restrict__ x, int64_t ldx,
                                             bool x_fast, float (&hi)[4][R], float (&lo)[4][R]) {
  using T = ScaledTraits<FMT>;
  constexpr int V = T::V;
  float xv[R][V];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const float* xp = x + (int64_t)r * ldx + c;
    if (x_fast || c + V <= N) {
      if (x_fast) {
#pragma unroll
        for (int v = 0; v < V; v += 4) {
          const float4 t = __ldg(reinterpret_cast<const float4*>(xp + v));
          xv[r][v] = t.x;
          xv[r][v + 1] = t.y;
          xv[r][v + 2] = t.z;
          xv[r][v + 3] = t.w;
        }
      } else {
#pragma unroll
        for (int v = 0; v < V; ++v) xv[r][v] = __ldg(xp + v);
      }
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) xv[r][v] = c + v < N ? __ldg(xp + v) : 0.f;
    }
  }
  const int64_t tcol = c / 128;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t row = row0 + i;
    if (row >= M) break;
    float f[V];
    T::decode(raw[i], f);
    if constexpr (FMT == 7) {  // products rounded one by one, summed without loss
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int v = 0; v < V; ++v) two_sum_acc(hi[i][r], lo[i][r], __fmul_rn(f[v], xv[r][v]));
      continue;
    }
    const float s = __ldg(scales + (row / 128) * TN + tcol);
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
      for (int g = 0; g < V; g += 4) {
        float p = f[g] * xv[r][g];
        p = fmaf(f[g + 1], xv[r][g + 1], p);
        p = fmaf(f[g + 2], xv[r][g + 2], p);
        p = fmaf(f[g + 3], xv[r][g + 3], p);
        const float ps = p * s;
        two_sum_acc(hi[i][r], lo[i][r], ps);
        lo[i][r] += fmaf(p, s, -ps);
      }
    }
  }
}

template <int FMT>
__device__ __forceinline__ void scaled_load(const uint8_t* __restrict__ payload, int64_t M, int64_t ld,
                                            int64_t row0, int64_t c, uint4 (&raw)[4]) {
  constexpr int EB = scaled_elem_bytes<FMT>();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t row = row0 + i;
    raw[i] = row < M ? __ldcs(reinterpret_cast<const uint4*>(payload + ((uint64_t)row * ld + c) * EB))
                     : make_uint4(0, 0, 0, 0);
  }
}

template <int FMT, int R>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
    scaled_range_kernel(const uint8_t* __restrict__ payload, const float* __restrict__ scales, int64_t M, int64_t N,
                        int64_t ld, int64_t TN, const float* __restrict__ x, int64_t ldx, bool x_vec_ok, int64_t L,
                        int maxseg, double* __restrict__ ws, double* __restrict__ y, int64_t ldy,
                        double* __restrict__ state, double decay, bool red32) {
  constexpr int V = ScaledTraits<FMT>::V;
  const int lane = threadIdx.x & 31;
  const int64_t g = (int64_t)blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5);
  const int64_t BM = (M + 3) / 4, CB = ld / V;  // bands, chunks per band
  const int64_t total = BM * CB;
  const bool x_fast = x_vec_ok && (N % 4 == 0) && (ld == N);
  int64_t b0 = g * L;
  const int64_t b1 = min(total, b0 + L);
  while (b0 < b1) {
    const int64_t I = b0 / CB;
    const int64_t piece_end = min(b1, (I + 1) * CB);
    const int64_t g_lo = (I * CB) / L, g_hi = ((I + 1) * CB - 1) / L;
    const int64_t row0 = 4 * I;
    float hi[4][R], lo[4][R];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int r = 0; r < R; ++r) hi[i][r] = lo[i][r] = 0.f;
    int64_t J = b0 - I * CB + lane;
    const int64_t J1 = piece_end - I * CB;
    for (; J + 32 < J1; J += 64) {  // two chunks in flight, processed in order
      uint4 r0[4], r1[4];
      scaled_load<FMT>(payload, M, ld, row0, J * V, r0);
      scaled_load<FMT>(payload, M, ld, row0, (J + 32) * V, r1);
      scaled_chunk<FMT, R>(payload, scales, M, N, ld, TN, row0, J * V, r0, x, ldx, x_fast, hi, lo);
      scaled_chunk<FMT, R>(payload, scales, M, N, ld, TN, row0, (J + 32) * V, r1, x, ldx, x_fast, hi, lo);
    }
    if (J < J1) {
      uint4 r0[4];
      scaled_load<FMT>(payload, M, ld, row0, J * V, r0);
      scaled_chunk<FMT, R>(payload, scales, M, N, ld, TN, row0, J * V, r0, x, ldx, x_fast, hi, lo);
    }
    if (g_lo == g_hi) {
      band_finish<0, R>(hi, lo, lane, row0, M, 0, 1, 4 * BM, ws, y, ldy, state, decay, red32);
    } else {
      band_finish<0, R>(hi, lo, lane, 4 * ((I * maxseg + (g - g_lo)) * R), M, 0, 2, 0, ws, y, ldy, state, decay,
                        red32);
    }
    b0 = piece_end;
  }
}

}  // namespace dev
}  // namespace whff
