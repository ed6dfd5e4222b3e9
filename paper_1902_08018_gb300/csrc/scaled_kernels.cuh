// scaled_kernels.cuh -- GEMV on the scaled element formats (BF16, FP16, FP8
// E4M3 with one FP32 scale per 128 x 128 tile): the precision layer.
//
// Same schedule as the fixed-allocation kernels: the warps of a persistent
// grid split the band-major sequence of 16-byte column chunks of all 4-row
// bands into equal contiguous ranges; a lane keeps two chunks (4 rows each) in
// flight; 8 consecutive products of one row are chained in FP32 and enter a
// TwoSum accumulator together with the exact rounding error of their sum's
// product with the tile scale.  Rows 2h and 2h+1 of a band share one packed
// FP32 pair instruction per step.  FP32 storage
// (FMT 7, unit scales) follows the paper's mixed precision instead (Sec. 4.4):
// every product is rounded to FP32 on its own and enters the TwoSum alone.
#pragma once
#include <cstdint>

#include "f32x2.cuh"
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
  // rows 2h and 2h+1 go through the packed FP32 pair instructions together;
  // rows past M hold zeros (their y is never written)
  float f[4][V];
#pragma unroll
  for (int i = 0; i < 4; ++i) T::decode(raw[i], f[i]);
  float2 hi2[2][R], lo2[2][R];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      hi2[h][r] = make_float2(hi[2 * h][r], hi[2 * h + 1][r]);
      lo2[h][r] = make_float2(lo[2 * h][r], lo[2 * h + 1][r]);
    }
  // A product that must stay rounded is a scalar mul.rn, which is never
  // fused into its consumer; a packed multiply feeding a packed add may be.
  if constexpr (FMT == 7) {  // products rounded one by one, summed without loss
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int h = 0; h < 2; ++h)
          two_sum_acc2(hi2[h][r], lo2[h][r],
                       make_float2(__fmul_rn(f[2 * h][v], xv[r][v]), __fmul_rn(f[2 * h + 1][v], xv[r][v])));
  } else {
    // the four rows of a band lie in one 128-row tile: one scale per chunk
    const float s = __ldg(scales + (row0 / 128) * TN + c / 128);
    const float2 s2 = make_float2(s, s);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      constexpr int G = 8;  // products per chain
#pragma unroll
      for (int g = 0; g < V; g += G) {
        float2 xx[G];
#pragma unroll
        for (int e = 0; e < G; ++e) xx[e] = make_float2(xv[r][g + e], xv[r][g + e]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float* fa = f[2 * h] + g;
          const float* fb = f[2 * h + 1] + g;
          float2 p = mul_f2(make_float2(fa[0], fb[0]), xx[0]);
#pragma unroll
          for (int e = 1; e < G; ++e) p = fma_f2(make_float2(fa[e], fb[e]), xx[e], p);
          const float2 ps = make_float2(__fmul_rn(p.x, s), __fmul_rn(p.y, s));
          two_sum_acc2(hi2[h][r], lo2[h][r], ps);
          lo2[h][r] = add_f2(lo2[h][r], fma_f2(p, s2, make_float2(-ps.x, -ps.y)));
        }
      }
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      hi[2 * h][r] = hi2[h][r].x;
      hi[2 * h + 1][r] = hi2[h][r].y;
      lo[2 * h][r] = lo2[h][r].x;
      lo[2 * h + 1][r] = lo2[h][r].y;
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

// Chunks [J, J1) of the band at row0, lane stride STRIDE (two in flight,
// processed in order) into the lane's TwoSum sums.
template <int FMT, int R, int STRIDE>
__device__ __forceinline__ void scaled_piece(const uint8_t* __restrict__ payload, const float* __restrict__ scales,
                                             int64_t M, int64_t N, int64_t ld, int64_t TN, int64_t row0, int64_t J,
                                             int64_t J1, const float* __restrict__ x, int64_t ldx, bool x_fast,
                                             float (&hi)[4][R], float (&lo)[4][R]) {
  constexpr int V = ScaledTraits<FMT>::V;
  for (; J + STRIDE < J1; J += 2 * STRIDE) {
    uint4 r0[4], r1[4];
    scaled_load<FMT>(payload, M, ld, row0, J * V, r0);
    scaled_load<FMT>(payload, M, ld, row0, (J + STRIDE) * V, r1);
    scaled_chunk<FMT, R>(payload, scales, M, N, ld, TN, row0, J * V, r0, x, ldx, x_fast, hi, lo);
    scaled_chunk<FMT, R>(payload, scales, M, N, ld, TN, row0, (J + STRIDE) * V, r1, x, ldx, x_fast, hi, lo);
  }
  if (J < J1) {
    uint4 r0[4];
    scaled_load<FMT>(payload, M, ld, row0, J * V, r0);
    scaled_chunk<FMT, R>(payload, scales, M, N, ld, TN, row0, J * V, r0, x, ldx, x_fast, hi, lo);
  }
}

// GL = 32: the warp takes one piece of a band at a time; GL = 8: four lane
// groups take the next four pieces at once (short bands, where a warp per
// band would spend its time folding).
template <int FMT, int R, int GL>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
    scaled_range_kernel(const uint8_t* __restrict__ payload, const float* __restrict__ scales, int64_t M, int64_t N,
                        int64_t ld, int64_t TN, const float* __restrict__ x, int64_t ldx, bool x_vec_ok, int64_t L,
                        int maxseg, double* __restrict__ ws, double* __restrict__ y, int64_t ldy,
                        double* __restrict__ state, double decay, bool red32) {
  constexpr int V = ScaledTraits<FMT>::V;
  constexpr int NG = 32 / GL;  // pieces taken at once
  const int lane = threadIdx.x & 31;
  const int gl = lane % GL;
  const int64_t g = (int64_t)blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5);
  const int64_t BM = (M + 3) / 4, CB = ld / V;  // bands, chunks per band
  const int64_t total = BM * CB;
  const bool x_fast = x_vec_ok && (N % 4 == 0) && (ld == N);
  int64_t b0 = g * L;
  const int64_t b1 = min(total, b0 + L);
  while (b0 < b1) {
    float hi[4][R], lo[4][R];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int r = 0; r < R; ++r) hi[i][r] = lo[i][r] = 0.f;
    if constexpr (GL == 32) {
      const int64_t I = b0 / CB;
      const int64_t piece_end = min(b1, (I + 1) * CB);
      const int64_t g_lo = (I * CB) / L, g_hi = ((I + 1) * CB - 1) / L;
      scaled_piece<FMT, R, 32>(payload, scales, M, N, ld, TN, 4 * I, b0 - I * CB + lane, piece_end - I * CB, x,
                               ldx, x_fast, hi, lo);
      if (g_lo == g_hi) {
        band_finish<0, R>(hi, lo, lane, 4 * I, M, 0, 1, 4 * BM, ws, y, ldy, state, decay, red32);
      } else {
        band_finish<0, R>(hi, lo, lane, 4 * ((I * maxseg + (g - g_lo)) * R), M, 0, 2, 0, ws, y, ldy, state, decay,
                          red32);
      }
      b0 = piece_end;
    } else {  // lane group lane / GL takes the piece of band b0 / CB + lane / GL
      const int64_t I = b0 / CB + lane / GL;
      const int64_t pb = max(b0, I * CB), pe = min(b1, (I + 1) * CB);
      const bool active = pb < pe;
      const int64_t g_lo = (I * CB) / L, g_hi = ((I + 1) * CB - 1) / L;
      if (active)
        scaled_piece<FMT, R, GL>(payload, scales, M, N, ld, TN, 4 * I, pb - I * CB + gl, pe - I * CB, x, ldx, x_fast,
                                 hi, lo);
      // one call for all groups (the folds shuffle across the whole warp)
      const bool whole = g_lo == g_hi;
      band_finish<0, R, GL>(hi, lo, gl, whole ? 4 * I : 4 * ((I * maxseg + (g - g_lo)) * R), M, 0, whole ? 1 : 2,
                            whole ? 4 * BM : 0, ws, y, ldy, state, decay, red32, active);
      b0 = min(b1, (b0 / CB + NG) * CB);
    }
  }
}

// One persistent launch over all matrices of a batch of one scaled format
// and right-hand-side count (units: the 16-byte column chunks of each 4-row
// band, BN of them per band; the entries' band-major orders one after
// another), split into contiguous warp ranges like scaled_range_kernel's.
template <int FMT, int R>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
    scaled_batched_kernel(const BatchEntry* __restrict__ entries, int nentries, int64_t total, int64_t L) {
  const int lane = threadIdx.x & 31;
  const int64_t g = (int64_t)blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5);
  int64_t b0 = g * L;
  const int64_t b1 = min(total, b0 + L);
  int ei = 0;
  while (b0 < b1) {
    while (ei + 1 < nentries && entries[ei + 1].block_begin <= b0) ++ei;  // warp-uniform
    const BatchEntry& e = entries[ei];
    const int64_t local = b0 - e.block_begin;
    const int64_t I = local / e.BN;
    const int64_t piece_end = min(b1, e.block_begin + (I + 1) * e.BN);
    int64_t g_lo, g_hi;
    batch_band_span(e, I, L, g_lo, g_hi);
    const bool x_vec_ok = (reinterpret_cast<uintptr_t>(e.x) % 16 == 0) && (e.ldx % 4 == 0);
    const bool x_fast = x_vec_ok && (e.N % 4 == 0) && (e.ld == e.N);
    float hi[4][R], lo[4][R];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int r = 0; r < R; ++r) hi[i][r] = lo[i][r] = 0.f;
    scaled_piece<FMT, R, 32>(e.stream, e.scales, e.M, e.N, e.ld, e.TN, 4 * I, local - I * e.BN + lane,
                             piece_end - e.block_begin - I * e.BN, e.x, e.ldx, x_fast, hi, lo);
    if (g_lo == g_hi) {
      band_finish<0, R>(hi, lo, lane, 4 * I, e.M, 0, 1, 4 * e.BM, e.ws, e.y, e.ldy, e.state, e.decay, false);
    } else {
      band_finish<0, R>(hi, lo, lane, 4 * ((I * e.maxseg + (g - g_lo)) * R), e.M, 0, 2, 0, e.ws, e.y, e.ldy,
                        e.state, e.decay, false);
    }
    b0 = piece_end;
  }
}

}  // namespace dev
}  // namespace whff
