// wz2_kernels.cuh -- the fixed-allocation variant ("WZ2") of the zfp-style
// fixed-rate format: decode-only and fused decode + GEMV kernels.
//
// Sec. 5.2 finds the zfp decoder sequential (52 % of the run time) and Sec. 6
// asks for GPU-friendly decompression.  WZ2 keeps the 4x4 block and its
// exponent but stores every coefficient in a field of fixed width W at a fixed
// bit offset, so a block decodes with a handful of shifts and masks whose
// positions are compile-time constants.  With the lift taken in its exact
// linear form A_blk = (2G) V (2G)^T * 2^(K+emax-30), the product needs no
// inverse transform per block: y_I = (2G) sum_J s_J V_J ((2G)^T x_J) * 2^-3,
// s_J = 2^(K_J+emax_J-27), so a lane multiplies the stored coefficients with
// the transformed x chunk and the (2G) mixing happens once per 4-row band in
// the FP64 epilogue.
#pragma once
#include <cstdint>
#include <utility>

#include "f32x2.cuh"
#include "gemv_kernels.cuh"
#include "wz2_batch.h"

namespace whff {
namespace dev {

template <int RATE>
struct Wz2Layout {
  static constexpr int kWords = RATE / 2;               // 32-bit words per block
  static constexpr int kW = (16 * RATE - 13) / 16;      // field width
  static constexpr uint32_t kMask = (1u << kW) - 1u;
  static constexpr float kBias = 8388608.0f + (float)(1u << (kW - 1));  // 2^23 + 2^(W-1)
  static_assert(kW >= 7 && kW <= 23, "WZ2 rates 8..24");
};

// Field k (offset-binary) -> float value v, exactly: the field is OR-ed into
// the mantissa of 2^23, then 2^23 + 2^(W-1) is subtracted (exact, |v| < 2^22).
template <int RATE, int K>
__device__ __forceinline__ float wz2_field(const uint32_t (&w)[Wz2Layout<RATE>::kWords]) {
  using L = Wz2Layout<RATE>;
  constexpr int off = 13 + L::kW * K;
  constexpr int wi = off / 32, sh = off % 32;
  uint32_t u;
  if constexpr (sh + L::kW <= 32) {
    u = (w[wi] >> sh) & L::kMask;
  } else {
    u = __funnelshift_r(w[wi], w[wi + 1], sh) & L::kMask;
  }
  return __uint_as_float(u | 0x4B000000u) - L::kBias;
}

template <int RATE>
__device__ __forceinline__ void wz2_fields(const uint32_t (&w)[Wz2Layout<RATE>::kWords], float (&f)[16]) {
  f[0] = wz2_field<RATE, 0>(w);
  f[1] = wz2_field<RATE, 1>(w);
  f[2] = wz2_field<RATE, 2>(w);
  f[3] = wz2_field<RATE, 3>(w);
  f[4] = wz2_field<RATE, 4>(w);
  f[5] = wz2_field<RATE, 5>(w);
  f[6] = wz2_field<RATE, 6>(w);
  f[7] = wz2_field<RATE, 7>(w);
  f[8] = wz2_field<RATE, 8>(w);
  f[9] = wz2_field<RATE, 9>(w);
  f[10] = wz2_field<RATE, 10>(w);
  f[11] = wz2_field<RATE, 11>(w);
  f[12] = wz2_field<RATE, 12>(w);
  f[13] = wz2_field<RATE, 13>(w);
  f[14] = wz2_field<RATE, 14>(w);
  f[15] = wz2_field<RATE, 15>(w);
}

template <int RATE>
__device__ __forceinline__ void wz2_load(const uint8_t* __restrict__ base, int64_t blk,
                                         uint32_t (&w)[Wz2Layout<RATE>::kWords]) {
  constexpr int NW = Wz2Layout<RATE>::kWords;
  const uint8_t* p = base + (uint64_t)blk * (uint64_t)(4 * NW);
  if constexpr (NW % 4 == 0) {
#pragma unroll
    for (int i = 0; i < NW / 4; ++i) {
      const uint4 v = __ldcs(reinterpret_cast<const uint4*>(p) + i);
      w[4 * i] = v.x;
      w[4 * i + 1] = v.y;
      w[4 * i + 2] = v.z;
      w[4 * i + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NW / 2; ++i) {
      const uint2 v = __ldcs(reinterpret_cast<const uint2*>(p) + i);
      w[2 * i] = v.x;
      w[2 * i + 1] = v.y;
    }
  }
}

// Field k of a block, already times the block scale s = 2^e: the field is
// OR-ed into the mantissa of 2^(e+23) (creg = its exponent bits) and
// 2^e (2^23 + 2^(W-1)) (bias) is subtracted -- both exact, so this is
// (field - 2^(W-1)) * s with one logic op and one add.  A zero block passes
// mreg = creg = 0 and bias = 0.
template <int RATE, int K>
__device__ __forceinline__ float wz2_field_scaled(const uint32_t (&w)[Wz2Layout<RATE>::kWords], uint32_t mreg,
                                                  uint32_t creg, float bias) {
  using Lay = Wz2Layout<RATE>;
  constexpr int off = 13 + Lay::kW * K;
  constexpr int wi = off / 32, sh = off % 32;
  uint32_t u;
  if constexpr (sh + Lay::kW <= 32) {
    u = w[wi] >> sh;
  } else {
    u = __funnelshift_r(w[wi], w[wi + 1], sh);
  }
  return __uint_as_float((u & mreg) | creg) - bias;
}

template <int RATE, int... Ks>
__device__ __forceinline__ void wz2_fields_scaled_impl(const uint32_t (&w)[Wz2Layout<RATE>::kWords], uint32_t mreg,
                                                       uint32_t creg, float bias, float (&f)[16],
                                                       std::integer_sequence<int, Ks...>) {
  ((f[Ks] = wz2_field_scaled<RATE, Ks>(w, mreg, creg, bias)), ...);
}

// The 16 coefficients of a block times its scale 2^(E+K-154): the exponent
// trick needs E + K - 4 <= 254 (|a| below about 2^103); larger blocks take
// the exact multiply.
template <int RATE>
__device__ __forceinline__ void wz2_fields_times_scale(const uint32_t (&w)[Wz2Layout<RATE>::kWords], float (&f)[16]) {
  using Lay = Wz2Layout<RATE>;
  const uint32_t E = w[0] & 0xFFu, K = (w[0] >> 8) & 31u;
  if (E + K <= 258u) {
    const uint32_t creg = E ? (E + K - 4u) << 23 : 0u;
    const uint32_t mreg = E ? Lay::kMask : 0u;
    const float bias = E ? __uint_as_float(creg | (1u << (Lay::kW - 1))) : 0.f;
    wz2_fields_scaled_impl<RATE>(w, mreg, creg, bias, f, std::make_integer_sequence<int, 16>{});
  } else {
    const float s = __uint_as_float((E + K - 27u) << 23);
    wz2_fields<RATE>(w, f);
#pragma unroll
    for (int k = 0; k < 16; ++k) f[k] *= s;
  }
}

// Coefficient matrix V (row-major 4x4, index 4a+b) from the fields: sequency
// order with the lift, row-major without.
template <bool LIFT>
__device__ __forceinline__ void wz2_unpermute(const float (&f)[16], float (&V)[16]) {
#pragma unroll
  for (int k = 0; k < 16; ++k) V[LIFT ? seq_index(k) : k] = f[k];
}

// Fold a band's FP64 sums and map them to y: MIX 1 = the lift's 2G mixing
// and 2^-3, MIX 2 = 2^3 (no transform), MIX 0 = identity (scaled formats).
template <bool LIFT, int R, int GL = 32>
__device__ __forceinline__ void wz2_finish(const float (&hi)[4][R], const float (&lo)[4][R], int lane, int64_t row0,
                                           int64_t M, int split, int ksplit, int64_t Mpad, double* __restrict__ ws,
                                           double* __restrict__ y, int64_t ldy, double* __restrict__ state,
                                           double decay, bool red32, bool active = true);

// red32: fold the lanes with the FP32 pair butterfly instead of FP64 (the
// same bar; another rounding).  GL: lanes per band (32, or 8 when a warp
// works on 4 bands at once); lane is the lane within its group, and a group
// with no piece (active = false) folds zeros and writes nothing.  All 32
// lanes must call it together.
template <int MIX, int R, int GL = 32>
__device__ __forceinline__ void band_finish(const float (&hi)[4][R], const float (&lo)[4][R], int lane, int64_t row0,
                                            int64_t M, int split, int ksplit, int64_t Mpad, double* __restrict__ ws,
                                            double* __restrict__ y, int64_t ldy, double* __restrict__ state,
                                            double decay, bool red32, bool active = true) {
  constexpr bool LIFT = MIX == 1;
  double z[4][R];
  if (red32) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int r = 0; r < R; ++r) z[i][r] = warp_sum_pair<GL>(hi[i][r], lo[i][r]);
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int r = 0; r < R; ++r) z[i][r] = warp_sum<GL>((double)hi[i][r] + (double)lo[i][r]);
  }
  if (!active) return;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    double t[4];
    if (LIFT) {  // y = (2G) z * 2^-3, 2G rows (2,-1,-1,0), (2,-1,1,0), (2,1,-1,-1), (2,1,1,1)
      const double a = 2.0 * z[0][r];
      t[0] = (a - z[1][r] - z[2][r]) * 0.125;
      t[1] = (a - z[1][r] + z[2][r]) * 0.125;
      t[2] = (a + z[1][r] - z[2][r] - z[3][r]) * 0.125;
      t[3] = (a + z[1][r] + z[2][r] + z[3][r]) * 0.125;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) t[i] = MIX == 2 ? z[i][r] * 8.0 : z[i][r];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) z[i][r] = t[i];
  }
  // lane (i*R + r) mod GL writes value (i, r)
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (lane != (i * R + r) % GL) continue;
      const int64_t row = row0 + i;
      if (ksplit == 2) {  // segment partial: ws[row0 + r*4 + i] (row0 = 4*(band*maxseg+seg)*R)
        ws[row0 + r * 4 + i] = z[i][r];
      } else if (ksplit > 1) {
        ws[((int64_t)split * R + r) * Mpad + row] = z[i][r];
      } else if (row < M) {
        y[(int64_t)r * ldy + row] = z[i][r];
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
        for (int r = 0; r < R; ++r) s = decay * s + z[i][r];
        state[row] = s;
      }
    }
  }
}

// One block's contribution, scaled: p[i][r] = s * sum_b V[i][b] xt_r[b].
template <bool LIFT, int R, int GL>
__device__ __forceinline__ void wz2_finish(const float (&hi)[4][R], const float (&lo)[4][R], int lane, int64_t row0,
                                           int64_t M, int split, int ksplit, int64_t Mpad, double* __restrict__ ws,
                                           double* __restrict__ y, int64_t ldy, double* __restrict__ state,
                                           double decay, bool red32, bool active) {
  band_finish<LIFT ? 1 : 2, R, GL>(hi, lo, lane, row0, M, split, ksplit, Mpad, ws, y, ldy, state, decay, red32,
                                   active);
}

// The stored-order field of row-major coefficient m (the inverse of seq_index).
__device__ __forceinline__ constexpr int seq_field(int m) {
  constexpr int t[16] = {0, 1, 4, 5, 2, 3, 8, 9, 6, 10, 12, 13, 7, 11, 14, 15};
  return t[m];
}

// Field k's bits with the block exponent OR-ed in (see wz2_field_scaled): a
// float of value 2^(e+23) + field * 2^e.
template <int RATE, int K>
__device__ __forceinline__ uint32_t wz2_field_bits(const uint32_t (&w)[Wz2Layout<RATE>::kWords], uint32_t mreg,
                                                   uint32_t creg) {
  using Lay = Wz2Layout<RATE>;
  constexpr int off = 13 + Lay::kW * K;
  constexpr int wi = off / 32, sh = off % 32;
  uint32_t u;
  if constexpr (sh + Lay::kW <= 32) {
    u = w[wi] >> sh;
  } else {
    u = __funnelshift_r(w[wi], w[wi + 1], sh);
  }
  return (u & mreg) | creg;
}

template <int RATE, int... Ks>
__device__ __forceinline__ void wz2_field_bits_impl(const uint32_t (&w)[Wz2Layout<RATE>::kWords], uint32_t mreg,
                                                    uint32_t creg, uint32_t (&u)[16], std::integer_sequence<int, Ks...>) {
  ((u[Ks] = wz2_field_bits<RATE, Ks>(w, mreg, creg)), ...);
}

// One block's partial for R right-hand sides: p[i][r] = s * sum_b V[i][b] xt_r[b],
// s = 2^(E+K-154) the block scale.  Two arithmetics, one per rate class, the
// same for every R and every kernel at a rate (so a column's bits never depend
// on the other columns of its pass):
//  * rates 8 and 12 (decode-bound: short blocks, many per byte): the scale is
//    folded into the field decode (the exponent trick of
//    wz2_fields_times_scale) and a row's four products are two packed FP32
//    pairs of columns, (V0 xt0 + V2 xt2) + (V1 xt1 + V3 xt3) -- 14 fewer
//    instructions per block and right-hand side.  Working on values scaled by a
//    power of two rounds exactly like scaling at the end.  Blocks above about
//    2^103 (the trick's exponent limit) decode unscaled and take s at the end.
//  * rates 16 and up (HBM-bound): fields by the 2^23 trick, the scalar chain
//    ((V0 xt0 + V1 xt1) + V2 xt2) + V3 xt3 with FMAs, then s (measured faster
//    there: the packed form needs more registers per block in flight).
// PRE: x already holds (2G)^T x per 4-column chunk (wz2_xt_kernel), so the
// lift's transform of x is not repeated per block.
template <int RATE>
__host__ __device__ constexpr bool wz2_packed() {
  return RATE <= 12;
}

template <int RATE, bool LIFT, int R, bool PRE = false>
__device__ __forceinline__ void wz2_block_partial(const uint32_t (&w)[Wz2Layout<RATE>::kWords],
                                                  const float* __restrict__ x, int64_t ldx, int64_t c0, int64_t N,
                                                  bool x_fast, bool x_vec_ok, float (&p)[4][R]) {
  using Lay = Wz2Layout<RATE>;
  const uint32_t E = w[0] & 0xFFu;
  const uint32_t K = (w[0] >> 8) & 31u;
  if constexpr (wz2_packed<RATE>()) {
    const bool trick = E + K <= 258u;
    // trick: the field OR-ed into the mantissa of 2^(e+23), e = E+K-154; else of
    // 2^23 (unscaled).  A zero block (E = 0) decodes to 0.
    const uint32_t creg = trick ? (E ? (E + K - 4u) << 23 : 0u) : 0x4B000000u;
    const uint32_t mreg = E ? Lay::kMask : 0u;
    const float bias = E ? __uint_as_float(creg | (1u << (Lay::kW - 1))) : 0.f;
    uint32_t u[16];
    wz2_field_bits_impl<RATE>(w, mreg, creg, u, std::make_integer_sequence<int, 16>{});
    const float2 b2 = make_float2(bias, bias);
    float2 P[4][2];  // P[i][h] = (V[i][2h], V[i][2h+1])
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m0 = 4 * i + 2 * h, m1 = m0 + 1;
        const int k0 = LIFT ? seq_field(m0) : m0, k1 = LIFT ? seq_field(m1) : m1;
        P[i][h] = sub_f2(make_float2(__uint_as_float(u[k0]), __uint_as_float(u[k1])), b2);
      }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float4 xv = x_fast ? __ldg(reinterpret_cast<const float4*>(x + (int64_t)r * ldx + c0))
                               : load_x4(x, ldx, r, c0, N, x_vec_ok);
      float2 X0, X1;
      if (LIFT && !PRE) {  // (2G)^T x
        const float a = xv.x + xv.y, b = xv.z + xv.w, c = xv.x + xv.z, d = xv.y + xv.w;
        X0 = make_float2(2.f * (a + b), b - a);
        X1 = make_float2(d - c, xv.w - xv.z);
      } else {
        X0 = make_float2(xv.x, xv.y);
        X1 = make_float2(xv.z, xv.w);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 q = fma_f2(P[i][1], X1, mul_f2(P[i][0], X0));
        p[i][r] = __fadd_rn(q.x, q.y);
      }
    }
    if (!trick) {
      const float s = __uint_as_float((E + K - 27u) << 23);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int r = 0; r < R; ++r) p[i][r] = __fmul_rn(p[i][r], s);
    }
  } else {
    // 2^(emax+K-27) is always a normal float; a zero block (E = 0) scales by 0
    const float s = E ? __uint_as_float((E + K - 27u) << 23) : 0.f;
    float f[16], V[16];
    wz2_fields<RATE>(w, f);
    wz2_unpermute<LIFT>(f, V);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float4 xv = x_fast ? __ldg(reinterpret_cast<const float4*>(x + (int64_t)r * ldx + c0))
                               : load_x4(x, ldx, r, c0, N, x_vec_ok);
      float xt[4];
      if (LIFT && !PRE) {  // (2G)^T x
        const float a = xv.x + xv.y, b = xv.z + xv.w, c = xv.x + xv.z, d = xv.y + xv.w;
        xt[0] = 2.f * (a + b);
        xt[1] = b - a;
        xt[2] = d - c;
        xt[3] = xv.w - xv.z;
      } else {
        xt[0] = xv.x;
        xt[1] = xv.y;
        xt[2] = xv.z;
        xt[3] = xv.w;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float q = V[4 * i] * xt[0];
        q = fmaf(V[4 * i + 1], xt[1], q);
        q = fmaf(V[4 * i + 2], xt[2], q);
        q = fmaf(V[4 * i + 3], xt[3], q);
        p[i][r] = q * s;
      }
    }
  }
}

// A pair of blocks' partials into the lane's TwoSum sums: (p0 + p1) per row
// and right-hand side.  At the packed rates the rows go in FP32 pairs (rows
// 0-1, 2-3); each half rounds as the scalar TwoSum, so the bits are the same.
template <int RATE, int R>
__device__ __forceinline__ void wz2_acc_pair(float (&hi)[4][R], float (&lo)[4][R], const float (&p0)[4][R],
                                             const float (&p1)[4][R]) {
  if constexpr (wz2_packed<RATE>()) {
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float2 H = make_float2(hi[2 * h][r], hi[2 * h + 1][r]), Lo = make_float2(lo[2 * h][r], lo[2 * h + 1][r]);
        two_sum_acc2(H, Lo, add_f2(make_float2(p0[2 * h][r], p0[2 * h + 1][r]), make_float2(p1[2 * h][r], p1[2 * h + 1][r])));
        hi[2 * h][r] = H.x, hi[2 * h + 1][r] = H.y, lo[2 * h][r] = Lo.x, lo[2 * h + 1][r] = Lo.y;
      }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int r = 0; r < R; ++r) two_sum_acc(hi[i][r], lo[i][r], p0[i][r] + p1[i][r]);
  }
}

// One block's partial alone (a lane's odd last block of a piece).
template <int RATE, int R>
__device__ __forceinline__ void wz2_acc_one(float (&hi)[4][R], float (&lo)[4][R], const float (&p0)[4][R]) {
  if constexpr (wz2_packed<RATE>()) {
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float2 H = make_float2(hi[2 * h][r], hi[2 * h + 1][r]), Lo = make_float2(lo[2 * h][r], lo[2 * h + 1][r]);
        two_sum_acc2(H, Lo, make_float2(p0[2 * h][r], p0[2 * h + 1][r]));
        hi[2 * h][r] = H.x, hi[2 * h + 1][r] = H.y, lo[2 * h][r] = Lo.x, lo[2 * h + 1][r] = Lo.y;
      }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int r = 0; r < R; ++r) two_sum_acc(hi[i][r], lo[i][r], p0[i][r]);
  }
}

// Accumulate the blocks [J0, J1) of one 4-row band (lane l takes J0+l,
// J0+l+32, ...) into the lane's TwoSum sums.  The arithmetic is fixed: the
// lane's blocks are taken in pairs (its 1st and 2nd, 3rd and 4th, ...), each
// pair's two scaled partials are added and the sum enters the TwoSum; an odd
// last block enters alone.  So every right-hand side gets the same rounding
// whatever R, UNROLL or the batch it is in.  UNROLL (2, 4 or 8) blocks per lane
// are kept in flight: their loads are issued before any is decoded.
template <int RATE, bool LIFT, int R, int UNROLL, int STRIDE = 32, bool PRE = false>
__device__ __forceinline__ void wz2_piece(const uint8_t* __restrict__ base, int64_t J0, int64_t J1, int lane,
                                          const float* __restrict__ x, int64_t ldx, int64_t N, bool x_fast,
                                          bool x_vec_ok, float (&hi)[4][R], float (&lo)[4][R]) {
  static_assert(UNROLL == 2 || UNROLL == 4 || UNROLL == 8, "blocks are consumed in pairs");
  constexpr int NW = Wz2Layout<RATE>::kWords;
  int64_t J = J0 + lane;
  for (; J + STRIDE * (UNROLL - 1) < J1; J += STRIDE * UNROLL) {
    uint32_t w[UNROLL][NW];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) wz2_load<RATE>(base, J + STRIDE * u, w[u]);
#pragma unroll
    for (int u = 0; u < UNROLL; u += 2) {
      float p0[4][R], p1[4][R];
      wz2_block_partial<RATE, LIFT, R, PRE>(w[u], x, ldx, 4 * (J + STRIDE * u), N, x_fast, x_vec_ok, p0);
      wz2_block_partial<RATE, LIFT, R, PRE>(w[u + 1], x, ldx, 4 * (J + STRIDE * (u + 1)), N, x_fast, x_vec_ok, p1);
      wz2_acc_pair<RATE, R>(hi, lo, p0, p1);
    }
  }
  for (; J + STRIDE < J1; J += 2 * STRIDE) {  // remaining whole pairs
    uint32_t w0[NW], w1[NW];
    wz2_load<RATE>(base, J, w0);
    wz2_load<RATE>(base, J + STRIDE, w1);
    float p0[4][R], p1[4][R];
    wz2_block_partial<RATE, LIFT, R, PRE>(w0, x, ldx, 4 * J, N, x_fast, x_vec_ok, p0);
    wz2_block_partial<RATE, LIFT, R, PRE>(w1, x, ldx, 4 * (J + STRIDE), N, x_fast, x_vec_ok, p1);
    wz2_acc_pair<RATE, R>(hi, lo, p0, p1);
  }
  if (J < J1) {  // odd last block
    uint32_t w0[NW];
    wz2_load<RATE>(base, J, w0);
    float p0[4][R];
    wz2_block_partial<RATE, LIFT, R, PRE>(w0, x, ldx, 4 * J, N, x_fast, x_vec_ok, p0);
    wz2_acc_one<RATE, R>(hi, lo, p0);
  }
}

// (2G)^T x_J for every 4-column chunk J and right-hand side r, once per pass:
// xt[r * ldt + 4J + i], the same FP32 operations in the same order as the
// per-block transform, so the results do not change.  Thread per (r, J).
static __global__ void wz2_xt_kernel(const float* __restrict__ x, int64_t ldx, int64_t N, int R, int64_t BN,
                                     float* __restrict__ xt, int64_t ldt) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)R * BN) return;
  const int r = (int)(q / BN);
  const int64_t J = q - (int64_t)r * BN;
  float xv[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) xv[c] = 4 * J + c < N ? x[(int64_t)r * ldx + 4 * J + c] : 0.f;
  const float a = xv[0] + xv[1], b = xv[2] + xv[3], c = xv[0] + xv[2], d = xv[1] + xv[3];
  *reinterpret_cast<float4*>(xt + (int64_t)r * ldt + 4 * J) = make_float4(2.f * (a + b), b - a, d - c, xv[3] - xv[2]);
}

// Persistent kernel with exact balance: the G warps of the grid split the
// band-major sequence of all BM*BN blocks into G contiguous ranges of L
// blocks.  A range covers pieces of one to a few 4-row bands; for every piece
// the lanes' sums are folded and either y (and the state) is written
// directly, when the band lies inside one range, or the piece's partial goes
// to ws[band][segment] for wz2_segment_epilogue, which adds a band's segments
// in order.  GL = 32: the warp takes one piece at a time; GL = 8: four lane
// groups take the next four pieces at once (short bands, where a warp per
// band would spend its time folding).  With the lift, x is the transformed
// vector of wz2_xt_kernel (4 BN floats per right-hand side).
template <int RATE, bool LIFT, int R, int UNROLL, int GL>
__device__ __forceinline__ void wz2_gemv_body(const uint8_t* __restrict__ stream, int64_t M, int64_t N, int64_t BM,
                                              int64_t BN, const float* __restrict__ x, int64_t ldx, bool x_vec_ok,
                                              int64_t L, int maxseg, double* __restrict__ ws, double* __restrict__ y,
                                              int64_t ldy, double* __restrict__ state, double decay, bool red32) {
  constexpr int64_t kBlockBytes = 4 * Wz2Layout<RATE>::kWords;
  constexpr int NG = 32 / GL;  // pieces taken at once
  const int lane = threadIdx.x & 31;
  const int gl = lane % GL;
  const int64_t g = (int64_t)blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5);
  const int64_t total = BM * BN;
  const bool x_fast = x_vec_ok && (N % 4 == 0);
  int64_t b0 = g * L;
  const int64_t b1 = min(total, b0 + L);
  while (b0 < b1) {
    float hi[4][R], lo[4][R];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int r = 0; r < R; ++r) hi[i][r] = lo[i][r] = 0.f;
    if constexpr (GL == 32) {  // the warp takes the piece starting at b0
      const int64_t I = b0 / BN;
      const int64_t piece_end = min(b1, (I + 1) * BN);
      const int64_t g_lo = (I * BN) / L, g_hi = ((I + 1) * BN - 1) / L;
      wz2_piece<RATE, LIFT, R, UNROLL, 32, LIFT>(stream + (uint64_t)(I * BN) * kBlockBytes, b0 - I * BN,
                                                 piece_end - I * BN, lane, x, ldx, N, x_fast, x_vec_ok, hi, lo);
      if (g_lo == g_hi) {  // the whole band is in this range: finish it here
        wz2_finish<LIFT, R>(hi, lo, lane, 4 * I, M, 0, 1, 4 * BM, ws, y, ldy, state, decay, red32);
      } else {  // one segment of a shared band: ws[(band * maxseg + seg) * R + r][i]
        wz2_finish<LIFT, R>(hi, lo, lane, 4 * ((I * maxseg + (g - g_lo)) * R), M, 0, 2, 0, ws, y, ldy, state,
                            decay, red32);
      }
      b0 = piece_end;
    } else {  // lane group lane / GL takes the piece of band b0 / BN + lane / GL
      const int64_t I = b0 / BN + lane / GL;
      const int64_t pb = max(b0, I * BN), pe = min(b1, (I + 1) * BN);
      const bool active = pb < pe;
      const int64_t g_lo = (I * BN) / L, g_hi = ((I + 1) * BN - 1) / L;
      if (active)
        wz2_piece<RATE, LIFT, R, UNROLL, GL, LIFT>(stream + (uint64_t)(I * BN) * kBlockBytes, pb - I * BN,
                                                   pe - I * BN, gl, x, ldx, N, x_fast, x_vec_ok, hi, lo);
      // one call for all groups (the folds shuffle across the whole warp)
      const bool whole = g_lo == g_hi;
      wz2_finish<LIFT, R, GL>(hi, lo, gl, whole ? 4 * I : 4 * ((I * maxseg + (g - g_lo)) * R), M, 0, whole ? 1 : 2,
                              whole ? 4 * BM : 0, ws, y, ldy, state, decay, red32, active);
      b0 = min(b1, (b0 / BN + NG) * BN);
    }
  }
}

// The persistent kernel (body above).  Its packed unroll-4 instantiation
// (rates 8 and 12) is held to 3 resident CTAs per SM; every other one keeps
// the compiler's default register budget.
template <int RATE, bool LIFT, int R, int UNROLL, int GL>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
    wz2_gemv_kernel(const uint8_t* __restrict__ stream, int64_t M, int64_t N, int64_t BM, int64_t BN,
                    const float* __restrict__ x, int64_t ldx, bool x_vec_ok, int64_t L, int maxseg,
                    double* __restrict__ ws, double* __restrict__ y, int64_t ldy, double* __restrict__ state,
                    double decay, bool red32) {
  wz2_gemv_body<RATE, LIFT, R, UNROLL, GL>(stream, M, N, BM, BN, x, ldx, x_vec_ok, L, maxseg, ws, y, ldy, state,
                                           decay, red32);
}

template <int RATE, bool LIFT, int R, int UNROLL, int GL>
__global__ void __launch_bounds__(kWarpsPerCta * 32, 3)
    wz2_gemv_kernel_o3(const uint8_t* __restrict__ stream, int64_t M, int64_t N, int64_t BM, int64_t BN,
                       const float* __restrict__ x, int64_t ldx, bool x_vec_ok, int64_t L, int maxseg,
                       double* __restrict__ ws, double* __restrict__ y, int64_t ldy, double* __restrict__ state,
                       double decay, bool red32) {
  wz2_gemv_body<RATE, LIFT, R, UNROLL, GL>(stream, M, N, BM, BN, x, ldx, x_vec_ok, L, maxseg, ws, y, ldy, state,
                                           decay, red32);
}

// The instantiation a launch uses.
template <int RATE, bool LIFT, int R, int UNROLL, int GL>
constexpr auto wz2_gemv_entry() {
  if constexpr (wz2_packed<RATE>() && R == 1 && UNROLL == 4)
    return &wz2_gemv_kernel_o3<RATE, LIFT, R, UNROLL, GL>;
  else
    return &wz2_gemv_kernel<RATE, LIFT, R, UNROLL, GL>;
}

// sum_{k < n} p[k * stride], added in k order; the loads of eight terms are
// issued before their additions (a band split over many warp ranges -- a slit
// of a long matrix -- has dozens of segments, and one load per dependent add
// would serialise their latencies).  Same rounding as the plain loop.
__device__ __forceinline__ double seq_sum_strided(const double* __restrict__ p, int64_t n, int64_t stride) {
  double t = 0.0;
  int64_t k = 0;
  for (; k + 8 <= n; k += 8) {
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = p[(k + j) * stride];
#pragma unroll
    for (int j = 0; j < 8; ++j) t += v[j];
  }
  for (; k < n; ++k) t += p[k * stride];
  return t;
}

// Sum the segments of bands shared by several warp ranges, then the state
// update (bands inside one range were finished by the kernel).  The shared
// bands are exactly those with a range boundary b = g L strictly inside them
// (b not a multiple of BN); each is taken by the warp of its first such
// boundary, so the launch has a warp per boundary (segment_epilogue_threads),
// not a thread per row.  In that warp, 8 lanes per row of the band: lane j
// adds segments j, j + 8, ... in order, then a fixed xor tree over the eight
// (the same order every time, so the result is deterministic; with one or two
// segments it is the plain sum).  A slit of a long matrix has dozens of
// segments per band: eight lanes keep their loads in flight together.
__host__ __device__ inline int64_t segment_epilogue_threads(int64_t M, int64_t BN, int64_t L) {
  const int64_t total = ((M + 3) / 4) * BN, ranges = (total + L - 1) / L;
  return ranges > 1 ? 32 * (ranges - 1) : 0;
}

static __global__ void wz2_segment_epilogue(const double* __restrict__ ws, int64_t M, int64_t BN, int64_t L,
                                            int maxseg, int R, double* __restrict__ y, int64_t ldy,
                                            double* __restrict__ state, double decay) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t g = 1 + (q >> 5);  // the boundary of this warp (warp-uniform)
  const int i = (int)((q & 31) >> 3), j = (int)(q & 7);
  const int64_t b = g * L, total = ((M + 3) / 4) * BN;
  const int64_t I = b / BN;
  // a boundary inside band I, and the first one there (the previous one is not inside I)
  const bool mine = b < total && b % BN != 0 && (g - 1) * L <= I * BN;
  const int64_t row = 4 * I + i;
  const bool valid = mine && row < M;
  const int64_t g_lo = (I * BN) / L, g_hi = ((I + 1) * BN - 1) / L;
  double s = (valid && state) ? state[row] : 0.0;
  for (int r = 0; r < R; ++r) {
    double t = 0.0;
    if (valid)
      for (int64_t seg = j; seg <= g_hi - g_lo; seg += 8) t += ws[((I * maxseg + seg) * R + r) * 4 + i];
#pragma unroll
    for (int o = 4; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (valid && j == 0) {
      y[(int64_t)r * ldy + row] = t;
      s = decay * s + t;
    }
  }
  if (valid && j == 0 && state) state[row] = s;
}

// ------------------------------------------------------------- batched launch
// First global block of band I of entry e, and its warp-range span.
__device__ __forceinline__ void batch_band_span(const BatchEntry& e, int64_t I, int64_t L, int64_t& g_lo,
                                                int64_t& g_hi) {
  const int64_t first = e.block_begin + I * e.BN;
  g_lo = first / L;
  g_hi = (first + e.BN - 1) / L;
}

// One persistent launch over all matrices of a batch that share a format,
// rate and right-hand-side count: the global block order is the entries'
// band-major orders one after another, split into contiguous warp ranges
// exactly as for a single matrix.
template <int RATE, bool LIFT, int R, int UNROLL>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
    wz2_batched_kernel(const BatchEntry* __restrict__ entries, int nentries, int64_t total, int64_t L) {
  constexpr int64_t kBlockBytes = 4 * Wz2Layout<RATE>::kWords;
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
    const bool x_fast = x_vec_ok && (e.N % 4 == 0);
    float hi[4][R], lo[4][R];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int r = 0; r < R; ++r) hi[i][r] = lo[i][r] = 0.f;
    wz2_piece<RATE, LIFT, R, UNROLL>(e.stream + (uint64_t)(I * e.BN) * kBlockBytes, local - I * e.BN,
                                     piece_end - e.block_begin - I * e.BN, lane, e.x, e.ldx, e.N, x_fast, x_vec_ok,
                                     hi, lo);
    if (g_lo == g_hi) {
      wz2_finish<LIFT, R>(hi, lo, lane, 4 * I, e.M, 0, 1, 4 * e.BM, e.ws, e.y, e.ldy, e.state, e.decay, false);
    } else {
      wz2_finish<LIFT, R>(hi, lo, lane, 4 * ((I * e.maxseg + (g - g_lo)) * R), e.M, 0, 2, 0, e.ws, e.y, e.ldy,
                          e.state, e.decay, false);
    }
    b0 = piece_end;
  }
}

// State update of a batch, after every column group has written y: thread per
// (matrix, row), rows of matrix k are global rows [row_begin[k], +M_k).
static __global__ void wz2_batched_state(const BatchState* __restrict__ st, const int64_t* __restrict__ row_begin,
                                         int n, int64_t total_rows) {
  const int64_t grow = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (grow >= total_rows) return;
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (row_begin[mid] <= grow) lo = mid; else hi = mid - 1;
  }
  const BatchState& b = st[lo];
  if (!b.state) return;
  const int64_t row = grow - row_begin[lo];
  double s = b.state[row];
  for (int r = 0; r < b.R; ++r) s = b.decay * s + b.y[(int64_t)r * b.ldy + row];
  b.state[row] = s;
}

// Segment epilogue of a batch: thread per (entry, row); rows of entry e are
// global rows [row_begin[e], row_begin[e] + M_e).
static __global__ void wz2_batched_epilogue(const BatchEntry* __restrict__ entries, const int64_t* __restrict__ row_begin,
                                            int nentries, int64_t total_rows, int64_t L, int R) {
  const int64_t grow = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (grow >= total_rows) return;
  int lo = 0, hi = nentries - 1;  // last entry with row_begin <= grow
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (row_begin[mid] <= grow) lo = mid; else hi = mid - 1;
  }
  const BatchEntry& e = entries[lo];
  const int64_t row = grow - row_begin[lo];
  const int64_t I = row / 4;
  const int i = (int)(row % 4);
  int64_t g_lo, g_hi;
  batch_band_span(e, I, L, g_lo, g_hi);
  if (g_lo == g_hi) return;
  double s = e.state ? e.state[row] : 0.0;
  for (int r = 0; r < R; ++r) {
    const double t = seq_sum_strided(e.ws + ((I * e.maxseg) * R + r) * 4 + i, g_hi - g_lo + 1, (int64_t)R * 4);
    e.y[(int64_t)r * e.ldy + row] = t;
    s = e.decay * s + t;
  }
  if (e.state) e.state[row] = s;
}

template <int RATE, bool LIFT>
__global__ void wz2_decompress_kernel(const uint8_t* __restrict__ stream, int64_t M, int64_t N, int64_t BN,
                                      int64_t nblocks, double* __restrict__ out, int64_t ldo) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblocks) return;
  const int64_t I = b / BN, J = b - (b / BN) * BN;
  uint32_t w[Wz2Layout<RATE>::kWords];
  wz2_load<RATE>(stream, b, w);
  const int E = (int)(w[0] & 0xFFu);
  const int K = (int)((w[0] >> 8) & 31u);
  float f[16], Vf[16];
  wz2_fields<RATE>(w, f);
  wz2_unpermute<LIFT>(f, Vf);
  int32_t T[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) T[i] = (int32_t)Vf[i];  // exact: |v| < 2^22
  double scale;
  if (LIFT) {
    // T = (2G) V (2G)^T, integers below 2^27: columns, then rows
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int s0 = pass ? 1 : 4, s1 = pass ? 4 : 1;  // pass 0: along a (stride 4); pass 1: along b
        int32_t& v0 = T[j * s1];
        int32_t& v1 = T[j * s1 + s0];
        int32_t& v2 = T[j * s1 + 2 * s0];
        int32_t& v3 = T[j * s1 + 3 * s0];
        const int32_t a = 2 * v0;
        const int32_t r0 = a - v1 - v2, r1 = a - v1 + v2, r2 = a + v1 - v2 - v3, r3 = a + v1 + v2 + v3;
        v0 = r0;
        v1 = r1;
        v2 = r2;
        v3 = r3;
      }
    }
    scale = ldexp(1.0, K + (E - 127) - 30);
  } else {
    scale = ldexp(1.0, K + (E - 127) - 24);
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t row = 4 * I + r;
    if (row >= M) break;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t col = 4 * J + c;
      if (col < N) out[row * ldo + col] = E ? (double)T[4 * r + c] * scale : 0.0;
    }
  }
}

}  // namespace dev
}  // namespace whff
