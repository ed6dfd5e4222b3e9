// wz3_kernels.cuh -- zfp's fixed-accuracy mode read GPU-first ("WZ3"):
// decode and fused decode + GEMV kernels.
//
// A WZ3 matrix keeps WZ2's blocks (block exponent, shift K, lifted
// coefficients in sequency order, offset-binary fields) but chooses K per
// block for an absolute tolerance and one field width W per run of up to 32
// blocks of a band.  A run is exactly what one warp takes in one iteration:
// lane l decodes block 32 run + l, and since W is the same for the whole run
// the warp switches once, uniformly, onto a field extractor compiled for that
// width (no per-lane prefix sums, no dynamic register indexing).  The run's
// first byte comes from one index entry (offset | W << 56) that every lane
// reads, and its words are interleaved across its blocks (word k of block b
// at word k nb + b), so each of the warp's loads is one coalesced sweep.
// As for WZ2 with the lift, the product works in the transform domain:
// y_band = (2G) sum_J s_J V_J ((2G)^T x_J) 2^-3 with s_J = 2^(E+K-154), the
// (2G) mixing once per band in FP64 (band_finish with the lift's mix).
#pragma once
#include <cstdint>

#include "wz2_kernels.cuh"

namespace whff {
namespace dev {

__host__ __device__ constexpr int wz3_block_bytes(int W) { return 8 * ((13 + 16 * W + 63) / 64); }

template <int W>
struct Wz3Layout {
  static constexpr int kWords = wz3_block_bytes(W) / 4;  // 32-bit words of a block
  static constexpr uint32_t kMask = (1u << W) - 1u;
  static_assert(W >= 1 && W <= 31, "WZ3 field widths are 1..31");
};

template <int W, int K, int NW>
__device__ __forceinline__ uint32_t wz3_field(const uint32_t (&w)[NW]) {
  constexpr int off = 13 + W * K;
  constexpr int wi = off / 32, sh = off % 32;
  if constexpr (sh + W <= 32) {
    return (w[wi] >> sh) & Wz3Layout<W>::kMask;
  } else {
    return __funnelshift_r(w[wi], w[wi + 1], sh) & Wz3Layout<W>::kMask;
  }
}

// The 16 fields of a width-W block, placed in block order (t[4 i + j] for
// coefficient (i, j)): up to 23 bits already OR'd into the mantissa of 2^23
// (so that one packed subtraction of 2^23 + 2^(W-1) gives the exact value),
// wider ones raw.  Only this part depends on W at compile time, so the code a
// run's width selects stays small.
template <int W, int... Ks>
__device__ __forceinline__ void wz3_fields_to(const uint32_t (&w)[16], uint32_t (&t)[16],
                                              std::integer_sequence<int, Ks...>) {
  constexpr uint32_t kOr = W <= 23 ? 0x4B000000u : 0u;
  ((t[seq_index(Ks)] = wz3_field<W, Ks>(w) | kOr), ...);
}

// Fields for the run's width W (1..31), a switch that is uniform over the warp.
__device__ __forceinline__ void wz3_fields_w(int W, const uint32_t (&w)[16], uint32_t (&t)[16]) {
  switch (W) {
#define WZ3_F(WW) \
  case WW:        \
    wz3_fields_to<WW>(w, t, std::make_integer_sequence<int, 16>{}); \
    break;
    WZ3_F(1) WZ3_F(2) WZ3_F(3) WZ3_F(4) WZ3_F(5) WZ3_F(6) WZ3_F(7) WZ3_F(8) WZ3_F(9) WZ3_F(10) WZ3_F(11) WZ3_F(12)
    WZ3_F(13) WZ3_F(14) WZ3_F(15) WZ3_F(16) WZ3_F(17) WZ3_F(18) WZ3_F(19) WZ3_F(20) WZ3_F(21) WZ3_F(22) WZ3_F(23)
    WZ3_F(24) WZ3_F(25) WZ3_F(26) WZ3_F(27) WZ3_F(28) WZ3_F(29) WZ3_F(30)
    default:  // 31 (wider runs are refused when the matrix is made resident)
      wz3_fields_to<31>(w, t, std::make_integer_sequence<int, 16>{});
#undef WZ3_F
  }
}

// The lane's block of a run of nb blocks (word-interleaved: word k of block
// b at word k nb + b of the run), so that each load instruction of the warp
// reads 8 nb consecutive bytes.  An idle lane (past the band's end) and every
// lane of a zero run load nothing.
__device__ __forceinline__ void wz3_load_run(const uint8_t* __restrict__ area, uint64_t e, int lane, int nb,
                                             bool active, uint32_t (&w)[16]) {
  const int W = (int)(e >> 56);
  const int nw = wz3_block_bytes(W) / 8;  // 64-bit words of a block (uniform over the warp)
  const uint2* p = reinterpret_cast<const uint2*>(area + (e & 0x00FFFFFFFFFFFFFFull)) + lane;
  if (active && W != 0) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < nw) {
        const uint2 v = __ldcs(p + k * nb);
        w[2 * k] = v.x;
        w[2 * k + 1] = v.y;
      }
  }
}

// A block's products added into the lane's sums: for each r,
// p_i = s * sum_b V[i][b] xt_r[b] (xt the transformed x of the block's column
// chunk J, ldt floats per column), then hi/lo[i][r] += p_i by TwoSum.  Rows
// (0, 1) and (2, 3) go in packed FP32 pairs; each half rounds as the scalar
// chain (product, three FMAs in b order, the scale, TwoSum) would.
template <int R>
__device__ __forceinline__ void wz3_accumulate(const uint32_t (&w)[16], int W, const float* __restrict__ xt,
                                               int64_t ldt, int J, float (&hi)[4][R], float (&lo)[4][R]) {
  uint32_t t[16];
  wz3_fields_w(W, w, t);
  float2 V[2][4];  // V[h][b] = (value (2h, b), value (2h + 1, b))
  if (W <= 23) {  // exact: (2^23 + field) - (2^23 + 2^(W-1))
    const float bias = 8388608.0f + (float)(1u << (W - 1));
    const float2 b2 = make_float2(bias, bias);
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        V[h][b] = sub_f2(make_float2(__uint_as_float(t[8 * h + b]), __uint_as_float(t[8 * h + 4 + b])), b2);
  } else {  // the integer conversion, round to nearest
    const uint32_t half = 1u << (W - 1);
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        V[h][b] = make_float2(__int2float_rn((int32_t)(t[8 * h + b] - half)),
                              __int2float_rn((int32_t)(t[8 * h + 4 + b] - half)));
  }
  const uint32_t E = w[0] & 0xFFu, K = (w[0] >> 8) & 31u;
  const float s = E ? __uint_as_float((E + K - 27u) << 23) : 0.f;  // 2^(E+K-154); E >= 28 for a nonzero block
  const float2 s2 = make_float2(s, s);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(xt + (int64_t)r * ldt + 4 * J));
    const float2 x0 = make_float2(x.x, x.x), x1 = make_float2(x.y, x.y), x2 = make_float2(x.z, x.z),
                 x3 = make_float2(x.w, x.w);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float2 q = mul_f2(V[h][0], x0);
      q = fma_f2(V[h][1], x1, q);
      q = fma_f2(V[h][2], x2, q);
      q = fma_f2(V[h][3], x3, q);
      float2 H = make_float2(hi[2 * h][r], hi[2 * h + 1][r]), Lo = make_float2(lo[2 * h][r], lo[2 * h + 1][r]);
      two_sum_acc2(H, Lo, mul_f2(q, s2));
      hi[2 * h][r] = H.x, hi[2 * h + 1][r] = H.y, lo[2 * h][r] = Lo.x, lo[2 * h + 1][r] = Lo.y;
    }
  }
}

// Persistent warp ranges over the runs in band-major order (units = runs):
// warp g takes runs [g L, (g + 1) L) of the pass's bands, band I of the pass
// being band0 + I of the matrix (index points at band0's first entry).  A
// band whose runs all lie in the range is finished here (y, state); a band
// shared by several ranges leaves one FP64 partial per range in
// ws[(I maxseg + seg) R + r][4] for the segment epilogue.  The index entry of
// the next run is read while the lanes decode the current one.
template <int R>
__global__ void __launch_bounds__(kWarpsPerCta * 32, R == 1 ? 4 : 1)
    wz3_gemv_kernel(const uint64_t* __restrict__ index, const uint8_t* __restrict__ area, int64_t M, int64_t BM,
                    int BN, int RB, const float* __restrict__ xt, int64_t ldt, int64_t L, int maxseg,
                    double* __restrict__ ws, double* __restrict__ y, int64_t ldy, double* __restrict__ state,
                    double decay) {
  const int lane = threadIdx.x & 31;
  const int64_t g = (int64_t)blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5);
  const int64_t total = BM * RB;
  const int64_t u0 = g * L, u1 = min(total, u0 + L);
  if (u0 >= u1) return;  // warp-uniform; nothing below synchronises across warps
  int64_t I = u0 / RB;  // band of the current piece
  float hi[4][R], lo[4][R];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int r = 0; r < R; ++r) hi[i][r] = lo[i][r] = 0.f;
  uint64_t e_nxt = __ldg(index + u0);  // the same word for every lane
  for (int64_t ub = u0; ub < u1;) {  // the range's piece of band I: runs [ub, ue)
    const int64_t ue = min(u1, (I + 1) * RB);
#pragma unroll 1
    for (int64_t u = ub; u < ue; ++u) {
      const uint64_t e = e_nxt;
      if (u + 1 < u1) e_nxt = __ldg(index + u + 1);
      const int q = (int)(u - I * RB);  // run within the band
      const int nb = min(32, BN - 32 * q);
      const int W = (int)(e >> 56);
      uint32_t w[16];
      wz3_load_run(area, e, lane, nb, lane < nb, w);
      if (W != 0 && lane < nb) wz3_accumulate<R>(w, W, xt, ldt, 32 * q + lane, hi, lo);  // a zero run adds 0
    }
    const int64_t g_lo = (I * RB) / L, g_hi = ((I + 1) * RB - 1) / L;
    if (g_lo == g_hi)
      band_finish<1, R>(hi, lo, lane, 4 * I, M, 0, 1, 4 * BM, ws, y, ldy, state, decay, false);
    else
      band_finish<1, R>(hi, lo, lane, 4 * ((I * maxseg + (g - g_lo)) * R), M, 0, 2, 0, ws, y, ldy, state, decay,
                        false);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int r = 0; r < R; ++r) hi[i][r] = lo[i][r] = 0.f;
    ++I;
    ub = ue;
  }
}

// Decode: thread per block, the exact definition -- T = (2G) V (2G)^T in
// integers, times 2^(K+emax-30) in FP64 (exact) -- written row-major (ldo),
// rows and columns past M, N dropped.
static __global__ void wz3_decompress_kernel(const uint64_t* __restrict__ index, const uint8_t* __restrict__ area,
                                             int64_t M, int64_t N, int64_t BN, int64_t RB, int64_t nblocks,
                                             double* __restrict__ out, int64_t ldo) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblocks) return;
  const int64_t I = b / BN, J = b - I * BN, run = J / 32;
  const uint64_t e = index[I * RB + run];
  const int W = (int)(e >> 56);
  int64_t T[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) T[k] = 0;
  int scale_exp = 0;
  bool zero = W == 0;
  if (!zero) {
    const int nw = wz3_block_bytes(W) / 8;
    const int64_t nb = min((int64_t)32, BN - 32 * run);
    // word-interleaved run: word k of block b at word k nb + b
    const uint64_t* wp = reinterpret_cast<const uint64_t*>(area + (e & 0x00FFFFFFFFFFFFFFull)) + (J - 32 * run);
    uint64_t w[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) w[k] = k < nw ? wp[k * nb] : 0ull;
    const int E = (int)(w[0] & 0xFF), K = (int)((w[0] >> 8) & 31);
    zero = E == 0;
    scale_exp = K + (E - 127) - 30;
    const uint64_t mask = (1ull << W) - 1ull;
    int64_t V[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int o = 13 + W * k, wi = o >> 6, sh = o & 63;
      uint64_t u = w[wi] >> sh;
      if (sh + W > 64) u |= w[wi + 1] << (64 - sh);
      V[seq_index(k)] = (int64_t)(u & mask) - ((int64_t)1 << (W - 1));
    }
    // (2G) applied to the columns, then to the rows
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t s2 = 2 * V[j], x = V[4 + j], yv = V[8 + j], z = V[12 + j];
      V[j] = s2 - x - yv, V[4 + j] = s2 - x + yv, V[8 + j] = s2 + x - yv - z, V[12 + j] = s2 + x + yv + z;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int64_t s2 = 2 * V[4 * r], x = V[4 * r + 1], yv = V[4 * r + 2], z = V[4 * r + 3];
      T[4 * r] = s2 - x - yv, T[4 * r + 1] = s2 - x + yv, T[4 * r + 2] = s2 + x - yv - z,
            T[4 * r + 3] = s2 + x + yv + z;
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t gi = 4 * I + r, gj = 4 * J + c;
      if (gi < M && gj < N) out[gi * ldo + gj] = zero ? 0.0 : ldexp((double)T[4 * r + c], scale_exp);
    }
}

}  // namespace dev
}  // namespace whff
