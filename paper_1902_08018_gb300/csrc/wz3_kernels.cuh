// wz3_kernels.cuh -- zfp's fixed-accuracy mode read GPU-first ("WZ3"):
// decode and fused decode + GEMV kernels.
//
// A WZ3 matrix keeps WZ2's blocks (block exponent, shift K, lifted
// coefficients in sequency order, offset-binary fields) but chooses K per
// block for an absolute tolerance and one field width W per run of up to 32
// blocks of a band.  A run is exactly what one warp takes in one iteration:
// lane l decodes block 32 run + l, and since W is the same for the whole run
// the warp switches once, uniformly, onto a decoder compiled for that width
// (no per-lane prefix sums, no dynamic register indexing).  The run's first
// byte comes from one index entry (offset | W << 56) that every lane reads.
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

// The 16 raw fields of a width-W block in sequency order (offset binary, no
// conversion): the only part of the decode that depends on W at compile time,
// so the code that a run's width selects stays small.
template <int W, int... Ks>
__device__ __forceinline__ void wz3_raw_impl(const uint32_t (&w)[16], uint32_t (&u)[16],
                                             std::integer_sequence<int, Ks...>) {
  ((u[Ks] = wz3_field<W, Ks>(w)), ...);
}

// Raw fields for the run's width W (1..31), a switch that is uniform over the warp.
__device__ __forceinline__ void wz3_raw(int W, const uint32_t (&w)[16], uint32_t (&u)[16]) {
  switch (W) {
#define WZ3_RAW(WW) \
  case WW:          \
    wz3_raw_impl<WW>(w, u, std::make_integer_sequence<int, 16>{}); \
    break;
    WZ3_RAW(1) WZ3_RAW(2) WZ3_RAW(3) WZ3_RAW(4) WZ3_RAW(5) WZ3_RAW(6) WZ3_RAW(7) WZ3_RAW(8) WZ3_RAW(9) WZ3_RAW(10)
    WZ3_RAW(11) WZ3_RAW(12) WZ3_RAW(13) WZ3_RAW(14) WZ3_RAW(15) WZ3_RAW(16) WZ3_RAW(17) WZ3_RAW(18) WZ3_RAW(19)
    WZ3_RAW(20) WZ3_RAW(21) WZ3_RAW(22) WZ3_RAW(23) WZ3_RAW(24) WZ3_RAW(25) WZ3_RAW(26) WZ3_RAW(27) WZ3_RAW(28)
    WZ3_RAW(29) WZ3_RAW(30)
    default:  // 31 (wider runs are refused when the matrix is made resident)
      wz3_raw_impl<31>(w, u, std::make_integer_sequence<int, 16>{});
#undef WZ3_RAW
  }
}

// Offset-binary fields -> values in block order: exact through the 2^23
// mantissa up to 23 bits, else the integer conversion (round to nearest; the
// FP32 product rounds anyway).
__device__ __forceinline__ void wz3_values(int W, const uint32_t (&u)[16], float (&V)[16]) {
  const uint32_t half = 1u << (W - 1);
  if (W <= 23) {
    const float bias = 8388608.0f + (float)half;
#pragma unroll
    for (int k = 0; k < 16; ++k) V[seq_index(k)] = __uint_as_float(u[k] | 0x4B000000u) - bias;
  } else {
#pragma unroll
    for (int k = 0; k < 16; ++k) V[seq_index(k)] = __int2float_rn((int32_t)(u[k] - half));
  }
}

// The lane's block of a run: its words (zeros past the block or for an idle lane).
__device__ __forceinline__ void wz3_load_run(const uint8_t* __restrict__ area, uint64_t e, int lane, bool active,
                                             uint32_t (&w)[16]) {
  const int W = (int)(e >> 56);
  const int nw2 = wz3_block_bytes(W) / 8;  // 8-byte words of the block
  const uint2* p = reinterpret_cast<const uint2*>(area + (e & 0x00FFFFFFFFFFFFFFull) +
                                                  (uint64_t)lane * (uint64_t)wz3_block_bytes(W));
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    uint2 v = make_uint2(0u, 0u);
    if (active && i < nw2) v = __ldcs(p + i);
    w[2 * i] = v.x;
    w[2 * i + 1] = v.y;
  }
}

// A block's products added into the lane's sums: for each r,
// p_i = s * sum_b V[i][b] xt_r[b] (xt the transformed x of the block's column
// chunk J, ldt floats per column), then hi/lo[i][r] += p_i by TwoSum.
template <int R>
__device__ __forceinline__ void wz3_accumulate(const uint32_t (&w)[16], int W, const float* __restrict__ xt,
                                               int64_t ldt, int64_t J, float (&hi)[4][R], float (&lo)[4][R]) {
  uint32_t u[16];
  wz3_raw(W, w, u);
  float V[16];
  wz3_values(W, u, V);
  const uint32_t E = w[0] & 0xFFu, K = (w[0] >> 8) & 31u;
  const float s = E ? __uint_as_float((E + K - 27u) << 23) : 0.f;  // 2^(E+K-154); E >= 28 for a nonzero block
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(xt + (int64_t)r * ldt + 4 * J));
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float q = __fmul_rn(V[4 * i], x.x);
      q = fmaf(V[4 * i + 1], x.y, q);
      q = fmaf(V[4 * i + 2], x.z, q);
      q = fmaf(V[4 * i + 3], x.w, q);
      two_sum_acc(hi[i][r], lo[i][r], __fmul_rn(q, s));
    }
  }
}

// A warp per (band, split): band I of this pass (band0 + I of the matrix),
// runs [split chunk, split chunk + chunk) of it, R right-hand sides (1 or 8).
// With one right-hand side the loop is software-pipelined: while the lanes
// decode run r, the words of run r + 1 are on their way and the index entry
// of run r + 2 is read (with eight, the products hide the loads).
// ksplit > 1: the band's mixed partial goes to ws[(split R + r) Mpad + row]
// (the split-K epilogue adds the splits in order and applies the state).
template <int R>
__global__ void __launch_bounds__(kWarpsPerCta * 32, R == 1 ? 4 : 2)
    wz3_gemv_kernel(const uint64_t* __restrict__ index, const uint8_t* __restrict__ area, int64_t band0, int64_t M,
                    int64_t BM, int64_t BN, int64_t RB, const float* __restrict__ xt, int64_t ldt, int ksplit,
                    int64_t chunk, double* __restrict__ ws, double* __restrict__ y, int64_t ldy,
                    double* __restrict__ state, double decay) {
  constexpr bool kPipe = R == 1;
  const int lane = threadIdx.x & 31;
  const int64_t I = (int64_t)blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5);
  if (I >= BM) return;  // warp-uniform; nothing below synchronises across warps
  const int split = (int)blockIdx.y;
  const int64_t r0 = (int64_t)split * chunk, r1 = min(RB, r0 + chunk);
  const uint64_t* idx = index + (band0 + I) * RB;  // one entry per run, the same word for every lane
  float hi[4][R], lo[4][R];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int r = 0; r < R; ++r) hi[i][r] = lo[i][r] = 0.f;
  uint64_t e_cur = r0 < r1 ? __ldg(idx + r0) : 0ull;
  uint64_t e_nxt = kPipe && r0 + 1 < r1 ? __ldg(idx + r0 + 1) : 0ull;
  uint32_t w_cur[16];
  if constexpr (kPipe) wz3_load_run(area, e_cur, lane, r0 < r1 && 32 * r0 + lane < BN, w_cur);
  for (int64_t run = r0; run < r1; ++run) {
    uint32_t w_nxt[16];
    uint64_t e_after = 0;
    if constexpr (kPipe) {
      wz3_load_run(area, e_nxt, lane, run + 1 < r1 && 32 * (run + 1) + lane < BN, w_nxt);
      e_after = run + 2 < r1 ? __ldg(idx + run + 2) : 0ull;
    } else {
      e_cur = __ldg(idx + run);
      wz3_load_run(area, e_cur, lane, 32 * run + lane < BN, w_cur);
    }
    const int W = (int)(e_cur >> 56);
    const int64_t J = 32 * run + lane;
    if (W != 0 && J < BN) wz3_accumulate<R>(w_cur, W, xt, ldt, J, hi, lo);  // a zero run decodes to zeros
    if constexpr (kPipe) {
#pragma unroll
      for (int k = 0; k < 16; ++k) w_cur[k] = w_nxt[k];
      e_cur = e_nxt;
      e_nxt = e_after;
    }
  }
  band_finish<1, R>(hi, lo, lane, 4 * I, M, split, ksplit, 4 * BM, ws, y, ldy, state, decay, false);
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
    const int bb = wz3_block_bytes(W);
    const uint64_t* wp =
        reinterpret_cast<const uint64_t*>(area + (e & 0x00FFFFFFFFFFFFFFull) + (uint64_t)(J - 32 * run) * bb);
    uint64_t w[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) w[k] = k < bb / 8 ? wp[k] : 0ull;
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
