// wz1_decode.cuh -- per-thread decoder of one WZ1 block (zfp-style fixed rate,
// Sec. 4.3), entirely in registers.
//
// Steps: header (nonzero flag, biased exponent) -> embedded plane decode up
// to the 16*rate-9 bit budget (verbatim prefix bits + group tests, last
// coefficient implied) -> 32x16 bit-matrix transpose of the plane words into
// one word per coefficient -> negabinary to two's complement -> inverse lift
// (columns, then rows; mod 2^32, arithmetic shifts) -> 16 int32 values q.
// The decoded matrix entry is (float)q * 2^(emax-26) (round to nearest even).
//
// Sec. 5.2 observes that zfp decoding is sequential within a stream and that
// the only parallelism is to give chunks to threads; in fixed-rate mode every
// 4x4 block is such a chunk, so one thread owns one block.
#pragma once
#include <cstdint>

namespace whff {
namespace dev {

// Row-major index 4*i + j of the k-th coefficient in sequency order.
__device__ __forceinline__ constexpr int seq_index(int k) {
  constexpr int t[16] = {0, 1, 4, 5, 2, 3, 8, 12, 6, 7, 9, 13, 10, 11, 14, 15};
  return t[k];
}

__device__ __forceinline__ uint32_t asr1(uint32_t v) { return (uint32_t)((int32_t)v >> 1); }

// Inverse lift of one 4-vector (s, d, d0, e) -> (x0, x1, x2, x3), mod 2^32.
__device__ __forceinline__ void inv_lift(uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d) {
  uint32_t s = a, dd = b, d0 = c, e = d;
  uint32_t d1 = e + d0;
  uint32_t s0 = s - asr1(dd);
  uint32_t s1 = dd + s0;
  a = s0 - asr1(d0);
  b = d0 + a;
  c = s1 - asr1(d1);
  d = d1 + c;
}

// Delta swap of bit groups between two words of a bit matrix.
__device__ __forceinline__ void dswap(uint32_t& a, uint32_t& b, int s, uint32_t m) {
  uint32_t t = ((a >> s) ^ b) & m;
  b ^= t;
  a ^= t << s;
}

// Decode the plane stream (starting after the 9 header bits) of one block
// whose NW32 little-endian 32-bit words are in w[0..NW32) followed by two zero
// words.  Returns the 16 negabinary words u[k] in sequency order.
//
// The plane loop is not unrolled (one small loop body instead of 32 copies:
// the unrolled form spent its time on instruction-cache misses), so the plane
// words go to the thread's own column of a shared-memory array, Ps[j * ps]
// for plane kmax - j, and come back for the bit-matrix transpose.
template <int NW32>
__device__ __forceinline__ void decode_planes(const uint32_t (&w)[NW32 + 2], uint32_t* __restrict__ Ps, int ps,
                                              uint32_t (&u)[16]) {
  constexpr int kMaxBits = 16 * NW32 * 2 - 9;  // 16*rate - 9, rate = 2*NW32
  uint64_t win = ((uint64_t)w[1] << 32 | w[0]) >> 9;
  int avail = 55;  // valid bits in win
  int widx = 2;    // next word to append
  int bits = kMaxBits;
  auto refill = [&]() {
    if (avail <= 32) {
      win |= (uint64_t)w[widx] << avail;
      ++widx;
      avail += 32;
    }
  };
  auto skip = [&](int c) {
    win >>= c;
    avail -= c;
    bits -= c;
  };

  // Leading empty planes (a single zero group test each, while nothing is
  // significant yet).  kmax = the first plane with a positive test.
  int z0 = (uint32_t)win ? __ffs((uint32_t)win) - 1 : 32;
  z0 = min(z0, bits);
  skip(z0);
  const int kmax = 31 - z0;

  int n = 0, j = 0;
#pragma unroll 1
  for (; j <= kmax && bits > 0; ++j) {
    refill();
    const int m = min(n, bits);
    uint32_t p = (uint32_t)win & ((1u << m) - 1u);
    skip(m);
#pragma unroll 1
    while (n < 16 && bits > 0) {
      refill();
      const uint32_t v = (uint32_t)win;
      if (!(v & 1u)) {  // negative group test: plane done
        skip(1);
        break;
      }
      const int avl = bits - 1;  // bits left after the test bit
      const int run = 15 - n;    // explicit positions n..14 (15 is implied)
      const uint32_t rest = v >> 1;
      const int z = rest ? __ffs(rest) - 1 : 31;
      if (z < run) {
        if (z + 1 <= avl) {
          p |= 1u << (n + z);
          n += z + 1;
          skip(z + 2);
          continue;
        }
        skip(1 + avl);  // budget ends inside the zero run
        break;
      }
      if (run <= avl) {  // positions n..14 zero, 15 implied one
        p |= 1u << 15;
        n = 16;
        skip(1 + run);
      } else {
        skip(1 + avl);
      }
      break;
    }
    Ps[j * ps] = p;
  }

  // Transpose the 32 (plane) x 16 (coefficient) bit matrix: A[i] bit j = P[j] bit i
  // (planes past the last decoded one are zero).
  uint32_t P[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) P[k] = k < j ? Ps[k * ps] : 0u;
  uint32_t A[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) A[i] = __byte_perm(P[i], P[i + 16], 0x5410);
#pragma unroll
  for (int k = 0; k < 8; ++k) dswap(A[k], A[k + 8], 8, 0x00FF00FFu);
#pragma unroll
  for (int k = 0; k < 16; ++k)
    if (!(k & 4)) dswap(A[k], A[k + 4], 4, 0x0F0F0F0Fu);
#pragma unroll
  for (int k = 0; k < 16; ++k)
    if (!(k & 2)) dswap(A[k], A[k + 2], 2, 0x33333333u);
#pragma unroll
  for (int k = 0; k < 16; ++k)
    if (!(k & 1)) dswap(A[k], A[k + 1], 1, 0x55555555u);
  // A[i] bit j is plane kmax - j: reverse and align so that bit k is plane k.
  const int sh = 31 - kmax;  // 0..32
#pragma unroll
  for (int i = 0; i < 16; ++i) u[i] = sh >= 32 ? 0u : (__brev(A[i]) >> sh);
}

// Shared memory the decoder needs: one 32-word column per thread of a block
// of kDecodeThreads threads.
constexpr int kDecodeThreads = 256;
constexpr int kPlaneWords = 32 * kDecodeThreads;

// Decode one block: q (row-major) after the inverse transform, emax, nonzero.
// Ps: the thread's column of a kPlaneWords-word shared array (stride kDecodeThreads).
template <int NW32>
__device__ __forceinline__ bool decode_block(const uint32_t (&w)[NW32 + 2], uint32_t* __restrict__ Ps, int32_t (&q)[16],
                                             int& emax) {
  const bool nz = w[0] & 1u;
  emax = (int)((w[0] >> 1) & 0xFFu) - 127;
  uint32_t u[16];
  decode_planes<NW32>(w, Ps, kDecodeThreads, u);
  uint32_t c[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) c[seq_index(k)] = (u[k] ^ 0xAAAAAAAAu) - 0xAAAAAAAAu;
#pragma unroll
  for (int j = 0; j < 4; ++j) inv_lift(c[j], c[4 + j], c[8 + j], c[12 + j]);
#pragma unroll
  for (int r = 0; r < 4; ++r) inv_lift(c[4 * r], c[4 * r + 1], c[4 * r + 2], c[4 * r + 3]);
#pragma unroll
  for (int i = 0; i < 16; ++i) q[i] = nz ? (int32_t)c[i] : 0;
  return nz;
}

// Load one block's words (2*rate bytes at a 2*rate-byte-aligned address).
template <int NW32>
__device__ __forceinline__ void load_block(const uint8_t* __restrict__ base, int64_t blk, uint32_t (&w)[NW32 + 2]) {
  const uint8_t* p = base + (uint64_t)blk * (uint64_t)(4 * NW32);
  if constexpr (NW32 % 4 == 0) {
#pragma unroll
    for (int i = 0; i < NW32 / 4; ++i) {
      uint4 v = __ldcs(reinterpret_cast<const uint4*>(p) + i);
      w[4 * i] = v.x;
      w[4 * i + 1] = v.y;
      w[4 * i + 2] = v.z;
      w[4 * i + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NW32 / 2; ++i) {
      uint2 v = __ldcs(reinterpret_cast<const uint2*>(p) + i);
      w[2 * i] = v.x;
      w[2 * i + 1] = v.y;
    }
  }
  w[NW32] = 0;
  w[NW32 + 1] = 0;
}

}  // namespace dev
}  // namespace whff
