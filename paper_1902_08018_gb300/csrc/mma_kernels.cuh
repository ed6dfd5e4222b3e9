// mma_kernels.cuh -- many right-hand sides on the 5th-generation tensor cores.
//
// With R right-hand sides the step Y = A X is a dense contraction (Sec. 4.4's
// GEMV becomes a GEMM), so for R >= 4 (the default crossover) the WZ2 kernels run
// it on tcgen05.  In the transform domain the contraction is
//     Z_band = sum_J (s_J V_J) ((2G)^T X_J),   Y_band = (2G) Z_band * 2^-3,
// a GEMM whose A operand is the stored integer coefficients times a
// power-of-two block scale, and whose B operand is the transformed x.
//
// Precision (the 1e-6 bar): a coefficient of a W-bit field has at most W-1
// significant bits, so A splits EXACTLY into PA = ceil((W-1)/8) BF16 pieces
// (1 at rate 8, 2 at rates 12 and 16, 3 at 20 and 24); B (FP32) into three
// BF16 pieces (8+8+8 bits, exact).  The products A_p B_q with p+q <= 2 are
// issued (kind::f16, BF16 in, FP32 accumulate in TMEM); the dropped ones are
// below 2^-24 of |a||x|.  The tensor cores' FP32 accumulate is not a
// round-to-nearest sum, so the products go to three accumulators by size:
// A_0 B_0; the 2^-8 terms A_0 B_1 + A_1 B_0; the 2^-16 terms A_0 B_2 + A_1 B_1
// + A_2 B_0.  With the B pieces side by side along N, one instruction
// A_p [B_0 .. B_{2-p}] (N = (3-p) NR) writes accumulators p..2, so a K step
// takes PA instructions.  The accumulators cover at most kMmaDrainStages
// stages of one tile (16 blocks = 64 columns of K each) and are then added
// and drained into TwoSum FP32 registers, so FP32 rounding never sees long
// sums.
//
// CTA = 8 warps = 256 threads, persistent: the grid splits the sequence of
// (tile, stage) items -- tile = 32 bands = 128 coefficient rows, stage = 16
// blocks of K -- into equal contiguous ranges.  Two stages are in flight:
// while the tensor cores multiply stage k (A and B tiles of buffer k % 2),
// the threads decode stage k+1 into the other A tile and drain the other TMEM
// accumulator when stage k-1 closed its group; the words of stage k+2 are already
// being loaded, and one thread brings the prebuilt B tile of stage k+1 in with
// a bulk copy (cp.async.bulk) tracked by an mbarrier.  A tile row m holds
// coefficient row a of band b as m = 32a + b, which makes every warp's tile
// stores bank-conflict free.  At the end of a tile piece the FP32 sums go to
// the workspace as one FP64 segment partial; wz2_mma_finish adds a band's
// segments in order and mixes with 2G, wz2_mma_state applies the state.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>
#include <utility>

#include "whff.h"
#include "bulk.cuh"
#include "wz2_kernels.cuh"

namespace whff {
namespace dev {

constexpr int kMmaThreads = 256;       // 8 warps; warps w and w+4 share TMEM lanes 32(w%4)..
constexpr int kMmaBands = 32;         // 128 coefficient rows per tile
constexpr int kMmaStageBlocks = 16;   // K = 64 per stage
constexpr int kMmaKSteps = 4;         // K = 16 per instruction
constexpr int kMmaDrainStages = 2;    // stages of one tile accumulated in TMEM between drains


// 64-bit shared-memory matrix descriptor: start >> 4 (bits 0-13), leading
// byte offset >> 4 (16-29), stride byte offset >> 4 (32-45), descriptor
// version 1 (bit 46), no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor, kind::f16: F32 accumulator (bits 4-5 = 1), A and B
// BF16 (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at 24.
__device__ __forceinline__ constexpr uint32_t mma_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// The same with A and B FP16 (bits 7-9 and 10-12 = 0).
__device__ __forceinline__ constexpr uint32_t mma_idesc_f16(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// Byte offset of element (row, k) in a 16-wide K-step tile (no swizzle,
// K-major): core matrix (row/8, k/8) of 8 rows x 16 bytes, 2 along K.
__device__ __forceinline__ uint32_t tile_off(int row, int k) {
  return (uint32_t)(((row >> 3) * 2 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Exact split of a float with at most 24 significant bits into three BF16.
__device__ __forceinline__ void split3(float v, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(a);
  b = __float2bfloat16_rn(r1);
  c = __float2bfloat16_rn(r1 - __bfloat162float(b));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// BF16 pieces of one A coefficient: its field has at most W-1 significant bits.
template <int RATE>
struct MmaPieces {
  static constexpr int kBits = Wz2Layout<RATE>::kW - 1;
  static constexpr int kA = kBits <= 8 ? 1 : kBits <= 16 ? 2 : 3;
};

// B operand of one stage: per K step, the 3 pieces one after another along N
// (a 3 NR x 16 BF16 tile).
template <int NR>
struct MmaBTile {
  static constexpr int kBTile = NR * 16 * 2;  // one piece, one K step
  static constexpr int kB = 3 * kMmaKSteps * kBTile;
};

// TMEM columns: two accumulator groups of three NR-column accumulators,
// rounded up to the power of two that tcgen05.alloc takes.
template <int NR>
__host__ __device__ constexpr uint32_t mma_tmem_cols() {
  return 6 * NR <= 32 ? 32u : 6 * NR <= 64 ? 64u : 6 * NR <= 128 ? 128u : 256u;
}

// Shared memory: A and B tiles of two stages, then 4 mbarriers, the TMEM slot,
// flags and thread 0's B-copy cursor; the member table follows kBytes.
template <int RATE, int NR>
struct MmaSmem {
  static constexpr int kATile = 128 * 16 * 2;  // one piece, one K step
  static constexpr int kA = MmaPieces<RATE>::kA * kMmaKSteps * kATile;
  static constexpr int kB = MmaBTile<NR>::kB;
  static constexpr int kBars = 2 * (kA + kB);
  static constexpr int kBytes = kBars + 80;  // 4 mbarriers, TMEM slot, flags, cursors
};



// Eight columns of the three accumulators at ta, ta + stride, ta + 2 stride,
// summed big + (small + smaller): one wait for the three loads, tied to their
// registers so no use can move above it.
__device__ __forceinline__ void tmem_load_sum8(uint32_t ta, uint32_t stride, float (&v)[8]) {
  uint32_t a[8], b[8], c[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
               : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7])
               : "r"(ta));
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
               : "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]), "=r"(b[7])
               : "r"(ta + stride));
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
               : "=r"(c[0]), "=r"(c[1]), "=r"(c[2]), "=r"(c[3]), "=r"(c[4]), "=r"(c[5]), "=r"(c[6]), "=r"(c[7])
               : "r"(ta + 2 * stride));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n"
               : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]),
                 "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7]),
                 "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3]), "+r"(c[4]), "+r"(c[5]), "+r"(c[6]), "+r"(c[7])
               :
               : "memory");
#pragma unroll
  for (int i = 0; i < 8; i += 2) {  // packed pairs: each half rounds as a + (b + c) would
    const float2 bc = add_f2(make_float2(__uint_as_float(b[i]), __uint_as_float(b[i + 1])),
                             make_float2(__uint_as_float(c[i]), __uint_as_float(c[i + 1])));
    const float2 t = add_f2(make_float2(__uint_as_float(a[i]), __uint_as_float(a[i + 1])), bc);
    v[i] = t.x;
    v[i + 1] = t.y;
  }
}


// The B operand of every stage, built once per step: for column block J and
// right-hand side r, (2G)^T x_J (or x_J without the lift) in three BF16
// pieces, already in the shared-memory tile layout of its 16-block stage:
// out[stage][piece][kstep] = NR x 16 BF16 tile.  Thread per (stage, J, r).
// The pass of thread q in a launch-wide grid: `single` when table is null,
// else the entry with the largest begin <= q (begin = bt_begin or fin_begin).
template <bool FIN>
__device__ __forceinline__ MmaPass pass_of(const MmaPass& single, const MmaPass* __restrict__ table, int n,
                                           int64_t q) {
  if (!table) return single;
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((FIN ? table[mid].fin_begin : table[mid].bt_begin) <= q) lo = mid;
    else hi = mid - 1;
  }
  return table[lo];
}

// B tiles of every pass: for stage st, column block J and right-hand side r,
// (2G)^T x_J (or x_J without the lift) in three BF16 pieces, already in the
// shared-memory tile layout of the stage: out[st][kstep][piece] = NR x 16 BF16.
// Thread per (pass, stage, J in the stage, r); total threads given.
template <bool LIFT, int NR>
__global__ void wz2_mma_btiles(MmaPass single, const MmaPass* __restrict__ table, int n, int64_t threads) {
  using S = MmaBTile<NR>;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= threads) return;
  const MmaPass ps = pass_of<false>(single, table, n, q);
  const int64_t ql = q - ps.bt_begin;
  if (ql >= (int64_t)ps.S * kMmaStageBlocks * NR) return;
  const int r = (int)(ql % NR);
  const int jl = (int)((ql / NR) % kMmaStageBlocks);
  const int64_t stage = ql / ((int64_t)NR * kMmaStageBlocks);
  const int64_t J = stage * kMmaStageBlocks + jl;
  float xt[4] = {0.f, 0.f, 0.f, 0.f};
  if (r < ps.R) {
    float xv[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) xv[c] = 4 * J + c < ps.N ? __ldg(ps.x + (int64_t)r * ps.ldx + 4 * J + c) : 0.f;
    if (LIFT) {
      const float aa = xv[0] + xv[1], bb = xv[2] + xv[3], cc = xv[0] + xv[2], dd = xv[1] + xv[3];
      xt[0] = 2.f * (aa + bb);
      xt[1] = bb - aa;
      xt[2] = dd - cc;
      xt[3] = xv[3] - xv[2];
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) xt[c] = xv[c];
    }
  }
  __nv_bfloat16 p[3][4];
#pragma unroll
  for (int b = 0; b < 4; ++b) split3(xt[b], p[0][b], p[1][b], p[2][b]);
  const int kstep = jl >> 2, kk = (jl & 3) * 4;
  uint8_t* base = ps.btiles + stage * (int64_t)S::kB;
#pragma unroll
  for (int pc = 0; pc < 3; ++pc)
    *reinterpret_cast<uint2*>(base + (kstep * 3 + pc) * S::kBTile + tile_off(r, kk)) =
        make_uint2(pack2(p[pc][0], p[pc][1]), pack2(p[pc][2], p[pc][3]));
}


// cvt.rn.bf16x2.f32: the packed pair (lo in bits 0-15, hi in bits 16-31).
__device__ __forceinline__ uint32_t bf16x2_rn(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;\n" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
__device__ __forceinline__ float bf16_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t u) { return __uint_as_float(u & 0xFFFF0000u); }

// The 16 coefficients of a block times its scale 2^(E+K-154), as packed pairs
// in tile-row order: P[a][h] = (V[a][2h], V[a][2h+1]).  The field is OR-ed into
// the mantissa of 2^(e+23) and one packed subtraction per pair gives the scaled
// value exactly (wz2_fields_times_scale's values, two per instruction); blocks
// beyond the trick's exponent range (|a| >= 2^103) decode unscaled and take s
// by an exact packed multiply.  A zero block decodes to zeros.
template <int RATE, bool LIFT>
__device__ __forceinline__ void mma_block_pairs(const uint32_t (&w)[Wz2Layout<RATE>::kWords], float2 (&P)[4][2]) {
  using Lay = Wz2Layout<RATE>;
  const uint32_t E = w[0] & 0xFFu, K = (w[0] >> 8) & 31u;
  const bool trick = E + K <= 258u;
  const uint32_t creg = trick ? (E ? (E + K - 4u) << 23 : 0u) : 0x4B000000u;
  const uint32_t mreg = E ? Lay::kMask : 0u;
  const float bias = E ? __uint_as_float(creg | (1u << (Lay::kW - 1))) : 0.f;
  uint32_t u[16];
  wz2_field_bits_impl<RATE>(w, mreg, creg, u, std::make_integer_sequence<int, 16>{});
  const float2 b2 = make_float2(bias, bias);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m0 = 4 * a + 2 * h, m1 = m0 + 1;
      const int k0 = LIFT ? seq_field(m0) : m0, k1 = LIFT ? seq_field(m1) : m1;
      P[a][h] = sub_f2(make_float2(__uint_as_float(u[k0]), __uint_as_float(u[k1])), b2);
    }
  if (!trick) {
    const float s = __uint_as_float((E + K - 27u) << 23);
    const float2 s2 = make_float2(s, s);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int h = 0; h < 2; ++h) P[a][h] = mul_f2(P[a][h], s2);
  }
}

// Exact split of a pair of values (at most 8 PA significant bits each) into PA
// BF16 pairs, d[p] = piece p of (v.x, v.y): round to BF16, subtract, repeat --
// the two subtractions of each step in one packed instruction.
template <int PA>
__device__ __forceinline__ void split_pair(float2 v, uint32_t (&d)[PA]) {
#pragma unroll
  for (int p = 0; p < PA; ++p) {
    d[p] = bf16x2_rn(v.x, v.y);
    if (p + 1 < PA) v = sub_f2(v, make_float2(bf16_lo(d[p]), bf16_hi(d[p])));
  }
}

// Persistent grid over the item sequence of one or more passes (members):
// member k owns items [item_begin, item_begin + tiles S), item = item_begin +
// tile S + stage; CTA g takes items [g L, g L + L).  ws[((tile * maxseg + seg)
// * R + r) * 128 + m] of a member receives the FP64 partial of tile row m
// (= 32a + band) for the CTA's segment seg = g - (item_begin + tile S) / L.
// `single` is the only member when table is null (one matrix); otherwise the
// nmem members of the table (a batch) are copied to shared memory.
template <int RATE, bool LIFT, int NR, bool TABLE>
__global__ void __launch_bounds__(kMmaThreads, MmaPieces<RATE>::kA == 3 ? 1 : 2)  // 3 A pieces: 120 KB of tiles
    wz2_mma_kernel(MmaMember single, const MmaMember* __restrict__ table, int nmem, int64_t total, int64_t L,
                   int* __restrict__ status, uint32_t spin) {
  using SM = MmaSmem<RATE, NR>;
  constexpr int PA = MmaPieces<RATE>::kA;
  constexpr int NW = Wz2Layout<RATE>::kWords;
  constexpr int HALF = NR / 2;  // TMEM columns drained by each of the two warps on a lane quarter
  constexpr uint32_t kCols = mma_tmem_cols<NR>();  // two groups of three accumulators
  extern __shared__ __align__(1024) uint8_t smem[];
  const uint32_t s_base = smem_addr(smem);
  const uint32_t mma_bar = s_base + SM::kBars;  // two mbarriers: MMAs of buffer 0, 1 done
  const uint32_t b_bar = mma_bar + 16;          // two mbarriers: B tile of buffer 0, 1 landed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + SM::kBars + 32);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + SM::kBars + 36);
  int64_t* last_commit = reinterpret_cast<int64_t*>(smem + SM::kBars + 48);  // last stage whose MMAs were committed
  int64_t* last_copy = reinterpret_cast<int64_t*>(smem + SM::kBars + 56);    // last stage whose B copy was started
  MmaMember* tab = reinterpret_cast<MmaMember*>(smem + SM::kBytes);          // the members

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int64_t it0 = (int64_t)blockIdx.x * L;
  const int64_t n = max((int64_t)0, min(total, it0 + L) - it0);
  if constexpr (TABLE)
    for (int i = t; i < nmem; i += kMmaThreads) tab[i] = table[i];
  // member m (TABLE: of the batch's table; else the one matrix)
  auto mb = [&](int m) -> const MmaMember& {
    if constexpr (TABLE) return tab[m];
    return single;
  };

  if (t == 0) {
    mbar_init(mma_bar, 1);
    mbar_init(mma_bar + 8, 1);
    mbar_init(b_bar, 1);
    mbar_init(b_bar + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *abort_flag = 0;
    *last_commit = *last_copy = -1;
  }
  if (warp == 0) {  // TMEM: six accumulators of NR fp32 columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(tslot)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;

  // decode assignment: band 8(warp%4) + lane%8 of the tile, blocks jl and jl+4
  // of the stage, jl = 8(warp/4) + lane/8
  const int band_l = 8 * (warp & 3) + (lane & 7);
  const int jl0 = 8 * (warp >> 2) + (lane >> 3);
  // drain assignment: tile row 32(warp%4) + lane, accumulator columns HALF(warp/4)..
  const int m_row = 32 * (warp & 3) + lane;
  const int c0 = HALF * (warp >> 2);

  // Cursors (member, tile, stage) of the next item to fetch, to copy B for
  // and to issue; they advance in item order, so the loop has no divisions.
  int mem0 = 0;
  if constexpr (TABLE)
    while (mem0 + 1 < nmem && tab[mem0 + 1].item_begin <= it0) ++mem0;
  const int tile0 = (int)((it0 - mb(mem0).item_begin) / mb(mem0).S);
  const int st0 = (int)(it0 - mb(mem0).item_begin - (int64_t)tile0 * mb(mem0).S);
  int f_m = mem0, f_tile = tile0, f_st = st0;  // fetch
  int m_m = mem0, m_tile = tile0, m_st = st0;  // issue
  // the B-copy cursor (member, tile, stage) is thread 0's alone: it lives in
  // shared memory, not in every thread's registers
  int* b_cur = reinterpret_cast<int*>(smem + SM::kBars + 64);
  if (t == 0) b_cur[0] = mem0, b_cur[1] = tile0, b_cur[2] = st0;
  auto advance = [&](int& m, int& tile, int& st) {
    if (++st == mb(m).S) {
      st = 0, ++tile;
      if constexpr (TABLE)
        if (tile == tab[m].tiles) tile = 0, ++m;
    }
  };

  uint32_t w[2][2][NW];  // compressed words of two stages (ring), 2 blocks each
  constexpr int64_t kBlockBytes = 4 * NW;
  // this thread's first block of the next fetch: band 32 f_tile + band_l, block 16 f_st + jl0
  bool f_band_ok = false;
  const uint8_t* f_ptr = nullptr;
  auto fetch_at = [&]() {
    const int64_t band = 32 * (int64_t)f_tile + band_l;
    f_band_ok = band < mb(f_m).BM;
    f_ptr = mb(f_m).stream + (band * mb(f_m).BN + 16 * (int64_t)f_st + jl0) * kBlockBytes;
  };
  if (n > 0) fetch_at();
  auto fetch = [&](int slot) {
    const int64_t J = 16 * (int64_t)f_st + jl0;
    const int64_t BN = mb(f_m).BN;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (f_band_ok && J + 4 * u < BN) {
        wz2_load<RATE>(f_ptr, 4 * u, w[slot][u]);
      } else {
#pragma unroll
        for (int i = 0; i < NW; ++i) w[slot][u][i] = 0u;  // a zero block: E = 0, scale 0
      }
    }
    const int m_before = f_m, t_before = f_tile;
    advance(f_m, f_tile, f_st);
    if (f_m != m_before || f_tile != t_before) {
      if (f_m < nmem) fetch_at();
    } else {
      f_ptr += 16 * kBlockBytes;
    }
  };
  auto b_copy = [&](int64_t k) {  // thread 0: B tile of stage k into buffer k % 2
    const int buf = (int)(k & 1);
    int bm = b_cur[0], bt = b_cur[1], bs = b_cur[2];
    bulk_copy_g2s(s_base + 2 * SM::kA + buf * SM::kB, mb(bm).btiles + (int64_t)bs * SM::kB, (uint32_t)SM::kB,
                  b_bar + 8 * buf);
    advance(bm, bt, bs);
    b_cur[0] = bm, b_cur[1] = bt, b_cur[2] = bs;
    *last_copy = k;
  };
  auto fail = [&]() {  // a wait ran out: the CTA stops at its next barrier
    atomicExch(status, WHFF_ETIMEOUT);
    *abort_flag = 1;
  };

  float hi[HALF], lo[HALF];
#pragma unroll
  for (int r = 0; r < HALF; ++r) hi[r] = lo[r] = 0.f;
  int cur_m = mem0, cur_tile = tile0;  // member and tile of the sums in hi/lo
  auto flush = [&]() {
    const MmaMember& me = mb(cur_m);
    const int64_t seg = (int64_t)blockIdx.x - (me.item_begin + (int64_t)cur_tile * me.S) / L;
    double* dst = me.ws + (((int64_t)cur_tile * me.maxseg + seg) * me.R) * 128 + m_row;
#pragma unroll
    for (int r = 0; r < HALF; ++r) {
      if (c0 + r < me.R) dst[(int64_t)(c0 + r) * 128] = (double)hi[r] + (double)lo[r];
      hi[r] = lo[r] = 0.f;
    }
  };
  // drain accumulator group `acc` (its three accumulators, added), which holds
  // a group of stages of tile `tile` of member `mem`
  auto drain = [&](int acc, int mem, int tile) {
    if (mem != cur_m || tile != cur_tile) {
      flush();
      cur_m = mem;
      cur_tile = tile;
    }
    const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(3 * acc * NR + c0);
#pragma unroll
    for (int h = 0; h < HALF; h += 8) {
      float v[8];
      tmem_load_sum8(ta + h, NR, v);
#pragma unroll
      for (int r = 0; r < 8; r += 2) {  // TwoSum on packed pairs of columns (the same bits per half)
        float2 H = make_float2(hi[h + r], hi[h + r + 1]), Lo = make_float2(lo[h + r], lo[h + r + 1]);
        two_sum_acc2(H, Lo, make_float2(v[r], v[r + 1]));
        hi[h + r] = H.x, hi[h + r + 1] = H.y, lo[h + r] = Lo.x, lo[h + r + 1] = Lo.y;
      }
    }
  };

  const uint64_t a_desc0 = smem_desc(s_base, 128, 256);
  const uint64_t b_desc0 = smem_desc(s_base + 2 * SM::kA, 128, 256);
  bool ok = true;  // this thread's waits all ended in time
  // accumulator groups: up to kMmaDrainStages consecutive stages of one tile
  // share a TMEM accumulator pair (alternating 0, 1); a group is drained after
  // its last stage's MMAs complete
  int gpos = 0, gacc = 0;
  bool p_ends = false;  // stage k-1 closed its group ...
  int p_acc = 0, p_m = mem0, p_tile = tile0;  // ... in accumulator pair p_acc, of member p_m's tile p_tile
  if (n > 0) {
    fetch(0);
    if (t == 0) b_copy(0);
  }
  if (n > 1) fetch(1);

  // one stage; `buf` is a literal at every call, so the ring stays in registers
  auto stage = [&](const int buf, const int64_t k) -> bool {
    uint8_t* As = smem + buf * SM::kA;
    // ---- A tile: this thread's 2 blocks
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int jl = jl0 + 4 * u;
      float2 P[4][2];
      mma_block_pairs<RATE, LIFT>(w[buf][u], P);
      const int kstep = jl >> 2, kk = (jl & 3) * 4;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        uint32_t d0[PA], d1[PA];
        split_pair<PA>(P[a][0], d0);
        split_pair<PA>(P[a][1], d1);
        const uint32_t off = tile_off(32 * a + band_l, kk);
#pragma unroll
        for (int p = 0; p < PA; ++p)
          *reinterpret_cast<uint2*>(As + (p * kMmaKSteps + kstep) * SM::kATile + off) = make_uint2(d0[p], d1[p]);
      }
    }
    // this ring slot is free: the words of stage k+2 are on their way from here
    // on, through the barrier, the MMA issue and the drain
    if (k + 2 < n) fetch(buf);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic writes -> tensor-core reads
    if (!__syncthreads_and(ok ? 1 : 0)) return false;
    // group bookkeeping of stage k (the same in every thread)
    const bool init = gpos == 0;
    const int acc = gacc;
    const int tile_k = m_tile, mem_k = m_m;
    const bool ends = ++gpos == kMmaDrainStages || m_st == mb(m_m).S - 1 || k == n - 1;
    if (ends) gpos = 0, gacc ^= 1;
    advance(m_m, m_tile, m_st);
    if (t == 0) {
      if (!mbar_wait(b_bar + 8 * buf, (uint32_t)((k >> 1) & 1), spin)) {
        ok = false;
        fail();
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint64_t ad0 = a_desc0 + (uint64_t)((buf * SM::kA) >> 4);
        const uint64_t bd0 = b_desc0 + (uint64_t)((buf * SM::kB) >> 4);
        const uint32_t d0 = tmem + (uint32_t)(3 * acc * NR);
        // A_p [B_0 .. B_{2-p}] into accumulators p..2; A_0 of the first K step
        // of a group starts all three
#pragma unroll
        for (int ks = 0; ks < kMmaKSteps; ++ks) {
#pragma unroll
          for (int pa = 0; pa < PA; ++pa) {
            const uint64_t ad = ad0 + (uint64_t)(((pa * kMmaKSteps + ks) * SM::kATile) >> 4);
            const uint64_t bd = bd0 + (uint64_t)((3 * ks * MmaBTile<NR>::kBTile) >> 4);
            const uint32_t accumulate = (init && ks == 0 && pa == 0) ? 0u : 1u;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d0 + (uint32_t)(pa * NR)),
                "l"(ad), "l"(bd), "r"(mma_idesc((3 - pa) * NR)), "r"(accumulate));
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         mma_bar + 8 * buf)
                     : "memory");
        *last_commit = k;
      }
    }
    if (k >= 1) {  // stage k-1 (other buffer): wait for its MMAs; drain its group if it closed one
      const bool done =
          __all_sync(0xFFFFFFFFu, mbar_wait(mma_bar + 8 * (buf ^ 1), (uint32_t)(((k - 1) >> 1) & 1), spin));
      if (!done) {
        if (ok && lane == 0) fail();
        ok = false;
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (t == 0 && ok && k + 1 < n) b_copy(k + 1);  // its B tile buffer is free now
        if (p_ends) drain(p_acc, p_m, p_tile);
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      }
    } else if (t == 0 && ok && k + 1 < n) {
      b_copy(k + 1);
    }
    p_ends = ends;
    p_acc = acc;
    p_m = mem_k;
    p_tile = tile_k;
    return true;
  };

  bool alive = true;
  for (int64_t k = 0; k < n && alive; k += 2) {
    alive = stage(0, k);
    if (alive && k + 1 < n) alive = stage(1, k + 1);
  }
  if (alive && n > 0) alive = __syncthreads_and(ok ? 1 : 0) != 0;
  if (alive && n > 0) {  // the last stage, which always closes its group
    const int buf = (int)((n - 1) & 1);
    if (__all_sync(0xFFFFFFFFu, mbar_wait(mma_bar + 8 * buf, (uint32_t)(((n - 1) >> 1) & 1), spin))) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      drain(p_acc, p_m, p_tile);
      flush();
    } else if (lane == 0) {
      fail();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (t == 0 && *abort_flag) {  // give the MMAs and the copy in flight a second bounded chance
    const int64_t c = *last_commit, b = *last_copy;
    if (c >= 0) (void)mbar_wait(mma_bar + 8 * (int)(c & 1), (uint32_t)((c >> 1) & 1));
    if (b >= 0) (void)mbar_wait(b_bar + 8 * (int)(b & 1), (uint32_t)((b >> 1) & 1));
  }
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols));
  }
}

// Sum each band's segment partials in order and map its 4 coefficient rows to
// y (2G mix and 2^-3 with the lift, 2^3 without).  Thread per (pass, tile,
// column, band of the tile), the band fastest, so a warp reads 32 consecutive
// partials of one row and writes 32 consecutive 4-row groups of y.
template <bool LIFT>
__global__ void wz2_mma_finish(MmaPass single, const MmaPass* __restrict__ table, int n, int64_t threads, int64_t L) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= threads) return;
  const MmaPass ps = pass_of<true>(single, table, n, q);
  const int64_t ql = q - ps.fin_begin;
  const int bl = (int)(ql & 31);
  const int64_t tr = ql >> 5;  // tile * R + r
  const int r = (int)(tr % ps.R);
  const int64_t tile = tr / ps.R;
  const int64_t I = 32 * tile + bl;
  if (tile >= ps.tiles || 4 * I >= ps.M) return;
  const int64_t first = ps.item_begin + tile * ps.S;
  const int nseg = (int)((first + ps.S - 1) / L - first / L + 1);
  double z[4];
  for (int a = 0; a < 4; ++a)
    z[a] = seq_sum_strided(ps.ws + ((tile * ps.maxseg) * ps.R + r) * 128 + 32 * a + bl, nseg, (int64_t)ps.R * 128);
  double yy[4];
  if (LIFT) {
    const double a = 2.0 * z[0];
    yy[0] = (a - z[1] - z[2]) * 0.125;
    yy[1] = (a - z[1] + z[2]) * 0.125;
    yy[2] = (a + z[1] - z[2] - z[3]) * 0.125;
    yy[3] = (a + z[1] + z[2] + z[3]) * 0.125;
  } else {
    for (int i = 0; i < 4; ++i) yy[i] = z[i] * 8.0;
  }
  for (int i = 0; i < 4; ++i)
    if (4 * I + i < ps.M) ps.y[(int64_t)r * ps.ldy + 4 * I + i] = yy[i];
}

// state <- decay * state + y[:, r] for r = 0..R-1 in order.  Thread per row.
static __global__ void wz2_mma_state(const double* __restrict__ y, int64_t ldy, int R, int64_t M,
                                     double* __restrict__ state, double decay) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= M) return;
  double s = state[row];
  for (int r = 0; r < R; ++r) s = decay * s + y[(int64_t)r * ldy + row];
  state[row] = s;
}

}  // namespace dev
}  // namespace whff
