// scaled_mma_tma.cuh -- the tensor-core pass for BF16 storage with the A tile
// brought in by the TMA unit (cp.async.bulk.tensor) instead of the threads.
//
// BF16 values are their own BF16 piece, so the A tile of a stage (128 rows x 64
// columns) needs no decode at all; the register-fed kernel still spends its
// threads on 16-byte global loads and shared stores and waits on them (long
// scoreboard).  Here the roles are split:
//  * one thread (warp 8, lane 0) issues, per stage, one 2-D TMA load of the
//    64-column x 128-row box with 128-byte swizzling -- whole 128-byte rows
//    from HBM, landing in the K-major SWIZZLE_128B layout (8-row x 128-byte
//    atoms, 1024 bytes apart along M) that the MMA reads directly, one K step
//    32 bytes further along the row -- and the bulk copy of the prebuilt B
//    tile, both completing on the stage's mbarrier;
//    then, once the stage has landed, the stage's MMAs (one per K step, A
//    times the three B pieces side by side), committed to the slot's "freed"
//    barrier and, at the end of a 128-column scale group, to the group's
//    barrier; it refills a slot as soon as the MMAs reading it are done.
//  * warps 0-7 only drain: they wait for a group's barrier, add its three
//    accumulators, scale and TwoSum them exactly as the register-fed kernel,
//    and release the TMEM group through its "free" barrier (one arrival per
//    warp).  The same MMAs in the same order and the same drain: the results
//    are those of scaled_mma_kernel<BF16>, bit for bit.
// The ring holds kNS stages; two CTAs share an SM (measured: one CTA with a
// seven-deep ring was 5 % slower).  Every wait is bounded; a
// wait that runs out records WHFF_ETIMEOUT and raises the CTA's abort flag,
// which every other wait watches; the load thread then waits (full limit) for
// its last MMAs and for every copy still in flight before TMEM is freed.
#pragma once
#include <cuda.h>

#include "scaled_mma.cuh"

namespace whff {
namespace dev {

constexpr int kTmaThreads = 288;  // warps 0-7 drain, warp 8 loads and issues

template <int NR>
struct TmaSmem {
  static constexpr int kA = 128 * 128;                // the stage's box: 128 rows x 64 BF16 (128 bytes)
  static constexpr int kB = MmaBTile<NR>::kB;
  static constexpr int kNS = NR <= 16 ? 4 : 3;        // ring depth (two CTAs per SM)
  static constexpr int kBars = kNS * (kA + kB);       // barriers after the ring
  static constexpr int kBytes = kBars + (2 * kNS + 4) * 8 + 64;
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

// 2-D tiled TMA load of the box at (x, y) (x: column, a multiple of 64 BF16 =
// 128 bytes; y: row) into shared memory (1024-byte aligned for the 128-byte
// swizzle); completes bytes on bar.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// 1-D bulk copy whose bytes the caller has already announced on bar.
__device__ __forceinline__ void bulk_g2s_tx(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst), "l"(src),
      "r"(bytes), "r"(bar)
      : "memory");
}

// Shared-memory descriptor of a K-major SWIZZLE_128B operand: 8-row x 128-byte
// atoms 1024 bytes apart along M (stride byte offset), the leading byte offset
// unused (1), descriptor version 1 (bit 46), layout type 2 = 128-byte swizzle
// (bits 61-63).  A K step of 16 BF16 starts 32 bytes further into the atom;
// the swizzle is applied on the absolute address, so the tile base is
// 1024-byte aligned.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}

// Bounded wait that also gives up when the CTA's abort flag is raised:
// 1 done, 0 timed out, -1 aborted elsewhere.
__device__ __forceinline__ int mbar_wait_or_abort(uint32_t bar, uint32_t parity, uint32_t limit,
                                                  const volatile int* abort_flag) {
  for (uint32_t it = 0; it < limit; ++it) {
    if (mbar_try_wait(bar, parity)) return 1;
    if (*abort_flag) return -1;
  }
  return 0;
}

// Same items, segments and workspace layout as scaled_mma_kernel<BF16, NR>;
// tmap covers the whole stored matrix (M_total x ld BF16, box 8 x 128), and
// row0 is the first row of this pass (a row view's offset, a multiple of 128).
// F16: FP16 storage with FP16 B pieces (kind::f16 takes A and B of one type;
// the B tiles are then the FP16 pieces of x scaled per column, see
// f16_mma_btiles); otherwise BF16 storage and BF16 pieces.
template <int NR, bool F16>
__global__ void __launch_bounds__(kTmaThreads, 2)
    scaled_mma_tma_kernel(const __grid_constant__ CUtensorMap tmap, int64_t row0, const float* __restrict__ scales,
                          int64_t TN, const uint8_t* __restrict__ btiles, double* __restrict__ ws, int S, int R,
                          int maxseg, int64_t total, int64_t L, int* __restrict__ status, uint32_t spin) {
  using SM = TmaSmem<NR>;
  constexpr int NS = SM::kNS;
  constexpr int HALF = NR / 2;  // TMEM columns drained by each of the two warps on a lane quarter
  constexpr uint32_t kCols = mma_tmem_cols<NR>();
  extern __shared__ __align__(1024) uint8_t smem[];
  const uint32_t s_base = smem_addr(smem);
  const uint32_t a_base = s_base, b_base = s_base + NS * SM::kA;
  const uint32_t full = s_base + SM::kBars;  // NS: the stage in the slot has landed
  const uint32_t freed = full + 8 * NS;      // NS: the MMAs reading the slot are done
  const uint32_t gfull = freed + 8 * NS;     // 2: the accumulator group is complete
  const uint32_t gfree = gfull + 16;         // 2: the accumulator group has been drained (8 arrivals)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + SM::kBars + (2 * NS + 4) * 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int64_t it0 = (int64_t)blockIdx.x * L;
  const int64_t n = max((int64_t)0, min(total, it0 + L) - it0);
  if (t == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      mbar_init(full + 8 * s, 1);
      mbar_init(freed + 8 * s, 1);
    }
    mbar_init(gfull, 1);
    mbar_init(gfull + 8, 1);
    mbar_init(gfree, 8);
    mbar_init(gfree + 8, 8);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *abort_flag = 0;
  }
  if (warp == 8) {  // TMEM: two groups of three NR-column accumulators
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(tslot)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;
  auto fail = [&]() {
    atomicExch(status, WHFF_ETIMEOUT);
    *abort_flag = 1;
  };
  const int tile0 = (int)(it0 / S), st0 = (int)(it0 - (int64_t)tile0 * S);
  auto advance = [&](int& tile, int& st) {
    if (++st == S) st = 0, ++tile;
  };

  int64_t issued = 0, consumed = 0, last_commit = -1;  // the load thread's bookkeeping
  if (warp == 8 && lane == 0 && n > 0) {
    int l_tile = tile0, l_st = st0;  // load cursor
    auto load = [&](int64_t k) {     // stage k into slot k % NS
      const int slot = (int)(k % NS);
      const uint32_t bar = full + 8 * slot;
      mbar_expect_tx(bar, (uint32_t)(SM::kA + SM::kB));
      tma_load_2d(a_base + slot * SM::kA, &tmap, 64 * l_st, (int)(row0 + 128 * (int64_t)l_tile), bar);
      bulk_g2s_tx(b_base + slot * SM::kB, btiles + (int64_t)l_st * SM::kB, (uint32_t)SM::kB, bar);
      advance(l_tile, l_st);
      ++issued;
    };
    for (int64_t k = 0; k < n && k < NS; ++k) load(k);
    int m_st = st0, m_tile = tile0, gpos = 0, gacc = 0;
    int64_t gi = 0;  // index of the accumulator group being built
    for (int64_t k = 0; k < n; ++k) {
      const int slot = (int)(k % NS);
      int r = mbar_wait_or_abort(full + 8 * slot, (uint32_t)((k / NS) & 1), spin, abort_flag);
      if (r <= 0) {
        if (r == 0) fail();
        break;
      }
      ++consumed;
      const bool init = gpos == 0;
      const int acc = gacc;
      const bool ends = ++gpos == kMmaDrainStages || (m_st & 1) || m_st == S - 1 || k == n - 1;
      if (init && gi >= 2) {  // the group two back in this accumulator pair must have been drained
        r = mbar_wait_or_abort(gfree + 8 * acc, (uint32_t)(((gi - 2) >> 1) & 1), spin, abort_flag);
        if (r <= 0) {
          if (r == 0) fail();
          break;
        }
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t d0 = tmem + (uint32_t)(3 * acc * NR);
#pragma unroll
      for (int ks = 0; ks < kMmaKSteps; ++ks) {
        const uint64_t ad = smem_desc_sw128(a_base + slot * SM::kA + ks * 32);
        const uint64_t bd = smem_desc(b_base + slot * SM::kB + 3 * ks * MmaBTile<NR>::kBTile, 128, 256);
        const uint32_t accumulate = (init && ks == 0) ? 0u : 1u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d0),
            "l"(ad), "l"(bd), "r"(F16 ? mma_idesc_f16(3 * NR) : mma_idesc(3 * NR)), "r"(accumulate));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(freed +
                                                                                                      8 * slot)
                   : "memory");
      last_commit = k;
      if (ends) {
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(gfull +
                                                                                                        8 * acc)
                     : "memory");
        gpos = 0;
        gacc ^= 1;
        ++gi;
      }
      advance(m_tile, m_st);
      if (k >= 1 && k - 1 + NS < n) {  // refill the previous stage's slot once its MMAs are done
        const int ps = (int)((k - 1) % NS);
        r = mbar_wait_or_abort(freed + 8 * ps, (uint32_t)(((k - 1) / NS) & 1), spin, abort_flag);
        if (r <= 0) {
          if (r == 0) fail();
          break;
        }
        load(k - 1 + NS);
      }
    }
  }

  if (warp < 8 && n > 0) {  // drain: tile row 32(warp%4) + lane, accumulator columns HALF(warp/4)..
    const int m_row = 32 * (warp & 3) + lane;
    const int c0 = HALF * (warp >> 2);
    float hi[HALF], lo[HALF];
#pragma unroll
    for (int r = 0; r < HALF; ++r) hi[r] = lo[r] = 0.f;
    int cur_tile = tile0;
    auto flush = [&]() {
      const int64_t seg = (int64_t)blockIdx.x - ((int64_t)cur_tile * S) / L;
      double* dst = ws + (((int64_t)cur_tile * maxseg + seg) * R) * 128 + m_row;
#pragma unroll
      for (int r = 0; r < HALF; ++r) {
        if (c0 + r < R) dst[(int64_t)(c0 + r) * 128] = (double)hi[r] + (double)lo[r];
        hi[r] = lo[r] = 0.f;
      }
    };
    int m_st = st0, m_tile = tile0, gpos = 0;
    int64_t gi = 0;
    bool alive = true;
    for (int64_t k = 0; k < n && alive; ++k) {
      const int tile_k = m_tile, st_k = m_st;
      const bool ends = ++gpos == kMmaDrainStages || (m_st & 1) || m_st == S - 1 || k == n - 1;
      advance(m_tile, m_st);
      if (!ends) continue;
      gpos = 0;
      const int acc = (int)(gi & 1);
      const float s = __ldg(scales + (int64_t)tile_k * TN + (st_k >> 1));
      const int r = mbar_wait_or_abort(gfull + 8 * acc, (uint32_t)((gi >> 1) & 1), spin, abort_flag);
      const bool timed_out = __any_sync(0xFFFFFFFFu, r == 0);
      if (!__all_sync(0xFFFFFFFFu, r > 0)) {
        if (lane == 0 && timed_out) fail();
        alive = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      if (tile_k != cur_tile) {
        flush();
        cur_tile = tile_k;
      }
      const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(3 * acc * NR + c0);
#pragma unroll
      for (int h = 0; h < HALF; h += 8) {
        float v[8];
        tmem_load_sum8(ta + h, NR, v);
#pragma unroll
        for (int q = 0; q < 8; q += 2) {  // packed pairs of columns: each half rounds as the scalar steps
          const float2 ps = make_float2(__fmul_rn(v[q], s), __fmul_rn(v[q + 1], s));
          float2 H = make_float2(hi[h + q], hi[h + q + 1]), Lo = make_float2(lo[h + q], lo[h + q + 1]);
          two_sum_acc2(H, Lo, ps);
          Lo = add_f2(Lo, fma_f2(make_float2(v[q], v[q + 1]), make_float2(s, s), make_float2(-ps.x, -ps.y)));
          hi[h + q] = H.x, hi[h + q + 1] = H.y, lo[h + q] = Lo.x, lo[h + q + 1] = Lo.y;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(gfree + 8 * acc);
      ++gi;
    }
    if (alive) flush();
  }

  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 8 && lane == 0 && *abort_flag) {  // let the MMAs and the copies in flight end (bounded)
    if (last_commit >= 0) (void)mbar_wait(freed + 8 * (int)(last_commit % NS), (uint32_t)((last_commit / NS) & 1));
    for (int64_t k = consumed; k < issued; ++k) (void)mbar_wait(full + 8 * (int)(k % NS), (uint32_t)((k / NS) & 1));
  }
  __syncwarp();
  if (warp == 8) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols));
  }
}

}  // namespace dev
}  // namespace whff
