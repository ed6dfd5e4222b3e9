// wz2_stream.cuh -- the fused WZ2 decode + GEMV for one right-hand side with
// the compressed blocks staged through shared memory by the copy engine.
//
// The register-fed kernel (wz2_gemv_kernel) keeps UNROLL blocks per lane in
// flight in registers; at low rates (16-byte blocks at rate 8) that is too few
// bytes in flight per SM to cover HBM latency, and the kernel waits on its
// loads (long-scoreboard stalls).  Here every warp streams its contiguous
// block range through a ring of kNS shared-memory slots: lane 0 starts a 1-D
// bulk copy (cp.async.bulk, completion on an mbarrier) of each stage of
// 32*kU consecutive blocks, kNS - 1 stages ahead of the lanes that decode,
// so the bytes in flight no longer cost registers.  A stage never crosses a
// band: the sequence of stages follows the pieces (the parts of 4-row bands
// inside the range) exactly like wz2_piece, and lane l takes blocks
// l, l + 32, ... of each stage -- the same blocks, pairs and additions as the
// register-fed kernel, so the results are the same bit for bit.
//
// Bulk copies start on a 16-byte boundary: a stage whose first block does not
// (24- and 40-byte blocks, rates 12 and 20) is copied from the boundary below
// and read 8 bytes into its slot; the copy may run up to 15 bytes past the
// piece, which the handle's stream allocation covers with its padding
// (kStreamPad).  The host launches this kernel only on streams at least
// 16-byte (8-byte for 24- and 40-byte blocks) aligned.
// Every wait is bounded: a wait that runs out records WHFF_ETIMEOUT, waits
// (bounded) for the warp's copies still in flight and leaves.
#pragma once
#include <cstdint>

#include "bulk.cuh"
#include "whff.h"
#include "wz2_kernels.cuh"

namespace whff {
namespace dev {

template <int RATE>
struct Wz2Stream {
  static constexpr int kBB = 2 * RATE;                      // bytes per block
  static constexpr int kU = RATE <= 8 ? 4 : 2;              // blocks per lane per stage (even: pairs)
  static constexpr int kStageBlocks = 32 * kU;
  static constexpr int kSlotBytes = kStageBlocks * kBB + 16;  // + room for the 16-byte alignment shift
  static constexpr int kNS = RATE <= 16 ? 4 : 3;            // ring depth per warp
  static constexpr int kRingBytes = kNS * kSlotBytes;
  static constexpr int kSmemBytes = kWarpsPerCta * (kRingBytes + 8 * kNS);
};

// Words of lane block `b` of a slot (8-byte aligned in shared memory).
template <int RATE>
__device__ __forceinline__ void wz2_lds(const uint8_t* p, uint32_t (&w)[Wz2Layout<RATE>::kWords]) {
  constexpr int NW = Wz2Layout<RATE>::kWords;
  if constexpr (Wz2Stream<RATE>::kBB % 16 == 0) {
#pragma unroll
    for (int i = 0; i < NW / 4; ++i) {
      const uint4 v = *reinterpret_cast<const uint4*>(p + 16 * i);
      w[4 * i] = v.x, w[4 * i + 1] = v.y, w[4 * i + 2] = v.z, w[4 * i + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NW / 2; ++i) {
      const uint2 v = *reinterpret_cast<const uint2*>(p + 8 * i);
      w[2 * i] = v.x, w[2 * i + 1] = v.y;
    }
  }
}

// The warp's position in its sequence of stages: band I, blocks [J, Jend) of
// the band still to stream (Jend = the end of the range's piece of band I).
struct StageCursor {
  int64_t I, J, Jend;
};

__device__ __forceinline__ void cursor_begin(StageCursor& c, int64_t b0, int64_t b1, int64_t BN) {
  c.I = b0 / BN;
  c.J = b0 - c.I * BN;
  c.Jend = min(BN, b1 - c.I * BN);
}

// Advance past a stage of n blocks; at the end of a piece move to the next band.
__device__ __forceinline__ void cursor_next(StageCursor& c, int n, int64_t b1, int64_t BN) {
  c.J += n;
  if (c.J >= c.Jend) {
    ++c.I;
    c.J = 0;
    c.Jend = min(BN, b1 - c.I * BN);
  }
}

template <int RATE, bool LIFT>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
    wz2_stream_kernel(const uint8_t* __restrict__ stream, int64_t M, int64_t N, int64_t BM, int64_t BN,
                      const float* __restrict__ x, int64_t ldx, bool x_vec_ok, int64_t L, int maxseg,
                      double* __restrict__ ws, double* __restrict__ y, int64_t ldy, double* __restrict__ state,
                      double decay, bool red32, int* __restrict__ status) {
  using S = Wz2Stream<RATE>;
  constexpr int NW = Wz2Layout<RATE>::kWords;
  extern __shared__ __align__(128) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t g = (int64_t)blockIdx.x * kWarpsPerCta + warp;
  const int64_t total = BM * BN;
  const int64_t b0 = g * L, b1 = min(total, b0 + L);
  if (b0 >= b1) return;  // no cross-warp synchronisation in this kernel
  uint8_t* ring = smem + warp * S::kRingBytes;
  const uint32_t ring_s = smem_addr(ring);
  const uint32_t bar0 = smem_addr(smem + kWarpsPerCta * S::kRingBytes + warp * 8 * S::kNS);
  if (lane == 0) {
#pragma unroll
    for (int s = 0; s < S::kNS; ++s) mbar_init(bar0 + 8 * s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncwarp();
  const bool x_fast = x_vec_ok && (N % 4 == 0);

  // producer (lane 0 issues; every lane keeps the cursor, it is warp-uniform)
  StageCursor pc;
  cursor_begin(pc, b0, b1, BN);
  int64_t issued = 0;  // stages started so far
  auto issue = [&](int slot) {
    const int n = (int)min((int64_t)S::kStageBlocks, pc.Jend - pc.J);
    const uint8_t* src = stream + (uint64_t)(pc.I * BN + pc.J) * (uint64_t)S::kBB;
    const uint32_t shift = (uint32_t)(reinterpret_cast<uintptr_t>(src) & 15u);
    const uint32_t bytes = (shift + (uint32_t)n * S::kBB + 15u) & ~15u;
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // the slot's last reads before the copy
      bulk_copy_g2s(ring_s + slot * S::kSlotBytes, src - shift, bytes, bar0 + 8 * slot);
    }
    cursor_next(pc, n, b1, BN);
    ++issued;
  };
#pragma unroll
  for (int s = 0; s < S::kNS; ++s)
    if (pc.I * BN + pc.J < b1) issue(s);

  StageCursor cc;
  cursor_begin(cc, b0, b1, BN);
  int64_t consumed = 0;
  uint32_t parity = 0;  // bit s: phase of slot s
  float hi[4][1], lo[4][1];
#pragma unroll
  for (int i = 0; i < 4; ++i) hi[i][0] = lo[i][0] = 0.f;
  int slot = 0;
  while (cc.I * BN + cc.J < b1) {
    const int n = (int)min((int64_t)S::kStageBlocks, cc.Jend - cc.J);
    const bool ok = mbar_wait(bar0 + 8 * slot, (parity >> slot) & 1u);
    if (!__all_sync(0xFFFFFFFFu, ok)) {  // a copy did not land in time: report, drain, leave
      if (lane == 0) {
        atomicExch(status, WHFF_ETIMEOUT);
        for (int64_t t = consumed; t < issued; ++t) {
          const int s = (int)(t % S::kNS);
          (void)mbar_wait(bar0 + 8 * s, (uint32_t)((t / S::kNS) & 1));
        }
      }
      __syncwarp();
      return;
    }
    parity ^= 1u << slot;
    const uint8_t* src = stream + (uint64_t)(cc.I * BN + cc.J) * (uint64_t)S::kBB;
    const uint8_t* base = ring + slot * S::kSlotBytes + (reinterpret_cast<uintptr_t>(src) & 15u);
    const int64_t J0 = cc.J;
#pragma unroll
    for (int u = 0; u < S::kU; u += 2) {
      const int j0 = lane + 32 * u, j1 = j0 + 32;
      if (j1 < n) {  // a whole pair
        uint32_t w0[NW], w1[NW];
        wz2_lds<RATE>(base + j0 * S::kBB, w0);
        wz2_lds<RATE>(base + j1 * S::kBB, w1);
        float p0[4][1], p1[4][1];
        wz2_block_partial<RATE, LIFT, 1, LIFT>(w0, x, ldx, 4 * (J0 + j0), N, x_fast, x_vec_ok, p0);
        wz2_block_partial<RATE, LIFT, 1, LIFT>(w1, x, ldx, 4 * (J0 + j1), N, x_fast, x_vec_ok, p1);
#pragma unroll
        for (int i = 0; i < 4; ++i) two_sum_acc(hi[i][0], lo[i][0], p0[i][0] + p1[i][0]);
      } else if (j0 < n) {  // the lane's odd last block of the piece
        uint32_t w0[NW];
        wz2_lds<RATE>(base + j0 * S::kBB, w0);
        float p0[4][1];
        wz2_block_partial<RATE, LIFT, 1, LIFT>(w0, x, ldx, 4 * (J0 + j0), N, x_fast, x_vec_ok, p0);
#pragma unroll
        for (int i = 0; i < 4; ++i) two_sum_acc(hi[i][0], lo[i][0], p0[i][0]);
      }
    }
    __syncwarp();  // every lane has read the slot
    ++consumed;
    if (pc.I * BN + pc.J < b1) issue(slot);
    slot = slot + 1 == S::kNS ? 0 : slot + 1;
    const int64_t I = cc.I;
    cursor_next(cc, n, b1, BN);
    if (cc.I != I) {  // the piece of band I is complete: fold it as wz2_gemv_kernel does
      const int64_t g_lo = (I * BN) / L, g_hi = ((I + 1) * BN - 1) / L;
      if (g_lo == g_hi) {
        wz2_finish<LIFT, 1>(hi, lo, lane, 4 * I, M, 0, 1, 4 * BM, ws, y, ldy, state, decay, red32);
      } else {
        wz2_finish<LIFT, 1>(hi, lo, lane, 4 * ((I * maxseg + (g - g_lo)) * 1), M, 0, 2, 0, ws, y, ldy, state, decay,
                            red32);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) hi[i][0] = lo[i][0] = 0.f;
    }
  }
}

}  // namespace dev
}  // namespace whff
