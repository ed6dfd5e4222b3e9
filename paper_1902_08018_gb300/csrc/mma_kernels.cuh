// mma_kernels.cuh -- many right-hand sides on the 5th-generation tensor cores.
//
// With R right-hand sides the step Y = A X is a dense contraction (Sec. 4.4's
// GEMV becomes a GEMM), so for R >= 16 the fixed-allocation (WZ2) kernels run
// it on tcgen05.  In the transform domain the contraction is
//     Z_band = sum_J (s_J V_J) ((2G)^T X_J),   Y_band = (2G) Z_band * 2^-3,
// a GEMM whose A operand is the stored integer coefficients (|v| < 2^22)
// times a power-of-two block scale, and whose B operand is the transformed x.
//
// Precision (the 1e-6 bar): A splits EXACTLY into three BF16 pieces (8+8+6
// bits); B (FP32) into three BF16 pieces (8+8+8 bits, exact).  Six products
// A_p B_q with p+q <= 2 are issued (kind::f16, BF16 in, FP32 accumulate in
// TMEM); the dropped ones are below 2^-24 of |a||x|.  The TMEM accumulator
// covers one stage (16 blocks = 64 columns of K) and is drained into TwoSum
// FP32 registers after every stage, so FP32 rounding never sees long sums.
//
// CTA = 8 warps = 256 threads; tile = 32 bands (128 coefficient rows) x NR
// right-hand sides x a column range of the matrix.  Per stage every thread
// decodes 2 blocks into the A tile (shared memory, canonical no-swizzle
// K-major layout: 8x16-byte core matrices, 128 B apart along K and 256 B
// apart along M/N) and copies its part of the B tile, which a small kernel
// builds once per step for all stages; one thread issues the 24 MMAs and
// commits them to an mbarrier; the next stage's blocks are loaded meanwhile;
// all threads wait (bounded) and drain TMEM (warps w and w+4 share the lanes
// 32(w%4).. and take half the columns each).  Partials go to a workspace per
// column split; mma_finish sums splits, mixes with 2G and applies the state.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

#include "whff.h"
#include "wz2_kernels.cuh"

namespace whff {
namespace dev {

constexpr int kMmaThreads = 256;       // 8 warps; warps w and w+4 share TMEM lanes 32(w%4)..
constexpr int kMmaBands = 32;         // 128 coefficient rows per tile
constexpr int kMmaStageBlocks = 16;   // K = 64 per stage
constexpr int kMmaKSteps = 4;         // K = 16 per instruction
constexpr uint32_t kMmaSpinLimit = 1u << 22;  // try_wait polls: bounded to seconds

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 64-bit shared-memory matrix descriptor: start >> 4 (bits 0-13), leading
// byte offset >> 4 (16-29), stride byte offset >> 4 (32-45), descriptor
// version 1 (bit 46), no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor, kind::f16: F32 accumulator (bits 4-5 = 1), A and B
// BF16 (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at 24.
template <int NR>
__device__ __forceinline__ constexpr uint32_t mma_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NR >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
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

template <int NR>
struct MmaSmem {
  static constexpr int kATile = 128 * 16 * 2;  // one piece, one K step
  static constexpr int kBTile = NR * 16 * 2;
  static constexpr int kA = 3 * kMmaKSteps * kATile;
  static constexpr int kB = 3 * kMmaKSteps * kBTile;
  static constexpr int kBytes = kA + kB + 64;  // + mbarrier and TMEM slot
};

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < kMmaSpinLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

template <int NR>
__device__ __forceinline__ void tmem_load_row(uint32_t taddr, float (&v)[NR]);

template <>
__device__ __forceinline__ void tmem_load_row<32>(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tmem_load_row<8>(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tmem_load_row<16>(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// The B operand of every stage, built once per step: for column block J and
// right-hand side r, (2G)^T x_J (or x_J without the lift) in three BF16
// pieces, already in the shared-memory tile layout of its 16-block stage:
// out[stage][piece][kstep] = NR x 16 BF16 tile.  Thread per (stage, J, r).
template <bool LIFT, int NR>
__global__ void wz2_mma_btiles(const float* __restrict__ x, int64_t ldx, int64_t N, int R, int64_t nstages,
                               uint8_t* __restrict__ out) {
  using S = MmaSmem<NR>;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nstages * kMmaStageBlocks * NR) return;
  const int r = (int)(q % NR);
  const int jl = (int)((q / NR) % kMmaStageBlocks);
  const int64_t stage = q / ((int64_t)NR * kMmaStageBlocks);
  const int64_t J = stage * kMmaStageBlocks + jl;
  float xt[4] = {0.f, 0.f, 0.f, 0.f};
  if (r < R) {
    float xv[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) xv[c] = 4 * J + c < N ? __ldg(x + (int64_t)r * ldx + 4 * J + c) : 0.f;
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
  uint8_t* base = out + stage * (int64_t)S::kB;
#pragma unroll
  for (int pc = 0; pc < 3; ++pc)
    *reinterpret_cast<uint2*>(base + (pc * kMmaKSteps + kstep) * S::kBTile + tile_off(r, kk)) =
        make_uint2(pack2(p[pc][0], p[pc][1]), pack2(p[pc][2], p[pc][3]));
}

// Grid: (ceil(BM/32), ksplit).  ws[(split * R + r) * Mpad + coefficient row]
// receives the split's FP64 partial of Z (coefficient rows, not yet mixed).
// Thread t decodes blocks (t & 7) and (t & 7) + 8 of band t >> 3 in every
// stage; the next stage's compressed words are loaded while the MMAs of the
// current one run.
template <int RATE, bool LIFT, int NR>
__global__ void __launch_bounds__(kMmaThreads, 2)
    wz2_mma_kernel(const uint8_t* __restrict__ stream, int64_t BM, int64_t BN, const uint8_t* __restrict__ btiles,
                   int R, int64_t jchunk, double* __restrict__ ws, int64_t Mpad, int* __restrict__ status) {
  using S = MmaSmem<NR>;
  constexpr int NW = Wz2Layout<RATE>::kWords;
  constexpr int HALF = NR / 2;  // TMEM columns drained by each of the two warps on a lane quarter
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* As = smem;
  uint8_t* Bs = smem + S::kA;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S::kA + S::kB);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::kA + S::kB + 16);

  const int t = threadIdx.x, warp = t >> 5;
  const int64_t band0 = (int64_t)blockIdx.x * kMmaBands;
  const int split = blockIdx.y;
  const int64_t J0 = (int64_t)split * jchunk;  // a multiple of the 16-block stage
  const int64_t J1 = min(BN, J0 + jchunk);
  const uint32_t bar_a = smem_addr(bar);

  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_a));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {  // TMEM: NR fp32 columns (at least 32)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(tslot)),
                 "r"(NR < 32 ? 32 : NR));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;

  float hi[HALF], lo[HALF];
#pragma unroll
  for (int r = 0; r < HALF; ++r) hi[r] = lo[r] = 0.f;

  const int my_band = t >> 3;
  const int my_sub = t & 7;
  const int64_t band = band0 + my_band;
  constexpr int kBVec = S::kB / 16;                              // uint4 in a B tile
  constexpr int BV = (kBVec + kMmaThreads - 1) / kMmaThreads;    // per thread (the last one guarded)
  // two stages of compressed words in flight (ring of 2), one B tile ahead
  uint32_t w[2][2][NW];
  uint4 bnext[BV];
  auto fetch = [&](int slot, int64_t Js) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t J = Js + my_sub + 8 * u;
      if (band < BM && J < J1) {
        wz2_load<RATE>(stream, band * BN + J, w[slot][u]);
      } else {
#pragma unroll
        for (int i = 0; i < NW; ++i) w[slot][u][i] = 0u;  // a zero block: E = 0, scale 0
      }
    }
  };
  auto fetch_b = [&](int64_t Js) {
    const uint4* src = reinterpret_cast<const uint4*>(btiles + (Js / kMmaStageBlocks) * (int64_t)S::kB);
#pragma unroll
    for (int i = 0; i < BV; ++i)
      if (t + i * kMmaThreads < kBVec) bnext[i] = __ldg(src + t + i * kMmaThreads);
  };
  // The descriptors of a stage never change: base descriptors of the A and B
  // tiles plus a compile-time offset in 16-byte units in the start-address
  // field (shared addresses stay below 256 KB, so the field cannot carry).
  const uint64_t a_base = smem_desc(smem_addr(As), 128, 256);
  const uint64_t b_base = smem_desc(smem_addr(Bs), 128, 256);
  if (J0 < J1) {
    fetch(0, J0);
    fetch_b(J0);
  }
  if (J0 + kMmaStageBlocks < J1) fetch(1, J0 + kMmaStageBlocks);
  bool ok = true;
  uint32_t phase = 0;
  // one stage; `slot` is a literal at every call, so the ring stays in registers
  auto stage = [&](const int slot, const int64_t Js) -> bool {
    // ---- A tile: this thread's 2 blocks of its band
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int jl = my_sub + 8 * u;
      uint32_t (&wu)[NW] = w[slot][u];
      const uint32_t E = wu[0] & 0xFFu, K = (wu[0] >> 8) & 31u;
      const float s = E ? __uint_as_float((E + K - 27u) << 23) : 0.f;
      float f[16], V[16];
      wz2_fields<RATE>(wu, f);
      wz2_unpermute<LIFT>(f, V);
      const int kstep = jl >> 2, kk = (jl & 3) * 4;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int row = 4 * my_band + a;
        __nv_bfloat16 p[3][4];
#pragma unroll
        for (int b = 0; b < 4; ++b) split3(V[4 * a + b] * s, p[0][b], p[1][b], p[2][b]);
#pragma unroll
        for (int pc = 0; pc < 3; ++pc)
          *reinterpret_cast<uint2*>(As + (pc * kMmaKSteps + kstep) * S::kATile + tile_off(row, kk)) =
              make_uint2(pack2(p[pc][0], p[pc][1]), pack2(p[pc][2], p[pc][3]));
      }
    }
    // ---- B tile: this stage's prebuilt pieces (fetched one stage ahead)
    {
      uint4* dst = reinterpret_cast<uint4*>(Bs);
#pragma unroll
      for (int i = 0; i < BV; ++i)
        if (t + i * kMmaThreads < kBVec) dst[t + i * kMmaThreads] = bnext[i];
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic writes -> tensor-core reads
    __syncthreads();
    if (t == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      constexpr uint32_t idesc = mma_idesc<NR>();
      uint32_t acc = 0;
#pragma unroll
      for (int ks = 0; ks < kMmaKSteps; ++ks) {
#pragma unroll
        for (int m = 0; m < 6; ++m) {
          // products A_p B_q with p + q <= 2: (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
          const int pa = m == 2 || m == 4 ? 1 : m == 5 ? 2 : 0;
          const int pb = m == 1 || m == 4 ? 1 : m == 3 ? 2 : 0;
          const uint64_t ad = a_base + (uint64_t)(((pa * kMmaKSteps + ks) * S::kATile) >> 4);
          const uint64_t bd = b_base + (uint64_t)(((pb * kMmaKSteps + ks) * S::kBTile) >> 4);
          asm volatile(
              "{\n\t.reg .pred p;\n\t"
              "setp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          acc = 1;
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar_a)
                   : "memory");
    }
    // loads in flight while the tensor cores work: the B tile of the next stage
    // and the compressed blocks of the stage after it (this slot is now free)
    if (Js + kMmaStageBlocks < J1) fetch_b(Js + kMmaStageBlocks);
    if (Js + 2 * kMmaStageBlocks < J1) fetch(slot, Js + 2 * kMmaStageBlocks);
    // every thread waits (bounded) for the commit; the CTA then agrees on the
    // outcome, so a timeout is a uniform exit and never a barrier deadlock
    if (!__syncthreads_and(mbar_wait(bar_a, phase) ? 1 : 0)) {
      ok = false;
      if (t == 0) atomicExch(status, WHFF_ETIMEOUT);
      (void)mbar_wait(bar_a, phase);  // give the MMAs in flight a second bounded chance
      return false;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    float v[HALF];
    // lane quarter (warp % 4), column half (warp / 4)
    tmem_load_row<HALF>(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(HALF * (warp >> 2)), v);
#pragma unroll
    for (int r = 0; r < HALF; ++r) two_sum_acc(hi[r], lo[r], v[r]);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();  // the next stage overwrites the tiles and the accumulator
    return true;
  };
  for (int64_t Js = J0; Js < J1 && ok; Js += 2 * kMmaStageBlocks) {
    ok = stage(0, Js);
    if (ok && Js + kMmaStageBlocks < J1) ok = stage(1, Js + kMmaStageBlocks);
  }
  if (ok) {
    const int64_t row = 4 * band0 + 32 * (warp & 3) + (t & 31);  // coefficient row of the tile
    const int c0 = HALF * (warp >> 2);
    if (row < Mpad) {
#pragma unroll
      for (int r = 0; r < HALF; ++r)
        if (c0 + r < R) ws[((int64_t)split * R + c0 + r) * Mpad + row] = (double)hi[r] + (double)lo[r];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NR < 32 ? 32 : NR));
  }
}

// Sum the column splits of Z in order, map each band's 4 coefficient rows to
// y (2G mix and 2^-3 with the lift, 2^3 without) and update the state in
// column order.  Thread per band.
template <bool LIFT>
__global__ void wz2_mma_finish(const double* __restrict__ ws, int ksplit, int R, int64_t Mpad, int64_t M,
                               double* __restrict__ y, int64_t ldy, double* __restrict__ state, double decay) {
  const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (4 * I >= M) return;
  double s[4] = {0, 0, 0, 0};
  if (state)
    for (int i = 0; i < 4; ++i)
      if (4 * I + i < M) s[i] = state[4 * I + i];
  for (int r = 0; r < R; ++r) {
    double z[4];
    for (int i = 0; i < 4; ++i) {
      double t = 0.0;
      for (int k = 0; k < ksplit; ++k) t += ws[((int64_t)k * R + r) * Mpad + 4 * I + i];
      z[i] = t;
    }
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
      if (4 * I + i < M) {
        y[(int64_t)r * ldy + 4 * I + i] = yy[i];
        s[i] = decay * s[i] + yy[i];
      }
  }
  if (state)
    for (int i = 0; i < 4; ++i)
      if (4 * I + i < M) state[4 * I + i] = s[i];
}

}  // namespace dev
}  // namespace whff
