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
// CTA = 4 warps = 128 threads; tile = 32 bands (128 coefficient rows) x NR
// right-hand sides x a column range of the matrix.  Per stage every thread
// decodes 4 blocks into the A tile and transforms 4 x-chunks into the B tile
// (shared memory, canonical no-swizzle K-major layout: 8x16-byte core
// matrices, 128 B apart along K and 256 B apart along M/N); one thread issues
// the 24 MMAs and commits them to an mbarrier; all threads wait (bounded),
// drain their TMEM lane, and go on.  Partials go to a workspace per column
// split; mma_finish sums splits, mixes with 2G and applies the state.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

#include "whff.h"
#include "wz2_kernels.cuh"

namespace whff {
namespace dev {

constexpr int kMmaThreads = 128;
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

// Grid: (ceil(BM/32), ksplit).  ws[(split * R + r) * Mpad4 + coefficient row]
// receives the split's FP64 partial of Z (coefficient rows, not yet mixed).
template <int RATE, bool LIFT, int NR>
__global__ void __launch_bounds__(kMmaThreads)
    wz2_mma_kernel(const uint8_t* __restrict__ stream, int64_t N, int64_t BM, int64_t BN, const float* __restrict__ x,
                   int64_t ldx, int R, int64_t jchunk, double* __restrict__ ws, int64_t Mpad,
                   int* __restrict__ status) {
  using S = MmaSmem<NR>;
  constexpr int NW = Wz2Layout<RATE>::kWords;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* As = smem;
  uint8_t* Bs = smem + S::kA;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S::kA + S::kB);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::kA + S::kB + 16);

  const int t = threadIdx.x, warp = t >> 5;
  const int64_t band0 = (int64_t)blockIdx.x * kMmaBands;
  const int split = blockIdx.y;
  const int64_t J0 = (int64_t)split * jchunk;
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

  float hi[NR], lo[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) hi[r] = lo[r] = 0.f;

  const int my_band = t >> 2;     // decode: thread -> band (32 bands x 4 threads)
  const int my_sub = t & 3;       // its blocks in a stage: my_sub + 4u, u = 0..3
  const int64_t band = band0 + my_band;
  bool ok = true;
  uint32_t phase = 0;
  for (int64_t Js = J0; Js < J1 && ok; Js += kMmaStageBlocks) {
    // ---- A tile: this thread's 4 blocks of its band
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int jl = my_sub + 4 * u;  // block within the stage, 0..15
      const int64_t J = Js + jl;
      float V[16];
      float s = 0.f;
      if (band < BM && J < J1) {
        uint32_t w[NW];
        wz2_load<RATE>(stream, band * BN + J, w);
        const uint32_t E = w[0] & 0xFFu, K = (w[0] >> 8) & 31u;
        s = E ? __uint_as_float((E + K - 27u) << 23) : 0.f;
        float f[16];
        wz2_fields<RATE>(w, f);
        wz2_unpermute<LIFT>(f, V);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) V[i] = 0.f;
      }
      const int kstep = jl >> 2;          // 4 blocks (16 K) per MMA step
      const int kk = (jl & 3) * 4;        // K offset inside the step
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int row = 4 * my_band + a;
        __nv_bfloat16 p[3][4];
#pragma unroll
        for (int b = 0; b < 4; ++b) split3(V[4 * a + b] * s, p[0][b], p[1][b], p[2][b]);
#pragma unroll
        for (int pc = 0; pc < 3; ++pc) {
          uint8_t* dst = As + (pc * kMmaKSteps + kstep) * S::kATile + tile_off(row, kk);
          *reinterpret_cast<uint2*>(dst) = make_uint2(pack2(p[pc][0], p[pc][1]), pack2(p[pc][2], p[pc][3]));
        }
      }
    }
    // ---- B tile: (2G)^T x for 16 column blocks x NR right-hand sides
    for (int q = t; q < kMmaStageBlocks * NR; q += kMmaThreads) {
      const int jl = q % kMmaStageBlocks, r = q / kMmaStageBlocks;
      const int64_t J = Js + jl;
      float xt[4] = {0.f, 0.f, 0.f, 0.f};
      if (r < R && J < J1) {
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
          xt[0] = xv[0];
          xt[1] = xv[1];
          xt[2] = xv[2];
          xt[3] = xv[3];
        }
      }
      __nv_bfloat16 p[3][4];
#pragma unroll
      for (int b = 0; b < 4; ++b) split3(xt[b], p[0][b], p[1][b], p[2][b]);
      const int kstep = jl >> 2, kk = (jl & 3) * 4;
#pragma unroll
      for (int pc = 0; pc < 3; ++pc) {
        uint8_t* dst = Bs + (pc * kMmaKSteps + kstep) * S::kBTile + tile_off(r, kk);
        *reinterpret_cast<uint2*>(dst) = make_uint2(pack2(p[pc][0], p[pc][1]), pack2(p[pc][2], p[pc][3]));
      }
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
          const uint64_t ad = smem_desc(smem_addr(As + (pa * kMmaKSteps + ks) * S::kATile), 128, 256);
          const uint64_t bd = smem_desc(smem_addr(Bs + (pb * kMmaKSteps + ks) * S::kBTile), 128, 256);
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
    // every thread waits (bounded) for the commit; the CTA then agrees on the
    // outcome, so a timeout is a uniform exit and never a barrier deadlock
    if (!__syncthreads_and(mbar_wait(bar_a, phase) ? 1 : 0)) {
      ok = false;
      if (t == 0) atomicExch(status, WHFF_ETIMEOUT);
      (void)mbar_wait(bar_a, phase);  // give the MMAs in flight a second bounded chance
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    float v[NR];
    tmem_load_row<NR>(tmem + ((uint32_t)(32 * warp) << 16), v);  // lane = row t of the tile
#pragma unroll
    for (int r = 0; r < NR; ++r) two_sum_acc(hi[r], lo[r], v[r]);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();  // the next stage overwrites the tiles and the accumulator
  }
  if (ok) {
    const int64_t row = 4 * band0 + t;  // coefficient row of the tile
    if (row < Mpad) {
#pragma unroll
      for (int r = 0; r < NR; ++r)
        if (r < R) ws[((int64_t)split * R + r) * Mpad + row] = (double)hi[r] + (double)lo[r];
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
