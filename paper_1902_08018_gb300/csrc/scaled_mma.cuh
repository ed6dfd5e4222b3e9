// scaled_mma.cuh -- many right-hand sides on the tensor cores for the scaled
// element formats (BF16, FP16, FP8 E4M3 with one FP32 scale per 128 x 128
// tile).
//
// Y = A X with A stored as element values q times the tile scale s: inside
// one 128 x 128 scale tile the contraction is s (Q X), so the tensor cores
// multiply the stored values themselves and the scale is applied when the
// tile's columns have all been accumulated.  Q is exact in BF16 pieces (one
// piece for BF16 and FP8 E4M3, two for FP16's 11 significant bits); X is split
// into three BF16 pieces as in the fixed-allocation kernel, the products
// Q_p X_q with p + q <= 2 go to three TMEM accumulators by size, and every
// two stages (128 columns: exactly one scale tile) the accumulators are added,
// multiplied by s (the product's rounding error kept exactly with an FMA) and
// drained into TwoSum FP32 registers.
//
// Same persistent pipeline as wz2_mma_kernel: items are (tile of 128 rows,
// stage of 64 columns), CTA g takes items [g L, g L + L), two stages in
// flight (A and B tiles of buffer k % 2), the B tiles prebuilt per pass and
// brought in with cp.async.bulk.  The A tile needs no decode for BF16: a
// thread moves 16 bytes (8 values of one row) from HBM to one 16-byte row of
// a core matrix; lanes take 8 consecutive rows, so every warp store fills
// whole core matrices without bank conflicts.
#pragma once
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "mma_kernels.cuh"

namespace whff {
namespace dev {

template <int FMT>
struct ScaledMmaTraits {
  static constexpr int kEB = FMT == 4 ? 1 : 2;          // bytes per element
  static constexpr int kPA = FMT == 3 ? 2 : 1;          // BF16 pieces of a value
  static constexpr int kLoads = kEB == 2 ? 4 : 2;       // 16-byte loads per thread and stage
  static_assert(FMT == 2 || FMT == 3 || FMT == 4, "BF16, FP16 or FP8 E4M3 storage");
};

template <int FMT, int NR>
struct ScaledMmaSmem {
  static constexpr int kATile = 128 * 16 * 2;  // one piece, one K step
  static constexpr int kA = ScaledMmaTraits<FMT>::kPA * kMmaKSteps * kATile;
  static constexpr int kB = MmaBTile<NR>::kB;
  static constexpr int kBars = 2 * (kA + kB);
  static constexpr int kBytes = kBars + 64;  // 4 mbarriers, TMEM slot, flags
};

// 16 bytes of storage -> BF16 piece pairs in tile order: out[p][h] is piece p
// of elements 2h, 2h+1 of an 8-value chunk (FP8: two chunks, c = 0, 1).
template <int FMT>
__device__ __forceinline__ void scaled_mma_pieces(uint4 raw, uint32_t (&out)[2][ScaledMmaTraits<FMT>::kPA][4]) {
  const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
  if constexpr (FMT == 2) {  // BF16: the stored bits are the piece
#pragma unroll
    for (int h = 0; h < 4; ++h) out[0][0][h] = w[h];
  } else if constexpr (FMT == 3) {  // FP16 -> FP32 -> two exact BF16 pieces
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      __half2_raw hr;
      hr.x = (unsigned short)(w[h] & 0xFFFF);
      hr.y = (unsigned short)(w[h] >> 16);
      const float2 v = __half22float2(__half2(hr));
      const uint32_t p0 = bf16x2_rn(v.x, v.y);
      out[0][0][h] = p0;
      out[0][1][h] = bf16x2_rn(v.x - bf16_lo(p0), v.y - bf16_hi(p0));
    }
  } else {  // FP8 E4M3 -> FP16 -> FP32 -> BF16 (exact: 4 significant bits)
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint32_t pair = (w[q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
      const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)pair, __NV_E4M3);
      const float2 v = __half22float2(__half2(hr));
      out[q >> 2][0][q & 3] = bf16x2_rn(v.x, v.y);
    }
  }
}

// Persistent grid over the (tile, stage) items of one matrix: tiles of 128
// rows, stages of 64 columns, S stages per tile.  ws[((tile * maxseg + seg) *
// R + r) * 128 + m] receives the FP64 partial of tile row m for the CTA's
// segment seg = g - (tile S) / L.
template <int FMT, int NR>
__global__ void __launch_bounds__(kMmaThreads, 2)
    scaled_mma_kernel(const uint8_t* __restrict__ payload, const float* __restrict__ scales, int64_t M, int64_t ld,
                      int64_t TN, const uint8_t* __restrict__ btiles, double* __restrict__ ws, int S, int R,
                      int maxseg, int64_t total, int64_t L, int* __restrict__ status, uint32_t spin) {
  using SM = ScaledMmaSmem<FMT, NR>;
  using TR = ScaledMmaTraits<FMT>;
  constexpr int PA = TR::kPA, NL = TR::kLoads, EB = TR::kEB;
  constexpr int HALF = NR / 2;  // TMEM columns drained by each of the two warps on a lane quarter
  constexpr uint32_t kCols = mma_tmem_cols<NR>();
  extern __shared__ __align__(1024) uint8_t smem[];
  const uint32_t s_base = smem_addr(smem);
  const uint32_t mma_bar = s_base + SM::kBars;  // two mbarriers: MMAs of buffer 0, 1 done
  const uint32_t b_bar = mma_bar + 16;          // two mbarriers: B tile of buffer 0, 1 landed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + SM::kBars + 32);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + SM::kBars + 36);
  int64_t* last_commit = reinterpret_cast<int64_t*>(smem + SM::kBars + 40);
  int64_t* last_copy = reinterpret_cast<int64_t*>(smem + SM::kBars + 48);

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int64_t it0 = (int64_t)blockIdx.x * L;
  const int64_t n = max((int64_t)0, min(total, it0 + L) - it0);
  if (t == 0) {
    mbar_init(mma_bar, 1);
    mbar_init(mma_bar + 8, 1);
    mbar_init(b_bar, 1);
    mbar_init(b_bar + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *abort_flag = 0;
    *last_commit = *last_copy = -1;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(tslot)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;

  // load assignment: lane l takes row 8G + l%8 of the tile; 16-bit formats:
  // load u covers group G = (4 warp + u) / 2, chunk 4((4 warp + u) % 2) + l/8
  // (8 columns); FP8: group G = 2 warp + u, columns 16 (l/8) .. + 15
  const int r8 = lane & 7, q8 = lane >> 3;
  // drain assignment: tile row 32(warp%4) + lane, accumulator columns HALF(warp/4)..
  const int m_row = 32 * (warp & 3) + lane;
  const int c0 = HALF * (warp >> 2);
  auto load_row = [&](int u) { return EB == 2 ? 8 * ((4 * warp + u) >> 1) + r8 : 8 * (2 * warp + u) + r8; };
  auto load_col = [&](int u) { return EB == 2 ? 8 * (4 * ((4 * warp + u) & 1) + q8) : 16 * q8; };

  const int tile0 = (int)(it0 / S), st0 = (int)(it0 - (int64_t)tile0 * S);
  int f_tile = tile0, f_st = st0;  // fetch
  int m_tile = tile0, m_st = st0;  // issue
  int b_st = st0;                  // thread 0: the next B copy's stage
  auto advance = [&](int& tile, int& st) {
    if (++st == S) st = 0, ++tile;
  };

  uint4 w[2][NL];  // storage of two stages (ring)
  auto fetch = [&](int slot) {
#pragma unroll
    for (int u = 0; u < NL; ++u) {
      const int64_t row = 128 * (int64_t)f_tile + load_row(u);
      const int64_t col = 64 * (int64_t)f_st + load_col(u);  // first element of the 16 bytes
      w[slot][u] = (row < M && col < ld)
                       ? __ldcs(reinterpret_cast<const uint4*>(payload + ((uint64_t)row * ld + col) * EB))
                       : make_uint4(0u, 0u, 0u, 0u);
    }
    advance(f_tile, f_st);
  };
  auto b_copy = [&](int64_t k) {  // thread 0: B tile of stage k into buffer k % 2
    const int buf = (int)(k & 1);
    bulk_copy_g2s(s_base + 2 * SM::kA + buf * SM::kB, btiles + (int64_t)b_st * SM::kB, (uint32_t)SM::kB,
                  b_bar + 8 * buf);
    if (++b_st == S) b_st = 0;
    *last_copy = k;
  };
  auto fail = [&]() {
    atomicExch(status, WHFF_ETIMEOUT);
    *abort_flag = 1;
  };

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
  // drain accumulator group `acc` of tile `tile`, whose tile scale is s:
  // s (sum of the three accumulators) enters the TwoSum sums with the exact
  // rounding error of the product
  auto drain = [&](int acc, int tile, float s) {
    if (tile != cur_tile) {
      flush();
      cur_tile = tile;
    }
    const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(3 * acc * NR + c0);
#pragma unroll
    for (int h = 0; h < HALF; h += 8) {
      float v[8];
      tmem_load_sum8(ta + h, NR, v);
#pragma unroll
      for (int r = 0; r < 8; r += 2) {  // packed pairs of columns: each half rounds as the scalar steps
        const float2 ps = make_float2(__fmul_rn(v[r], s), __fmul_rn(v[r + 1], s));
        float2 H = make_float2(hi[h + r], hi[h + r + 1]), Lo = make_float2(lo[h + r], lo[h + r + 1]);
        two_sum_acc2(H, Lo, ps);
        Lo = add_f2(Lo, fma_f2(make_float2(v[r], v[r + 1]), make_float2(s, s), make_float2(-ps.x, -ps.y)));
        hi[h + r] = H.x, hi[h + r + 1] = H.y, lo[h + r] = Lo.x, lo[h + r + 1] = Lo.y;
      }
    }
  };

  const uint64_t a_desc0 = smem_desc(s_base, 128, 256);
  const uint64_t b_desc0 = smem_desc(s_base + 2 * SM::kA, 128, 256);
  bool ok = true;
  // accumulator groups: the stages of one scale tile column (2 stages = 128
  // columns) of one tile share an accumulator group (alternating 0, 1)
  int gpos = 0, gacc = 0;
  bool p_ends = false;
  int p_acc = 0, p_tile = tile0;
  float p_s = 0.f;  // the closed group's tile scale, loaded a stage before its drain
  if (n > 0) {
    fetch(0);
    if (t == 0) b_copy(0);
  }
  if (n > 1) fetch(1);

  auto stage = [&](const int buf, const int64_t k) -> bool {
    uint8_t* As = smem + buf * SM::kA;
#pragma unroll
    for (int u = 0; u < NL; ++u) {
      uint32_t d[2][PA][4];
      scaled_mma_pieces<FMT>(w[buf][u], d);
      const int row = load_row(u);
#pragma unroll
      for (int c = 0; c < (EB == 2 ? 1 : 2); ++c) {
        const int k0 = load_col(u) + 8 * c;  // first of 8 columns within the stage
        const uint32_t off = (uint32_t)((((row >> 3) * 2 + ((k0 >> 3) & 1)) * 128) + (row & 7) * 16);
#pragma unroll
        for (int p = 0; p < PA; ++p)
          *reinterpret_cast<uint4*>(As + (p * kMmaKSteps + (k0 >> 4)) * SM::kATile + off) =
              make_uint4(d[c][p][0], d[c][p][1], d[c][p][2], d[c][p][3]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    if (!__syncthreads_and(ok ? 1 : 0)) return false;
    const bool init = gpos == 0;
    const int acc = gacc;
    const int tile_k = m_tile, tc_k = m_st >> 1;
    const bool ends = ++gpos == kMmaDrainStages || (m_st & 1) || m_st == S - 1 || k == n - 1;
    if (ends) gpos = 0, gacc ^= 1;
    advance(m_tile, m_st);
    if (t == 0) {
      if (!mbar_wait(b_bar + 8 * buf, (uint32_t)((k >> 1) & 1), spin)) {
        ok = false;
        fail();
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint64_t ad0 = a_desc0 + (uint64_t)((buf * SM::kA) >> 4);
        const uint64_t bd0 = b_desc0 + (uint64_t)((buf * SM::kB) >> 4);
        const uint32_t d0 = tmem + (uint32_t)(3 * acc * NR);
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
    if (k + 2 < n) fetch(buf);
    if (k >= 1) {
      const bool done =
          __all_sync(0xFFFFFFFFu, mbar_wait(mma_bar + 8 * (buf ^ 1), (uint32_t)(((k - 1) >> 1) & 1), spin));
      if (!done) {
        if (ok && lane == 0) fail();
        ok = false;
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (t == 0 && ok && k + 1 < n) b_copy(k + 1);
        if (p_ends) drain(p_acc, p_tile, p_s);
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      }
    } else if (t == 0 && ok && k + 1 < n) {
      b_copy(k + 1);
    }
    p_ends = ends;
    p_acc = acc;
    p_tile = tile_k;
    if (ends) p_s = __ldg(scales + (int64_t)tile_k * TN + tc_k);
    return true;
  };

  bool alive = true;
  for (int64_t k = 0; k < n && alive; k += 2) {
    alive = stage(0, k);
    if (alive && k + 1 < n) alive = stage(1, k + 1);
  }
  if (alive && n > 0) alive = __syncthreads_and(ok ? 1 : 0) != 0;
  if (alive && n > 0) {
    const int buf = (int)((n - 1) & 1);
    if (__all_sync(0xFFFFFFFFu, mbar_wait(mma_bar + 8 * buf, (uint32_t)(((n - 1) >> 1) & 1), spin))) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      drain(p_acc, p_tile, p_s);
      flush();
    } else if (lane == 0) {
      fail();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (t == 0 && *abort_flag) {  // let the MMAs and the copy in flight end (bounded) before the CTA exits
    const int64_t c = *last_commit, b = *last_copy;
    if (c >= 0) (void)mbar_wait(mma_bar + 8 * (int)(c & 1), (uint32_t)((c >> 1) & 1));
    if (b >= 0) (void)mbar_wait(b_bar + 8 * (int)(b & 1), (uint32_t)((b >> 1) & 1));
  }
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols));
  }
}

// y[r][128 tile + m] = the tile's segment partials of row m, added in order.
// Thread per (tile, column, row of the tile), the row fastest.
// Per column r of x (FP16 passes): e_r with max |x_r| * 2^e_r < 2^15, so that
// the scaled column's FP16 pieces stay below the FP16 maximum (0 for a zero
// column).  A block per column.
static __global__ void f16_colexp_kernel(const float* __restrict__ x, int64_t ldx, int64_t N, int R,
                                         int* __restrict__ colexp) {
  const int r = (int)blockIdx.x;
  float m = 0.f;
  if (r < R)
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) m = fmaxf(m, fabsf(__ldg(x + (int64_t)r * ldx + i)));
  __shared__ float red[32];
#pragma unroll
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) m = fmaxf(m, red[k]);
    int e = 0;
    if (m > 0.f) (void)frexpf(m, &e);  // m < 2^e
    colexp[r] = m > 0.f ? 15 - e : 0;
  }
}

// B tiles of an FP16 pass: x_J * 2^e_r in three FP16 pieces (exact: 11 + 11 +
// 11 significant bits cover FP32's 24; the scale keeps the first below 2^15),
// in the tile layout of wz2_mma_btiles.  Thread per (stage, J, r).
template <int NR>
static __global__ void f16_mma_btiles(MmaPass ps, const int* __restrict__ colexp, int64_t threads) {
  using S = MmaBTile<NR>;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= threads) return;
  const int r = (int)(q % NR);
  const int jl = (int)((q / NR) % kMmaStageBlocks);
  const int64_t stage = q / ((int64_t)NR * kMmaStageBlocks);
  const int64_t J = stage * kMmaStageBlocks + jl;
  __half p[3][4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float v = 0.f;
    if (r < ps.R && 4 * J + c < ps.N) v = ldexpf(__ldg(ps.x + (int64_t)r * ps.ldx + 4 * J + c), colexp[r]);
    const __half h0 = __float2half_rn(v);
    const float r1 = v - __half2float(h0);
    const __half h1 = __float2half_rn(r1);
    p[0][c] = h0;
    p[1][c] = h1;
    p[2][c] = __float2half_rn(r1 - __half2float(h1));
  }
  const int kstep = jl >> 2, kk = (jl & 3) * 4;
  uint8_t* base = ps.btiles + stage * (int64_t)S::kB;
#pragma unroll
  for (int pc = 0; pc < 3; ++pc) {
    const uint32_t lo = (uint32_t)__half_as_ushort(p[pc][0]) | ((uint32_t)__half_as_ushort(p[pc][1]) << 16);
    const uint32_t hi = (uint32_t)__half_as_ushort(p[pc][2]) | ((uint32_t)__half_as_ushort(p[pc][3]) << 16);
    *reinterpret_cast<uint2*>(base + (kstep * 3 + pc) * S::kBTile + tile_off(r, kk)) = make_uint2(lo, hi);
  }
}

// colexp (FP16 passes, else null): y of column r is the sum times 2^-e_r (exact).
static __global__ void scaled_mma_finish(const double* __restrict__ ws, int64_t M, int S, int R, int maxseg,
                                         int64_t tiles, int64_t L, double* __restrict__ y, int64_t ldy,
                                         const int* __restrict__ colexp) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= tiles * R * 128) return;
  const int m = (int)(q & 127);
  const int64_t tr = q >> 7;
  const int r = (int)(tr % R);
  const int64_t tile = tr / R;
  const int64_t row = 128 * tile + m;
  if (row >= M) return;
  const int64_t first = tile * S;
  const int nseg = (int)((first + S - 1) / L - first / L + 1);
  double acc = 0.0;
  for (int g = 0; g < nseg; ++g) acc += ws[((tile * maxseg + g) * R + r) * 128 + m];
  y[(int64_t)r * ldy + row] = colexp ? ldexp(acc, -colexp[r]) : acc;
}

}  // namespace dev
}  // namespace whff
