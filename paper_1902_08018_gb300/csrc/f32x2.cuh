// f32x2.cuh -- packed FP32 pairs (add/sub/mul/fma .f32x2: one instruction
// for two lanes of data on GB300) and a TwoSum accumulator on pairs.
#pragma once

namespace whff {
namespace dev {

// Packed FP32 pairs (add/sub/mul/fma .f32x2, one instruction for two lanes
// of data): each half rounds exactly like the scalar instruction.  The
// compiler may fuse a packed multiply into a packed add that consumes it, so
// a product whose rounding matters is formed with scalar __fmul_rn instead.
__device__ __forceinline__ float2 add_f2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 a, b, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
      "add.rn.f32x2 d, a, b;\n\tmov.b64 {%0, %1}, d;\n\t}\n"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 sub_f2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 a, b, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
      "sub.rn.f32x2 d, a, b;\n\tmov.b64 {%0, %1}, d;\n\t}\n"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 mul_f2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 a, b, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
      "mul.rn.f32x2 d, a, b;\n\tmov.b64 {%0, %1}, d;\n\t}\n"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 fma_f2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 a, b, c, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
      "mov.b64 c, {%6, %7};\n\tfma.rn.f32x2 d, a, b, c;\n\tmov.b64 {%0, %1}, d;\n\t}\n"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

// two_sum_acc on a pair of accumulators
__device__ __forceinline__ void two_sum_acc2(float2& hi, float2& lo, float2 p) {
  const float2 s = add_f2(hi, p);
  const float2 bp = sub_f2(s, hi);
  const float2 err = add_f2(sub_f2(hi, sub_f2(s, bp)), sub_f2(p, bp));
  hi = s;
  lo = add_f2(lo, err);
}

}  // namespace dev
}  // namespace whff
