// Packed FP32 complex arithmetic for sm_103a: fma.rn.f32x2 does two FP32
// FMAs in one instruction (it occupies the FMA pipe as two, but takes one
// issue slot).  A complex multiply-add acc += a b becomes two packed FMAs,
//   acc += (b.x, b.x) (a.x, a.y) + (-b.y, b.y) (a.y, a.x),
// with the operator entry b stored as the quad (b.x, b.x, -b.y, b.y).
#pragma once

#include <cuda_runtime.h>

namespace qf {
namespace dev {

typedef unsigned long long f32x2;  // two packed floats (x in the low word)

__device__ __forceinline__ f32x2 ffma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f32x2 pk2(float x, float y) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ float2 upk2(f32x2 a) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(a));
  return r;
}
__device__ __forceinline__ f32x2 pswap(f32x2 a) {  // (x, y) -> (y, x)
  const float2 v = upk2(a);
  return pk2(v.y, v.x);
}

// Operator entry b as two packed pairs: (b.x, b.x) and (-b.y, b.y).
struct OpE {
  f32x2 re, im;
};
__device__ __forceinline__ OpE load_op(const float4* ops, int i) {
  const float4 v = ops[i];
  return OpE{pk2(v.x, v.y), pk2(v.z, v.w)};
}
// The same from shared memory as one 16-byte load into the two pairs.  The
// asm is volatile so that the compiler reloads the entry at every use
// instead of hoisting a whole operator into registers out of a loop.
__device__ __forceinline__ OpE lds_op(const float4* ops, int i) {
  OpE e;
  asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];"
               : "=l"(e.re), "=l"(e.im)
               : "r"((unsigned)__cvta_generic_to_shared(ops + i)));
  return e;
}
__device__ __forceinline__ float4 op_quad(double2 b) {
  return make_float4((float)b.x, (float)b.x, (float)-b.y, (float)b.y);
}
// acc += a * b, a_sw = pswap(a)
__device__ __forceinline__ f32x2 cmad2(f32x2 acc, f32x2 a, f32x2 a_sw, OpE b) {
  return ffma2(b.im, a_sw, ffma2(b.re, a, acc));
}

}  // namespace dev
}  // namespace qf
