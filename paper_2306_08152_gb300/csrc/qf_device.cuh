// Device helpers shared by the QFactor kernels: complex arithmetic on
// float2 / double2, index deposits, and lane-cooperative 4x4 products.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace qf {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

// Double-float ("df64") reals: a value is the unevaluated sum hi + lo of two
// floats, |lo| <= ulp(hi)/2 after normalisation, about 48 significant bits
// (Dekker 1971; the error-free transformations TwoSum (Knuth) and TwoProd
// via FMA).  A complex df64 tensor entry is 16 bytes: (re.hi, im.hi) then
// (re.lo, im.lo), so the hi and lo parts are each a float2.
struct DF {};
struct __align__(16) dfc {
  float2 h, l;
};

template <typename R> struct Cplx;
template <> struct Cplx<float> { typedef float2 T; };
template <> struct Cplx<double> { typedef double2 T; };
template <> struct Cplx<DF> { typedef dfc T; };

// Accumulation type of sums over tensor entries (environment, trace).
template <typename R> struct Acc { typedef R T; };
template <> struct Acc<DF> { typedef double T; };

__device__ __forceinline__ float2 cmake(double2 v, float) {
  return make_float2((float)v.x, (float)v.y);
}
__device__ __forceinline__ double2 cmake(double2 v, double) { return v; }
__device__ __forceinline__ dfc cmake(double2 v, DF) {
  dfc r;
  r.h = make_float2((float)v.x, (float)v.y);
  r.l = make_float2((float)(v.x - (double)r.h.x), (float)(v.y - (double)r.h.y));
  return r;
}

__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(dfc v) {
  return make_double2((double)v.h.x + (double)v.l.x, (double)v.h.y + (double)v.l.y);
}
// an entry in its accumulation type
__device__ __forceinline__ float2 to_acc(float2 v) { return v; }
__device__ __forceinline__ double2 to_acc(double2 v) { return v; }
__device__ __forceinline__ double2 to_acc(dfc v) { return to_d2(v); }
__device__ __forceinline__ float2 to_f2(double2 v) { return make_float2((float)v.x, (float)v.y); }

// c + a*b
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y);
  c.y = fmaf(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}
// c + conj(a)*b
__device__ __forceinline__ float2 cfma_cj(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y);
  c.y = fmaf(-a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double2 cfma_cj(double2 a, double2 b, double2 c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(-a.y, b.x, c.y);
  return c;
}
template <typename C2> __device__ __forceinline__ C2 czero();
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ dfc czero<dfc>() {
  dfc r;
  r.h = make_float2(0.f, 0.f);
  r.l = make_float2(0.f, 0.f);
  return r;
}

// df64: s + err = a + b exactly (TwoSum, 6 operations, any magnitudes)
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}
// c + x1*y1 + x2*y2 for df64 reals: the hi*hi products exactly (TwoProd),
// their sum with TwoSum; the rounding errors, the hi*lo cross terms and c's
// lo part gather in lo (lo*lo terms, about 2^-48 relative, are dropped).
// The result is not renormalised (cfinish does that once per sum).
__device__ __forceinline__ void df_dot2_acc(float& ch, float& cl, float x1h, float x1l, float y1h,
                                            float y1l, float x2h, float x2l, float y2h, float y2l) {
  const float p1 = __fmul_rn(x1h, y1h);
  const float e1 = __fmaf_rn(x1h, y1h, -p1);
  const float p2 = __fmul_rn(x2h, y2h);
  const float e2 = __fmaf_rn(x2h, y2h, -p2);
  float t1, t2;
  float s = two_sum(ch, p1, t1);
  s = two_sum(s, p2, t2);
  float lo = __fadd_rn(cl, __fadd_rn(__fadd_rn(t1, t2), __fadd_rn(e1, e2)));
  lo = __fmaf_rn(x1h, y1l, lo);
  lo = __fmaf_rn(x1l, y1h, lo);
  lo = __fmaf_rn(x2h, y2l, lo);
  lo = __fmaf_rn(x2l, y2h, lo);
  ch = s;
  cl = lo;
}
// c + a*b, complex df64
__device__ __forceinline__ dfc cfma(dfc a, dfc b, dfc c) {
  df_dot2_acc(c.h.x, c.l.x, a.h.x, a.l.x, b.h.x, b.l.x, -a.h.y, -a.l.y, b.h.y, b.l.y);
  df_dot2_acc(c.h.y, c.l.y, a.h.x, a.l.x, b.h.y, b.l.y, a.h.y, a.l.y, b.h.x, b.l.x);
  return c;
}
// Renormalise a sum built by cfma (identity for float2 / double2).
__device__ __forceinline__ float2 cfinish(float2 v) { return v; }
__device__ __forceinline__ double2 cfinish(double2 v) { return v; }
__device__ __forceinline__ dfc cfinish(dfc v) {
  const float hx = __fadd_rn(v.h.x, v.l.x), hy = __fadd_rn(v.h.y, v.l.y);
  v.l = make_float2(__fsub_rn(v.l.x, __fsub_rn(hx, v.h.x)), __fsub_rn(v.l.y, __fsub_rn(hy, v.h.y)));
  v.h = make_float2(hx, hy);
  return v;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

__device__ __forceinline__ float2 shfl(float2 v, int src) {
  return make_float2(__shfl_sync(kFull, v.x, src), __shfl_sync(kFull, v.y, src));
}
__device__ __forceinline__ double2 shfl(double2 v, int src) {
  return make_double2(__shfl_sync(kFull, v.x, src), __shfl_sync(kFull, v.y, src));
}
__device__ __forceinline__ dfc shfl(dfc v, int src) {
  dfc r;
  r.h = shfl(v.h, src);
  r.l = shfl(v.l, src);
  return r;
}

// Insert a zero bit at position p into x.
__device__ __forceinline__ unsigned dep1(unsigned x, int p) {
  return ((x >> p) << (p + 1)) | (x & ((1u << p) - 1u));
}
// Insert zero bits at positions lo < hi into x.
__device__ __forceinline__ unsigned dep2(unsigned x, int lo, int hi) {
  return dep1(dep1(x, lo), hi);
}

// ---------------------------------------------------------------------------
// Lane-cooperative 4x4 complex products.  A warp holds a 4x4 matrix one
// element per lane: lane l owns element (i, j) = ((l >> 2) & 3, l & 3);
// lanes 16..31 hold a duplicate of lanes 0..15, so every lane can take part
// in shuffles without masks.

struct Lane {
  int l, i, j, base;
  __device__ __forceinline__ Lane() {
    l = threadIdx.x & 31;
    i = (l >> 2) & 3;
    j = l & 3;
    base = l & 16;
  }
  __device__ __forceinline__ int at(int r, int c) const { return base | (r << 2) | c; }
};

// (A B)[i][j]
template <typename C2>
__device__ __forceinline__ C2 wmm(const Lane& L, C2 a, C2 b) {
  C2 acc = czero<C2>();
#pragma unroll
  for (int k = 0; k < 4; ++k) acc = cfma(shfl(a, L.at(L.i, k)), shfl(b, L.at(k, L.j)), acc);
  return acc;
}
// (A^dagger B)[i][j] = sum_k conj(A[k][i]) B[k][j]
template <typename C2>
__device__ __forceinline__ C2 wmm_dn(const Lane& L, C2 a, C2 b) {
  C2 acc = czero<C2>();
#pragma unroll
  for (int k = 0; k < 4; ++k) acc = cfma_cj(shfl(a, L.at(k, L.i)), shfl(b, L.at(k, L.j)), acc);
  return acc;
}
// (A B^dagger)[i][j] = sum_k A[i][k] conj(B[j][k])
template <typename C2>
__device__ __forceinline__ C2 wmm_nd(const Lane& L, C2 a, C2 b) {
  C2 acc = czero<C2>();
#pragma unroll
  for (int k = 0; k < 4; ++k) acc = cfma_cj(shfl(b, L.at(L.j, k)), shfl(a, L.at(L.i, k)), acc);
  return acc;
}
// FP64 versions: GB300 issues an FP64 warp instruction only about every
// 33 ns per SM sub-partition, however many lanes are active, so the k sum
// is split between the half-warps (k = 0, 1 on lanes 0-15, k = 2, 3 on lanes
// 16-31) and the halves are added with one shuffle: 10 FP64 instructions
// and two dependent multiply-adds per product instead of 16 and four.  Both
// halves end with the same value (the two partial sums added in either
// order), so lanes 16-31 still mirror lanes 0-15.
__device__ __forceinline__ double2 half_sum(double2 acc) {
  acc.x += __shfl_xor_sync(kFull, acc.x, 16);
  acc.y += __shfl_xor_sync(kFull, acc.y, 16);
  return acc;
}
template <>
__device__ __forceinline__ double2 wmm<double2>(const Lane& L, double2 a, double2 b) {
  const int k0 = (L.l >> 3) & 2;
  double2 acc = cfma(shfl(a, L.at(L.i, k0)), shfl(b, L.at(k0, L.j)), czero<double2>());
  acc = cfma(shfl(a, L.at(L.i, k0 + 1)), shfl(b, L.at(k0 + 1, L.j)), acc);
  return half_sum(acc);
}
template <>
__device__ __forceinline__ double2 wmm_dn<double2>(const Lane& L, double2 a, double2 b) {
  const int k0 = (L.l >> 3) & 2;
  double2 acc = cfma_cj(shfl(a, L.at(k0, L.i)), shfl(b, L.at(k0, L.j)), czero<double2>());
  acc = cfma_cj(shfl(a, L.at(k0 + 1, L.i)), shfl(b, L.at(k0 + 1, L.j)), acc);
  return half_sum(acc);
}
template <>
__device__ __forceinline__ double2 wmm_nd<double2>(const Lane& L, double2 a, double2 b) {
  const int k0 = (L.l >> 3) & 2;
  double2 acc = cfma_cj(shfl(b, L.at(L.j, k0)), shfl(a, L.at(L.i, k0)), czero<double2>());
  acc = cfma_cj(shfl(b, L.at(L.j, k0 + 1)), shfl(a, L.at(L.i, k0 + 1)), acc);
  return half_sum(acc);
}

// A^dagger[i][j] = conj(A[j][i])
template <typename C2>
__device__ __forceinline__ C2 wdag(const Lane& L, C2 a) {
  return cconj(shfl(a, L.at(L.j, L.i)));
}

// 1/sqrt(q) for a positive normal double q by Newton's iteration
// r <- r (3 - q r^2) / 2 from an FP32 seed.  q = m 4^k with m in [1, 4), so
// the seed rsqrtf(m) 2^-k neither under- nor overflows in FP32; its relative
// error (~1e-7) squares with each step, so two steps reach FP64 rounding.
// No FP64 division or square root (long instruction sequences on the FP64
// pipe).
__device__ __forceinline__ double rsqrt_d(double q) {
  const int k = (((__double2hiint(q) >> 20) & 0x7ff) - 1023) >> 1;  // floor(log2(q) / 2)
  const double m = q * __hiloint2double((1023 - 2 * k) << 20, 0);
  double r = (double)rsqrtf((float)m) * __hiloint2double((1023 - k) << 20, 0);
  r = r * (1.5 - 0.5 * q * r * r);
  r = r * (1.5 - 0.5 * q * r * r);
  return r;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, h));
  return v;
}

}  // namespace dev
}  // namespace qf
