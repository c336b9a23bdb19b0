// Device helpers shared by the QFactor kernels: complex arithmetic on
// float2 / double2, index deposits, and lane-cooperative 4x4 products.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace qf {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

template <typename R> struct Cplx;
template <> struct Cplx<float> { typedef float2 T; };
template <> struct Cplx<double> { typedef double2 T; };

__device__ __forceinline__ float2 cmake(double2 v, float) {
  return make_float2((float)v.x, (float)v.y);
}
__device__ __forceinline__ double2 cmake(double2 v, double) { return v; }

__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
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
// A^dagger[i][j] = conj(A[j][i])
template <typename C2>
__device__ __forceinline__ C2 wdag(const Lane& L, C2 a) {
  return cconj(shfl(a, L.at(L.j, L.i)));
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, h));
  return v;
}

}  // namespace dev
}  // namespace qf
