// Warp-level 8x8 complex math of the three-qubit update (OptimizeGate,
// Sec. III-A1, Eq. opt_u, for a 2^3 x 2^3 environment): the lane layout,
// warp products, one-sided Jacobi (FP32, then FP64 polishing) and the warp
// polar factor.  Shared by the sweep's environment kernel and the batched
// kernel.
#pragma once

#include "qf_device.cuh"

namespace qf {
namespace {  // internal linkage in every translation unit that includes this
namespace w8 {

using namespace dev;

// ------------------------------------------------------------ warp 8x8 math
//
// A warp holds an 8x8 complex matrix with lane l = 8*g + j owning the
// elements (g, j) and (g + 4, j), g = 0..3, j = 0..7.

struct L8 {
  int l, g, j;
  __device__ __forceinline__ L8() {
    l = threadIdx.x & 31;
    g = l >> 3;
    j = l & 7;
  }
};

__device__ __forceinline__ int src8(int row, int col) { return ((row & 3) << 3) | col; }

// element (row, col) of the matrix (v0, v1) for every lane; `row` may differ
// between lanes.  C2 is float2 or double2 here and in the products below.
template <typename C2>
__device__ __forceinline__ C2 get8(C2 v0, C2 v1, int row, int col) {
  const C2 a = shfl(v0, src8(row, col));
  const C2 b = shfl(v1, src8(row, col));
  return row < 4 ? a : b;
}

__device__ __forceinline__ double2 cmuld(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <typename C2>
__device__ __forceinline__ C2 conj8(C2 v) {
  v.y = -v.y;
  return v;
}

// C = A B
template <typename C2>
__device__ __forceinline__ void mm8(const L8& L, C2 a0, C2 a1, C2 b0, C2 b1, C2& c0, C2& c1) {
  C2 s0 = czero<C2>(), s1 = s0;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const C2 x0 = shfl(a0, src8(L.g, m)), x1 = shfl(a1, src8(L.g, m));  // A[g][m], A[g+4][m]
    const C2 bm = m < 4 ? shfl(b0, src8(m, L.j)) : shfl(b1, src8(m, L.j));  // B[m][j]
    s0 = cfma(x0, bm, s0);
    s1 = cfma(x1, bm, s1);
  }
  c0 = s0;
  c1 = s1;
}

// C = A B^dagger
template <typename C2>
__device__ __forceinline__ void mm8_nd(const L8& L, C2 a0, C2 a1, C2 b0, C2 b1, C2& c0, C2& c1) {
  C2 s0 = czero<C2>(), s1 = s0;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const C2 x0 = shfl(a0, src8(L.g, m)), x1 = shfl(a1, src8(L.g, m));
    const C2 cb = conj8(get8(b0, b1, L.j, m));  // conj(B[j][m])
    s0 = cfma(x0, cb, s0);
    s1 = cfma(x1, cb, s1);
  }
  c0 = s0;
  c1 = s1;
}

// C = A^dagger B
template <typename C2>
__device__ __forceinline__ void mm8_dn(const L8& L, C2 a0, C2 a1, C2 b0, C2 b1, C2& c0, C2& c1) {
  C2 s0 = czero<C2>(), s1 = s0;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    // A^dagger[i][m] = conj(A[m][i]) for i = g and g + 4
    const C2 ami0 = m < 4 ? shfl(a0, src8(m, L.g)) : shfl(a1, src8(m, L.g));
    const C2 ami1 = m < 4 ? shfl(a0, src8(m, L.g + 4)) : shfl(a1, src8(m, L.g + 4));
    const C2 bm = m < 4 ? shfl(b0, src8(m, L.j)) : shfl(b1, src8(m, L.j));
    s0 = cfma(conj8(ami0), bm, s0);
    s1 = cfma(conj8(ami1), bm, s1);
  }
  c0 = s0;
  c1 = s1;
}

// (v0, v1) <- its conjugate transpose
template <typename C2>
__device__ __forceinline__ void dag8(const L8& L, C2& v0, C2& v1) {
  const C2 t0 = get8(v0, v1, L.j, L.g), t1 = get8(v0, v1, L.j, L.g + 4);
  v0 = conj8(t0);
  v1 = conj8(t1);
}

__device__ __forceinline__ double wmaxd(double v) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, h));
  return v;
}
template <typename T>
__device__ __forceinline__ T colsum(T v) {  // over the 4 row groups
  v += __shfl_xor_sync(kFull, v, 8);
  v += __shfl_xor_sync(kFull, v, 16);
  return v;
}

// Rare path: some singular value is below 1e-3 of the largest, so X is built
// by modified Gram-Schmidt in FP64 (lane 0) over the columns of W in order
// of decreasing singular value (columns below 1e-13 of the largest are
// numerically zero), falling back to standard basis vectors for an
// orthonormal completion.  sm: 128 double2 of shared scratch for this warp.
__device__ __noinline__ void complete8(const L8& L, double2 w0, double2 w1, const double* sig,
                                              double smax, double2* sm, double2& x0, double2& x1) {
  sm[L.g * 8 + L.j] = w0;
  sm[(L.g + 4) * 8 + L.j] = w1;
  __syncwarp();
  if (L.l == 0) {
    int ord[8];
    for (int a = 0; a < 8; ++a) ord[a] = a;
    for (int a = 0; a < 8; ++a)
      for (int b = 0; b < 7 - a; ++b)
        if (sig[ord[b]] < sig[ord[b + 1]]) {
          const int t = ord[b];
          ord[b] = ord[b + 1];
          ord[b + 1] = t;
        }
    double2* X = sm + 64;
    bool done[8];
    for (int a = 0; a < 8; ++a) done[a] = false;
    for (int e = 0; e < 64; ++e) X[e] = make_double2(0.0, 0.0);
    for (int oi = 0; oi < 8; ++oi) {
      const int k = ord[oi];
      for (int att = 0; att < 9; ++att) {
        double2 v[8];
        if (att == 0) {
          if (!(sig[k] > 1e-13 * smax)) continue;  // numerically zero: complete instead
          for (int i = 0; i < 8; ++i) v[i] = make_double2(sm[i * 8 + k].x / sig[k], sm[i * 8 + k].y / sig[k]);
        } else {
          for (int i = 0; i < 8; ++i) v[i] = make_double2(i == att - 1 ? 1.0 : 0.0, 0.0);
        }
        for (int pass = 0; pass < 2; ++pass)  // twice is enough (Kahan)
          for (int jj = 0; jj < 8; ++jj) {
            if (!done[jj]) continue;
            double2 d = make_double2(0.0, 0.0);
            for (int i = 0; i < 8; ++i) d = cfma_cj(X[i * 8 + jj], v[i], d);
            for (int i = 0; i < 8; ++i) {
              const double2 pr = cmuld(d, X[i * 8 + jj]);
              v[i].x -= pr.x;
              v[i].y -= pr.y;
            }
          }
        double nv = 0.0;
        for (int i = 0; i < 8; ++i) nv += v[i].x * v[i].x + v[i].y * v[i].y;
        nv = sqrt(nv);
        if (nv > 0.3) {  // among e_0..e_7 one keeps a residual of at least 1/sqrt(8)
          for (int i = 0; i < 8; ++i) X[i * 8 + k] = make_double2(v[i].x / nv, v[i].y / nv);
          done[k] = true;
          break;
        }
      }
    }
  }
  __syncwarp();
  x0 = sm[64 + L.g * 8 + L.j];
  x1 = sm[64 + (L.g + 4) * 8 + L.j];
  __syncwarp();
}

// One-sided Jacobi sweeps on the lane-distributed 8x8 pair (W, Y): each
// sweep pairs column j with j ^ r for r = 1..7 (four disjoint pairs per
// round) and rotates W[:,p], W[:,q] (and Y's) so that they become
// orthogonal.  Stops when the largest |g_pq| / (|W_p| |W_q|) is below tol
// or after max_sweeps.  R is float or double.
template <typename R, typename C2>
__device__ __forceinline__ void jacobi8(const L8& L, C2& w0, C2& w1, C2& y0, C2& y1, R tol,
                                        int max_sweeps) {
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    R off = R(0);
#pragma unroll 1
    for (int r = 1; r <= 7; ++r) {
      const int q = L.j ^ r;
      const bool isP = L.j < q;
      const int src = L.l ^ r;
      const C2 wq0 = shfl(w0, src), wq1 = shfl(w1, src);
      const C2 yq0 = shfl(y0, src), yq1 = shfl(y1, src);
      R n2 = w0.x * w0.x + w0.y * w0.y + w1.x * w1.x + w1.y * w1.y;
      n2 += __shfl_xor_sync(kFull, n2, 8);
      n2 += __shfl_xor_sync(kFull, n2, 16);
      const R n2q = __shfl_sync(kFull, n2, src);
      const C2 cp0 = isP ? w0 : wq0, cq0 = isP ? wq0 : w0;
      const C2 cp1 = isP ? w1 : wq1, cq1 = isP ? wq1 : w1;
      // g = conj(W[:,p]) . W[:,q]
      R gx = cp0.x * cq0.x + cp0.y * cq0.y + cp1.x * cq1.x + cp1.y * cq1.y;
      R gy = cp0.x * cq0.y - cp0.y * cq0.x + cp1.x * cq1.y - cp1.y * cq1.x;
      gx += __shfl_xor_sync(kFull, gx, 8);
      gx += __shfl_xor_sync(kFull, gx, 16);
      gy += __shfl_xor_sync(kFull, gy, 8);
      gy += __shfl_xor_sync(kFull, gy, 16);
      const R al = isP ? n2 : n2q, be = isP ? n2q : n2;
      // |g| with a scaled hypot: g can lie far below sqrt of the smallest normal
      const R gm0 = fmax(fabs(gx), fabs(gy));
      const R nrm = sqrt(al) * sqrt(be);
      const R tiny = sizeof(R) == 4 ? R(1e-12) : R(1e-200);
      if (gm0 > tol * R(0.01) * nrm && fmax(al, be) > tiny && gm0 > R(0)) {
        const float gxs = __fdividef(gx, gm0), gys = __fdividef(gy, gm0);
        const float rr = rsqrtf(gxs * gxs + gys * gys);
        const float gm = gm0 * (gxs * gxs + gys * gys) * rr;
        off = fmaxf(off, __fdividef(gm, nrm));
        const float zeta = 0.5f * __fdividef(be - al, gm), az = fabsf(zeta);
        const float t = az > 1e18f ? __fdividef(0.5f, zeta) : copysignf(__fdividef(1.f, az + sqrtf(1.f + az * az)), zeta);
        const float c = rsqrtf(1.f + t * t), sn = c * t;
        C2 e;  // conj(g) / |g|
        e.x = gxs * rr;
        e.y = -gys * rr;
        if (isP) {  // W[:,p] <- c W[:,p] - s e W[:,q]
          const C2 e0 = cmul(e, wq0), e1 = cmul(e, wq1), f0 = cmul(e, yq0), f1 = cmul(e, yq1);
          w0.x = c * w0.x - sn * e0.x; w0.y = c * w0.y - sn * e0.y;
          w1.x = c * w1.x - sn * e1.x; w1.y = c * w1.y - sn * e1.y;
          y0.x = c * y0.x - sn * f0.x; y0.y = c * y0.y - sn * f0.y;
          y1.x = c * y1.x - sn * f1.x; y1.y = c * y1.y - sn * f1.y;
        } else {  // W[:,q] <- s W[:,p] + c e W[:,q]
          const C2 e0 = cmul(e, w0), e1 = cmul(e, w1), f0 = cmul(e, y0), f1 = cmul(e, y1);
          w0.x = sn * wq0.x + c * e0.x; w0.y = sn * wq0.y + c * e0.y;
          w1.x = sn * wq1.x + c * e1.x; w1.y = sn * wq1.y + c * e1.y;
          y0.x = sn * yq0.x + c * f0.x; y0.y = sn * yq0.y + c * f0.y;
          y1.x = sn * yq1.x + c * f1.x; y1.y = sn * yq1.y + c * f1.y;
        }
      }
    }
    R m = off;
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, h));
    if (m < tol) break;
  }
}

// FP64 polishing sweeps after the FP32 stage, in which every column pair is
// already orthogonal to ~1e-6.  The inner products g = W_p^dagger W_q,
// |W_p|^2 and |W_q|^2 are FP64 sums; the rotation angle t = tan(theta) is
// taken in FP32 from zeta = (|W_q|^2 - |W_p|^2) / (2|g|) (an angle accurate
// to FP32 still shrinks g by ~1e-7 per sweep); the rotation applied is
// unitary to FP64 rounding: c = 1/sqrt(1 + t^2) and e = conj(g)/|g| by
// rsqrt_d, s = c t.  No FP64 division or square root (long instruction
// sequences on the FP64 pipe).  Stops once every pair has
// |g| <= tol |W_p| |W_q| (tested as g^2 <= tol^2 |W_p|^2 |W_q|^2).
__device__ __forceinline__ void polish8(const L8& L, double2& w0, double2& w1, double2& y0, double2& y1,
                                        double tol, int max_sweeps) {
  const double tol2 = tol * tol;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    bool open = false;
#pragma unroll 1
    for (int r = 1; r <= 7; ++r) {
      const int q = L.j ^ r;
      const bool isP = L.j < q;
      const int src = L.l ^ r;
      const double2 wq0 = shfl(w0, src), wq1 = shfl(w1, src);
      const double2 yq0 = shfl(y0, src), yq1 = shfl(y1, src);
      const double n2 = colsum(w0.x * w0.x + w0.y * w0.y + w1.x * w1.x + w1.y * w1.y);
      const double n2q = __shfl_sync(kFull, n2, src);
      const double2 cp0 = isP ? w0 : wq0, cq0 = isP ? wq0 : w0;
      const double2 cp1 = isP ? w1 : wq1, cq1 = isP ? wq1 : w1;
      const double gx = colsum(cp0.x * cq0.x + cp0.y * cq0.y + cp1.x * cq1.x + cp1.y * cq1.y);
      const double gy = colsum(cp0.x * cq0.y - cp0.y * cq0.x + cp1.x * cq1.y - cp1.y * cq1.x);
      const double al = isP ? n2 : n2q, be = isP ? n2q : n2;
      const double g2 = gx * gx + gy * gy, ab = al * be;
      open |= g2 > tol2 * ab;
      // rotate where |g| is above FP64 rounding of |W_p| |W_q| (and normal)
      if (g2 > 1e-4 * tol2 * ab && g2 > 1e-300) {
        const double rg = rsqrt_d(g2);
        const float z = (float)(0.5 * (be - al) * rg), az = fabsf(z);
        const float tf = copysignf(az > 1e18f ? 0.5f / az : 1.f / (az + sqrtf(1.f + az * az)), z);
        const double t = (double)tf;
        const double c = rsqrt_d(1.0 + t * t), sn = c * t;
        const double2 e = make_double2(gx * rg, -gy * rg);  // conj(g) / |g|
        if (isP) {  // W[:,p] <- c W[:,p] - s e W[:,q]
          const double2 e0 = cmuld(e, wq0), e1 = cmuld(e, wq1), f0 = cmuld(e, yq0), f1 = cmuld(e, yq1);
          w0 = make_double2(c * w0.x - sn * e0.x, c * w0.y - sn * e0.y);
          w1 = make_double2(c * w1.x - sn * e1.x, c * w1.y - sn * e1.y);
          y0 = make_double2(c * y0.x - sn * f0.x, c * y0.y - sn * f0.y);
          y1 = make_double2(c * y1.x - sn * f1.x, c * y1.y - sn * f1.y);
        } else {  // W[:,q] <- s W[:,p] + c e W[:,q]
          const double2 e0 = cmuld(e, w0), e1 = cmuld(e, w1), f0 = cmuld(e, y0), f1 = cmuld(e, y1);
          w0 = make_double2(sn * wq0.x + c * e0.x, sn * wq0.y + c * e0.y);
          w1 = make_double2(sn * wq1.x + c * e1.x, sn * wq1.y + c * e1.y);
          y0 = make_double2(sn * yq0.x + c * f0.x, sn * yq0.y + c * f0.y);
          y1 = make_double2(sn * yq1.x + c * f1.x, sn * yq1.y + c * f1.y);
        }
      }
    }
    if (!__any_sync(kFull, open)) break;
  }
}

// Rare path of the 8x8 update (some FP32 singular value is below 1e-3 of
// the largest): from the FP32 rotation (fy0, fy1), Y made unitary in FP64
// (two Newton-Schulz steps), W = A Y, FP64 polishing sweeps to 1e-15, X =
// W's normalised columns (or, with a singular value still below 1e-3 of the
// largest, complete8), u = Y X^dagger.  The polar factor of a nearly
// singular A is ill-conditioned (a perturbation dA moves it by up to about
// 2 ||dA|| / s_min, R.-C. Li's bound), so this path keeps the FP64 rounding
// of A as the only source of error.  Returns the sum of the singular values
// of the scaled A; y_io (if not null) receives the final rotation.
__device__ __noinline__ double polar8_rare(double2 as0, double2 as1, float2 fy0, float2 fy1, double2* sm,
                                           double2* u0, double2* u1, float2* y_io) {
  const L8 L;
  double2 y0 = to_d2(fy0), y1 = to_d2(fy1);
  for (int step = 0; step < 2; ++step) {
    double2 P0, P1;
    mm8_dn(L, y0, y1, y0, y1, P0, P1);
    const double2 Q0 = make_double2((L.g == L.j ? 1.5 : 0.0) - 0.5 * P0.x, -0.5 * P0.y);
    const double2 Q1 = make_double2((L.g + 4 == L.j ? 1.5 : 0.0) - 0.5 * P1.x, -0.5 * P1.y);
    mm8(L, y0, y1, Q0, Q1, y0, y1);
  }
  double2 w0, w1;
  mm8(L, as0, as1, y0, y1, w0, w1);
  polish8(L, w0, w1, y0, y1, 1e-15, 8);
  const double sj = sqrt(colsum(w0.x * w0.x + w0.y * w0.y + w1.x * w1.x + w1.y * w1.y));
  double s8[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) s8[k] = __shfl_sync(kFull, sj, k);
  double smax = 0.0, smin = s8[0], ssum = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    smax = fmax(smax, s8[k]);
    smin = fmin(smin, s8[k]);
    ssum += s8[k];
  }
  double2 x0, x1;
  if (smin > 1e-3 * smax) {
    x0 = make_double2(w0.x / sj, w0.y / sj);
    x1 = make_double2(w1.x / sj, w1.y / sj);
  } else {
    // a column of small norm s has its direction only to ~eps s_max / s, so
    // X is re-orthonormalised (Gram-Schmidt, in order of decreasing s)
    // rather than normalised, keeping u unitary to FP64 rounding
    complete8(L, w0, w1, s8, smax, sm, x0, x1);
  }
  mm8_nd(L, y0, y1, x0, x1, *u0, *u1);  // Y X^dagger
  if (y_io) {
    y_io[L.g * 8 + L.j] = to_f2(y0);
    y_io[L.g * 8 + L.j + 32] = to_f2(y1);
  }
  return ssum;
}

// Warp 8x8 polar update (OptimizeGate, Sec. III-A1, Eq. opt_u): with
// A = X D Y^dagger, u = Y X^dagger maximises Re Tr(A u); *sig = sum(D).
// The stages follow the 4x4 update, because GB300's FP64 rate is 1/64 of
// its FP32 rate and the warps of an SM share one FP64 pipe:
//   0. A is scaled by a power of two (exact) to a largest entry in [1, 2);
//   1. one-sided Jacobi in FP32 to an off-diagonal measure of 1e-6
//      (no FP64 work), from A, or from A Y0 with Y0 the rotation of the
//      previous update of the same gate (y_io, a warm start);
//   2. with every FP32 singular value above 1e-3 of the largest (the
//      common case), FP64 refinement rounds: Newton-Schulz
//      re-unitarisation of u (the small correction product in FP32),
//      M = A u (Hermitian positive definite at the optimum), and
//      u <- u (I - W + W^2 / 2) with W the solution of H W + W H = M - M^dagger
//      in X's eigenbasis (W'_ij = K'_ij / (d_i + d_j), FP32): each round
//      squares the error, two FP64 8x8 products a round; *sig = Re Tr(A u)
//      of the final u;
//   3. otherwise polar8_rare.
// y_io: nullptr, or the 64-entry row-major FP32 rotation of the previous
// update (read, then rewritten with this update's; lane (g, j) touches
// entries (g, j) and (g + 4, j) only).  Returns false for a non-finite A.
__device__ __noinline__ bool warp_polar8(double2 a0, double2 a1, double2* sm, double2* u0, double2* u1,
                                         double* sig, float2* y_io = nullptr) {
  const L8 L;
  const bool fin = __all_sync(kFull, isfinite(a0.x) && isfinite(a0.y) && isfinite(a1.x) && isfinite(a1.y));
  if (!fin) return false;
  const double amax = wmaxd(fmax(fmax(fabs(a0.x), fabs(a0.y)), fmax(fabs(a1.x), fabs(a1.y))));
  if (amax == 0.0) {  // A = 0: every unitary is optimal
    *u0 = make_double2(L.g == L.j ? 1.0 : 0.0, 0.0);
    *u1 = make_double2(L.g + 4 == L.j ? 1.0 : 0.0, 0.0);
    *sig = 0.0;
    return true;
  }
  int ex;
  frexp(amax, &ex);  // amax = m 2^ex, m in [0.5, 1)
  const double sc = ldexp(1.0, 1 - ex), unscale = ldexp(1.0, ex - 1);
  const double2 as0 = make_double2(a0.x * sc, a0.y * sc), as1 = make_double2(a1.x * sc, a1.y * sc);
  const float2 fa0 = to_f2(as0), fa1 = to_f2(as1);

  // ---- stage 1: FP32 Jacobi
  const int e0 = L.g * 8 + L.j, e1 = e0 + 32;
  float2 fw0, fw1, fy0, fy1;
  if (y_io) {
    fy0 = y_io[e0];
    fy1 = y_io[e1];
    mm8(L, fa0, fa1, fy0, fy1, fw0, fw1);  // W = A Y0
  } else {
    fw0 = fa0;
    fw1 = fa1;
    fy0 = make_float2(L.g == L.j ? 1.f : 0.f, 0.f);
    fy1 = make_float2(L.g + 4 == L.j ? 1.f : 0.f, 0.f);
  }
  jacobi8<float>(L, fw0, fw1, fy0, fy1, 1e-6f, 15);
  const float sj = sqrtf(colsum(fw0.x * fw0.x + fw0.y * fw0.y + fw1.x * fw1.x + fw1.y * fw1.y));
  float smax = 0.f, smin = 3.4e38f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float sk = __shfl_sync(kFull, sj, k);  // lane k holds column k
    smax = fmaxf(smax, sk);
    smin = fminf(smin, sk);
  }
  if (!(smin > 1e-3f * smax)) {  // ---- stage 3 (rare): A close to singular
    *sig = polar8_rare(as0, as1, fy0, fy1, sm, u0, u1, y_io) * unscale;
    return __all_sync(kFull, isfinite(u0->x) && isfinite(u0->y) && isfinite(u1->x) && isfinite(u1->y));
  }
  const float2 x0 = make_float2(fw0.x / sj, fw0.y / sj), x1 = make_float2(fw1.x / sj, fw1.y / sj);
  // d_i + d_j for rows g and g + 4 of this lane's column j (>= 2e-3 smax)
  const float den0 = __shfl_sync(kFull, sj, L.g) + sj, den1 = __shfl_sync(kFull, sj, L.g + 4) + sj;
  float2 v0, v1;
  mm8_nd(L, fy0, fy1, x0, x1, v0, v1);  // Y X^dagger
  double2 w0 = to_d2(v0), w1 = to_d2(v1);

  // ---- stage 2: FP64 refinement
  double2 M0 = make_double2(0.0, 0.0), M1 = M0;
  float2 D0 = make_float2(0.f, 0.f), D1 = D0;
  // the correction's first-order error is about 1e-7 smax / (d_i + d_j) of
  // its size: stop once that is below FP64 rounding of the result
  const float wtol = 3e-6f * fminf(1.f, 10.f * smin / smax);
  for (int round = 0; round < 5; ++round) {
    // Newton-Schulz: u <- u - u (u^dagger u - I) / 2
    double2 P0, P1;
    mm8_dn(L, w0, w1, w0, w1, P0, P1);
    const float2 Pm0 = make_float2((float)(P0.x - (L.g == L.j ? 1.0 : 0.0)), (float)P0.y);
    const float2 Pm1 = make_float2((float)(P1.x - (L.g + 4 == L.j ? 1.0 : 0.0)), (float)P1.y);
    float2 c0, c1;
    mm8(L, to_f2(w0), to_f2(w1), Pm0, Pm1, c0, c1);
    w0 = make_double2(w0.x - 0.5 * (double)c0.x, w0.y - 0.5 * (double)c0.y);
    w1 = make_double2(w1.x - 0.5 * (double)c1.x, w1.y - 0.5 * (double)c1.y);
    // M = A u, K = M - M^dagger
    mm8(L, as0, as1, w0, w1, M0, M1);
    double2 Md0 = M0, Md1 = M1;
    dag8(L, Md0, Md1);
    const float2 K0 = make_float2((float)(M0.x - Md0.x), (float)(M0.y - Md0.y));
    const float2 K1 = make_float2((float)(M1.x - Md1.x), (float)(M1.y - Md1.y));
    // H W + W H = K in the eigenbasis X of H: W = X (X^dagger K X ./ (d_i + d_j)) X^dagger
    float2 t0, t1, k0, k1;
    mm8(L, K0, K1, x0, x1, t0, t1);
    mm8_dn(L, x0, x1, t0, t1, k0, k1);
    k0 = make_float2(k0.x / den0, k0.y / den0);
    k1 = make_float2(k1.x / den1, k1.y / den1);
    mm8_nd(L, k0, k1, x0, x1, t0, t1);
    float2 W0, W1;
    mm8(L, x0, x1, t0, t1, W0, W1);
    float om = fmaxf(fmaxf(fabsf(W0.x), fabsf(W0.y)), fmaxf(fabsf(W1.x), fabsf(W1.y)));
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) om = fmaxf(om, __shfl_xor_sync(kFull, om, h));
    // u <- u (I - W + W^2 / 2)
    mm8(L, W0, W1, W0, W1, t0, t1);
    const float2 Z0 = make_float2(-W0.x + 0.5f * t0.x, -W0.y + 0.5f * t0.y);
    const float2 Z1 = make_float2(-W1.x + 0.5f * t1.x, -W1.y + 0.5f * t1.y);
    mm8(L, to_f2(w0), to_f2(w1), Z0, Z1, D0, D1);
    w0 = make_double2(w0.x + (double)D0.x, w0.y + (double)D0.y);
    w1 = make_double2(w1.x + (double)D1.x, w1.y + (double)D1.y);
    if (om < wtol) break;
  }
  {  // final Newton-Schulz step: unitary to FP64 rounding whatever the last D
    double2 P0, P1;
    mm8_dn(L, w0, w1, w0, w1, P0, P1);
    const float2 Pm0 = make_float2((float)(P0.x - (L.g == L.j ? 1.0 : 0.0)), (float)P0.y);
    const float2 Pm1 = make_float2((float)(P1.x - (L.g + 4 == L.j ? 1.0 : 0.0)), (float)P1.y);
    float2 c0, c1;
    mm8(L, to_f2(w0), to_f2(w1), Pm0, Pm1, c0, c1);
    w0 = make_double2(w0.x - 0.5 * (double)c0.x, w0.y - 0.5 * (double)c0.y);
    w1 = make_double2(w1.x - 0.5 * (double)c1.x, w1.y - 0.5 * (double)c1.y);
  }
  // sum of singular values = Re Tr(A u) of the final u, in FP64: the last
  // Newton-Schulz step moves Re Tr(A u) to first order in u's distance from
  // unitarity, which the FP32 correction leaves near FP64 rounding only
  {
    const double2 ut0 = get8(w0, w1, L.j, L.g), ut1 = get8(w0, w1, L.j, L.g + 4);  // u[j][g], u[j][g+4]
    double tr = as0.x * ut0.x - as0.y * ut0.y + as1.x * ut1.x - as1.y * ut1.y;
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) tr += __shfl_xor_sync(kFull, tr, h);
    *sig = tr * unscale;
  }
  *u0 = w0;
  *u1 = w1;
  if (y_io) {
    y_io[e0] = fy0;
    y_io[e1] = fy1;
  }
  return __all_sync(kFull, isfinite(w0.x) && isfinite(w0.y) && isfinite(w1.x) && isfinite(w1.y));
}

}  // namespace w8
}  // namespace
}  // namespace qf
