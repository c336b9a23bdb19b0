// Four-qubit gates (the paper's method with a 16 x 16 unitary as one
// variable, Sec. III and Sec. VI): the fused 16x16 pass, the band partial
// trace over the other qubits, and the 16x16 FP64 update (OptimizeGate,
// Eq. opt_u) on one CTA.
//
// A gate on qubits (q[0], q[1], q[2], q[3]) acts on the local index
// sum_i bit(q[i]) 2^(3-i) (q[0] is the most significant local bit).  Its
// operators are 16x16 row-major (256 FP64 complex values); a start's pass
// operators L, R sit at LR + s*512 (L first).
//
// The 16x16 update runs on a whole CTA of 256 threads (thread t holds
// element (t / 16, t % 16) of every shared matrix): one-sided Jacobi in FP32
// (eight disjoint column pairs per round, one warp per pair: lanes 0-15 hold
// the pair's rows of W, lanes 16-31 those of Y), then from W = A Y (Y made
// unitary in FP64) FP64 sweeps with angles from FP32 and exactly unitary
// FP64 rotations, X = W's normalised columns (re-orthonormalised by FP64
// Gram-Schmidt when a singular value is below 1e-3 of the largest, and
// completed below 1e-13), u = Y X^dagger.  The per-element FP64 work is
// spread over eight warps because GB300 issues FP64 at 1/64 of its FP32 rate.

#include <cuda_runtime.h>

#include <atomic>
#include <type_traits>

#include "qf_device.cuh"
#include "qf_internal.h"
#include "qf_tc.cuh"
#include "qfactor.h"

namespace qf {
namespace {

using namespace dev;

constexpr int kCta16 = 256;  // threads of every 16x16 kernel that runs the update

// Offset of local index v of a gate on bit positions p[0..3] (p[0]: the
// local index's most significant bit).
__device__ __forceinline__ unsigned off16(int v, const int* p) {
  return (((unsigned)v >> 3) & 1u) << p[0] | (((unsigned)v >> 2) & 1u) << p[1] |
         (((unsigned)v >> 1) & 1u) << p[2] | ((unsigned)v & 1u) << p[3];
}

// Insert zero bits at the four (ascending) positions qs[0..3].
__device__ __forceinline__ unsigned dep4(unsigned x, const int* qs) {
  return dep1(dep1(dep1(dep1(x, qs[0]), qs[1]), qs[2]), qs[3]);
}

__device__ __forceinline__ void sort4(const int* p, int* qs) {
  for (int i = 0; i < 4; ++i) qs[i] = p[i];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 3 - a; ++b)
      if (qs[b] > qs[b + 1]) {
        const int t = qs[b];
        qs[b] = qs[b + 1];
        qs[b + 1] = t;
      }
}

// ------------------------------------------------------ CTA 16x16 products
// C = op(A) op(B) on shared 16x16 matrices (FP64, or FP32 for the small
// corrections of the update), one element per thread (t = 16 i + j); C
// must not alias A or B.  Ends with a barrier.
enum MmOp { kMmNN = 0, kMmND = 1, kMmDN = 2 };  // A B, A B^dagger, A^dagger B

// Every shared 16x16 matrix of the update keeps entry (r, c) at
// 16 r + (c ^ r): a row and a column each hit 16 distinct positions mod 16,
// so the column accesses of the Jacobi rounds and of A B^dagger are free of
// bank conflicts.  swt(t) is the position of entry (t / 16, t % 16).
__device__ __forceinline__ int sw16(int r, int c) { return r * 16 + (c ^ r); }
__device__ __forceinline__ int swt(int t) { return t ^ (t >> 4); }

template <int OP, typename C2>
__device__ __forceinline__ void cta_mm(const C2* A, const C2* B, C2* C) {
  const int t = threadIdx.x, i = t >> 4, j = t & 15;
  C2 acc = czero<C2>();
#pragma unroll 4
  for (int k = 0; k < 16; ++k) {
    if (OP == kMmNN) {
      acc = cfma(A[sw16(i, k)], B[sw16(k, j)], acc);
    } else if (OP == kMmND) {  // A[i][k] conj(B[j][k])
      acc = cfma_cj(B[sw16(j, k)], A[sw16(i, k)], acc);
    } else {  // conj(A[k][i]) B[k][j]
      acc = cfma_cj(A[sw16(k, i)], B[sw16(k, j)], acc);
    }
  }
  C[swt(t)] = acc;
  __syncthreads();
}

// Two FP64 Newton-Schulz steps M <- M (3I - M^dagger M) / 2 on shared M
// (tmp, tmp2: shared scratch).
__device__ __forceinline__ void cta_newton_schulz(double2* M, double2* tmp, double2* tmp2, int steps) {
  const int t = threadIdx.x, i = t >> 4, j = t & 15;
  for (int s = 0; s < steps; ++s) {
    cta_mm<kMmDN>(M, M, tmp);
    tmp[swt(t)] = make_double2((i == j ? 1.5 : 0.0) - 0.5 * tmp[swt(t)].x, -0.5 * tmp[swt(t)].y);
    __syncthreads();
    cta_mm<kMmNN>(M, tmp, tmp2);
    M[swt(t)] = tmp2[swt(t)];
    __syncthreads();
  }
}

// The column pair of warp w in Jacobi round r = 1..15: (p, p ^ r), p < p ^ r;
// the eight pairs of a round are disjoint.
__device__ __forceinline__ int pair_col(int r, int w) {
  const int hb = 31 - __clz(r);
  return ((w >> hb) << (hb + 1)) | (w & ((1 << hb) - 1));
}

// ------------------------------------------------------ CTA 16x16 polar
// Shared workspace of the 16x16 update (29 KB).
struct Polar16Smem {
  double2 a[256];  // A, scaled in place by a power of two
  double2 w[256];  // W = A Y
  double2 y[256];  // Y
  double2 x[256];  // X, then the result u
  double2 t1[256], t2[256];
  float2 fw[256], fy[256];  // the FP32 stage's W and Y
  double s[16];             // column norms (singular values)
  unsigned emax;
  float off[2];
  double red[kCta16 / 32];  // per-warp partial sums
};

__device__ __forceinline__ unsigned expo_field(double v) {
  return (unsigned)(__double2hiint(v) >> 20) & 0x7ffu;
}

// Largest exponent field of the shared matrix a (every thread gets it).
__device__ __forceinline__ unsigned cta_max_exponent(Polar16Smem& S) {
  const int t = threadIdx.x;
  if (t == 0) S.emax = 0u;
  __syncthreads();
  const double2 v = S.a[swt(t)];
  const unsigned e = __reduce_max_sync(kFull, max(expo_field(v.x), expo_field(v.y)));
  if ((t & 31) == 0) atomicMax(&S.emax, e);
  __syncthreads();
  return S.emax;
}

// One-sided Jacobi round r on the lane-split pair (W, Y) in FP32: warp w
// rotates columns (p, p ^ r); lanes 0-15 hold rows of W, lanes 16-31 rows
// of Y.  Returns the pair's off-diagonal measure |g| / (|W_p| |W_q|).
__device__ __forceinline__ float jacobi16_round_f(Polar16Smem& S, int r) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int p = pair_col(r, w), q = p ^ r, row = lane & 15;
  const bool isW = lane < 16;
  float2* M = isW ? S.fw : S.fy;
  const float2 xp = M[sw16(row, p)], xq = M[sw16(row, q)];
  float al = isW ? xp.x * xp.x + xp.y * xp.y : 0.f;
  float be = isW ? xq.x * xq.x + xq.y * xq.y : 0.f;
  float gx = isW ? xp.x * xq.x + xp.y * xq.y : 0.f;  // conj(W[i][p]) W[i][q]
  float gy = isW ? xp.x * xq.y - xp.y * xq.x : 0.f;
#pragma unroll
  for (int h = 1; h < 16; h <<= 1) {
    al += __shfl_xor_sync(kFull, al, h);
    be += __shfl_xor_sync(kFull, be, h);
    gx += __shfl_xor_sync(kFull, gx, h);
    gy += __shfl_xor_sync(kFull, gy, h);
  }
  al = __shfl_sync(kFull, al, 0);
  be = __shfl_sync(kFull, be, 0);
  gx = __shfl_sync(kFull, gx, 0);
  gy = __shfl_sync(kFull, gy, 0);
  const float gm = fmaxf(fabsf(gx), fabsf(gy));
  const float nrm = sqrtf(al) * sqrtf(be);
  float off = 0.f;
  // columns below 1e-6 of A's largest entry are noise in FP32: the FP64
  // stage resolves them
  if (gm > 1e-7f * nrm && fmaxf(al, be) > 1e-12f && gm > 0.f) {
    const float gxs = __fdividef(gx, gm), gys = __fdividef(gy, gm);
    const float rr = rsqrtf(gxs * gxs + gys * gys);
    const float ag = gm * (gxs * gxs + gys * gys) * rr;
    off = __fdividef(ag, nrm);
    const float zeta = 0.5f * __fdividef(be - al, ag);
    const float az = fabsf(zeta);
    const float tt = az > 1e18f ? __fdividef(0.5f, zeta)
                                : copysignf(__fdividef(1.f, az + sqrtf(1.f + az * az)), zeta);
    const float c = rsqrtf(1.f + tt * tt), sn = c * tt;
    const float2 e = make_float2(gxs * rr, -gys * rr);  // conj(g) / |g|
    const float2 ex = cmul(e, xq);
    M[sw16(row, p)] = make_float2(c * xp.x - sn * ex.x, c * xp.y - sn * ex.y);
    M[sw16(row, q)] = make_float2(sn * xp.x + c * ex.x, sn * xp.y + c * ex.y);
  }
  return off;
}

// The same round in FP64 (after the FP32 stage), two column pairs per warp
// so that the FP64 pipe (1/64 of the FP32 rate) does no work for zeros:
// warp w < 4 takes pairs 2 w (lanes 0-15) and 2 w + 1 (lanes 16-31), lane
// l holding row l % 16 of W and of Y.  FP64 inner products over the
// half-warp, an FP32 rotation angle and a rotation unitary to FP64 rounding
// (rsqrt_d, no FP64 division or square root); pairs with
// |g| <= 1e-2 tol |W_p| |W_q| are left alone.
__device__ __forceinline__ void jacobi16_round_d(Polar16Smem& S, int r, double tol2) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w >= 4) return;
  const int p = pair_col(r, 2 * w + (lane >> 4)), q = p ^ r, row = lane & 15;
  const double2 xp = S.w[sw16(row, p)], xq = S.w[sw16(row, q)];
  double al = xp.x * xp.x + xp.y * xp.y;
  double be = xq.x * xq.x + xq.y * xq.y;
  double gx = xp.x * xq.x + xp.y * xq.y;  // conj(W[i][p]) W[i][q]
  double gy = xp.x * xq.y - xp.y * xq.x;
#pragma unroll
  for (int h = 1; h < 16; h <<= 1) {
    al += __shfl_xor_sync(kFull, al, h);
    be += __shfl_xor_sync(kFull, be, h);
    gx += __shfl_xor_sync(kFull, gx, h);
    gy += __shfl_xor_sync(kFull, gy, h);
  }
  const double g2 = gx * gx + gy * gy, ab = al * be;
  if (g2 > 1e-4 * tol2 * ab && g2 > 1e-300) {
    const double rg = rsqrt_d(g2);
    const float z = (float)(0.5 * (be - al) * rg), az = fabsf(z);
    const float tf = copysignf(az > 1e18f ? 0.5f / az : 1.f / (az + sqrtf(1.f + az * az)), z);
    const double tt = (double)tf;
    const double c = rsqrt_d(1.0 + tt * tt), sn = c * tt;
    const double2 e = make_double2(gx * rg, -gy * rg);  // conj(g) / |g|
    const double2 ex = cmul(e, xq);
    S.w[sw16(row, p)] = make_double2(c * xp.x - sn * ex.x, c * xp.y - sn * ex.y);
    S.w[sw16(row, q)] = make_double2(sn * xp.x + c * ex.x, sn * xp.y + c * ex.y);
    const double2 yp = S.y[sw16(row, p)], yq = S.y[sw16(row, q)];
    const double2 ey = cmul(e, yq);
    S.y[sw16(row, p)] = make_double2(c * yp.x - sn * ey.x, c * yp.y - sn * ey.y);
    S.y[sw16(row, q)] = make_double2(sn * yp.x + c * ey.x, sn * yp.y + c * ey.y);
  }
}

// Whether every column pair of W is orthogonal to |g| <= tol |W_p| |W_q|
// (the Gram matrix W^dagger W in FP64; t1 is scratch).
__device__ __forceinline__ bool cta_w_orthogonal(Polar16Smem& S, double tol2) {
  const int t = threadIdx.x, i = t >> 4, j = t & 15;
  cta_mm<kMmDN>(S.w, S.w, S.t1);
  const double2 g = S.t1[swt(t)];
  const double gii = S.t1[16 * i].x, gjj = S.t1[16 * j].x;
  const bool open = i != j && g.x * g.x + g.y * g.y > tol2 * gii * gjj;
  return !__syncthreads_or(open);
}

// X for a nearly singular A (warp 0; lane i < 16 holds row i): the columns
// of W in order of decreasing norm, normalised and orthogonalised (twice,
// Kahan) against those before; columns below 1e-13 of the largest norm are
// numerically zero and completed with standard basis vectors.
__device__ void gram_schmidt16(Polar16Smem& S, double smax) {
  const int lane = threadIdx.x & 31;
  int ord[16];
  for (int k = 0; k < 16; ++k) ord[k] = k;
  for (int a = 0; a < 16; ++a)
    for (int b = a + 1; b < 16; ++b)
      if (S.s[ord[b]] > S.s[ord[a]]) {
        const int tmp = ord[a];
        ord[a] = ord[b];
        ord[b] = tmp;
      }
  unsigned done = 0u;
  for (int oi = 0; oi < 16; ++oi) {
    const int k = ord[oi];
    for (int att = 0; att <= 16; ++att) {
      double2 v = make_double2(0.0, 0.0);
      if (att == 0) {
        if (!(S.s[k] > 1e-13 * smax)) continue;
        if (lane < 16) {
          const double inv = 1.0 / S.s[k];
          v = make_double2(S.w[sw16(lane, k)].x * inv, S.w[sw16(lane, k)].y * inv);
        }
      } else if (lane == att - 1) {
        v = make_double2(1.0, 0.0);
      }
      for (int pass = 0; pass < 2; ++pass)
        for (int jj = 0; jj < 16; ++jj) {
          if (!(done & (1u << jj))) continue;
          const double2 xj = lane < 16 ? S.x[sw16(lane, jj)] : make_double2(0.0, 0.0);
          double2 d = cfma_cj(xj, v, make_double2(0.0, 0.0));
#pragma unroll
          for (int h = 16; h >= 1; h >>= 1) {
            d.x += __shfl_xor_sync(kFull, d.x, h);
            d.y += __shfl_xor_sync(kFull, d.y, h);
          }
          const double2 pr = cmul(d, xj);
          v.x -= pr.x;
          v.y -= pr.y;
        }
      double nv = v.x * v.x + v.y * v.y;
#pragma unroll
      for (int h = 16; h >= 1; h >>= 1) nv += __shfl_xor_sync(kFull, nv, h);
      nv = sqrt(nv);
      // among e_0..e_15 one keeps a residual of at least 1/4
      if (nv > 0.24) {
        if (lane < 16) S.x[sw16(lane, k)] = make_double2(v.x / nv, v.y / nv);
        done |= 1u << k;
        break;
      }
    }
  }
  __syncwarp();
}

// Largest of a non-negative value over the CTA (every thread gets it).
__device__ __forceinline__ float cta_max_nonneg(Polar16Smem& S, float v) {
  __syncthreads();
  if (threadIdx.x == 0) S.emax = 0u;
  __syncthreads();
  const unsigned m = __reduce_max_sync(kFull, __float_as_uint(v));
  if ((threadIdx.x & 31) == 0) atomicMax(&S.emax, m);
  __syncthreads();
  return __uint_as_float(S.emax);
}

// Sum over the CTA in a fixed order (warps, then the warps' partials in
// order); every thread gets it.
__device__ __forceinline__ double cta_sum(Polar16Smem& S, double v) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) v += __shfl_xor_sync(kFull, v, h);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) S.red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
#pragma unroll
  for (int w = 0; w < kCta16 / 32; ++w) r += S.red[w];
  return r;
}

// One Newton-Schulz step on the FP64 u in S.x: u <- u - u (u^dagger u - I) / 2,
// u^dagger u in FP64 and the small correction product in FP32 (F0-F2: FP32
// scratch matrices).
__device__ __forceinline__ void cta_ns_step(Polar16Smem& S, float2* F0, float2* F1, float2* F2) {
  const int t = threadIdx.x, i = t >> 4, j = t & 15;
  cta_mm<kMmDN>(S.x, S.x, S.t1);
  const double2 pq = S.t1[swt(t)];
  F1[swt(t)] = make_float2((float)(pq.x - (i == j ? 1.0 : 0.0)), (float)pq.y);
  F0[swt(t)] = to_f2(S.x[swt(t)]);
  __syncthreads();
  cta_mm<kMmNN>(F0, F1, F2);
  const float2 c = F2[swt(t)];
  const double2 u = S.x[swt(t)];
  S.x[swt(t)] = make_double2(u.x - 0.5 * (double)c.x, u.y - 0.5 * (double)c.y);
  __syncthreads();
}

// OptimizeGate on a CTA of kCta16 threads: A in S.a (FP64, destroyed) ->
// u = Y X^dagger in S.x with A = X D Y^dagger, *sig = sum(D).  Returns false
// for a non-finite A.  Every thread must call it.
__device__ bool cta_polar16(Polar16Smem& S, double* sig) {
  const int t = threadIdx.x, i = t >> 4, j = t & 15;
  {
    const double2 a = S.a[swt(t)];
    if (__syncthreads_or(!(isfinite(a.x) && isfinite(a.y)))) return false;
  }
  // exact power-of-two scaling: the largest entry in [1, 4)
  unsigned em = cta_max_exponent(S);
  double pre = 1.0;
  if (em == 0u) {
    const double2 a = S.a[swt(t)];
    if (__syncthreads_and(a.x == 0.0 && a.y == 0.0)) {  // A = 0: every unitary is optimal
      S.x[swt(t)] = make_double2(i == j ? 1.0 : 0.0, 0.0);
      *sig = 0.0;
      __syncthreads();
      return true;
    }
    pre = __hiloint2double((1023 + 600) << 20, 0);  // 2^600: subnormal entries only
    S.a[swt(t)] = make_double2(a.x * pre, a.y * pre);
    em = cta_max_exponent(S);
  }
  if (em > 2045u) em = 2045u;
  const double sc = __hiloint2double((int)(2046u - em) << 20, 0);  // 2^(1023 - em)
  const double unscale =
      __hiloint2double((int)em << 20, 0) * (pre == 1.0 ? 1.0 : __hiloint2double((1023 - 600) << 20, 0));
  {
    const double2 a = S.a[swt(t)];
    S.a[swt(t)] = make_double2(a.x * sc, a.y * sc);
    S.fw[swt(t)] = make_float2((float)(a.x * sc), (float)(a.y * sc));
    S.fy[swt(t)] = make_float2(i == j ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  // stage 1: FP32 one-sided Jacobi to an off-diagonal measure of 1e-6
  for (int sweep = 0; sweep < 15; ++sweep) {
    if (t == 0) S.off[sweep & 1] = 0.f;
    __syncthreads();
    float off = 0.f;
    for (int r = 1; r <= 15; ++r) {
      off = fmaxf(off, jacobi16_round_f(S, r));
      __syncthreads();
    }
    if ((t & 31) == 0) atomicMax(reinterpret_cast<int*>(&S.off[sweep & 1]), __float_as_int(off));
    __syncthreads();
    if (S.off[sweep & 1] < 1e-6f) break;
  }
  // FP32 singular values: the column norms of W
  if (t < 16) {
    float s2 = 0.f;
    for (int r = 0; r < 16; ++r) {
      const float2 v = S.fw[sw16(r, t)];
      s2 += v.x * v.x + v.y * v.y;
    }
    S.s[t] = (double)sqrtf(s2);
  }
  __syncthreads();
  float fsmax = 0.f, fsmin = 3.4e38f;
  for (int k = 0; k < 16; ++k) {
    fsmax = fmaxf(fsmax, (float)S.s[k]);
    fsmin = fminf(fsmin, (float)S.s[k]);
  }
  if (fsmin > 1e-3f * fsmax) {
    // stage 2 (common): FP64 refinement rounds from u = Y X^dagger, as in
    // the 4x4 and 8x8 updates: a Newton-Schulz step, M = A u, and
    // u <- u (I - W + W^2 / 2) with H W + W H = M - M^dagger solved in X's
    // eigenbasis (W'_ij = K'_ij / (d_i + d_j), FP32); each round squares the
    // error.  FP32 scratch: t2 and y (unused on this path).
    float2* F0 = reinterpret_cast<float2*>(S.t2);
    float2* F1 = F0 + 256;
    float2* F2 = reinterpret_cast<float2*>(S.y);
    float2* F3 = F2 + 256;
    const float si = (float)S.s[i], sj = (float)S.s[j];
    {  // X = W's normalised columns, in place
      const float2 v = S.fw[swt(t)];
      S.fw[swt(t)] = make_float2(v.x / sj, v.y / sj);
    }
    __syncthreads();
    cta_mm<kMmND>(S.fy, S.fw, F0);  // Y X^dagger
    S.x[swt(t)] = to_d2(F0[swt(t)]);
    F3[swt(t)] = make_float2(0.f, 0.f);  // D
    __syncthreads();
    const float den = si + sj;  // >= 2e-3 of the largest singular value
    // the correction's first-order error is about 1e-7 smax / (d_i + d_j)
    // of its size: stop once that is below FP64 rounding of the result
    const float wtol = 3e-6f * fminf(1.f, 10.f * fsmin / fsmax);
    for (int round = 0; round < 5; ++round) {
      cta_ns_step(S, F0, F1, F2);
      cta_mm<kMmNN>(S.a, S.x, S.w);  // M = A u
      {
        const double2 m = S.w[swt(t)], mt = S.w[sw16(j, i)];
        F0[swt(t)] = make_float2((float)(m.x - mt.x), (float)(m.y + mt.y));  // K = M - M^dagger
      }
      __syncthreads();
      cta_mm<kMmNN>(F0, S.fw, F1);  // K X
      cta_mm<kMmDN>(S.fw, F1, F2);  // K' = X^dagger K X
      {
        const float2 v = F2[swt(t)];
        F2[swt(t)] = make_float2(v.x / den, v.y / den);  // W'
      }
      __syncthreads();
      cta_mm<kMmND>(F2, S.fw, F0);  // W' X^dagger
      cta_mm<kMmNN>(S.fw, F0, F1);  // W = X W' X^dagger
      const float2 wv = F1[swt(t)];
      const float om = cta_max_nonneg(S, fmaxf(fabsf(wv.x), fabsf(wv.y)));
      cta_mm<kMmNN>(F1, F1, F2);  // W^2
      {
        const float2 w2 = F2[swt(t)];
        F2[swt(t)] = make_float2(-wv.x + 0.5f * w2.x, -wv.y + 0.5f * w2.y);  // Z = -W + W^2 / 2
      }
      F0[swt(t)] = to_f2(S.x[swt(t)]);
      __syncthreads();
      cta_mm<kMmNN>(F0, F2, F3);  // D = u Z
      {
        const float2 d = F3[swt(t)];
        const double2 u = S.x[swt(t)];
        S.x[swt(t)] = make_double2(u.x + (double)d.x, u.y + (double)d.y);
      }
      __syncthreads();
      if (om < wtol) break;
    }
    cta_ns_step(S, F0, F1, F2);  // unitary to FP64 rounding whatever the last D
    // sum of singular values = Re Tr(A u), from the final u: the last
    // Newton-Schulz step moves Re Tr(A u) to first order in u's distance
    // from unitarity (FP32 rounding of D leaves ~1e-12 at 16x16), so the
    // trace is taken after it, in FP64 (one product per thread, summed in
    // a fixed order)
    const double2 u = S.x[swt(t)], ut = S.x[sw16(j, i)];  // u[i][j], u[j][i]
    const double2 av = S.a[swt(t)];                       // A[i][j]
    *sig = cta_sum(S, av.x * ut.x - av.y * ut.y) * unscale;
    return __syncthreads_and(isfinite(u.x) && isfinite(u.y));
  }
  // stage 2 (rare: a singular value below 1e-3 of the largest): Y unitary in
  // FP64, W = A Y, FP64 sweeps to 1e-15
  S.y[swt(t)] = to_d2(S.fy[swt(t)]);
  __syncthreads();
  cta_newton_schulz(S.y, S.t1, S.t2, 2);
  cta_mm<kMmNN>(S.a, S.y, S.w);
  const double tol2 = 1e-30;
  for (int sweep = 0; sweep < 8; ++sweep) {
    for (int r = 1; r <= 15; ++r) {
      jacobi16_round_d(S, r, tol2);
      __syncthreads();
    }
    if (cta_w_orthogonal(S, tol2)) break;
  }
  if (t < 16) {
    double s2 = 0.0;
    for (int r = 0; r < 16; ++r) s2 += S.w[sw16(r, t)].x * S.w[sw16(r, t)].x + S.w[sw16(r, t)].y * S.w[sw16(r, t)].y;
    S.s[t] = sqrt(s2);
  }
  __syncthreads();
  double smax = 0.0, smin = S.s[0], ssum = 0.0;
  for (int k = 0; k < 16; ++k) {
    smax = fmax(smax, S.s[k]);
    smin = fmin(smin, S.s[k]);
    ssum += S.s[k];
  }
  if (smin > 1e-3 * smax) {
    const double inv = 1.0 / S.s[j];
    S.x[swt(t)] = make_double2(S.w[swt(t)].x * inv, S.w[swt(t)].y * inv);
  } else if (t < 32) {  // rare: re-orthonormalise, complete the null space
    gram_schmidt16(S, smax);
  }
  __syncthreads();
  cta_mm<kMmND>(S.y, S.x, S.t1);  // u = Y X^dagger
  const double2 u = S.t1[swt(t)];
  S.x[swt(t)] = u;
  *sig = ssum * unscale;
  return __syncthreads_and(isfinite(u.x) && isfinite(u.y));
}

// ------------------------------------------------------------ environment
//
// P[x][y] = sum over the 2^(n-4) rests r of T[(r, x), (r, y)], taken from
// the tensor before the gate's removal (E = P u^dagger backward,
// u^dagger P forward, as for two-qubit gates).  Grid (B, S): thread
// t = 16 x + y of CTA b sums entry (x, y) over its CTA's slice of rests in
// the tensor's accumulation precision and writes it; the last CTA of the
// start (atomic ticket) adds the B partials in a fixed order and runs the
// 16x16 update.

template <typename R>
__global__ void __launch_bounds__(kCta16)
env16_kernel(const typename Cplx<R>::T* __restrict__ T, int n, int p0, int p1, int p2, int p3,
             int mode, double2* __restrict__ gates_k, long long gstride, double beta,
             double2* __restrict__ LR, double2* __restrict__ out, long long out_stride,
             double* __restrict__ sigma_out, int* __restrict__ status, double* __restrict__ part,
             unsigned* __restrict__ counters) {
  using CT = typename Cplx<R>::T;
  using Ar = typename Acc<R>::T;
  __shared__ Polar16Smem S;
  __shared__ bool is_last;
  const int s = blockIdx.y, B = gridDim.x, bb = blockIdx.x, t = threadIdx.x;
  const int i = t >> 4, j = t & 15;
  const int p[4] = {p0, p1, p2, p3};
  int qs[4];
  sort4(p, qs);
  const unsigned N = 1u << n;
  const unsigned nr = 1u << (n - 4);
  const unsigned chunk = (nr + B - 1) / B;
  const unsigned r_beg = bb * chunk, r_end = min(nr, r_beg + chunk);
  const CT* Ts = T + (size_t)s * N * N;
  const unsigned ox = off16(i, p), oy = off16(j, p);
  Ar vx = Ar(0), vy = Ar(0);
  for (unsigned r = r_beg; r < r_end; ++r) {
    const unsigned d = dep4(r, qs);
    const auto e = to_acc(Ts[(size_t)(d | ox) * N + (d | oy)]);
    vx += e.x;
    vy += e.y;
  }
  part[((size_t)s * B + bb) * 512 + 2 * t] = (double)vx;
  part[((size_t)s * B + bb) * 512 + 2 * t + 1] = (double)vy;
  __threadfence();
  __syncthreads();
  if (t == 0) {
    const unsigned ticket = atomicAdd(&counters[s], 1u);
    is_last = (ticket == (unsigned)B - 1u);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double2 P = make_double2(0.0, 0.0);
  for (int k = 0; k < B; ++k) {
    P.x += __ldcg(&part[((size_t)s * B + k) * 512 + 2 * t]);
    P.y += __ldcg(&part[((size_t)s * B + k) * 512 + 2 * t + 1]);
  }
  if (t == 0) counters[s] = 0u;
  if (mode == kTraceOnly) {
    out[s * out_stride + t] = P;
    return;
  }
  S.t1[swt(t)] = P;
  const double2 u = gates_k[s * gstride + t];
  S.t2[swt(t)] = u;
  __syncthreads();
  const double2 ud = cconj(S.t2[sw16(j, i)]);  // u^dagger[i][j]
  if (mode == kForward)
    cta_mm<kMmDN>(S.t2, S.t1, S.a);  // u^dagger P
  else
    cta_mm<kMmND>(S.t1, S.t2, S.a);  // P u^dagger
  const double2 E = S.a[swt(t)];
  if (out) out[s * out_stride + t] = E;
  double2* lr = LR + (size_t)s * 512;
  if (mode == kEnvOnly) {
    lr[t] = u;
    lr[256 + t] = ud;
    return;
  }
  if (beta != 0.0) S.a[swt(t)] = make_double2((1.0 - beta) * E.x + beta * ud.x, (1.0 - beta) * E.y + beta * ud.y);
  __syncthreads();
  double sg = 0.0;
  double2 un;
  if (cta_polar16(S, &sg)) {
    un = S.x[swt(t)];
  } else {
    if (t == 0) atomicCAS(status, 0, -4);
    un = u;  // keep the old gate: the tensor stays consistent
    sg = 0.0;
  }
  gates_k[s * gstride + t] = un;
  const bool bwd = mode == kBackward;
  lr[t] = bwd ? un : ud;
  lr[256 + t] = bwd ? ud : un;
  if (sigma_out && t == 0) sigma_out[s] = sg;
}

// One CTA per 16x16 matrix (qf_optimize_gates_k with dim 16).
__global__ void __launch_bounds__(kCta16) optimize16_kernel(const double2* __restrict__ E,
                                                            const double2* __restrict__ u_old,
                                                            double beta, double2* __restrict__ u_out,
                                                            double* __restrict__ sigma_out) {
  __shared__ Polar16Smem S;
  const int m = blockIdx.x, t = threadIdx.x, i = t >> 4, j = t & 15;
  double2 a = E[(size_t)m * 256 + t];
  if (beta != 0.0) {
    const double2 d = cconj(u_old[(size_t)m * 256 + j * 16 + i]);
    a = make_double2((1.0 - beta) * a.x + beta * d.x, (1.0 - beta) * a.y + beta * d.y);
  }
  S.a[swt(t)] = a;
  __syncthreads();
  double sg = 0.0;
  const bool ok = cta_polar16(S, &sg);
  u_out[(size_t)m * 256 + t] = ok ? S.x[swt(t)] : make_double2(NAN, NAN);
  if (sigma_out && t == 0) sigma_out[m] = ok ? sg : NAN;
}

// Re-unitarisation (reset_iter): three FP64 Newton-Schulz steps on every
// 16x16 gate of a circuit; CTA m takes gate m % p of start m / p and leaves
// gates of other sizes alone (desc[k] = (size, entry offset)).
__global__ void __launch_bounds__(kCta16) reunitarize16_kernel(double2* __restrict__ gates, long long gsz,
                                                               const int2* __restrict__ desc, int p) {
  __shared__ double2 M[256], t1[256], t2[256];
  const int m = blockIdx.x, s = m / p, k = m % p;
  const int2 d = desc[k];
  if (d.x != 4) return;  // the whole CTA leaves together
  double2* gp = gates + (size_t)s * gsz + d.y;
  M[swt(threadIdx.x)] = gp[threadIdx.x];
  __syncthreads();
  cta_newton_schulz(M, t1, t2, 3);
  gp[threadIdx.x] = M[swt(threadIdx.x)];
}

// ------------------------------------------------------------------ pass
//
// B <- L B R on every 16x16 block (Alg. 1 ApplyRight and ApplyLeft on four
// qubits, fused): 32 complex multiply-adds per entry against one read and
// one write.  A warp takes two blocks per group, lane 16 b + x holding row x
// of block b (consecutive blocks take consecutive column rests).  R acts
// along the row in registers and each output entry goes to a padded
// per-warp transpose buffer; the lane then takes column x of its block,
// applies L and writes the output entries of that column.  Every complex
// multiply-add takes one operator entry from shared memory (a broadcast).

constexpr int kPass16Threads = 128;
constexpr int kBlk16 = 16 * 17;  // padded 16x16 block in the transpose buffer

template <typename R, bool HL, bool HR>
__global__ void __launch_bounds__(kPass16Threads)
pass16_kernel(typename Cplx<R>::T* __restrict__ T, int n, int p0, int p1, int p2, int p3,
              const double2* __restrict__ L, long long Ls, const double2* __restrict__ Rm,
              long long Rs) {
  typedef typename Cplx<R>::T C;
  __shared__ C sL[256], sR[256];
  __shared__ C buf[kPass16Threads / 32][2 * kBlk16];
  const int s = blockIdx.y;
  for (int e = threadIdx.x; e < 256; e += kPass16Threads) {
    if (HL) sL[e] = cmake(L[s * Ls + e], R());
    if (HR) sR[e] = cmake(Rm[s * Rs + e], R());
  }
  __syncthreads();
  const int p[4] = {p0, p1, p2, p3};
  int qs[4];
  sort4(p, qs);
  unsigned off[16];  // constant indices only
#pragma unroll
  for (int v = 0; v < 16; ++v) off[v] = off16(v, p);
  const unsigned N = 1u << n;
  const int lnc = n - 4;
  const unsigned cmask = (1u << lnc) - 1u;
  const unsigned nblk = 1u << (2 * lnc);
  C* __restrict__ Ts = T + (size_t)s * N * N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = lane >> 4, x = lane & 15;
  const unsigned offx = off16(x, p);
  C* wb = buf[w] + b * kBlk16;
  const unsigned warps = gridDim.x * (kPass16Threads / 32);
  for (unsigned grp = blockIdx.x * (kPass16Threads / 32) + w; grp * 2u < nblk; grp += warps) {
    const unsigned blk = grp * 2u + (unsigned)b;
    const bool valid = blk < nblk;
    const unsigned r0 = dep4(blk >> lnc, qs), c0 = dep4(blk & cmask, qs);
    C row[16];
    if (valid) {
      const C* src = Ts + (size_t)(r0 | offx) * N + c0;
#pragma unroll
      for (int y = 0; y < 16; ++y) row[y] = src[off[y]];
    } else {
#pragma unroll
      for (int y = 0; y < 16; ++y) row[y] = czero<C>();
    }
    if (HR) {  // row <- row R
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        C acc = czero<C>();
#pragma unroll
        for (int k = 0; k < 16; ++k) acc = cfma(row[k], sR[k * 16 + c], acc);
        acc = cfinish(acc);
        if (HL)
          wb[x * 17 + c] = acc;
        else if (valid)
          Ts[(size_t)(r0 | offx) * N + (c0 | off[c])] = acc;
      }
    } else if (HL) {
#pragma unroll
      for (int y = 0; y < 16; ++y) wb[x * 17 + y] = row[y];
    }
    if (HL) {
      __syncwarp();
      C col[16];  // column x of the block
#pragma unroll
      for (int k = 0; k < 16; ++k) col[k] = wb[k * 17 + x];
      __syncwarp();  // the buffer is rewritten by the next group
      if (valid) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          C acc = czero<C>();
#pragma unroll
          for (int k = 0; k < 16; ++k) acc = cfma(sL[r * 16 + k], col[k], acc);
          Ts[(size_t)(r0 | off[r]) * N + (c0 | offx)] = cfinish(acc);
        }
      }
    }
  }
}

// complex64 version for the FP32 pipe.  In the kernel above every complex
// multiply-add waits on one shared-memory operator load, which keeps the
// FP32 pipe below a third busy.  Here a lane holds row x of two blocks of a
// four-block group and each 16-byte operator load brings two adjacent
// operator entries, so one load serves four complex multiply-adds (16
// FMAs): R is read as (R[k][c], R[k][c+1]) pairs, L from a transposed copy
// as (L[r][k], L[r+1][k]) pairs.  With kPair (no gate bit at 0, n >= 5) the
// lane's two blocks are adjacent column rests 2m and 2m + 1, whose entries
// sit side by side: every global load and store is one 16-byte access of
// both blocks.  Otherwise the blocks are b and b + 2 and take 8-byte
// accesses.  The output loops stay rolled: unrolled, the body overflows
// the instruction cache.
constexpr int kPass16cBlocks = 4;  // blocks per warp and group

template <bool HL, bool HR, bool kPair>
__global__ void __launch_bounds__(kPass16Threads)
pass16c_kernel(float2* __restrict__ T, int n, int p0, int p1, int p2, int p3,
               const double2* __restrict__ L, long long Ls, const double2* __restrict__ Rm,
               long long Rs) {
  __shared__ float4 sR2[16 * 8];   // [k][c/2]: (R[k][c], R[k][c+1])
  __shared__ float4 sLT2[16 * 8];  // [k][r/2]: (L[r][k], L[r+1][k])
  __shared__ float2 buf[kPass16Threads / 32][kPass16cBlocks * kBlk16];
  const int s = blockIdx.y;
  for (int e = threadIdx.x; e < 128; e += kPass16Threads) {
    const int k = e >> 3, c2 = (e & 7) * 2;
    if (HR) {
      const double2 a = Rm[s * Rs + k * 16 + c2], b = Rm[s * Rs + k * 16 + c2 + 1];
      sR2[e] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
    }
    if (HL) {
      const double2 a = L[s * Ls + c2 * 16 + k], b = L[s * Ls + (c2 + 1) * 16 + k];
      sLT2[e] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
    }
  }
  __syncthreads();
  const int p[4] = {p0, p1, p2, p3};
  int qs[4];
  sort4(p, qs);
  unsigned off[16];  // constant indices only
#pragma unroll
  for (int v = 0; v < 16; ++v) off[v] = off16(v, p);
  const unsigned N = 1u << n;
  const int lnc = n - 4;
  const unsigned cmask = (1u << lnc) - 1u;
  const unsigned nblk = 1u << (2 * lnc);
  float2* __restrict__ Ts = T + (size_t)s * N * N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = lane >> 4, x = lane & 15;
  const unsigned offx = off16(x, p);
  // the lane's blocks within the group: (2b, 2b + 1) paired, else (b, b + 2)
  const unsigned oa = kPair ? 2u * (unsigned)b : (unsigned)b, ob = kPair ? oa + 1u : oa + 2u;
  float2* wa = buf[w] + oa * kBlk16;
  float2* wbb = buf[w] + ob * kBlk16;
  const unsigned warps = gridDim.x * (kPass16Threads / 32);
  for (unsigned grp = blockIdx.x * (kPass16Threads / 32) + w; grp * kPass16cBlocks < nblk; grp += warps) {
    const unsigned ba = grp * kPass16cBlocks + oa, bb2 = grp * kPass16cBlocks + ob;
    const bool va = ba < nblk, vb = bb2 < nblk;  // both true with kPair (nblk >= 4)
    const unsigned ra = dep4(ba >> lnc, qs), ca = dep4(ba & cmask, qs);
    const unsigned rb = dep4(bb2 >> lnc, qs), cb = dep4(bb2 & cmask, qs);
    // with kPair: rb = ra and cb = ca + 1 (block 2m + 1 differs in column bit 0)
    float2 xa[16], xb[16];
    if (kPair) {
      const float2* sa = Ts + (size_t)(ra | offx) * N + ca;
#pragma unroll
      for (int y = 0; y < 16; ++y) {
        const float4 v = *reinterpret_cast<const float4*>(sa + off[y]);
        xa[y] = make_float2(v.x, v.y);
        xb[y] = make_float2(v.z, v.w);
      }
    } else {
      const float2* sa = Ts + (size_t)(ra | offx) * N + ca;
      const float2* sb = Ts + (size_t)(rb | offx) * N + cb;
#pragma unroll
      for (int y = 0; y < 16; ++y) {
        xa[y] = va ? sa[off[y]] : make_float2(0.f, 0.f);
        xb[y] = vb ? sb[off[y]] : make_float2(0.f, 0.f);
      }
    }
    if (HR) {  // rows <- rows R, two output columns per operator load
#pragma unroll 1
      for (int c = 0; c < 16; c += 2) {
        float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const float4 r = sR2[k * 8 + c / 2];
          const float2 r0 = make_float2(r.x, r.y), r1 = make_float2(r.z, r.w);
          a0 = cfma(xa[k], r0, a0);
          a1 = cfma(xa[k], r1, a1);
          b0 = cfma(xb[k], r0, b0);
          b1 = cfma(xb[k], r1, b1);
        }
        if (HL) {
          wa[x * 17 + c] = a0;
          wa[x * 17 + c + 1] = a1;
          wbb[x * 17 + c] = b0;
          wbb[x * 17 + c + 1] = b1;
        } else if (kPair) {
          const unsigned c0 = off16(c, p), c1 = off16(c + 1, p);
          *reinterpret_cast<float4*>(Ts + (size_t)(ra | offx) * N + (ca | c0)) = make_float4(a0.x, a0.y, b0.x, b0.y);
          *reinterpret_cast<float4*>(Ts + (size_t)(ra | offx) * N + (ca | c1)) = make_float4(a1.x, a1.y, b1.x, b1.y);
        } else {
          const unsigned c0 = off16(c, p), c1 = off16(c + 1, p);
          if (va) {
            Ts[(size_t)(ra | offx) * N + (ca | c0)] = a0;
            Ts[(size_t)(ra | offx) * N + (ca | c1)] = a1;
          }
          if (vb) {
            Ts[(size_t)(rb | offx) * N + (cb | c0)] = b0;
            Ts[(size_t)(rb | offx) * N + (cb | c1)] = b1;
          }
        }
      }
    } else if (HL) {
#pragma unroll
      for (int y = 0; y < 16; ++y) {
        wa[x * 17 + y] = xa[y];
        wbb[x * 17 + y] = xb[y];
      }
    }
    if (HL) {
      __syncwarp();
#pragma unroll
      for (int k = 0; k < 16; ++k) {  // column x of both blocks
        xa[k] = wa[k * 17 + x];
        xb[k] = wbb[k * 17 + x];
      }
      __syncwarp();  // the buffers are rewritten by the next group
#pragma unroll 1
      for (int r = 0; r < 16; r += 2) {
        float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const float4 l = sLT2[k * 8 + r / 2];
          const float2 l0 = make_float2(l.x, l.y), l1 = make_float2(l.z, l.w);
          a0 = cfma(l0, xa[k], a0);
          a1 = cfma(l1, xa[k], a1);
          b0 = cfma(l0, xb[k], b0);
          b1 = cfma(l1, xb[k], b1);
        }
        const unsigned r0o = off16(r, p), r1o = off16(r + 1, p);
        if (kPair) {
          *reinterpret_cast<float4*>(Ts + (size_t)(ra | r0o) * N + (ca | offx)) = make_float4(a0.x, a0.y, b0.x, b0.y);
          *reinterpret_cast<float4*>(Ts + (size_t)(ra | r1o) * N + (ca | offx)) = make_float4(a1.x, a1.y, b1.x, b1.y);
        } else {
          if (va) {
            Ts[(size_t)(ra | r0o) * N + (ca | offx)] = a0;
            Ts[(size_t)(ra | r1o) * N + (ca | offx)] = a1;
          }
          if (vb) {
            Ts[(size_t)(rb | r0o) * N + (cb | offx)] = b0;
            Ts[(size_t)(rb | r1o) * N + (cb | offx)] = b1;
          }
        }
      }
    }
  }
}

// ------------------------------------------- tensor-core 16x16 pass (tcgen05)
// Complex64 with both operators, n >= 7.  The block products of the pass
// are dense contractions (128 FP32 FMAs per entry, above what the FP32 pipe
// delivers at HBM speed), so they run on the fifth-generation tensor cores
// as real GEMMs in 3xTF32 form: each FP32 value x is split into TF32 parts
// hi + lo, and A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32
// accumulation in tensor memory (the dropped lo*lo term and the rounding of
// the parts stay near 2^-21 of |A B|).
//
// A tile is the 16 x 128 slab of one row rest's 16 row variants and the 128
// columns of the 8 column-rest blocks whose rests differ only in the 3
// lowest non-gate column bits: the tile's columns are all values of the 7
// column bits S = {gate bits} + {3 lowest non-gate bits} (tile column u:
// bit k of u is the k-th lowest position of S).  Inside the kernel a local
// gate index is in ascending-bit order (bit k <-> gate position qs[k]); the
// operators are permuted to that order when they are embedded.  Per tile:
//  0. (during the previous tile) the tile streams into a staging buffer as
//     16-byte copies of adjacent column pairs (column bit 0 is always in S);
//  1. thread m (tensor-memory lane m) takes tile column u = m from the
//     staging buffer, 16 entries, one per row variant, and stores it as
//     A[m][2 i + c] (row variant i, c = re / im) in TF32 hi (columns 0-31)
//     and lo (32-63);
//  2. one thread issues D = A Emb(L)^T (4 K steps of 8, three products:
//     12 MMAs of M = 128, N = 32; A from tensor memory, the embedded
//     operator from shared memory, K-major with the 128-byte swizzle) and
//     commits to an mbarrier; meanwhile the next tile starts streaming in;
//  3. thread m moves D (column u of L B) into the tile buffer;
//  4. thread m' = 16 b + i takes row i of block b from the buffer and the
//     same sequence applies Emb(R^T) (R on the column index);
//  5. thread m' puts its output row into the buffer, and the tile goes to
//     HBM as 16-byte column pairs.
// The tile buffer holds entry (i, u) at i * 128 + (u ^ i): every access
// pattern above hits each bank pair exactly twice per warp (a 16-byte
// access of a pair takes the pair swapped for odd i).  Emb(O) is the real
// 32 x 32 matrix with Emb[2 a + c'][2 b + c] = Re O[a][b] for c' = c, -Im
// for (0, 1) and +Im for (1, 0), so that out[a] = sum_b O[a][b] x[b].
// Tensor memory: 128 columns per CTA (A hi, A lo, D at 64-95); 52 KB of
// shared memory per CTA keep at most 4 CTAs (512 columns) on an SM.
// Every wait is bounded (wait_limit polls).  When one runs out, the CTA
// records QF_ETIMEOUT in *status (if given), writes NaN over the rest of its
// tiles, waits (bounded by the default limit) for its MMAs in flight, frees
// its tensor memory and ends.
constexpr int kTcThreads = 128;
constexpr uint32_t kTcCols = 128;
constexpr int kTcSmem = 52 * 1024;
constexpr int kTcChunk = 16;           // tiles per CTA at most
constexpr int kTcWaitLimit = 1 << 22;  // polls of one completion wait
std::atomic<int> g_tc_wait_limit{kTcWaitLimit};  // qf_set_tc_wait_limit

// Byte offset of element (row nn, column k) in a K-major, 128-byte-swizzled
// 32 x 32 TF32 tile (1024-byte aligned).
__device__ __forceinline__ uint32_t sw128_off(int nn, int k) {
  return (uint32_t)(nn * 128 + (((k >> 2) ^ (nn & 7)) << 4) + ((k & 3) << 2));
}

// D = A Emb^T in two halves, issued by one thread: with the operator tile
// [Emb_hi; Emb_lo] (64 rows: the lo tile follows the hi tile) one N = 64 MMA
// per K step gives A_hi Emb_hi^T (columns 64-95) and A_hi Emb_lo^T (96-127),
// and an N = 32 MMA adds A_lo Emb_hi^T to the first half: 8 MMAs, the sum
// of the halves is the 3xTF32 product.
__device__ __forceinline__ void tc_issue_stage(uint32_t tb, uint32_t op_hi, uint32_t bar) {
  constexpr uint32_t id64 = tc::idesc_tf32(128, 64), id32 = tc::idesc_tf32(128, 32);
  tc::fence_after_sync();
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const uint64_t bh = tc::desc_kmajor_sw128(op_hi + 32u * kk);
    tc::mma_tf32_ts(tb + 64u, tb + 8u * kk, bh, id64, kk > 0 ? 1u : 0u);
    tc::mma_tf32_ts(tb + 64u, tb + 32u + 8u * kk, bh, id32, 1u);
  }
  tc::commit(bar);
}

// Entries 8 h .. 8 h + 7 of this lane's D (the two halves summed).
__device__ __forceinline__ void tc_load_d(uint32_t ta, int h, float2 (&out)[8]) {
  uint32_t a[16], b[16];
  tc::ld16(ta + 64u + 16u * h, a);
  tc::ld16(ta + 96u + 16u * h, b);
#pragma unroll
  for (int e = 0; e < 8; ++e)
    out[e] = make_float2(__uint_as_float(a[2 * e]) + __uint_as_float(b[2 * e]),
                         __uint_as_float(a[2 * e + 1]) + __uint_as_float(b[2 * e + 1]));
}

// 16 complex values get(0..15) -> TF32 hi parts at columns 0-31 and lo
// parts at 32-63 of this thread's lane, eight values at a time.  The lo
// part x - hi goes in as FP32: the tensor core takes its leading TF32 bits,
// which keeps it to about 2^-10 of itself (2^-21 of x).
template <typename Get>
__device__ __forceinline__ void tc_store_a(uint32_t ta, Get get) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float2 z[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) z[e] = get(8 * h + e);
    uint32_t v[16];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      v[2 * e] = tc::tf32(z[e].x);
      v[2 * e + 1] = tc::tf32(z[e].y);
    }
    tc::st16(ta + 16u * h, v);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      v[2 * e] = __float_as_uint(z[e].x - __uint_as_float(v[2 * e]));
      v[2 * e + 1] = __float_as_uint(z[e].y - __uint_as_float(v[2 * e + 1]));
    }
    tc::st16(ta + 32u + 16u * h, v);
  }
}

// Rows 8 h .. 8 h + 7 of tile columns 2 pp and 2 pp + 1 (adjacent entries:
// column bit 0 is always in S) -> the staging buffer, as asynchronous
// 16-byte copies; `off` is the pair's entry offset in row variant 0.
__device__ __forceinline__ void tc_prefetch(float2* stage, const float2* Tp, unsigned off, const unsigned* rowoff,
                                            int pp, int h) {
#pragma unroll 4
  for (int e = 0; e < 8; ++e) {
    const int i = 8 * h + e;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_addr(stage + i * 128 + 2 * pp)),
                 "l"(Tp + off + rowoff[i])
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void tc_prefetch_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__global__ void __launch_bounds__(kTcThreads, 4)
pass16tc_kernel(float2* __restrict__ T, int n, int S, int p0, int p1, int p2, int p3,
                const double2* __restrict__ L, long long Ls, const double2* __restrict__ Rm, long long Rs,
                int* status, int wait_limit) {
  extern __shared__ unsigned char dsm[];
  const uint32_t dsm_s = tc::smem_addr(dsm);
  const uint32_t ops_s = (dsm_s + 1023u) & ~1023u;  // L hi, L lo, R hi, R lo: 4 KB each
  unsigned char* ops = dsm + (ops_s - dsm_s);
  float2* buf = reinterpret_cast<float2*>(ops + 4 * 4096);  // [16][128] complex, the tile
  float2* stage = buf + 16 * 128;  // [16][128]: the next tile, in flight
  uint64_t* bar = reinterpret_cast<uint64_t*>(stage + 16 * 128);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  unsigned* s_rowoff = tslot + 1;  // [16] row offset (entries) of ascending row variant i
  unsigned* s_uj = s_rowoff + 16;  // [16] tile-column bits of ascending gate index j
  const uint32_t bar_s = tc::smem_addr(bar);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int pp = tid & 63, ph = tid >> 6;  // copy role: column pair pp, rows 8 ph ..
  const unsigned N = 1u << n;

  if (warp == 0) tc::tmem_alloc(tc::smem_addr(tslot), kTcCols);
  if (tid == 0) tc::mbar_init(bar_s, 1);

  const int p[4] = {p0, p1, p2, p3};
  int qs[4];
  sort4(p, qs);
  int pidx[4];  // which of p[] is the k-th lowest gate position
#pragma unroll
  for (int k = 0; k < 4; ++k) pidx[k] = (p[0] == qs[k]) ? 0 : (p[1] == qs[k]) ? 1 : (p[2] == qs[k]) ? 2 : 3;
  // S, ascending: tile-column bit k <-> the k-th selected position (bit 0
  // is always selected: a gate bit or the lowest non-gate bit)
  unsigned gbits_u = 0;  // tile-column bits that are gate bits
  unsigned colm = 0;     // column offset of tile column u = tid
  unsigned colp = 0;     // column offset of tile column u = 2 pp
  {
    int cnt = 0, ng = 0;
    for (int pos = 0; cnt < 7; ++pos) {
      const bool g = pos == qs[0] || pos == qs[1] || pos == qs[2] || pos == qs[3];
      if (g || ng < 3) {
        if (g)
          gbits_u |= 1u << cnt;
        else
          ++ng;
        colm |= (((unsigned)tid >> cnt) & 1u) << pos;
        colp |= (((unsigned)(2 * pp) >> cnt) & 1u) << pos;
        ++cnt;
      }
    }
  }
  if (tid < 16) {
    const unsigned i = (unsigned)tid;
    s_rowoff[tid] = ((i & 1u) << qs[0] | ((i >> 1) & 1u) << qs[1] | ((i >> 2) & 1u) << qs[2] |
                     ((i >> 3) & 1u) << qs[3]) * N;
    unsigned v = 0;
    int gk = 0;
    for (int k = 0; k < 7; ++k)
      if ((gbits_u >> k) & 1u) v |= ((i >> gk++) & 1u) << k;
    s_uj[tid] = v;
  }
  // row role: thread m' = 16 b + i holds row i of block b (tile-column bits ub)
  const unsigned rb_i = (unsigned)tid & 15u;
  unsigned ub = 0;
  {
    int bk = 0;
    for (int k = 0; k < 7; ++k)
      if (!((gbits_u >> k) & 1u)) ub |= (((unsigned)tid >> (4 + bk++)) & 1u) << k;
  }

  const int lnc = n - 4;
  const unsigned cgbits = (unsigned)lnc - 3u;
  const unsigned tps = 1u << (2 * lnc - 3);  // tiles per start
  const unsigned total = tps * (unsigned)S;
  const unsigned chunk = (total + gridDim.x - 1) / gridDim.x;
  const unsigned t0 = blockIdx.x * chunk;
  const unsigned t1 = t0 + chunk < total ? t0 + chunk : total;
  const size_t NN = (size_t)N * N;

  // tile -> start, and the entry offset of the tile's row rest and column
  // base in row variant 0 of the start's tensor (below 2^30 for n <= 15)
  const auto geom = [&](unsigned tile, unsigned& s, unsigned& base) {
    s = tile >> (2 * lnc - 3);
    const unsigned t = tile & (tps - 1u);
    base = dep4(t >> cgbits, qs) * N + dep4((t & ((1u << cgbits) - 1u)) << 3, qs);
  };

  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tb = *tslot;
  const uint32_t ta = tb + ((uint32_t)(warp * 32) << 16);  // this warp's lanes

  // tile output (buffer) -> HBM as 16-byte column pairs; entry (i, u) sits
  // at u ^ i, so odd i find the pair swapped
  const auto store_tile = [&](float2* Tq, unsigned bq) {
#pragma unroll 4
    for (int e = 0; e < 8; ++e) {
      const int i = 8 * ph + e;
      const float4 v = *reinterpret_cast<const float4*>(buf + i * 128 + ((2 * pp) ^ (i & 14)));
      *reinterpret_cast<float4*>(Tq + bq + colp + s_rowoff[i]) = (i & 1) ? make_float4(v.z, v.w, v.x, v.y) : v;
    }
  };

  unsigned tile = t0, cur_s = 0xffffffffu, s_cur = 0, b_cur = 0;
  float2* prev_T = nullptr;  // the previous tile, its output still in the buffer
  unsigned prev_b = 0;
  uint32_t phase = 0;
  bool failed = false;
  if (tile < t1) {
    geom(tile, s_cur, b_cur);
    tc_prefetch(stage, T + s_cur * NN, b_cur + colp, s_rowoff, pp, ph);
  }
  tc_prefetch_wait();
  __syncthreads();  // the first tile has landed
  for (; tile < t1; ++tile) {
    const unsigned s = s_cur, base = b_cur;
    float2* Tp = T + s * NN;
    const bool more = tile + 1 < t1;
    if (more) geom(tile + 1, s_cur, b_cur);
    if (s != cur_s) {  // embed this start's operators (no MMA is in flight)
      cur_s = s;
      // one complex entry O[a][b] per thread and step -> the four real
      // entries (2 a + c', 2 b + c), hi and lo
#pragma unroll 1
      for (int e = tid; e < 512; e += kTcThreads) {
        const int which = e >> 8, a = (e >> 4) & 15, b = e & 15;
        int ga = 0, gb = 0;  // the gate's own local indices of a and b
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          ga |= ((a >> q) & 1) << (3 - pidx[q]);
          gb |= ((b >> q) & 1) << (3 - pidx[q]);
        }
        // O = L (a: output row) or R^T (a: output column); FP32 operators,
        // as the FMA kernels
        const double2 o = which == 0 ? L[s * Ls + ga * 16 + gb] : Rm[s * Rs + gb * 16 + ga];
        const float ore = (float)o.x, oim = (float)o.y;
        unsigned char* obase = ops + which * 8192;
#pragma unroll
        for (int cp = 0; cp < 2; ++cp)
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const float val = (cp == c) ? ore : (cp == 0 ? -oim : oim);
            const uint32_t hi = tc::tf32(val);
            const uint32_t lo = tc::tf32(val - __uint_as_float(hi));
            const uint32_t off = sw128_off(2 * a + cp, 2 * b + c);
            *reinterpret_cast<uint32_t*>(obase + off) = hi;
            *reinterpret_cast<uint32_t*>(obase + 4096 + off) = lo;
          }
      }
      tc::fence_async_smem();
    }
    // 1. tile column tid -> A
    tc_store_a(ta, [&](int i) { return stage[i * 128 + tid]; });
    tc::fence_before_sync();
    __syncthreads();
    // 2. L stage; meanwhile the next tile streams into the staging buffer and
    //    the previous tile's output goes to HBM
    if (tid == 0) tc_issue_stage(tb, ops_s, bar_s);
    if (more) tc_prefetch(stage, T + s_cur * NN, b_cur + colp, s_rowoff, pp, ph);
    if (prev_T) store_tile(prev_T, prev_b);
    const bool ok1 = tc::mbar_wait(bar_s, phase, wait_limit);
    phase ^= 1u;
    if (__syncthreads_or(!ok1)) {  // also frees the buffer
      failed = true;
      break;
    }
    tc::fence_after_sync();
    // 3. column tid of L B -> buffer
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float2 d[8];
      tc_load_d(ta, h, d);
#pragma unroll
      for (int e = 0; e < 8; ++e) buf[(8 * h + e) * 128 + (tid ^ (8 * h + e))] = d[e];
    }
    tc::fence_before_sync();
    __syncthreads();
    // 4. R stage on rows (b, i)
    tc_store_a(ta, [&](int j) { return buf[rb_i * 128 + ((ub | s_uj[j]) ^ rb_i)]; });
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) tc_issue_stage(tb, ops_s + 8192u, bar_s);
    const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(bar_s, phase, wait_limit));
    phase ^= 1u;
    tc::fence_after_sync();
    // 5. output rows -> buffer
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float2 d[8];
      if (ok) tc_load_d(ta, h, d);
#pragma unroll
      for (int e = 0; e < 8; ++e) buf[rb_i * 128 + ((ub | s_uj[8 * h + e]) ^ rb_i)] = d[e];
    }
    tc_prefetch_wait();  // the next tile is visible to every thread after the barrier
    tc::fence_before_sync();
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    prev_T = Tp;  // 6. stored during the next tile's L stage
    prev_b = base;
  }
  if (!failed && prev_T) store_tile(prev_T, prev_b);
  if (failed) {
    if (tid == 0 && status) atomicCAS(status, 0, QF_ETIMEOUT);
    const float nan = __int_as_float(0x7fc00000);
    for (; tile < t1; ++tile) {
      unsigned s, base;
      geom(tile, s, base);
      float2* Tp = T + s * NN;
#pragma unroll
      for (int i = 0; i < 16; ++i) Tp[base + colm + s_rowoff[i]] = make_float2(nan, nan);
    }
    tc::mbar_wait(bar_s, phase ^ 1u, kTcWaitLimit);  // the stage that ran out, should it still end
  }
  tc_prefetch_wait();
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tb, kTcCols);
}

template <typename R, bool HL, bool HR>
void pass16_launch(void* T, int n, int S, const int* p, const double2* L, long long Ls,
                   const double2* Rm, long long Rs, cudaStream_t st, int* status) {
  typedef typename Cplx<R>::T C;
  if constexpr (std::is_same<R, float>::value && HL && HR) {
    if (n >= 7) {
      static const bool attr = [] {  // once per process (thread-safe static)
        cudaFuncSetAttribute(pass16tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
        cudaFuncSetAttribute(pass16tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        return true;
      }();
      (void)attr;
      // chunks of at most kTcChunk tiles per CTA, over several waves: CTAs
      // that find their SM shared with other kernels then delay few tiles
      const long long tiles = (long long)S << (2 * (n - 4) - 3);
      const long long slots = (long long)sm_count() * 4;
      long long chunk = (tiles + slots - 1) / slots;
      if (chunk > kTcChunk) chunk = kTcChunk;
      pass16tc_kernel<<<(unsigned)((tiles + chunk - 1) / chunk), kTcThreads, kTcSmem, st>>>(
          (float2*)T, n, S, p[0], p[1], p[2], p[3], L, Ls, Rm, Rs, status, g_tc_wait_limit.load());
      return;
    }
  }
  const int per_group = std::is_same<R, float>::value ? kPass16cBlocks : 2;
  const long long groups = ((1ll << (2 * (n - 4))) + per_group - 1) / per_group;
  const long long want = (groups + 3) / 4;
  long long cap = ((long long)sm_count() * 8 + S - 1) / S;
  if (cap < 1) cap = 1;
  dim3 grid((unsigned)(want < cap ? want : cap), S);
  if constexpr (std::is_same<R, float>::value) {
    // adjacent block pairs when column bit 0 is a rest bit (and n >= 5)
    const bool pair = n >= 5 && p[0] != 0 && p[1] != 0 && p[2] != 0 && p[3] != 0;
    if (pair)
      pass16c_kernel<HL, HR, true><<<grid, kPass16Threads, 0, st>>>((float2*)T, n, p[0], p[1], p[2], p[3], L, Ls,
                                                                    Rm, Rs);
    else
      pass16c_kernel<HL, HR, false><<<grid, kPass16Threads, 0, st>>>((float2*)T, n, p[0], p[1], p[2], p[3], L,
                                                                     Ls, Rm, Rs);
  }
  else
    pass16_kernel<R, HL, HR><<<grid, kPass16Threads, 0, st>>>((C*)T, n, p[0], p[1], p[2], p[3], L, Ls, Rm, Rs);
}

template <typename R>
void pass16_ops(void* T, int n, int S, const int* p, const double2* L, long long Ls,
                const double2* Rm, long long Rs, cudaStream_t st, int* status) {
  if (L && Rm)
    pass16_launch<R, true, true>(T, n, S, p, L, Ls, Rm, Rs, st, status);
  else if (L)
    pass16_launch<R, true, false>(T, n, S, p, L, Ls, Rm, Rs, st, status);
  else if (Rm)
    pass16_launch<R, false, true>(T, n, S, p, L, Ls, Rm, Rs, st, status);
}

}  // namespace

// ================================================================ launchers

cudaError_t launch_pass16(void* T, int n, int S, const int* q, const double2* L, long long Ls,
                          const double2* R, long long Rs, int prec, cudaStream_t st, int* status) {
  if (!L && !R) return cudaSuccess;
  const int p[4] = {qubit_bit(n, q[0]), qubit_bit(n, q[1]), qubit_bit(n, q[2]), qubit_bit(n, q[3])};
  if (prec == 0)
    pass16_ops<double>(T, n, S, p, L, Ls, R, Rs, st, status);
  else if (prec == 2)
    pass16_ops<DF>(T, n, S, p, L, Ls, R, Rs, st, status);
  else
    pass16_ops<float>(T, n, S, p, L, Ls, R, Rs, st, status);
  return cudaGetLastError();
}

cudaError_t launch_update16(const void* T, int n, int S, const int* q, double2* gates_k,
                            long long gstride, int mode, double beta, double2* LR, double2* out,
                            long long out_stride, double* sigma_out, int* status, double* part,
                            unsigned* counters, int prec, cudaStream_t st) {
  const int p0 = qubit_bit(n, q[0]), p1 = qubit_bit(n, q[1]), p2 = qubit_bit(n, q[2]),
            p3 = qubit_bit(n, q[3]);
  dim3 grid(env_ctas(n), S);
  if (prec == 0)
    env16_kernel<double><<<grid, kCta16, 0, st>>>((const double2*)T, n, p0, p1, p2, p3, mode, gates_k,
                                                  gstride, beta, LR, out, out_stride, sigma_out, status,
                                                  part, counters);
  else if (prec == 2)
    env16_kernel<DF><<<grid, kCta16, 0, st>>>((const dfc*)T, n, p0, p1, p2, p3, mode, gates_k, gstride,
                                              beta, LR, out, out_stride, sigma_out, status, part,
                                              counters);
  else
    env16_kernel<float><<<grid, kCta16, 0, st>>>((const float2*)T, n, p0, p1, p2, p3, mode, gates_k,
                                                 gstride, beta, LR, out, out_stride, sigma_out, status,
                                                 part, counters);
  return cudaGetLastError();
}

cudaError_t launch_optimize16(const double2* E, const double2* u_old, double beta, int count,
                              double2* u_out, double* sigma_out, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  optimize16_kernel<<<count, kCta16, 0, st>>>(E, u_old, beta, u_out, sigma_out);
  return cudaGetLastError();
}

cudaError_t launch_reunitarize16(double2* gates, long long gsz, const int2* desc, int p, int S,
                                 cudaStream_t st) {
  if (p * S <= 0) return cudaSuccess;
  reunitarize16_kernel<<<p * S, kCta16, 0, st>>>(gates, gsz, desc, p);
  return cudaGetLastError();
}

}  // namespace qf

int qf_set_tc_wait_limit(int polls) {
  if (polls < 0) return qf::g_tc_wait_limit.load();
  return qf::g_tc_wait_limit.exchange(polls);
}
