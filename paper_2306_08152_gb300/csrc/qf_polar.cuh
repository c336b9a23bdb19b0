// Warp-cooperative 4x4 gate update (OptimizeGate, Sec. III-A1, Eq. opt_u).
//
// With A = X D Y^dagger the unitary maximising Re Tr(A u) is u = Y X^dagger.
// GB300 issues an FP64 warp instruction about every 33 ns (its FP64 rate is
// 1/64 of FP32), so the update is computed in stages on one warp
// (lane = matrix element):
//   0. A is scaled by a power of two (exact) so that its largest entry lies
//      in [1, 4): the FP32 stage neither under- nor overflows at any scale;
//   1. a one-sided Jacobi SVD in FP32 (rotations J with A J = W having
//      orthogonal columns; Y ~ J, X ~ W's normalised columns, D ~ their
//      norms), which costs no FP64 work;
//   2. when every FP32 singular value is above 1e-3 of the largest (the
//      common case), FP64 refinement: Newton-Schulz re-unitarisation of
//      u0 = Y X^dagger, M = A u (Hermitian positive semi-definite at the
//      optimum), and the correction u <- u (I - W + W^2/2) where W solves
//      H W + W H = M - M^dagger in X's eigenbasis (W_ij = K'_ij / (d_i + d_j)).
//      One round turns the FP32 error e into O(e^2); rounds repeat while
//      the correction is large;
//   3. otherwise (A close to singular; rare, out of line): FP64 one-sided
//      Jacobi from the FP32 rotation, columns below 1e-13 of the largest
//      singular value completed by FP64 Gram-Schmidt, and FP64
//      Newton-Schulz.  The polar factor of a nearly singular A is
//      ill-conditioned (a perturbation dA moves it by up to about
//      2 ||dA|| / s_min, R.-C. Li's bound for complex matrices), so this
//      path keeps the FP64 rounding of A as the only source of error, where
//      the FP32 eigenbasis of stage 2 would not resolve the small singular
//      directions.
// The sum of singular values (the new Re Tr(E u)) is returned with it.

#pragma once

#include "qf_device.cuh"

namespace qf {
namespace dev {

// Sum over the four rows of a lane-distributed 4x4 (lanes with equal j).
__device__ __forceinline__ double colsum4(double v) {
  v += __shfl_xor_sync(kFull, v, 4);
  v += __shfl_xor_sync(kFull, v, 8);
  return v;
}

// Power-of-two scaling of the warp's 4x4 A (exact): a <- a 2^-e with e the
// largest binary exponent among the entries, so that the largest entry lies
// in [1, 2) (in [2, 4) when e is the largest finite exponent); *unscale =
// 2^e.  A matrix of subnormal entries only is first multiplied by 2^600.
// Returns false for A = 0.
__device__ __forceinline__ bool pow2_scale(double2& a, double* unscale) {
  auto top = [&]() {
    const unsigned ex = (unsigned)(__double2hiint(a.x) >> 20) & 0x7ffu;
    const unsigned ey = (unsigned)(__double2hiint(a.y) >> 20) & 0x7ffu;
    return __reduce_max_sync(kFull, ex > ey ? ex : ey);
  };
  unsigned e = top();
  double pre = 1.0;
  if (e == 0u) {
    if (__all_sync(kFull, a.x == 0.0 && a.y == 0.0)) return false;
    pre = __hiloint2double((1023 + 600) << 20, 0);  // 2^600
    a.x *= pre;
    a.y *= pre;
    e = top();
  }
  if (e > 2045u) e = 2045u;  // keep 2^-e normal
  const double s = __hiloint2double((int)(2046u - e) << 20, 0);  // 2^(1023 - e)
  a.x *= s;
  a.y *= s;
  // 2^(e - 1023) / pre
  *unscale = __hiloint2double((int)e << 20, 0) * (pre == 1.0 ? 1.0 : __hiloint2double((1023 - 600) << 20, 0));
  return true;
}

// FP64 one-sided Jacobi sweeps on the lane-distributed pair (W, Y) (after
// the FP32 stage): each round r = 1..3 pairs column j with j ^ r (two
// disjoint pairs) and rotates both so that W[:,p] and W[:,q] become
// orthogonal.  The inner products g = W_p^dagger W_q, |W_p|^2 and |W_q|^2
// are FP64 sums; the rotation angle t = tan(theta) is taken in FP32 from
// zeta = (|W_q|^2 - |W_p|^2) / (2|g|) (an angle accurate to FP32 still
// shrinks g by ~1e-7 per sweep), and the rotation applied is unitary to
// FP64 rounding (c = 1/sqrt(1 + t^2) and e = conj(g)/|g| by rsqrt_d).
// Stops once every pair has |g| <= tol |W_p| |W_q|.
__device__ __forceinline__ void polish4(const Lane& L, double2& w, double2& y, double tol,
                                        int max_sweeps) {
  const double tol2 = tol * tol;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    bool open = false;
#pragma unroll 1
    for (int r = 1; r <= 3; ++r) {
      const int q = L.j ^ r;
      const bool isP = L.j < q;
      const int src = L.at(L.i, q);
      const double2 wq = shfl(w, src), yq = shfl(y, src);
      const double n2 = colsum4(w.x * w.x + w.y * w.y);
      const double n2q = __shfl_sync(kFull, n2, src);
      const double2 cp = isP ? w : wq, cq = isP ? wq : w;
      const double gx = colsum4(cp.x * cq.x + cp.y * cq.y);
      const double gy = colsum4(cp.x * cq.y - cp.y * cq.x);
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
          const double2 ew = cmul(e, wq), ey = cmul(e, yq);
          w = make_double2(c * w.x - sn * ew.x, c * w.y - sn * ew.y);
          y = make_double2(c * y.x - sn * ey.x, c * y.y - sn * ey.y);
        } else {  // W[:,q] <- s W[:,p] + c e W[:,q]
          const double2 ew = cmul(e, w), ey = cmul(e, y);
          w = make_double2(sn * wq.x + c * ew.x, sn * wq.y + c * ew.y);
          y = make_double2(sn * yq.x + c * ey.x, sn * yq.y + c * ey.y);
        }
      }
    }
    if (!__any_sync(kFull, open)) break;
  }
}

// a[k] for a warp-uniform k without a dynamically indexed (local) array
__device__ __forceinline__ double pick4(const double* a, int k) {
  return k == 0 ? a[0] : k == 1 ? a[1] : k == 2 ? a[2] : a[3];
}

// X for the rare path: the columns of W whose norm s[k] is above 1e-13 of
// the largest, normalised, in order of decreasing s, each orthogonalised
// (twice, Kahan) against those before it; the others completed to an
// orthonormal basis with the standard basis vectors.  FP64, on the lane
// layout: the candidate column is held by every lane as its row's entry
// v_i, column sums run over the rows with two shuffles, and the lanes of
// column k keep the result.  Returns the lane's element of X.
__device__ __forceinline__ double2 complete4(const Lane& L, double2 w, const double* s, double smax) {
  int ord[4] = {0, 1, 2, 3};
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 3 - a; ++b)
      if (pick4(s, ord[b]) < pick4(s, ord[b + 1])) {
        const int t = ord[b];
        ord[b] = ord[b + 1];
        ord[b + 1] = t;
      }
  double2 x = make_double2(0.0, 0.0);
  unsigned done = 0u;
#pragma unroll 1
  for (int oi = 0; oi < 4; ++oi) {
    const int k = oi == 0 ? ord[0] : oi == 1 ? ord[1] : oi == 2 ? ord[2] : ord[3];
    const double sk = pick4(s, k);
    const double2 wk = shfl(w, L.at(L.i, k));  // W[i][k]
#pragma unroll 1
    for (int att = 0; att < 5; ++att) {
      double2 v;
      if (att == 0) {
        if (!(sk > 1e-13 * smax)) continue;  // numerically zero: complete instead
        const double inv = 1.0 / sk;
        v = make_double2(wk.x * inv, wk.y * inv);
      } else {
        v = make_double2(L.i == att - 1 ? 1.0 : 0.0, 0.0);
      }
#pragma unroll 1
      for (int pass = 0; pass < 2; ++pass)
#pragma unroll 1
        for (int jj = 0; jj < 4; ++jj) {
          if (!(done & (1u << jj))) continue;
          const double2 xj = shfl(x, L.at(L.i, jj));  // X[i][jj]
          const double2 t = cfma_cj(xj, v, make_double2(0.0, 0.0));
          const double2 d = make_double2(colsum4(t.x), colsum4(t.y));
          const double2 pr = cmul(d, xj);
          v.x -= pr.x;
          v.y -= pr.y;
        }
      const double nv = sqrt(colsum4(v.x * v.x + v.y * v.y));
      if (nv > 0.4) {  // among e_0..e_3 one keeps a residual of at least 1/2
        if (L.j == k) x = make_double2(v.x / nv, v.y / nv);
        done |= 1u << k;
        break;
      }
    }
  }
  return x;
}

// Stage 3 (rare): A (scaled, FP64) has a singular value below 1e-3 of the
// largest.  From the FP32 rotation y32: Y made unitary in FP64 (two
// Newton-Schulz steps), W = A Y, FP64 Jacobi to 1e-15, X = complete4, then
// u = Y X^dagger, two FP64 Newton-Schulz steps, *sig = Re Tr(A u) (the sum
// of singular values).  *y_out receives the final rotation (FP32).
static __device__ __noinline__ void polar4_rare(Lane L, double2 as, float2 y32, double2* u_out,
                                                double* sig, float2* y_out) {
  double2 y = to_d2(y32);
  for (int k = 0; k < 2; ++k) {
    const double2 P = wmm_dn(L, y, y);
    y = wmm(L, y, make_double2((L.i == L.j ? 1.5 : 0.0) - 0.5 * P.x, -0.5 * P.y));
  }
  double2 w = wmm(L, as, y);
  polish4(L, w, y, 1e-15, 12);
  const double sj = sqrt(colsum4(w.x * w.x + w.y * w.y));
  double s4[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) s4[k] = __shfl_sync(kFull, sj, L.at(0, k));
  const double smax = fmax(fmax(s4[0], s4[1]), fmax(s4[2], s4[3]));
  const double2 x = complete4(L, w, s4, smax);
  double2 u = wmm_nd(L, y, x);  // Y X^dagger
  for (int k = 0; k < 2; ++k) {
    const double2 P = wmm_dn(L, u, u);
    u = wmm(L, u, make_double2((L.i == L.j ? 1.5 : 0.0) - 0.5 * P.x, -0.5 * P.y));
  }
  const double2 M = wmm(L, as, u);
  *sig = __shfl_sync(kFull, M.x, 0) + __shfl_sync(kFull, M.x, 5) + __shfl_sync(kFull, M.x, 10) +
         __shfl_sync(kFull, M.x, 15);
  *u_out = u;
  *y_out = to_f2(y);
}

// Warp-cooperative polar update.  Every lane passes element (L.i, L.j) of A
// (FP64) and receives element (L.i, L.j) of u = argmax Re Tr(A u); *sig gets
// the sum of singular values of A.  Returns false for a non-finite A.
// `sm` is unused (kept for the callers' per-warp scratch layout).
//
// y_io (optional, one element per lane): the Jacobi starts from A Y0 with
// Y0 = *y_io instead of A (a warm start from the previous update of the same
// gate, whose right singular vectors are close), and *y_io receives the
// final rotation.  The FP64 stages fix the result whatever the start.
static __device__ __forceinline__ bool warp_polar(const Lane& L, double2 a, float2* sm, double2* u_out, double* sig,
                                                  float2* y_io = nullptr) {
  (void)sm;
  const bool fin = __all_sync(kFull, isfinite(a.x) && isfinite(a.y));
  if (!fin) return false;
  double unscale = 1.0;
  if (!pow2_scale(a, &unscale)) {  // A = 0: every unitary is optimal
    *u_out = make_double2(L.i == L.j ? 1.0 : 0.0, 0.0);
    *sig = 0.0;
    return true;
  }

  // ---- stage 1: one-sided Jacobi in FP32 (two disjoint column pairs per round)
  float2 w = make_float2((float)a.x, (float)a.y);
  float2 y = make_float2(L.i == L.j ? 1.f : 0.f, 0.f);
  if (y_io) {  // W = A Y0
    y = *y_io;
    w = wmm(L, w, y);
  }
  for (int sweep = 0; sweep < 12; ++sweep) {
    float off = 0.f;
    // kept rolled: the batched kernel runs one copy of this code per warp
    // and its instruction fetch, not the loop overhead, is what costs
#pragma unroll 1
    for (int r = 1; r <= 3; ++r) {
      const int q = L.j ^ r;
      const bool isP = L.j < q;
      const int src = L.at(L.i, q);
      const float2 wq = shfl(w, src), yq = shfl(y, src);
      float n2 = w.x * w.x + w.y * w.y;
      const float2 cp = isP ? w : wq, cq = isP ? wq : w;
      float gx = cp.x * cq.x + cp.y * cq.y;  // conj(W[i][p]) W[i][q]
      float gy = cp.x * cq.y - cp.y * cq.x;
      n2 += __shfl_xor_sync(kFull, n2, 4);
      n2 += __shfl_xor_sync(kFull, n2, 8);
      gx += __shfl_xor_sync(kFull, gx, 4);
      gx += __shfl_xor_sync(kFull, gx, 8);
      gy += __shfl_xor_sync(kFull, gy, 4);
      gy += __shfl_xor_sync(kFull, gy, 8);
      const float n2q = __shfl_sync(kFull, n2, src);
      const float al = isP ? n2 : n2q, be = isP ? n2q : n2;
      // |g| and its phase with a scaled hypot: g can be far below sqrt(FLT_MIN)
      const float gm = fmaxf(fabsf(gx), fabsf(gy));
      const float nrm = sqrtf(al) * sqrtf(be);
      // columns below 1e-6 of A's largest entry are rounding noise here:
      // leave them alone (the FP64 stage 3 resolves them)
      if (gm > 1e-7f * nrm && fmaxf(al, be) > 1e-12f && gm > 0.f) {
        const float gxs = __fdividef(gx, gm), gys = __fdividef(gy, gm);
        const float rr = rsqrtf(gxs * gxs + gys * gys);
        const float ag = gm * (gxs * gxs + gys * gys) * rr;
        off = fmaxf(off, __fdividef(ag, nrm));
        const float zeta = 0.5f * __fdividef(be - al, ag);
        const float az = fabsf(zeta);
        const float t = az > 1e18f ? __fdividef(0.5f, zeta)
                                   : copysignf(__fdividef(1.f, az + sqrtf(1.f + az * az)), zeta);
        const float c = rsqrtf(1.f + t * t), sn = c * t;
        const float2 e = make_float2(gxs * rr, -gys * rr);  // conj(g) / |g|
        if (isP) {  // W[:,p] <- c W[:,p] - s e W[:,q]
          const float2 ew = cmul(e, wq), ey = cmul(e, yq);
          w = make_float2(c * w.x - sn * ew.x, c * w.y - sn * ew.y);
          y = make_float2(c * y.x - sn * ey.x, c * y.y - sn * ey.y);
        } else {  // W[:,q] <- s W[:,p] + c e W[:,q]
          const float2 ew = cmul(e, w), ey = cmul(e, y);
          w = make_float2(sn * wq.x + c * ew.x, sn * wq.y + c * ew.y);
          y = make_float2(sn * yq.x + c * ey.x, sn * yq.y + c * ey.y);
        }
      }
    }
    if (warp_max(off) < 1e-6f) break;
  }
  float n2 = w.x * w.x + w.y * w.y;
  n2 += __shfl_xor_sync(kFull, n2, 4);
  n2 += __shfl_xor_sync(kFull, n2, 8);
  const float sj = sqrtf(n2);  // singular value of column j
  float s4[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) s4[k] = __shfl_sync(kFull, sj, L.at(0, k));
  const float smax = fmaxf(fmaxf(s4[0], s4[1]), fmaxf(s4[2], s4[3]));
  const float smin = fminf(fminf(s4[0], s4[1]), fminf(s4[2], s4[3]));
  if (!(smin > 1e-3f * smax)) {  // ---- stage 3 (rare): A close to singular
    double sg = 0.0;
    float2 yo;
    polar4_rare(L, a, y, u_out, &sg, &yo);
    *sig = sg * unscale;
    if (y_io) *y_io = yo;
    return __all_sync(kFull, isfinite(u_out->x) && isfinite(u_out->y));
  }
  const float2 x = make_float2(w.x / sj, w.y / sj);
  const float si = s4[L.i], sjj = s4[L.j];
  const float2 u0 = wmm_nd(L, y, x);  // Y X^dagger

  // ---- stage 2: FP64 refinement
  double2 u = to_d2(u0);
  double2 M = make_double2(0.0, 0.0);
  float2 D = make_float2(0.f, 0.f);
  const float den = si + sjj;  // >= 2e-3 smax here
  // the correction's first-order error is about 1e-7 smax / (s_i + s_j) of
  // its size: stop once that is below FP64 rounding of the result
  const float wtol = 3e-6f * fminf(1.f, 10.f * smin / smax);
  for (int round = 0; round < 5; ++round) {
    // Newton-Schulz: u <- u (3I - u^dagger u) / 2 = u - u (u^dagger u - I) / 2,
    // with the small correction product in FP32
    const double2 P = wmm_dn(L, u, u);
    const float2 Pm = make_float2((float)(P.x - (L.i == L.j ? 1.0 : 0.0)), (float)P.y);
    const float2 cor = wmm(L, to_f2(u), Pm);
    u = make_double2(u.x - 0.5 * (double)cor.x, u.y - 0.5 * (double)cor.y);
    // M = A u, K = M - M^dagger
    M = wmm(L, a, u);
    const double2 Md = wdag(L, M);
    const float2 K = make_float2((float)(M.x - Md.x), (float)(M.y - Md.y));
    // H W + W H = K in the eigenbasis X of H = M's Hermitian part
    const float2 Kp = wmm_dn(L, x, wmm(L, K, x));
    const float2 Wp = make_float2(Kp.x / den, Kp.y / den);
    const float2 W = wmm(L, x, wmm_nd(L, Wp, x));
    const float om = warp_max(fmaxf(fabsf(W.x), fabsf(W.y)));
    // u <- u (I - W + W^2 / 2)
    const float2 W2 = wmm(L, W, W);
    const float2 Z = make_float2(-W.x + 0.5f * W2.x, -W.y + 0.5f * W2.y);
    D = wmm(L, to_f2(u), Z);
    u = make_double2(u.x + (double)D.x, u.y + (double)D.y);
    if (om < wtol) break;
  }
  // sum of singular values = Re Tr(A u) = Re Tr(M) + Re Tr(A D) (M from the
  // last round, before D was added; Tr(A D) is small, FP32 suffices)
  const float2 Dt = shfl(D, L.at(L.j, L.i));  // D[j][i]
  float trd = (float)a.x * Dt.x - (float)a.y * Dt.y;  // Re(A[i][j] D[j][i])
#pragma unroll
  for (int h = 8; h >= 1; h >>= 1) trd += __shfl_xor_sync(kFull, trd, h);
  const double trm = __shfl_sync(kFull, M.x, 0) + __shfl_sync(kFull, M.x, 5) +
                     __shfl_sync(kFull, M.x, 10) + __shfl_sync(kFull, M.x, 15);
  *sig = (trm + (double)trd) * unscale;
  {  // final Newton-Schulz step: unitary to FP64 rounding whatever the last D
    const double2 P = wmm_dn(L, u, u);
    const float2 Pm = make_float2((float)(P.x - (L.i == L.j ? 1.0 : 0.0)), (float)P.y);
    const float2 cor = wmm(L, to_f2(u), Pm);
    u = make_double2(u.x - 0.5 * (double)cor.x, u.y - 0.5 * (double)cor.y);
  }
  *u_out = u;
  if (y_io) *y_io = y;
  return __all_sync(kFull, isfinite(u.x) && isfinite(u.y));
}

}  // namespace dev
}  // namespace qf
