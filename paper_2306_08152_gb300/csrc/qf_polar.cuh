// Warp-cooperative 4x4 gate update (OptimizeGate, Sec. III-A1, Eq. opt_u).
//
// With A = X D Y^dagger the unitary maximising Re Tr(A u) is u = Y X^dagger.
// GB300 issues an FP64 warp instruction about every 33 ns (its FP64 rate is
// 1/64 of FP32), so the update is computed in two stages on one warp
// (lane = matrix element):
//   1. a one-sided Jacobi SVD in FP32 (rotations J with A J = W having
//      orthogonal columns; Y ~ J, X ~ W's normalised columns, D ~ their
//      norms), which costs no FP64 work;
//   2. FP64 refinement: Newton-Schulz re-unitarisation of u0 = Y X^dagger,
//      M = A u (Hermitian positive semi-definite at the optimum), and the
//      correction u <- u (I - W + W^2/2) where W solves H W + W H = M - M^dagger
//      in X's eigenbasis (W_ij = K'_ij / (d_i + d_j)).  One round turns the
//      FP32 error e into O(e^2); rounds repeat while the correction is large.
// The sum of singular values (the new Re Tr(E u)) is returned with it.

#pragma once

#include "qf_device.cuh"

namespace qf {
namespace dev {

// Rare path: some singular value is (numerically) zero, so X needs an
// orthonormal completion.  Lane 0 runs modified Gram-Schmidt over the
// columns of W in order of decreasing singular value, falling back to
// standard basis vectors; `sm` is 32 float2 of shared scratch for this warp.
static __device__ __noinline__ float2 complete_left_vectors(const Lane& L, float2 w, const float* s4, float smax,
                                        float2* sm) {
  if (L.l < 16) sm[L.l] = w;
  __syncwarp();
  if (L.l == 0) {
    int ord[4] = {0, 1, 2, 3};
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 3 - a; ++b)
        if (s4[ord[b]] < s4[ord[b + 1]]) {
          int t = ord[b];
          ord[b] = ord[b + 1];
          ord[b + 1] = t;
        }
    float2 X[16];
    bool done[4] = {false, false, false, false};
    for (int e = 0; e < 16; ++e) X[e] = make_float2(0.f, 0.f);
    for (int oi = 0; oi < 4; ++oi) {
      const int k = ord[oi];
      for (int att = 0; att < 5; ++att) {
        float2 v[4];
        if (att == 0) {
          if (!(s4[k] > 1e-5f * smax)) continue;  // noise column: complete instead
          for (int i = 0; i < 4; ++i)
            v[i] = make_float2(sm[i * 4 + k].x / s4[k], sm[i * 4 + k].y / s4[k]);
        } else {
          for (int i = 0; i < 4; ++i) v[i] = make_float2(i == att - 1 ? 1.f : 0.f, 0.f);
        }
        for (int jj = 0; jj < 4; ++jj) {
          if (!done[jj]) continue;
          float2 d = make_float2(0.f, 0.f);
          for (int i = 0; i < 4; ++i) d = cfma_cj(X[i * 4 + jj], v[i], d);
          for (int i = 0; i < 4; ++i) {
            float2 pr = cmul(d, X[i * 4 + jj]);
            v[i].x -= pr.x;
            v[i].y -= pr.y;
          }
        }
        float nv = 0.f;
        for (int i = 0; i < 4; ++i) nv += v[i].x * v[i].x + v[i].y * v[i].y;
        nv = sqrtf(nv);
        if (nv > 0.4f) {  // among e_0..e_3 one keeps a residual of at least 1/2
          for (int i = 0; i < 4; ++i) X[i * 4 + k] = make_float2(v[i].x / nv, v[i].y / nv);
          done[k] = true;
          break;
        }
      }
    }
    for (int e = 0; e < 16; ++e) sm[16 + e] = X[e];
  }
  __syncwarp();
  return sm[16 + (L.l & 15)];
}

// Warp-cooperative polar update.  Every lane passes element (L.i, L.j) of A
// (FP64) and receives element (L.i, L.j) of u = argmax Re Tr(A u); *sig gets
// the sum of singular values of A.  Returns false for a non-finite A.
//
// y_io (optional, one element per lane): the Jacobi starts from A Y0 with
// Y0 = *y_io instead of A (a warm start from the previous update of the same
// gate, whose right singular vectors are close), and *y_io receives the
// final rotation.  The FP64 refinement fixes the result whatever the start.
static __device__ __forceinline__ bool warp_polar(const Lane& L, double2 a, float2* sm, double2* u_out, double* sig,
                                                  float2* y_io = nullptr) {
  const bool fin = __all_sync(kFull, isfinite(a.x) && isfinite(a.y));
  if (!fin) return false;
  const float amax = warp_max(fmaxf(fabsf((float)a.x), fabsf((float)a.y)));
  if (amax == 0.f) {  // A = 0: every unitary is optimal
    *u_out = make_double2(L.i == L.j ? 1.0 : 0.0, 0.0);
    *sig = 0.0;
    return true;
  }
  const float sc = 1.f / amax;  // FP32 stage works on A / max|A_ij|

  // ---- stage 1: one-sided Jacobi in FP32 (two disjoint column pairs per round)
  float2 w = make_float2((float)a.x * sc, (float)a.y * sc);
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
      // columns below 1e-6 of A's largest entry are rounding noise: leave
      // them alone (their directions are fixed by the completion below)
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
  const float sj = sqrtf(n2);  // singular value of column j (scaled)
  float s4[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) s4[k] = __shfl_sync(kFull, sj, L.at(0, k));
  const float smax = fmaxf(fmaxf(s4[0], s4[1]), fmaxf(s4[2], s4[3]));
  const float smin = fminf(fminf(s4[0], s4[1]), fminf(s4[2], s4[3]));
  float2 x;
  if (smin > 1e-3f * smax) {
    x = make_float2(w.x / sj, w.y / sj);
  } else {
    x = complete_left_vectors(L, w, s4, smax, sm);
  }
  const float si = s4[L.i], sjj = s4[L.j];
  const float2 u0 = wmm_nd(L, y, x);  // Y X^dagger

  // ---- stage 2: FP64 refinement
  double2 u = to_d2(u0);
  double2 M = make_double2(0.0, 0.0);
  float2 D = make_float2(0.f, 0.f);
  const float den = si + sjj;
  const bool use = den > 1e-6f * smax;
  for (int round = 0; round < 4; ++round) {
    // Newton-Schulz: u <- u (3I - u^dagger u) / 2 = u - u (u^dagger u - I) / 2,
    // with the small correction product in FP32
    const double2 P = wmm_dn(L, u, u);
    const float2 Pm = make_float2((float)(P.x - (L.i == L.j ? 1.0 : 0.0)), (float)P.y);
    const float2 cor = wmm(L, to_f2(u), Pm);
    u = make_double2(u.x - 0.5 * (double)cor.x, u.y - 0.5 * (double)cor.y);
    // M = A u, K = M - M^dagger
    M = wmm(L, a, u);
    const double2 Md = wdag(L, M);
    const float2 K = make_float2((float)(M.x - Md.x) * sc, (float)(M.y - Md.y) * sc);
    // H W + W H = K in the eigenbasis X of H = M's Hermitian part
    const float2 Kp = wmm_dn(L, x, wmm(L, K, x));
    const float2 Wp = use ? make_float2(Kp.x / den, Kp.y / den) : make_float2(0.f, 0.f);
    const float2 W = wmm(L, x, wmm_nd(L, Wp, x));
    const float om = warp_max(fmaxf(fabsf(W.x), fabsf(W.y)));
    // u <- u (I - W + W^2 / 2)
    const float2 W2 = wmm(L, W, W);
    const float2 Z = make_float2(-W.x + 0.5f * W2.x, -W.y + 0.5f * W2.y);
    D = wmm(L, to_f2(u), Z);
    u = make_double2(u.x + (double)D.x, u.y + (double)D.y);
    if (om < 3e-6f) break;
  }
  // sum of singular values = Re Tr(A u) = Re Tr(M) + Re Tr(A D) (M from the
  // last round, before D was added; Tr(A D) is small, FP32 suffices)
  const float2 Dt = shfl(D, L.at(L.j, L.i));  // D[j][i]
  float trd = (float)a.x * Dt.x - (float)a.y * Dt.y;  // Re(A[i][j] D[j][i])
#pragma unroll
  for (int h = 8; h >= 1; h >>= 1) trd += __shfl_xor_sync(kFull, trd, h);
  const double trm = __shfl_sync(kFull, M.x, 0) + __shfl_sync(kFull, M.x, 5) +
                     __shfl_sync(kFull, M.x, 10) + __shfl_sync(kFull, M.x, 15);
  *sig = trm + (double)trd;
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
