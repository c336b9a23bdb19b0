// Environment and gate-update kernels of the QFactor sweep for sm_103a.
//
// CalcEnvMat (Alg. 1): the environment of gate k on (a, b) needs only the
// partial trace P = Tr_rest(T) over the 2^(n+2) "band" entries whose row and
// column agree outside (a, b).  It is taken from the tensor *before* gate k
// is removed, so E = P u^dagger (gate on the tensor's right) or u^dagger P
// (gate on its left), and the removal is fused into the following pass.
//
// OptimizeGate (Sec. III-A1, Eq. opt_u) runs on one warp of the last CTA
// (warp_polar, qf_polar.cuh).

#include "qf_device.cuh"
#include "qf_internal.h"
#include "qf_polar.cuh"

namespace qf {
namespace {

using namespace dev;

constexpr int kEnvThreads = 256;

// ------------------------------------------- parameterised gate updates
//
// Sec. III-A ("Specializing gate sets"): for a parameterised gate G(theta)
// the update is theta' = argmax Re Tr(A G(theta)) (A = E, or the damped
// (1 - beta) E + beta u^dagger), in closed form.  With A the 4x4 matrix of
// the gate's slot and, for one-qubit kinds, A1[x][y] = sum_r A[2x+r][2y+r]:
//   Rz:  Re Tr = Re A1[0][0] + Re(e^{i theta} z), z = A1[1][1];
//   GPI: Re Tr = Re(e^{i phi} z), z = A1[0][1] + conj A1[1][0];
//   MS:  sqrt 2 Re Tr = Re Tr A + Re(e^{i a} z_a) + Re(e^{i b} z_b),
//        a = phi0 + phi1, b = phi0 - phi1,
//        z_a = -i (A[0][3] - conj A[3][0]), z_b = -i (A[1][2] - conj A[2][1]);
// each angle is -arg of its z (kept where z = 0: every angle is optimal).

// Entry e = 4 i + j of the 4x4 slot matrix of gate kind with parameters
// (p0, p1); one-qubit kinds are G (x) I.
__device__ __forceinline__ double2 param_gate_entry(int kind, double p0, double p1, int e) {
  const int i = e >> 2, j = e & 3;
  if (kind == kGateMs) {
    const double h = 0.70710678118654752440;  // 1 / sqrt 2
    if (i == j) return make_double2(h, 0.0);
    if (i + j != 3) return make_double2(0.0, 0.0);
    // -i e^{i t} = (sin t, -cos t) with t = -a, -b, b, a for i = 0, 1, 2, 3
    const double t = (i == 0) ? -(p0 + p1) : (i == 1) ? -(p0 - p1) : (i == 2) ? (p0 - p1) : (p0 + p1);
    double sn, cs;
    sincos(t, &sn, &cs);
    return make_double2(h * sn, -h * cs);
  }
  if ((i & 1) != (j & 1)) return make_double2(0.0, 0.0);
  const int x = i >> 1, y = j >> 1;
  double sn, cs;
  if (kind == kGateRz) {
    if (x != y) return make_double2(0.0, 0.0);
    if (x == 0) return make_double2(1.0, 0.0);
    sincos(p0, &sn, &cs);
    return make_double2(cs, sn);
  }
  // GPI: [[0, e^{-i phi}], [e^{i phi}, 0]]
  if (x == y) return make_double2(0.0, 0.0);
  sincos(p0, &sn, &cs);
  return make_double2(cs, x == 0 ? -sn : sn);
}

// The warp's closed-form update: lane e (mod 16) holds A[e]; returns the new
// slot matrix's entry e and the maximum in *sg; prm (2 doubles) holds the
// old parameters and receives the new ones.  false (prm untouched) if the
// maximiser is not finite.
__device__ __noinline__ bool param_update(int kind, double2 A, double* prm, double2* un, double* sg) {
  const int l = threadIdx.x & 31, e = l & 15;
  double2 a[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) a[j] = shfl(A, j);
  const double o0 = prm[0], o1 = prm[1];
  __syncwarp();
  double p0 = o0, p1 = o1, best;
  if (kind == kGateMs) {
    const double2 wa = make_double2(a[3].x - a[12].x, a[3].y + a[12].y);  // A03 - conj A30
    const double2 wb = make_double2(a[6].x - a[9].x, a[6].y + a[9].y);    // A12 - conj A21
    const double2 za = make_double2(wa.y, -wa.x), zb = make_double2(wb.y, -wb.x);  // -i w
    double ta = o0 + o1, tb = o0 - o1;
    if (za.x != 0.0 || za.y != 0.0) ta = atan2(-za.y, za.x);
    if (zb.x != 0.0 || zb.y != 0.0) tb = atan2(-zb.y, zb.x);
    p0 = 0.5 * (ta + tb);
    p1 = 0.5 * (ta - tb);
    best = (a[0].x + a[5].x + a[10].x + a[15].x + hypot(za.x, za.y) + hypot(zb.x, zb.y)) *
           0.70710678118654752440;
  } else if (kind == kGateRz) {
    const double2 z = make_double2(a[10].x + a[15].x, a[10].y + a[15].y);
    if (z.x != 0.0 || z.y != 0.0) p0 = atan2(-z.y, z.x);
    best = a[0].x + a[5].x + hypot(z.x, z.y);
  } else {  // GPI
    const double2 z = make_double2(a[2].x + a[7].x + a[8].x + a[13].x, a[2].y + a[7].y - a[8].y - a[13].y);
    if (z.x != 0.0 || z.y != 0.0) p0 = atan2(-z.y, z.x);
    best = hypot(z.x, z.y);
  }
  if (!isfinite(p0) || !isfinite(p1)) return false;
  if (l == 0) {
    prm[0] = p0;
    prm[1] = p1;
  }
  *un = param_gate_entry(kind, p0, p1, e);
  *sg = best;
  return true;
}

// ----------------------------------------------------- environment kernel
//
// Grid (B, S): CTA b of start s sums the band entries of rests
// [b*chunk, (b+1)*chunk) and writes its 32 partial sums; the last CTA of the
// start to finish (atomic ticket, no waiting) adds the B partials in a fixed
// order, so results do not depend on timing, and runs the gate update.

// Look-ahead geometry: the environment of a gate on (pa, pb) taken from a
// tensor that still lacks the pending update (L1, R1) of the preceding gate
// on the disjoint pair (pa1, pb1).
struct LookGeom {
  int q[4];                 // the four gate bit positions, ascending
  int pa1, pb1;             // bit positions of the pending update's pair
  const double2 *L1, *R1;   // its pass operators, start stride `stride`
  long long stride;
};

template <typename R, bool kLook>
__global__ void __launch_bounds__(kEnvThreads) env_kernel(
    const typename Cplx<R>::T* __restrict__ T, int n, int plo, int phi, int pa, int pb,
    int mode, double2* __restrict__ gates_k, long long gstride, double beta,
    double2* __restrict__ LR, double2* __restrict__ out, long long out_stride,
    double* __restrict__ sigma_out, int* __restrict__ status, double* __restrict__ part,
    unsigned* __restrict__ counters, LookGeom lg, int kind, double* __restrict__ prm,
    long long prm_stride) {
  using CT = typename Cplx<R>::T;   // tensor entry
  using Ar = typename Acc<R>::T;    // accumulation real (FP32 for complex64, else FP64)
  using AT = typename Cplx<Ar>::T;
  __shared__ double red[32 * (kEnvThreads / 32)];
  __shared__ float2 scratch[32];
  __shared__ AT sM[16];
  __shared__ bool is_last;
  const int s = blockIdx.y, B = gridDim.x, b = blockIdx.x;
  const unsigned N = 1u << n;
  const unsigned nr = kLook ? N : 1u << (n - 2);
  const unsigned chunk = (nr + B - 1) / B;
  const unsigned r_beg = b * chunk;
  const unsigned r_end = min(nr, r_beg + chunk);
  const CT* Ts = T + (size_t)s * N * N;
  const unsigned o1 = 1u << pb, o2 = 1u << pa;
  const unsigned off[4] = {0u, o1, o2, o1 | o2};

  // band partial sums (FP32 accumulation for complex64, FP64 otherwise)
  Ar v[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = Ar(0);
  if (!kLook) {
    for (unsigned r = r_beg + threadIdx.x; r < r_end; r += blockDim.x) {
      const unsigned d = dep2(r, plo, phi);
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const unsigned rb = (d | off[x]) * N + d;
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const AT e = to_acc(Ts[rb | off[y]]);
          v[2 * (x * 4 + y)] += e.x;
          v[2 * (x * 4 + y) + 1] += e.y;
        }
      }
    }
  } else {
    // After the pending update T' = (L1 on pair 1) T (R1 on pair 1), so
    //   P[x][y] = sum_rest sum_i T'[(rest,i,x),(rest,i,y)]
    //           = sum_rest sum_{i,j} M[j][i] T[(rest,i,x),(rest,j,y)],
    // M = R1 L1: item (rest, i, j) reads 16 entries and weights them by M[j][i].
    if (threadIdx.x < 16) {
      const double2* l1 = lg.L1 + s * lg.stride;
      const double2* r1 = lg.R1 + s * lg.stride;
      const int r = threadIdx.x >> 2, c = threadIdx.x & 3;
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < 4; ++k) acc = cfma(r1[r * 4 + k], l1[k * 4 + c], acc);
      sM[threadIdx.x] = cmake(acc, Ar(0));
    }
    __syncthreads();
    const unsigned p1 = 1u << lg.pb1, p2 = 1u << lg.pa1;
    const unsigned off1[4] = {0u, p1, p2, p1 | p2};
    for (unsigned r = r_beg + threadIdx.x; r < r_end; r += blockDim.x) {
      const unsigned i = (r >> 2) & 3u, j = r & 3u;
      const unsigned d = dep1(dep1(dep1(dep1(r >> 4, lg.q[0]), lg.q[1]), lg.q[2]), lg.q[3]);
      const AT w = sM[j * 4 + i];
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const unsigned rb = (d | off1[i] | off[x]) * N + (d | off1[j]);
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const AT e = to_acc(Ts[rb | off[y]]);
          v[2 * (x * 4 + y)] += w.x * e.x - w.y * e.y;
          v[2 * (x * 4 + y) + 1] += w.x * e.y + w.y * e.x;
        }
      }
    }
  }
  // warp reduce-scatter: after the step with offset h, lanes with bit h set
  // keep the upper half; lane l ends with value l
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const Ar keep = up ? v[i + h] : v[i];
      const Ar send = up ? v[i] : v[i + h];
      v[i] = keep + __shfl_xor_sync(kFull, send, h);
    }
  }
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  red[wid * 32 + lane] = (double)v[0];
  __syncthreads();
  if (threadIdx.x < 32) {
    double acc = 0.0;
    for (int k = 0; k < nw; ++k) acc += red[k * 32 + threadIdx.x];
    part[((size_t)s * B + b) * 32 + threadIdx.x] = acc;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned ticket = atomicAdd(&counters[s], 1u);
    is_last = (ticket == (unsigned)B - 1u);
  }
  __syncthreads();
  if (!is_last || threadIdx.x >= 32) return;
  __threadfence();

  // the last CTA: fixed-order sum of the B partials, then the update
  double acc = 0.0;
  for (int k = 0; k < B; ++k) acc += __ldcg(&part[((size_t)s * B + k) * 32 + threadIdx.x]);
  if (threadIdx.x == 0) counters[s] = 0u;  // ready for the next launch
  const Lane L;
  const int e = L.l & 15;
  const double2 P = make_double2(__shfl_sync(kFull, acc, 2 * e), __shfl_sync(kFull, acc, 2 * e + 1));
  if (mode == kTraceOnly) {
    if (L.l < 16) out[s * out_stride + e] = P;
    return;
  }
  const double2 u = gates_k[s * gstride + e];
  const double2 ud = wdag(L, u);
  // E = P u^dagger (gate on the right) or u^dagger P (gate on the left)
  const double2 E = (mode == kForward) ? wmm_dn(L, u, P) : wmm_nd(L, P, u);
  if (out && L.l < 16) out[s * out_stride + e] = E;
  double2* lr = LR + (size_t)s * 32;
  if (mode == kEnvOnly) {
    if (L.l < 16) {
      lr[e] = u;
      lr[16 + e] = ud;
    }
    return;
  }
  double2 A = E;
  if (beta != 0.0)
    A = make_double2((1.0 - beta) * E.x + beta * ud.x, (1.0 - beta) * E.y + beta * ud.y);
  double2 un;
  double sg = 0.0;
  const bool ok = kind == kGateGeneral ? warp_polar(L, A, scratch, &un, &sg)
                                       : param_update(kind, A, prm + s * prm_stride, &un, &sg);
  if (!ok) {
    if (L.l == 0) atomicCAS(status, 0, -4);
    un = u;  // keep the old gate: the tensor stays consistent
    sg = 0.0;
  }
  if (L.l < 16) {
    gates_k[s * gstride + e] = un;
    if (mode == kBackward) {
      lr[e] = un;
      lr[16 + e] = ud;
    } else {
      lr[e] = ud;
      lr[16 + e] = un;
    }
  }
  if (sigma_out && L.l == 0) sigma_out[s] = sg;
}

// The slot matrices of the parameterised gates from their parameters, one
// thread per entry.
__global__ void param_gates_kernel(double2* __restrict__ gates, long long gsz, const int2* __restrict__ tab,
                                   const double* __restrict__ params, long long prm_stride, int p, int S) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)S * p * 16) return;
  const int e = (int)(idx & 15);
  const long long sg = idx >> 4;
  const int g = (int)(sg % p), s = (int)(sg / p);
  const int2 t = tab[g];
  if (t.x == kGateGeneral) return;
  const double* pr = params + s * prm_stride + 2 * g;
  gates[s * gsz + t.y + e] = param_gate_entry(t.x, pr[0], pr[1], e);
}

// One warp per matrix.
__global__ void __launch_bounds__(128) optimize_kernel(const double2* __restrict__ E,
                                                       const double2* __restrict__ u_old,
                                                       double beta, int count,
                                                       double2* __restrict__ u_out,
                                                       double* __restrict__ sigma_out) {
  __shared__ float2 scratch[4][32];
  const int wid = threadIdx.x >> 5;
  const int m = blockIdx.x * 4 + wid;
  if (m >= count) return;  // whole warps leave together
  const Lane L;
  const int e = L.l & 15;
  double2 A = E[(size_t)m * 16 + e];
  if (beta != 0.0) {
    const double2 ud = wdag(L, u_old[(size_t)m * 16 + e]);
    A = make_double2((1.0 - beta) * A.x + beta * ud.x, (1.0 - beta) * A.y + beta * ud.y);
  }
  double2 un;
  double sg;
  if (!warp_polar(L, A, scratch[wid], &un, &sg)) {
    un = make_double2(NAN, NAN);
    sg = NAN;
  }
  if (L.l < 16) u_out[(size_t)m * 16 + e] = un;
  if (sigma_out && L.l == 0) sigma_out[m] = sg;
}

// grad[s][k] = -(t_s / (N |t_s|)) E[s][k]^dagger, in place, one thread per
// 4x4 matrix: the gradient of cost = 1 - |t|/N, t = Tr(V^dagger C) = Tr(E_k u_k),
// in the d/dRe + i d/dIm convention.  |t| = 0 gives a zero gradient.
__global__ void grad_from_env_kernel(double2* __restrict__ env, const double2* __restrict__ tr,
                                     double inv_n, int S, int p) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= S * p) return;
  const int s = m / p;
  const double2 t = tr[s];
  const double at = sqrt(t.x * t.x + t.y * t.y);
  const double2 f = at > 0.0 ? make_double2(-t.x * inv_n / at, -t.y * inv_n / at)
                             : make_double2(0.0, 0.0);
  double2 e[16];
  double2* E = env + (size_t)m * 16;
#pragma unroll
  for (int i = 0; i < 16; ++i) e[i] = E[i];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) E[i * 4 + j] = cmul(f, cconj(e[j * 4 + i]));
}

// The same for a circuit of 2-, 3- and 4-qubit gates: CTA (k, s) turns the
// d x d environment of gate k of set s (desc[k] = (qubits, entry offset),
// d = 2^qubits, set stride gsz) into -(t/(N|t|)) E^dagger in place; thread
// e owns the unordered pair of entries (i, j), (j, i) with i <= j.
__global__ void grad_from_env_k_kernel(double2* __restrict__ env, const double2* __restrict__ tr,
                                       double inv_n, long long gsz, const int2* __restrict__ desc) {
  const int k = blockIdx.x, s = blockIdx.y;
  const int2 dk = desc[k];
  const int d = 1 << dk.x;
  const double2 t = tr[s];
  const double at = sqrt(t.x * t.x + t.y * t.y);
  const double2 f = at > 0.0 ? make_double2(-t.x * inv_n / at, -t.y * inv_n / at)
                             : make_double2(0.0, 0.0);
  double2* E = env + (size_t)s * gsz + dk.y;
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
    const int i = e / d, j = e % d;
    if (i > j) continue;
    const double2 a = E[i * d + j], b = E[j * d + i];
    E[i * d + j] = cmul(f, cconj(b));
    E[j * d + i] = cmul(f, cconj(a));
  }
}

// Periodic re-unitarisation of gates in FP64 (reset_iter, Sec. III-A2): three
// Newton-Schulz steps u <- u (3I - u^dagger u) / 2 per gate, one warp per gate.
// Each step squares the deviation from unitarity; on gates that are already
// unitary to FP64 rounding they change nothing beyond rounding.
__global__ void __launch_bounds__(128) reunitarize_kernel(double2* __restrict__ gates, int count) {
  const int m = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (m >= count) return;  // whole warps leave together
  const Lane L;
  const int e = L.l & 15;
  double2 u = gates[(size_t)m * 16 + e];
  for (int step = 0; step < 3; ++step) {
    const double2 P = wmm_dn(L, u, u);
    const double2 Q = make_double2((L.i == L.j ? 1.5 : 0.0) - 0.5 * P.x, -0.5 * P.y);
    u = wmm(L, u, Q);
  }
  if (L.l < 16) gates[(size_t)m * 16 + e] = u;
}

}  // namespace

// ================================================================ launchers

cudaError_t launch_reunitarize(double2* gates, int count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  reunitarize_kernel<<<(count + 3) / 4, 128, 0, st>>>(gates, count);
  return cudaGetLastError();
}

cudaError_t launch_grad_from_env(double2* env, const double2* tr, int n, int S, int p,
                                 cudaStream_t st) {
  const int count = S * p;
  grad_from_env_kernel<<<(count + 127) / 128, 128, 0, st>>>(env, tr, 1.0 / (double)(1 << n), S, p);
  return cudaGetLastError();
}

cudaError_t launch_grad_from_env_k(double2* env, const double2* tr, int n, int S, long long gsz,
                                   const int2* desc, int p, cudaStream_t st) {
  if (S * p <= 0) return cudaSuccess;
  grad_from_env_k_kernel<<<dim3(p, S), 128, 0, st>>>(env, tr, 1.0 / (double)(1 << n), gsz, desc);
  return cudaGetLastError();
}

cudaError_t launch_update_lookahead(const void* T, int n, int S, int a1, int b1, const double2* L1,
                                    const double2* R1, long long stride1, int a, int b, double2* gates_k, long long gstride, int mode,
                                    double beta, double2* LR, double2* out, long long out_stride,
                                    double* sigma_out, int* status, double* part,
                                    unsigned* counters, int prec, cudaStream_t st) {
  const int pa = qubit_bit(n, a), pb = qubit_bit(n, b);
  LookGeom lg;
  lg.pa1 = qubit_bit(n, a1);
  lg.pb1 = qubit_bit(n, b1);
  lg.L1 = L1;
  lg.R1 = R1;
  lg.stride = stride1;
  int q[4] = {pa, pb, lg.pa1, lg.pb1};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 3 - i; ++j)
      if (q[j] > q[j + 1]) {
        const int t = q[j];
        q[j] = q[j + 1];
        q[j + 1] = t;
      }
  for (int i = 0; i < 4; ++i) lg.q[i] = q[i];
  dim3 grid(env_ctas(n), S);
  if (prec == 0)
    env_kernel<double, true><<<grid, kEnvThreads, 0, st>>>(
        (const double2*)T, n, 0, 0, pa, pb, mode, gates_k, gstride, beta, LR, out, out_stride,
        sigma_out, status, part, counters, lg, kGateGeneral, nullptr, 0);
  else if (prec == 2)
    env_kernel<DF, true><<<grid, kEnvThreads, 0, st>>>(
        (const dfc*)T, n, 0, 0, pa, pb, mode, gates_k, gstride, beta, LR, out, out_stride,
        sigma_out, status, part, counters, lg, kGateGeneral, nullptr, 0);
  else
    env_kernel<float, true><<<grid, kEnvThreads, 0, st>>>(
        (const float2*)T, n, 0, 0, pa, pb, mode, gates_k, gstride, beta, LR, out, out_stride,
        sigma_out, status, part, counters, lg, kGateGeneral, nullptr, 0);
  return cudaGetLastError();
}

int env_ctas(int n) {
  const unsigned rests = 1u << (n - 2);
  int b = (int)(rests / 256u);
  if (b < 1) b = 1;
  if (b > 32) b = 32;
  return b;
}

cudaError_t launch_update(const void* T, int n, int S, int a, int b, double2* gates_k,
                          long long gstride, int mode, double beta, double2* LR, double2* out,
                          long long out_stride, double* sigma_out, int* status, double* part,
                          unsigned* counters, int prec, cudaStream_t st, int kind, double* prm,
                          long long prm_stride) {
  const int pa = qubit_bit(n, a), pb = qubit_bit(n, b);
  const int plo = pa < pb ? pa : pb, phi = pa < pb ? pb : pa;
  dim3 grid(env_ctas(n), S);
  if (prec == 0)
    env_kernel<double, false><<<grid, kEnvThreads, 0, st>>>(
        (const double2*)T, n, plo, phi, pa, pb, mode, gates_k, gstride, beta, LR, out, out_stride,
        sigma_out, status, part, counters, LookGeom{}, kind, prm, prm_stride);
  else if (prec == 2)
    env_kernel<DF, false><<<grid, kEnvThreads, 0, st>>>(
        (const dfc*)T, n, plo, phi, pa, pb, mode, gates_k, gstride, beta, LR, out, out_stride,
        sigma_out, status, part, counters, LookGeom{}, kind, prm, prm_stride);
  else
    env_kernel<float, false><<<grid, kEnvThreads, 0, st>>>(
        (const float2*)T, n, plo, phi, pa, pb, mode, gates_k, gstride, beta, LR, out, out_stride,
        sigma_out, status, part, counters, LookGeom{}, kind, prm, prm_stride);
  return cudaGetLastError();
}

cudaError_t launch_param_gates(double2* gates, long long gsz, const int2* tab, const double* params,
                               long long prm_stride, int p, int S, cudaStream_t st) {
  const long long count = (long long)S * p * 16;
  if (count <= 0) return cudaSuccess;
  param_gates_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(gates, gsz, tab, params, prm_stride,
                                                                      p, S);
  return cudaGetLastError();
}

cudaError_t launch_optimize(const double2* E, const double2* u_old, double beta, int count,
                            double2* u_out, double* sigma_out, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  optimize_kernel<<<(count + 3) / 4, 128, 0, st>>>(E, u_old, beta, count, u_out, sigma_out);
  return cudaGetLastError();
}

}  // namespace qf
