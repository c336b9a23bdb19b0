// QFactor sweep kernels for sm_103a.
//
// Layout: a circuit tensor T is N x N row-major (N = 2^n), interleaved
// complex (float2 for complex64, double2 for complex128); start s occupies
// entries [s*N*N, (s+1)*N*N).  Qubit q is bit n-1-q of a row index and of a
// column index.  A gate on (a, b) therefore touches row bits {pa, pb} and
// column bits {pa, pb} with pa = n-1-a, pb = n-1-b, and its local index is
// x = 2*bit_pa + bit_pb.
//
// Every 16 entries that share all non-gate row and column bits form one 4x4
// block B (rows x = local row index, columns y = local column index).  The
// fused update of Alg. 1 (remove the old gate on one side, apply the new one
// on the other) is B <- L B R for every block: one read and one write of T.
//
// The 4x4 work is not a dense contraction worth tensor cores (32 complex
// FMAs per 16 entries); the pass is bound by HBM for complex64 and by the
// FP64 pipe for complex128.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "qf_internal.h"

namespace qf {
namespace {

// ---------------------------------------------------------------- complex

template <typename R> struct Cplx;
template <> struct Cplx<float> { typedef float2 T; };
template <> struct Cplx<double> { typedef double2 T; };

__device__ __forceinline__ float2 cmake(double2 v, float) {
  return make_float2((float)v.x, (float)v.y);
}
__device__ __forceinline__ double2 cmake(double2 v, double) { return v; }

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
__device__ __forceinline__ float2 czero(float) { return make_float2(0.f, 0.f); }
__device__ __forceinline__ double2 czero(double) { return make_double2(0.0, 0.0); }

__device__ __forceinline__ double2 dmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 dconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 dadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 dscale(double s, double2 a) {
  return make_double2(s * a.x, s * a.y);
}
__device__ __forceinline__ double dabs2(double2 a) { return a.x * a.x + a.y * a.y; }

__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }

// Insert zero bits at positions lo < hi (the gate's two bit positions) into
// the (n-2)-bit "rest" index x.
__device__ __forceinline__ unsigned dep2(unsigned x, int lo, int hi) {
  x = ((x >> lo) << (lo + 1)) | (x & ((1u << lo) - 1u));
  x = ((x >> hi) << (hi + 1)) | (x & ((1u << hi) - 1u));
  return x;
}

// ------------------------------------------------------ InitCircuitTensor
//
// T_s <- V^dagger: conjugate transpose through a 32 x 33 shared tile so that
// both the read of V and the write of T are coalesced.

template <typename R>
__global__ void __launch_bounds__(256) conj_transpose_kernel(
    const double2* __restrict__ V, typename Cplx<R>::T* __restrict__ T, int N) {
  __shared__ double2 tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  const int s = blockIdx.z;
  // read V rows by..by+31, columns bx..bx+31
  for (int j = threadIdx.y; j < 32; j += 8) {
    int r = by + j, c = bx + threadIdx.x;
    if (r < N && c < N) tile[j][threadIdx.x] = V[(size_t)r * N + c];
  }
  __syncthreads();
  typename Cplx<R>::T* Ts = T + (size_t)s * N * N;
  // write T rows bx..bx+31 (= V columns), columns by..by+31
  for (int j = threadIdx.y; j < 32; j += 8) {
    int r = bx + j, c = by + threadIdx.x;
    if (r < N && c < N) {
      double2 v = tile[threadIdx.x][j];
      v.y = -v.y;
      Ts[(size_t)r * N + c] = cmake(v, R());
    }
  }
}

// ------------------------------------------------------------- the pass
//
// One thread owns one 4x4 block per loop trip.  Consecutive threads take
// consecutive values of the column rest index, so each of the 16 loads of a
// warp reads 32 entries spaced by the rest-index stride: contiguous when the
// gate's column bits are above bit 4, and sector-shared with the partner
// loads of the same thread otherwise.

constexpr int kPassThreads = 256;

template <typename R, bool HL, bool HR>
__global__ void __launch_bounds__(kPassThreads, (sizeof(R) == 4 ? 3 : 1))
pass_kernel(typename Cplx<R>::T* __restrict__ T, int n, int plo, int phi,
            int pa, int pb, const double2* __restrict__ L, long long Ls,
            const double2* __restrict__ Rm, long long Rs) {
  typedef typename Cplx<R>::T C;
  __shared__ C sL[16], sR[16];
  const int s = blockIdx.y;
  if (threadIdx.x < 16) {
    if (HL) sL[threadIdx.x] = cmake(L[s * Ls + threadIdx.x], R());
    if (HR) sR[threadIdx.x] = cmake(Rm[s * Rs + threadIdx.x], R());
  }
  __syncthreads();

  const unsigned N = 1u << n;
  const int lnc = n - 2;
  const unsigned cmask = (1u << lnc) - 1u;
  const unsigned nblk = 1u << (2 * lnc);
  C* __restrict__ Ts = T + (size_t)s * N * N;
  const unsigned o1 = 1u << pb, o2 = 1u << pa;
  const unsigned off[4] = {0u, o1, o2, o1 | o2};

  for (unsigned blk = blockIdx.x * blockDim.x + threadIdx.x; blk < nblk;
       blk += gridDim.x * blockDim.x) {
    const unsigned r0 = dep2(blk >> lnc, plo, phi);
    const unsigned c0 = dep2(blk & cmask, plo, phi);
    C bm[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const unsigned rb = (r0 | off[x]) * N;
#pragma unroll
      for (int y = 0; y < 4; ++y) bm[x][y] = Ts[rb + (c0 | off[y])];
    }
    if (HR) {  // B <- B R, one row at a time
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        C t[4];
#pragma unroll
        for (int y = 0; y < 4; ++y) t[y] = czero(R());
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int y = 0; y < 4; ++y) t[y] = cfma(bm[x][k], sR[k * 4 + y], t[y]);
#pragma unroll
        for (int y = 0; y < 4; ++y) bm[x][y] = t[y];
      }
    }
    if (HL) {  // B <- L B, one column at a time
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        C t[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          C acc = czero(R());
#pragma unroll
          for (int k = 0; k < 4; ++k) acc = cfma(sL[x * 4 + k], bm[k][y], acc);
          t[x] = acc;
        }
#pragma unroll
        for (int x = 0; x < 4; ++x) bm[x][y] = t[x];
      }
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const unsigned rb = (r0 | off[x]) * N;
#pragma unroll
      for (int y = 0; y < 4; ++y) Ts[rb + (c0 | off[y])] = bm[x][y];
    }
  }
}

// ------------------------------------------------------ band partial trace
//
// P[x][y] = sum_r T[(d(r)|off x), (d(r)|off y)], r over the 2^(n-2) rest
// indices: only the 2^(n+2) "band" entries are read.  Each thread keeps 32
// FP64 partial sums; a warp reduce-scatter (31 shuffles) leaves lane l with
// value l, then the warps' results are added through shared memory.

constexpr int kTraceThreads = 256;

template <typename R>
__device__ void band_trace(const typename Cplx<R>::T* __restrict__ Ts, int n,
                           int plo, int phi, int pa, int pb,
                           double* __restrict__ out /* smem, 32 doubles */,
                           double* __restrict__ red /* smem, 32*nwarps */) {
  const unsigned N = 1u << n;
  const unsigned nr = 1u << (n - 2);
  const unsigned o1 = 1u << pb, o2 = 1u << pa;
  const unsigned off[4] = {0u, o1, o2, o1 | o2};
  double v[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = 0.0;
  for (unsigned r = threadIdx.x; r < nr; r += blockDim.x) {
    const unsigned d = dep2(r, plo, phi);
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const typename Cplx<R>::T* row = Ts + (size_t)(d | off[x]) * N + d;
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        double2 e = to_d2(row[off[y]]);
        v[2 * (x * 4 + y)] += e.x;
        v[2 * (x * 4 + y) + 1] += e.y;
      }
    }
  }
  // reduce-scatter across the warp: after the step with offset h, lanes
  // with bit h set keep the upper half of their values.
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      double keep = up ? v[i + h] : v[i];
      double send = up ? v[i] : v[i + h];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  // lane l now holds the warp total of value index l
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  red[w * 32 + lane] = v[0];
  __syncthreads();
  if (threadIdx.x < 32) {
    double acc = 0.0;
    for (int k = 0; k < nw; ++k) acc += red[k * 32 + threadIdx.x];
    out[threadIdx.x] = acc;
  }
  __syncthreads();
}

// ------------------------------------------------------------ 4x4 update
//
// OptimizeGate (Sec. III-A1, Eq. opt_u) in FP64: with A = X D Y^dagger the
// maximiser of Re Tr(A u) over unitaries is u = Y X^dagger.  The SVD is a
// one-sided (Hestenes) Jacobi iteration on the columns of A: complex plane
// rotations J with A J = W having orthogonal columns, so Y = J, D = column
// norms of W and X = normalised columns of W.  X is then made exactly
// unitary by modified Gram-Schmidt in order of decreasing singular value,
// completing it from the standard basis where a singular value vanishes (a
// rank-deficient A has several optimal u; any completion is one of them).

__device__ bool polar_update(const double2* __restrict__ A, double2* __restrict__ U,
                             double* sig_sum) {
  double2 W[16], J[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    W[i] = A[i];
    J[i] = make_double2((i % 5 == 0) ? 1.0 : 0.0, 0.0);
  }
  bool finite = true;
#pragma unroll
  for (int i = 0; i < 16; ++i) finite = finite && isfinite(A[i].x) && isfinite(A[i].y);
  if (!finite) return false;

  for (int sweep = 0; sweep < 40; ++sweep) {
    bool rotated = false;
#pragma unroll
    for (int p = 0; p < 3; ++p) {
#pragma unroll
      for (int q = p + 1; q < 4; ++q) {
        double al = 0.0, be = 0.0;
        double2 g = make_double2(0.0, 0.0);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          double2 wp = W[i * 4 + p], wq = W[i * 4 + q];
          al += dabs2(wp);
          be += dabs2(wq);
          g = dadd(g, dmul(dconj(wp), wq));
        }
        const double ag = sqrt(dabs2(g));
        if (ag > 1e-15 * sqrt(al * be) && ag > 1e-300) {
          rotated = true;
          const double zeta = (be - al) / (2.0 * ag);
          double t;
          if (fabs(zeta) > 1e100) {
            t = 0.5 / zeta;
          } else {
            t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          }
          const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
          const double2 e = make_double2(g.x / ag, -g.y / ag);  // conj(g)/|g|
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            double2 wp = W[i * 4 + p], ewq = dmul(e, W[i * 4 + q]);
            W[i * 4 + p] = make_double2(c * wp.x - sn * ewq.x, c * wp.y - sn * ewq.y);
            W[i * 4 + q] = make_double2(sn * wp.x + c * ewq.x, sn * wp.y + c * ewq.y);
            double2 jp = J[i * 4 + p], ejq = dmul(e, J[i * 4 + q]);
            J[i * 4 + p] = make_double2(c * jp.x - sn * ejq.x, c * jp.y - sn * ejq.y);
            J[i * 4 + q] = make_double2(sn * jp.x + c * ejq.x, sn * jp.y + c * ejq.y);
          }
        }
      }
    }
    if (!rotated) break;
  }

  double sig[4];
  double smax = 0.0, ssum = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double s2 = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) s2 += dabs2(W[i * 4 + k]);
    sig[k] = sqrt(s2);
    smax = fmax(smax, sig[k]);
    ssum += sig[k];
  }
  // order of decreasing singular value
  int ord[4] = {0, 1, 2, 3};
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 3 - i; ++j)
      if (sig[ord[j]] < sig[ord[j + 1]]) {
        int tmp = ord[j];
        ord[j] = ord[j + 1];
        ord[j + 1] = tmp;
      }
  double2 X[16];  // column k of X = left singular vector of column k of J
#pragma unroll
  for (int i = 0; i < 16; ++i) X[i] = make_double2(0.0, 0.0);
  bool done[4] = {false, false, false, false};
  for (int oi = 0; oi < 4; ++oi) {
    const int k = ord[oi];
    double2 v[4];
    bool ok = sig[k] > 1e-13 * smax && sig[k] > 1e-300;
    if (ok) {
      for (int i = 0; i < 4; ++i) v[i] = dscale(1.0 / sig[k], W[i * 4 + k]);
    }
    for (int attempt = 0; attempt < 5; ++attempt) {
      if (!ok) {  // candidate standard basis vector e_(attempt-1 or 0..3)
        int m = attempt == 0 ? oi : attempt - 1;
        for (int i = 0; i < 4; ++i) v[i] = make_double2(i == m ? 1.0 : 0.0, 0.0);
      }
      for (int j = 0; j < 4; ++j) {
        if (!done[j]) continue;
        double2 d = make_double2(0.0, 0.0);
        for (int i = 0; i < 4; ++i) d = dadd(d, dmul(dconj(X[i * 4 + j]), v[i]));
        for (int i = 0; i < 4; ++i) {
          double2 pr = dmul(d, X[i * 4 + j]);
          v[i].x -= pr.x;
          v[i].y -= pr.y;
        }
      }
      double nv = 0.0;
      for (int i = 0; i < 4; ++i) nv += dabs2(v[i]);
      nv = sqrt(nv);
      if (nv > 0.4) {  // >= 1/2 exists among the basis vectors
        for (int i = 0; i < 4; ++i) X[i * 4 + k] = dscale(1.0 / nv, v[i]);
        done[k] = true;
        break;
      }
      ok = false;
    }
  }
  // u = Y X^dagger = J X^dagger
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      double2 acc = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 4; ++k) acc = dadd(acc, dmul(J[i * 4 + k], dconj(X[j * 4 + k])));
      U[i * 4 + j] = acc;
    }
  *sig_sum = ssum;
  bool fin = isfinite(ssum);
  for (int i = 0; i < 16; ++i) fin = fin && isfinite(U[i].x) && isfinite(U[i].y);
  return fin;
}

// ---------------------------------------------------- env + update kernel
//
// One CTA per start: band partial trace P of the tensor *before* gate k is
// removed, E from P and the current gate u (P u^dagger when u sits on the
// right, u^dagger P when it sits on the left), then the FP64 update and the
// two pass operators.

template <typename R>
__global__ void __launch_bounds__(kTraceThreads) update_kernel(
    const typename Cplx<R>::T* __restrict__ T, int n, int plo, int phi, int pa,
    int pb, double2* __restrict__ gates_k, long long gstride, int mode,
    double beta, double2* __restrict__ LR, double2* __restrict__ env_out,
    long long env_stride, double* __restrict__ sigma_out, int* __restrict__ status) {
  __shared__ double Pd[32];
  __shared__ double red[32 * (kTraceThreads / 32)];
  const int s = blockIdx.x;
  const size_t NN = (size_t)1 << (2 * n);
  band_trace<R>(T + s * NN, n, plo, phi, pa, pb, Pd, red);
  if (threadIdx.x != 0) return;

  double2 P[16], u[16], E[16];
  double2* g = gates_k + s * gstride;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    P[i] = make_double2(Pd[2 * i], Pd[2 * i + 1]);
    u[i] = g[i];
  }
  // E = P u^dagger (gate on the right) or u^dagger P (gate on the left)
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      double2 acc = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (mode == kForward)
          acc = dadd(acc, dmul(dconj(u[k * 4 + i]), P[k * 4 + j]));
        else
          acc = dadd(acc, dmul(P[i * 4 + k], dconj(u[j * 4 + k])));
      }
      E[i * 4 + j] = acc;
    }
  if (env_out) {
    double2* eo = env_out + s * env_stride;
    for (int i = 0; i < 16; ++i) eo[i] = E[i];
  }
  double2* lr = LR + (size_t)s * 32;
  if (mode == kEnvOnly) {
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        lr[i * 4 + j] = u[i * 4 + j];
        lr[16 + i * 4 + j] = dconj(u[j * 4 + i]);
      }
    return;
  }
  double2 A[16], un[16];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      double2 e = E[i * 4 + j];
      if (beta != 0.0) {
        double2 ud = dconj(u[j * 4 + i]);
        e = make_double2((1.0 - beta) * e.x + beta * ud.x, (1.0 - beta) * e.y + beta * ud.y);
      }
      A[i * 4 + j] = e;
    }
  double ssum = 0.0;
  if (!polar_update(A, un, &ssum)) {
    atomicExch(status, -4);
    // keep the old gate so that the tensor stays consistent
    for (int i = 0; i < 16; ++i) un[i] = u[i];
    ssum = 0.0;
  }
  for (int i = 0; i < 16; ++i) g[i] = un[i];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double2 ud = dconj(u[j * 4 + i]);
      if (mode == kBackward) {
        lr[i * 4 + j] = un[i * 4 + j];
        lr[16 + i * 4 + j] = ud;
      } else {
        lr[i * 4 + j] = ud;
        lr[16 + i * 4 + j] = un[i * 4 + j];
      }
    }
  if (sigma_out) sigma_out[s] = ssum;
}

template <typename R>
__global__ void __launch_bounds__(kTraceThreads) partial_trace_kernel(
    const typename Cplx<R>::T* __restrict__ T, int n, int plo, int phi, int pa,
    int pb, double2* __restrict__ P) {
  __shared__ double Pd[32];
  __shared__ double red[32 * (kTraceThreads / 32)];
  const int s = blockIdx.x;
  const size_t NN = (size_t)1 << (2 * n);
  band_trace<R>(T + s * NN, n, plo, phi, pa, pb, Pd, red);
  if (threadIdx.x < 16)
    P[(size_t)s * 16 + threadIdx.x] = make_double2(Pd[2 * threadIdx.x], Pd[2 * threadIdx.x + 1]);
}

__global__ void optimize_kernel(const double2* __restrict__ E,
                                const double2* __restrict__ u_old, double beta,
                                int count, double2* __restrict__ u_out,
                                double* __restrict__ sigma_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double2 A[16], un[16];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      double2 e = E[(size_t)i * 16 + r * 4 + c];
      if (beta != 0.0) {
        double2 ud = dconj(u_old[(size_t)i * 16 + c * 4 + r]);
        e = make_double2((1.0 - beta) * e.x + beta * ud.x, (1.0 - beta) * e.y + beta * ud.y);
      }
      A[r * 4 + c] = e;
    }
  double ssum = 0.0;
  if (!polar_update(A, un, &ssum)) {
    for (int k = 0; k < 16; ++k) un[k] = make_double2(NAN, NAN);
    ssum = NAN;
  }
  for (int k = 0; k < 16; ++k) u_out[(size_t)i * 16 + k] = un[k];
  if (sigma_out) sigma_out[i] = ssum;
}

// ----------------------------------------------------------------- trace

template <typename R>
__global__ void __launch_bounds__(kTraceThreads) trace_kernel(
    const typename Cplx<R>::T* __restrict__ T, int n, double2* __restrict__ tr) {
  __shared__ double red[2 * (kTraceThreads / 32)];
  const int s = blockIdx.x;
  const size_t N = (size_t)1 << n;
  const typename Cplx<R>::T* Ts = T + (size_t)s * N * N;
  double re = 0.0, im = 0.0;
  for (size_t i = threadIdx.x; i < N; i += blockDim.x) {
    double2 e = to_d2(Ts[i * (N + 1)]);
    re += e.x;
    im += e.y;
  }
  for (int h = 16; h >= 1; h >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, h);
    im += __shfl_xor_sync(0xffffffffu, im, h);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[2 * w] = re;
    red[2 * w + 1] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += red[2 * k];
      b += red[2 * k + 1];
    }
    tr[s] = make_double2(a, b);
  }
}

__global__ void set_identity_kernel(double2* __restrict__ M, int n) {
  const size_t N = (size_t)1 << n;
  const size_t NN = N * N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < NN;
       i += (size_t)gridDim.x * blockDim.x)
    M[i] = make_double2((i / N == i % N) ? 1.0 : 0.0, 0.0);
}

}  // namespace

// ================================================================ launchers

cudaError_t launch_set_identity(double2* M, int n, cudaStream_t st) {
  const size_t NN = (size_t)1 << (2 * n);
  size_t blocks = (NN + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  set_identity_kernel<<<(unsigned)blocks, 256, 0, st>>>(M, n);
  return cudaGetLastError();
}

int sm_count() {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
      v = 152;
    cached = v;
  }
  return cached;
}

cudaError_t launch_conj_transpose(const double2* V, void* T, int n, int S, int prec,
                                  cudaStream_t st) {
  const int N = 1 << n;
  dim3 grid((N + 31) / 32, (N + 31) / 32, S), block(32, 8);
  if (prec == 0)
    conj_transpose_kernel<double><<<grid, block, 0, st>>>(V, (double2*)T, N);
  else
    conj_transpose_kernel<float><<<grid, block, 0, st>>>(V, (float2*)T, N);
  return cudaGetLastError();
}

template <typename R>
static void pass_dispatch(void* T, int n, int S, int plo, int phi, int pa, int pb,
                          const double2* L, long long Ls, const double2* Rm, long long Rs,
                          cudaStream_t st) {
  typedef typename Cplx<R>::T C;
  const unsigned nblk = 1u << (2 * (n - 2));
  const int per_sm = sizeof(R) == 4 ? 3 : 1;
  long long want = (nblk + kPassThreads - 1) / kPassThreads;
  long long cap = ((long long)sm_count() * per_sm + S - 1) / S;
  if (cap < 1) cap = 1;
  int gx = (int)(want < cap ? want : cap);
  dim3 grid(gx, S);
  C* t = (C*)T;
  if (L && Rm)
    pass_kernel<R, true, true><<<grid, kPassThreads, 0, st>>>(t, n, plo, phi, pa, pb, L, Ls, Rm, Rs);
  else if (L)
    pass_kernel<R, true, false><<<grid, kPassThreads, 0, st>>>(t, n, plo, phi, pa, pb, L, Ls, Rm, Rs);
  else if (Rm)
    pass_kernel<R, false, true><<<grid, kPassThreads, 0, st>>>(t, n, plo, phi, pa, pb, L, Ls, Rm, Rs);
}

cudaError_t launch_pass(void* T, int n, int S, int a, int b, const double2* L,
                        long long Lstride, const double2* R, long long Rstride, int prec,
                        cudaStream_t st) {
  if (!L && !R) return cudaSuccess;
  const int pa = qubit_bit(n, a), pb = qubit_bit(n, b);
  const int plo = pa < pb ? pa : pb, phi = pa < pb ? pb : pa;
  if (prec == 0)
    pass_dispatch<double>(T, n, S, plo, phi, pa, pb, L, Lstride, R, Rstride, st);
  else
    pass_dispatch<float>(T, n, S, plo, phi, pa, pb, L, Lstride, R, Rstride, st);
  return cudaGetLastError();
}

cudaError_t launch_update(const void* T, int n, int S, int a, int b, double2* gates_k,
                          long long gstride, int mode, double beta, double2* LR,
                          double2* env_out, long long env_stride, double* sigma_out,
                          int* status, int prec, cudaStream_t st) {
  const int pa = qubit_bit(n, a), pb = qubit_bit(n, b);
  const int plo = pa < pb ? pa : pb, phi = pa < pb ? pb : pa;
  if (prec == 0)
    update_kernel<double><<<S, kTraceThreads, 0, st>>>((const double2*)T, n, plo, phi, pa, pb,
                                                      gates_k, gstride, mode, beta, LR, env_out,
                                                      env_stride, sigma_out, status);
  else
    update_kernel<float><<<S, kTraceThreads, 0, st>>>((const float2*)T, n, plo, phi, pa, pb,
                                                     gates_k, gstride, mode, beta, LR, env_out,
                                                     env_stride, sigma_out, status);
  return cudaGetLastError();
}

cudaError_t launch_partial_trace(const void* T, int n, int S, int a, int b, double2* P,
                                 int prec, cudaStream_t st) {
  const int pa = qubit_bit(n, a), pb = qubit_bit(n, b);
  const int plo = pa < pb ? pa : pb, phi = pa < pb ? pb : pa;
  if (prec == 0)
    partial_trace_kernel<double><<<S, kTraceThreads, 0, st>>>((const double2*)T, n, plo, phi,
                                                             pa, pb, P);
  else
    partial_trace_kernel<float><<<S, kTraceThreads, 0, st>>>((const float2*)T, n, plo, phi, pa,
                                                            pb, P);
  return cudaGetLastError();
}

cudaError_t launch_optimize(const double2* E, const double2* u_old, double beta, int count,
                            double2* u_out, double* sigma_out, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int threads = 64;
  optimize_kernel<<<(count + threads - 1) / threads, threads, 0, st>>>(E, u_old, beta, count,
                                                                       u_out, sigma_out);
  return cudaGetLastError();
}

cudaError_t launch_trace(const void* T, int n, int S, double2* tr, int prec, cudaStream_t st) {
  if (prec == 0)
    trace_kernel<double><<<S, kTraceThreads, 0, st>>>((const double2*)T, n, tr);
  else
    trace_kernel<float><<<S, kTraceThreads, 0, st>>>((const float2*)T, n, tr);
  return cudaGetLastError();
}

}  // namespace qf
