// Batched instantiation of many small circuits in one persistent launch.
//
// Each warp runs a whole Qfactor (Alg. 1) for one (instance, start) problem:
// InitCircuitTensor, TwoSidedSweeps, the cost after every sweep, the
// stopping rules and the periodic rebuild, with the circuit tensor in the
// warp's own slice of shared memory (4^n entries: 1 KB at 3 qubits, 16 KB at
// 5 qubits in complex128).  Warps take problems from an atomic work counter,
// instance-major, so the starts of an instance run side by side.  Starts of
// one instance meet only through two per-instance words in global memory:
// a "converged" flag and a plateau count (Sec. IV-A: stop when any start
// converges, or once every start has met a plateau test).  Nothing waits on
// them; a warp reads them at its sweep boundaries.
//
// The gate update is the warp polar of qf_polar.cuh; in QF_C64_REFINE64 the
// bulk sweeps run on a complex64 tensor and the warp switches to a
// complex128 tensor rebuilt from the target and its FP64 gates.

#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "qf_device.cuh"
#include "qf_internal.h"
#include "qf_polar.cuh"
#include "qf_warp8.cuh"
#include "qfactor.h"

namespace qf {
namespace {

using namespace dev;

struct BatchInst {
  int n, p;
  long long loc_off;   // first location of the instance
  long long tgt_off;   // first target entry
  long long gate_off;  // first gate entry of start 0 ([start][p][16])
};

constexpr int kRing = 128;  // cost history kept per warp (long plateau window)

struct BatchParams {
  const BatchInst* inst;
  const int* order;  // instances in the order their problems are handed out
  int n_inst, S;
  const int2* locs;
  const double2* targets;
  double2* gates;
  float2* yprev;  // per gate entry: the last Jacobi rotation (warm start of the next update)
  double* cost_out;
  int* sweeps_out;
  int* c64_out;
  int* reason_out;
  int* conv_flag;
  int* plat_count;
  int* status;
  unsigned* work;
  double dist_tol, diff_a, diff_r, long_r, beta, switch_tol;
  int max_sweeps, min_sweeps, reset_iter, long_L, precision, max_c64;
  double* hist;    // optional cost history [instance][start][sweep], row hist_row
  int hist_row;
  int tmax_bytes;  // tensor capacity of a warp slice (complex128, largest n)
  int warp_bytes;  // whole warp slice
};

// One out-of-line copy of the warp polar for the whole kernel: inlined at
// every call site of both precisions the kernel outgrew the instruction cache.
__device__ __noinline__ bool polar_once(double2 a, float2* scratch, double2* u_out, double* sig,
                                        float2* y_io) {
  const Lane L;
  return warp_polar(L, a, scratch, u_out, sig, y_io);
}

template <typename R>
struct W {
  typedef typename Cplx<R>::T C;

  // T <- V^dagger
  static __device__ void conj_transpose(C* T, const double2* __restrict__ V, int n) {
    const int NN = 1 << (2 * n);
    const int lane = threadIdx.x & 31;
    for (int idx = lane; idx < NN; idx += 32) {
      const int r = idx >> n, c = idx & ((1 << n) - 1);
      const double2 v = V[idx];
      T[(c << n) | r] = cmake(make_double2(v.x, -v.y), R());
    }
    __syncwarp();
  }

  // T <- (L on (a,b)) T (R on (a,b)); operators in shared memory.  The
  // tensor lives in the warp's shared memory, so the two products run as
  // two in-place stages: R on every block row (item = (row x, block); a
  // lane reads the row's 4 entries and writes 4), then L on every block
  // column.  A lane holds one row or column at a time (a whole 4x4 block in
  // registers set the kernel's register count, and with it the warps per
  // SM), and 4 items per block give small circuits 4 times the active lanes.
  template <bool HL, bool HR>
  static __device__ void pass(C* T, int n, int pa, int pb, const C* Lm, const C* Rm) {
    const int lane = threadIdx.x & 31;
    const int plo = pa < pb ? pa : pb, phi = pa < pb ? pb : pa;
    const int lnc = n - 2;
    const unsigned N = 1u << n, cmask = (1u << lnc) - 1u, nblk = 1u << (2 * lnc);
    const unsigned o1 = 1u << pb, o2 = 1u << pa;
    const unsigned items = 4u * nblk;
    auto offv = [&](unsigned v) { return ((v & 2u) ? o2 : 0u) | ((v & 1u) ? o1 : 0u); };
    // N is a multiple of 16 entries, so an entry's bank is set by its column.
    // Row stage: lanes with the same c0 take the row's entries in the order
    // y ^ s, s = (it >> lnc) & 3 (off is GF(2)-linear: off(y ^ s) =
    // off(y) ^ off(s), and R's entry (k ^ s, y ^ s) is index (4k + y) ^ 5s),
    // so the lanes of a step touch distinct columns.
    if (HR) {  // row (r0 | off[x]) of block (r0, c0) <- row R
      for (unsigned it = lane; it < items; it += 32) {
        const unsigned blk = it & (nblk - 1u), x = it >> (2 * lnc);
        const unsigned r0 = dep2(blk >> lnc, plo, phi), c0 = dep2(blk & cmask, plo, phi);
        const unsigned sk = (it >> lnc) & 3u, os = offv(sk), s5 = 5u * sk;
        C* row = T + (size_t)(r0 | offv(x)) * N + c0;
        C v[4];
#pragma unroll
        for (int y = 0; y < 4; ++y) v[y] = row[offv(y) ^ os];
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          C acc = czero<C>();
#pragma unroll
          for (int k = 0; k < 4; ++k) acc = cfma(v[k], Rm[(k * 4 + y) ^ s5], acc);
          row[offv(y) ^ os] = acc;
        }
      }
      __syncwarp();
    }
    // Column stage: the gate column y varies fastest over the lanes, then
    // the block column, so a step's lanes cover distinct columns.
    if (HL) {  // column (c0 | off[y]) of block (r0, c0) <- L column
      for (unsigned it = lane; it < items; it += 32) {
        const unsigned y = it & 3u, cb = (it >> 2) & cmask, rb = it >> (2 + lnc);
        const unsigned r0 = dep2(rb, plo, phi), c0 = dep2(cb, plo, phi);
        C* col = T + (size_t)r0 * N + (c0 | offv(y));
        C v[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) v[x] = col[(size_t)offv(x) * N];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          C acc = czero<C>();
#pragma unroll
          for (int k = 0; k < 4; ++k) acc = cfma(Lm[x * 4 + k], v[k], acc);
          col[(size_t)offv(x) * N] = acc;
        }
      }
      __syncwarp();
    }
  }

  // Band partial trace on (a, b): P[x][y] = sum over the rests r of
  // T[(r, x), (r, y)].  Lane 16 h + 4 x + y sums entry (x, y) over the rests
  // r = h, h + 2, ... in the tensor's precision; the two half-warps are
  // added in FP64 with one shuffle (the same sum on both halves).  Returns
  // P[i][j] on lane (i, j).
  static __device__ double2 band(const C* T, int n, int pa, int pb, const Lane& L) {
    const int plo = pa < pb ? pa : pb, phi = pa < pb ? pb : pa;
    const unsigned N = 1u << n, nr = 1u << (n - 2);
    const unsigned o1 = 1u << pb, o2 = 1u << pa;
    const unsigned ox = ((L.i & 2) ? o2 : 0u) | ((L.i & 1) ? o1 : 0u);
    const unsigned oy = ((L.j & 2) ? o2 : 0u) | ((L.j & 1) ? o1 : 0u);
    R vx = R(0), vy = R(0);
    for (unsigned r = (unsigned)L.l >> 4; r < nr; r += 2) {
      const unsigned d = dep2(r, plo, phi);
      const C e = T[(d | ox) * N + (d | oy)];
      vx += e.x;
      vy += e.y;
    }
    const double px = (double)vx, py = (double)vy;
    return make_double2(px + __shfl_xor_sync(kFull, px, 16), py + __shfl_xor_sync(kFull, py, 16));
  }

  // 1 - |Tr T| / N (FP64 sum)
  static __device__ double cost(const C* T, int n) {
    const int N = 1 << n, lane = threadIdx.x & 31;
    double re = 0.0, im = 0.0;
    for (int i = lane; i < N; i += 32) {
      const double2 e = to_d2(T[i * (N + 1)]);
      re += e.x;
      im += e.y;
    }
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
      re += __shfl_xor_sync(kFull, re, h);
      im += __shfl_xor_sync(kFull, im, h);
    }
    return 1.0 - sqrt(re * re + im * im) / (double)N;
  }

  // InitCircuitTensor: T <- V^dagger, then T <- T (u_k on loc_k) for all k.
  static __device__ __noinline__ void build(C* T, C* LRs, const double2* V, const double2* g,
                                            const int2* locs,
                               int n, int p, const Lane& L) {
    conj_transpose(T, V, n);
    for (int k = 0; k < p; ++k) {
      if (L.l < 16) LRs[16 + L.l] = cmake(g[k * 16 + L.l], R());
      __syncwarp();
      const int2 lc = locs[k];
      pass<false, true>(T, n, n - 1 - lc.x, n - 1 - lc.y, LRs, LRs + 16);
    }
  }

  // One gate update: environment from the band, the FP64 warp polar, the
  // pass operators into shared memory, then the fused pass.
  static __device__ __noinline__ void update(C* T, C* LRs, float2* scratch, double2* g, float2* yp,
                                             int2 lc,
                                             int n,
                                bool forward, double beta, const Lane& L, int* bad) {
    const int pa = n - 1 - lc.x, pb = n - 1 - lc.y;
    const double2 P = band(T, n, pa, pb, L);
    const int e = L.l & 15;
    const double2 u = g[e];
    const double2 ud = wdag(L, u);
    const double2 E = forward ? wmm_dn(L, u, P) : wmm_nd(L, P, u);
    double2 A = E;
    if (beta != 0.0)
      A = make_double2((1.0 - beta) * E.x + beta * ud.x, (1.0 - beta) * E.y + beta * ud.y);
    double2 un;
    double sg;
    float2 y = yp[e];  // the gate's last Jacobi rotation: a warm start
    if (!polar_once(A, scratch, &un, &sg, &y)) {
      *bad = 1;
      un = u;
      y = make_float2(L.i == L.j ? 1.f : 0.f, 0.f);
    }
    if (L.l < 16) {
      g[e] = un;
      yp[e] = y;
      LRs[e] = cmake(forward ? ud : un, R());
      LRs[16 + e] = cmake(forward ? un : ud, R());
    }
    __syncwarp();
    pass<true, true>(T, n, pa, pb, LRs, LRs + 16);
  }

  // TwoSidedSweep (Alg. 1).
  static __device__ __noinline__ void sweep(C* T, C* LRs, float2* scratch, double2* g, float2* yp,
                                            const int2* locs,
                               int n, int p, double beta, const Lane& L, int* bad) {
    for (int k = p - 1; k >= 0; --k)
      update(T, LRs, scratch, g + k * 16, yp + k * 16, locs[k], n, false, beta, L, bad);
    for (int k = 0; k < p; ++k)
      update(T, LRs, scratch, g + k * 16, yp + k * 16, locs[k], n, true, beta, L, bad);
  }
};

// Periodic re-unitarisation (reset_iter): three FP64 Newton-Schulz steps per
// gate, u <- u (3I - u^dagger u) / 2.
__device__ void reunitarize(double2* g, int p, const Lane& L) {
  const int e = L.l & 15;
  for (int k = 0; k < p; ++k) {
    double2 u = g[k * 16 + e];
    for (int step = 0; step < 3; ++step) {
      const double2 P = wmm_dn(L, u, u);
      const double2 Q = make_double2((L.i == L.j ? 1.5 : 0.0) - 0.5 * P.x, -0.5 * P.y);
      u = wmm(L, u, Q);
    }
    __syncwarp();
    if (L.l < 16) g[k * 16 + e] = u;
    __syncwarp();
  }
}

__device__ bool plateau_test(const double* ring, int len, int it, const BatchParams& bp) {
  const double c = ring[(len - 1) % kRing];
  if ((bp.diff_a > 0.0 || bp.diff_r > 0.0) && len >= 2) {
    if (ring[(len - 2) % kRing] - c <= bp.diff_a + bp.diff_r * c) return true;
  }
  if (bp.long_L > 0 && it >= bp.long_L) {
    const double old = ring[(len - 1 - bp.long_L) % kRing];
    if (old - c < bp.long_r * old) return true;
  }
  return false;
}

// A complex64 start whose cost stalls at or below this switches to FP64
// (the stall is then the complex64 noise floor, ~1e-7); above it the stall
// is the method's own plateau and the start stays in complex64.
constexpr double kStallSwitchCost = 1e-5;

// The per-warp problem loop of the batched kernels: each warp takes the next
// (instance, start) from the work counter, runs Qfactor on it (Alg. 1) with
// the stopping rules of Sec. III-A2 and the multistart rule of Sec. IV-A,
// and writes its outputs.  Ops supplies the steps for its kind of circuit:
//   load(in, s)            gate pointers of start s; warm-start rotations reset
//   build<R>()             InitCircuitTensor into the warp's tensor
//   sweep<R>(bad)          one TwoSidedSweep
//   reunit()               the periodic re-unitarisation of the gates
// with R = float for the complex64 tensor and double for complex128.
template <typename Ops>
__device__ __forceinline__ void run_problems(const BatchParams& bp, Ops ops, void* Tbuf, double* ring) {
  const Lane L;
  const unsigned total = (unsigned)bp.n_inst * (unsigned)bp.S;
  for (;;) {
    unsigned prob = 0;
    if (L.l == 0) prob = atomicAdd(bp.work, 1u);
    prob = __shfl_sync(kFull, prob, 0);
    if (prob >= total) break;
    const int i = bp.order[prob / bp.S], s = (int)(prob % bp.S);
    const BatchInst in = bp.inst[i];
    const int n = in.n;
    ops.load(in, i, s);
    __syncwarp();
    volatile int* conv = bp.conv_flag + i;
    volatile int* plat = bp.plat_count + i;
    bool c64 = bp.precision != QF_C128;
    const bool refine = bp.precision == QF_C64_REFINE64;
    int bad = 0;
    if (c64)
      ops.template build<float>();
    else
      ops.template build<double>();
    double c = c64 ? W<float>::cost((float2*)Tbuf, n) : W<double>::cost((double2*)Tbuf, n);
    double* hist = bp.hist ? bp.hist + ((long long)i * bp.S + s) * bp.hist_row : nullptr;
    int len = 0;
    if (L.l == 0) ring[0] = c;
    if (hist && L.l == 0) hist[0] = c;
    len = 1;
    __syncwarp();
    int it = 0, c64_sw = 0, reason = QF_STOP_MAX_SWEEPS;
    bool plateaued = false;
    for (it = 1; it <= bp.max_sweeps; ++it) {
      if (*conv) {  // another start of this instance reached dist_tol
        reason = QF_STOP_CONVERGED;
        --it;
        break;
      }
      if (c64)
        ops.template sweep<float>(&bad);
      else
        ops.template sweep<double>(&bad);
      if (bp.reset_iter > 0 && it % bp.reset_iter == 0) {
        ops.reunit();
        if (c64)
          ops.template build<float>();
        else
          ops.template build<double>();
      }
      c = c64 ? W<float>::cost((float2*)Tbuf, n) : W<double>::cost((double2*)Tbuf, n);
      if (c64 && refine) {
        ++c64_sw;
        // leave complex64 once the cost is below switch_tol, or once ten c64
        // sweeps have lowered it by less than the complex64 noise floor while
        // the cost is near that floor (<= kStallSwitchCost); a stall at a
        // larger cost is the method's own plateau, which FP64 sweeps do not
        // lift, so the start stays in complex64
        const bool stalled = len > 10 && ring[(len - 10) % kRing] - c < 1e-7;
        if (c <= bp.switch_tol || (stalled && c <= kStallSwitchCost) || c64_sw >= bp.max_c64) {
          // rebuild in complex128 from the target and the FP64 gates
          ops.template build<double>();
          c = W<double>::cost((double2*)Tbuf, n);
          c64 = false;
        } else {
          if (L.l == 0) ring[len % kRing] = c;
          if (hist && L.l == 0) hist[it] = c;
          ++len;
          __syncwarp();
          if (it >= bp.min_sweeps && !plateaued && plateau_test(ring, len, it, bp)) {
            plateaued = true;
            if (L.l == 0) atomicAdd(bp.plat_count + i, 1);
          }
          __syncwarp();
          if (*plat >= bp.S) {  // every start of the instance plateaued
            reason = QF_STOP_PLATEAU;
            break;
          }
          continue;
        }
      }
      if (L.l == 0) ring[len % kRing] = c;
      if (hist && L.l == 0) hist[it] = c;
      ++len;
      __syncwarp();
      if (it >= bp.min_sweeps) {
        if (c <= bp.dist_tol) {
          if (L.l == 0) atomicExch(bp.conv_flag + i, 1);
          reason = QF_STOP_CONVERGED;
          break;
        }
        if (!plateaued && plateau_test(ring, len, it, bp)) {
          plateaued = true;
          if (L.l == 0) atomicAdd(bp.plat_count + i, 1);
        }
        __syncwarp();
        if (*plat >= bp.S) {
          reason = QF_STOP_PLATEAU;
          break;
        }
      }
    }
    if (it > bp.max_sweeps) it = bp.max_sweeps;
    if (c64) {  // report an FP64 cost: rebuild the tensor in complex128 once
      ops.template build<double>();
      c = W<double>::cost((double2*)Tbuf, n);
    }
    if (L.l == 0) {
      const long long q = (long long)i * bp.S + s;  // outputs in instance order
      bp.cost_out[q] = c;
      bp.sweeps_out[q] = it;
      bp.c64_out[q] = c64_sw;
      bp.reason_out[q] = reason;
      if (bad) atomicExch(bp.status, QF_ENONFINITE);
    }
    __syncwarp();
  }
}

// Steps of a circuit of two-qubit gates (gate k: 16 entries at k * 16).
struct Ops2 {
  double2* gates;
  float2* yprev;
  const double2* targets;
  const int2* all_locs;
  double beta;
  void* T;
  double2* LR;      // 32 x 16 B: the pass operators (complex64 or complex128)
  float2* scratch;  // 32 x 8 B
  Lane L;
  const double2* V;
  double2* g;
  float2* yp;
  const int2* locs;
  int n, p;
  __device__ __forceinline__ Ops2(const BatchParams& b, void* t, double2* lr, float2* sc)
      : gates(b.gates), yprev(b.yprev), targets(b.targets), all_locs(b.locs), beta(b.beta), T(t), LR(lr),
        scratch(sc) {}
  __device__ __forceinline__ void load(const BatchInst& in, int, int s) {
    n = in.n;
    p = in.p;
    g = gates + in.gate_off + (long long)s * p * 16;
    yp = yprev + in.gate_off + (long long)s * p * 16;
    V = targets + in.tgt_off;
    locs = all_locs + in.loc_off;
    if (L.l < 16)
      for (int k = 0; k < p; ++k) yp[k * 16 + L.l] = make_float2(L.i == L.j ? 1.f : 0.f, 0.f);
  }
  template <typename R>
  __device__ __forceinline__ void build() {
    typedef typename Cplx<R>::T C;
    W<R>::build((C*)T, (C*)LR, V, g, locs, n, p, L);
  }
  template <typename R>
  __device__ __forceinline__ void sweep(int* bad) {
    typedef typename Cplx<R>::T C;
    W<R>::sweep((C*)T, (C*)LR, scratch, g, yp, locs, n, p, beta, L, bad);
  }
  __device__ __forceinline__ void reunit() { reunitarize(g, p, L); }
};

__global__ void __maxnreg__(168) batched_kernel(BatchParams bp) {
  extern __shared__ __align__(256) unsigned char smem[];
  unsigned char* ws = smem + (size_t)(threadIdx.x >> 5) * bp.warp_bytes;
  unsigned char* after = ws + bp.tmax_bytes;
  Ops2 ops(bp, ws, reinterpret_cast<double2*>(after), reinterpret_cast<float2*>(after + 512));
  run_problems(bp, ops, ws, reinterpret_cast<double*>(after + 768));  // ring: kRing x 8 B
}


// ------------------------------------------------------ circuits of 2- and 3-qubit gates
//
// The same per-warp Qfactor for circuits that mix two- and three-qubit
// gates (Sec. III: a k-qubit unitary is one variable with a 2^k x 2^k
// environment).  Gate k of an instance is gk[k] = (size, q0, q1, q2) and
// starts at entry goff[k] of the start's gate block (4^size entries each,
// row-major in the gate's local index 4 bit(q0) + 2 bit(q1) + bit(q2)).  A
// three-qubit update is the band sum over 8x8 blocks, E = P u^dagger
// (backward) or u^dagger P (forward), the warp 8x8 polar of qf_warp8.cuh
// (lane 8 g + j holds entries (g, j) and (g + 4, j)) and the fused pass on
// 8x8 blocks; two-qubit gates take the routines above.

struct BatchParamsK {
  BatchParams b;
  const int4* gk;       // per gate: (size, q0, q1, q2)
  const int* goff;      // per gate: entry offset in the start's gate block
  const int* inst_ge;   // per instance: gate entries per start
};

template <typename R>
struct WK {
  typedef typename Cplx<R>::T C;

  // offset of local index v of a three-qubit gate on bit positions (p0, p1, p2)
  static __device__ __forceinline__ unsigned off8(unsigned v, int p0, int p1, int p2) {
    return ((v & 4u) ? 1u << p0 : 0u) | ((v & 2u) ? 1u << p1 : 0u) | ((v & 1u) ? 1u << p2 : 0u);
  }
  // zero bits inserted at three ascending positions
  static __device__ __forceinline__ unsigned dep3(unsigned x, int a, int b, int c) {
    return dep1(dep1(dep1(x, a), b), c);
  }
  static __device__ __forceinline__ void sort3(int p0, int p1, int p2, int& a, int& b, int& c) {
    a = p0, b = p1, c = p2;
    if (a > b) { const int t = a; a = b; b = t; }
    if (b > c) { const int t = b; b = c; c = t; }
    if (a > b) { const int t = a; a = b; b = t; }
  }

  // T <- (L on the gate) T (R on the gate) on every 8x8 block, as two
  // in-place stages (R along each block row, then L along each block column)
  template <bool HL, bool HR>
  static __device__ void pass8(C* T, int n, int p0, int p1, int p2, const C* Lm, const C* Rm) {
    const int lane = threadIdx.x & 31;
    int a, b, c;
    sort3(p0, p1, p2, a, b, c);
    const int lnc = n - 3;
    const unsigned N = 1u << n, cmask = (1u << lnc) - 1u, nblk = 1u << (2 * lnc);
    const unsigned items = 8u * nblk;
    // Bank-conflict-free order, as in the 4x4 pass: the row stage takes a
    // row's entries in the order y ^ s, s = (it >> lnc) & 7 (R's entry
    // (k ^ s, y ^ s) is index (8k + y) ^ 9s); the column stage maps the
    // gate column y to the lowest lane bits.
    if (HR) {
      for (unsigned it = lane; it < items; it += 32) {
        const unsigned blk = it & (nblk - 1u), x = it >> (2 * lnc);
        const unsigned r0 = dep3(blk >> lnc, a, b, c), c0 = dep3(blk & cmask, a, b, c);
        const unsigned sk = (it >> lnc) & 7u, os = off8(sk, p0, p1, p2), s9 = 9u * sk;
        C* row = T + (size_t)(r0 | off8(x, p0, p1, p2)) * N + c0;
        C v[8];
#pragma unroll
        for (int y = 0; y < 8; ++y) v[y] = row[off8(y, p0, p1, p2) ^ os];
#pragma unroll
        for (int y = 0; y < 8; ++y) {
          C acc = czero<C>();
#pragma unroll
          for (int k = 0; k < 8; ++k) acc = cfma(v[k], Rm[(k * 8 + y) ^ s9], acc);
          row[off8(y, p0, p1, p2) ^ os] = acc;
        }
      }
      __syncwarp();
    }
    if (HL) {
      for (unsigned it = lane; it < items; it += 32) {
        const unsigned y = it & 7u, cb = (it >> 3) & cmask, rb = it >> (3 + lnc);
        const unsigned r0 = dep3(rb, a, b, c), c0 = dep3(cb, a, b, c);
        C* col = T + (size_t)r0 * N + (c0 | off8(y, p0, p1, p2));
        C v[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) v[x] = col[(size_t)off8(x, p0, p1, p2) * N];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
          C acc = czero<C>();
#pragma unroll
          for (int k = 0; k < 8; ++k) acc = cfma(Lm[x * 8 + k], v[k], acc);
          col[(size_t)off8(x, p0, p1, p2) * N] = acc;
        }
      }
      __syncwarp();
    }
  }

  // P[x][y] = sum over the rests r of T[(r, x), (r, y)] for a three-qubit
  // gate; lane (g, j) gets P[g][j] and P[g + 4][j] (FP64 from the tensor's
  // precision)
  static __device__ void band8(const C* T, int n, int p0, int p1, int p2, const w8::L8& L, double2& P0,
                               double2& P1) {
    int a, b, c;
    sort3(p0, p1, p2, a, b, c);
    const unsigned N = 1u << n, nr = 1u << (n - 3);
    const unsigned ox0 = off8((unsigned)L.g, p0, p1, p2), ox1 = off8((unsigned)L.g + 4u, p0, p1, p2);
    const unsigned oy = off8((unsigned)L.j, p0, p1, p2);
    R v0x = R(0), v0y = R(0), v1x = R(0), v1y = R(0);
    for (unsigned r = 0; r < nr; ++r) {
      const unsigned d = dep3(r, a, b, c);
      const C e0 = T[(size_t)(d | ox0) * N + (d | oy)], e1 = T[(size_t)(d | ox1) * N + (d | oy)];
      v0x += e0.x;
      v0y += e0.y;
      v1x += e1.x;
      v1y += e1.y;
    }
    P0 = make_double2((double)v0x, (double)v0y);
    P1 = make_double2((double)v1x, (double)v1y);
  }

  // InitCircuitTensor: T <- V^dagger, then every gate on the right in order.
  static __device__ __noinline__ void build(C* T, C* LRs, const double2* V, const double2* g,
                                            const int4* gk, const int* goff, int n, int p, const Lane& L) {
    W<R>::conj_transpose(T, V, n);
    for (int k = 0; k < p; ++k) {
      const int4 d = gk[k];
      const double2* gp = g + goff[k];
      if (d.x == 3) {
        for (int e = L.l; e < 64; e += 32) LRs[64 + e] = cmake(gp[e], R());
        __syncwarp();
        pass8<false, true>(T, n, n - 1 - d.y, n - 1 - d.z, n - 1 - d.w, LRs, LRs + 64);
      } else {
        if (L.l < 16) LRs[64 + L.l] = cmake(gp[L.l], R());
        __syncwarp();
        W<R>::template pass<false, true>(T, n, n - 1 - d.y, n - 1 - d.z, LRs, LRs + 64);
      }
    }
  }

  // One three-qubit update: band, E, the warp 8x8 polar (warm-started from
  // the gate's previous rotation yp), the operators, the fused pass.
  static __device__ __noinline__ void update8(C* T, C* LRs, double2* sm8, double2* g, float2* yp, int4 d,
                                              int n, bool forward, double beta, int* bad) {
    const w8::L8 L;
    const int p0 = n - 1 - d.y, p1 = n - 1 - d.z, p2 = n - 1 - d.w;
    double2 P0, P1;
    band8(T, n, p0, p1, p2, L, P0, P1);
    const double2 u0 = g[L.g * 8 + L.j], u1 = g[(L.g + 4) * 8 + L.j];
    double2 E0, E1;
    if (forward)
      w8::mm8_dn(L, u0, u1, P0, P1, E0, E1);  // u^dagger P
    else
      w8::mm8_nd(L, P0, P1, u0, u1, E0, E1);  // P u^dagger
    double2 ud0 = u0, ud1 = u1;
    w8::dag8(L, ud0, ud1);
    double2 A0 = E0, A1 = E1;
    if (beta != 0.0) {
      A0 = make_double2((1.0 - beta) * E0.x + beta * ud0.x, (1.0 - beta) * E0.y + beta * ud0.y);
      A1 = make_double2((1.0 - beta) * E1.x + beta * ud1.x, (1.0 - beta) * E1.y + beta * ud1.y);
    }
    double2 n0, n1;
    double sg = 0.0;
    if (!w8::warp_polar8(A0, A1, sm8, &n0, &n1, &sg, yp)) {
      *bad = 1;
      n0 = u0;  // keep the old gate: the tensor stays consistent
      n1 = u1;
    }
    __syncwarp();
    g[L.g * 8 + L.j] = n0;
    g[(L.g + 4) * 8 + L.j] = n1;
    LRs[L.g * 8 + L.j] = cmake(forward ? ud0 : n0, R());
    LRs[(L.g + 4) * 8 + L.j] = cmake(forward ? ud1 : n1, R());
    LRs[64 + L.g * 8 + L.j] = cmake(forward ? n0 : ud0, R());
    LRs[64 + (L.g + 4) * 8 + L.j] = cmake(forward ? n1 : ud1, R());
    __syncwarp();
    pass8<true, true>(T, n, p0, p1, p2, LRs, LRs + 64);
  }

  // TwoSidedSweep (Alg. 1) over the mixed circuit.
  static __device__ __noinline__ void sweep(C* T, C* LRs, float2* scratch, double2* sm8, double2* g,
                                            float2* yp, const int4* gk, const int* goff, int n, int p,
                                            double beta, const Lane& L, int* bad) {
    for (int h = 0; h < 2; ++h)
      for (int i = 0; i < p; ++i) {
        const int k = h == 0 ? p - 1 - i : i;
        const int4 d = gk[k];
        if (d.x == 3)
          update8(T, LRs, sm8, g + goff[k], yp + goff[k], d, n, h == 1, beta, bad);
        else
          W<R>::update(T, LRs, scratch, g + goff[k], yp + goff[k], make_int2(d.y, d.z), n, h == 1, beta, L,
                       bad);
      }
  }
};

// Re-unitarisation of a mixed circuit: three FP64 Newton-Schulz steps per gate.
__device__ void reunitarize_k(double2* g, const int4* gk, const int* goff, int p, const Lane& L) {
  for (int k = 0; k < p; ++k) {
    double2* gp = g + goff[k];
    if (gk[k].x == 3) {
      const w8::L8 L8;
      double2 u0 = gp[L8.g * 8 + L8.j], u1 = gp[(L8.g + 4) * 8 + L8.j];
      for (int step = 0; step < 3; ++step) {
        double2 P0, P1;
        w8::mm8_dn(L8, u0, u1, u0, u1, P0, P1);
        const double2 Q0 = make_double2((L8.g == L8.j ? 1.5 : 0.0) - 0.5 * P0.x, -0.5 * P0.y);
        const double2 Q1 = make_double2((L8.g + 4 == L8.j ? 1.5 : 0.0) - 0.5 * P1.x, -0.5 * P1.y);
        w8::mm8(L8, u0, u1, Q0, Q1, u0, u1);
      }
      __syncwarp();
      gp[L8.g * 8 + L8.j] = u0;
      gp[(L8.g + 4) * 8 + L8.j] = u1;
      __syncwarp();
    } else {
      const int e = L.l & 15;
      double2 u = gp[e];
      for (int step = 0; step < 3; ++step) {
        const double2 P = wmm_dn(L, u, u);
        const double2 Q = make_double2((L.i == L.j ? 1.5 : 0.0) - 0.5 * P.x, -0.5 * P.y);
        u = wmm(L, u, Q);
      }
      __syncwarp();
      if (L.l < 16) gp[e] = u;
      __syncwarp();
    }
  }
}

// Steps of a circuit of 2- and 3-qubit gates (gate k: gk[k], entries from goff[k]).
struct OpsK {
  double2* gates;
  float2* yprev;
  const double2* targets;
  const int4* all_gk;
  const int* all_goff;
  const int* inst_ge;
  double beta;
  void* T;
  double2* LR;      // 128 x 16 B: the pass operators
  double2* sm8;     // 128 x 16 B: scratch of the 8x8 update
  float2* scratch;  // 32 x 8 B
  Lane L;
  const double2* V;
  double2* g;
  float2* yp;
  const int4* gk;
  const int* goff;
  int n, p;
  __device__ __forceinline__ OpsK(const BatchParamsK& b, void* t, double2* lr, double2* s8, float2* sc)
      : gates(b.b.gates), yprev(b.b.yprev), targets(b.b.targets), all_gk(b.gk), all_goff(b.goff),
        inst_ge(b.inst_ge), beta(b.b.beta), T(t), LR(lr), sm8(s8), scratch(sc) {}
  __device__ __forceinline__ void load(const BatchInst& in, int i, int s) {
    const int ge = inst_ge[i];
    n = in.n;
    p = in.p;
    g = gates + in.gate_off + (long long)s * ge;
    yp = yprev + in.gate_off + (long long)s * ge;
    V = targets + in.tgt_off;
    gk = all_gk + in.loc_off;
    goff = all_goff + in.loc_off;
    for (int k = 0; k < p; ++k) {  // warm-start rotations: the identity
      if (gk[k].x == 2) {
        if (L.l < 16) yp[goff[k] + L.l] = make_float2(L.i == L.j ? 1.f : 0.f, 0.f);
      } else {
        yp[goff[k] + L.l] = make_float2((L.l >> 3) == (L.l & 7) ? 1.f : 0.f, 0.f);
        yp[goff[k] + L.l + 32] = make_float2(((L.l + 32) >> 3) == (L.l & 7) ? 1.f : 0.f, 0.f);
      }
    }
  }
  template <typename R>
  __device__ __forceinline__ void build() {
    typedef typename Cplx<R>::T C;
    WK<R>::build((C*)T, (C*)LR, V, g, gk, goff, n, p, L);
  }
  template <typename R>
  __device__ __forceinline__ void sweep(int* bad) {
    typedef typename Cplx<R>::T C;
    WK<R>::sweep((C*)T, (C*)LR, scratch, sm8, g, yp, gk, goff, n, p, beta, L, bad);
  }
  __device__ __forceinline__ void reunit() { reunitarize_k(g, gk, goff, p, L); }
};

__global__ void __maxnreg__(168) batched_k_kernel(BatchParamsK pk) {
  extern __shared__ __align__(256) unsigned char smem[];
  unsigned char* ws = smem + (size_t)(threadIdx.x >> 5) * pk.b.warp_bytes;
  unsigned char* after = ws + pk.b.tmax_bytes;
  OpsK ops(pk, ws, reinterpret_cast<double2*>(after), reinterpret_cast<double2*>(after + 2048),
           reinterpret_cast<float2*>(after + 4096));
  run_problems(pk.b, ops, ws, reinterpret_cast<double*>(after + 4352));  // ring: kRing x 8 B
}

// ------------------------------------------------------------------ host

struct DevMem {
  void* p = nullptr;
  ~DevMem() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t b) { return cudaMalloc(&p, b ? b : 16); }
};

bool is_dev(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Autotuner: warps per CTA chosen by timing a short run (two sweeps of a
// prefix of the problems) for every candidate that fits in shared memory,
// cached per (largest qubit count, precision).
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int>, int> g_tuned;

cudaError_t launch_batch(const BatchParams& bp, int wpc, int smem_limit, cudaStream_t st,
                         int* ctas_out) {
  const int smem = wpc * bp.warp_bytes;
  cudaError_t e = cudaFuncSetAttribute(batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem_limit);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel, 32 * wpc, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long problems = (long long)bp.n_inst * bp.S;
  long long ctas = (long long)sm_count() * per_sm;
  const long long need = (problems + wpc - 1) / wpc;
  if (ctas > need) ctas = need;
  if (ctas < 1) ctas = 1;
  if (ctas_out) *ctas_out = (int)ctas;
  batched_kernel<<<(unsigned)ctas, 32 * wpc, smem, st>>>(bp);
  return cudaGetLastError();
}

cudaError_t launch_batch_k(const BatchParamsK& pk, int wpc, int smem_limit, cudaStream_t st,
                           int* ctas_out) {
  const int smem = wpc * pk.b.warp_bytes;
  cudaError_t e = cudaFuncSetAttribute(batched_k_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem_limit);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_k_kernel, 32 * wpc, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long problems = (long long)pk.b.n_inst * pk.b.S;
  long long ctas = (long long)sm_count() * per_sm;
  const long long need = (problems + wpc - 1) / wpc;
  if (ctas > need) ctas = need;
  if (ctas < 1) ctas = 1;
  if (ctas_out) *ctas_out = (int)ctas;
  batched_k_kernel<<<(unsigned)ctas, 32 * wpc, smem, st>>>(pk);
  return cudaGetLastError();
}

}  // namespace
}  // namespace qf

using namespace qf;

namespace {

// The batched call for circuits of two-qubit gates (`locations`) or of two-
// and three-qubit gates (`klocations`, the mixed kernel); exactly one is set.
int batched_impl(int n_instances, const int32_t* n_qubits, const int32_t* n_gates,
                 const qf_loc* locations, const qf_gate_loc* klocations, const qf_c128* targets,
                 int n_starts, const qf_c128* initial_gates, const qf_options* opts, qf_c128* out_gates,
                 double* out_costs, int32_t* out_sweeps, int32_t* out_best, qf_batch_stats* stats,
                 void* stream) {
  const bool kmode = klocations != nullptr;
  qf_options o;
  qf_options_default(&o);
  if (opts) o = *opts;
  if (n_instances < 1 || n_starts < 1)
    return qf_internal_set_error(QF_EINVAL, "n_instances and n_starts must be >= 1", "");
  if (!n_qubits || !n_gates || !(locations || klocations) || !targets || !initial_gates || !out_gates ||
      !out_costs)
    return qf_internal_set_error(QF_EINVAL, "NULL argument", "");
  if (o.max_sweeps < 1) return qf_internal_set_error(QF_EINVAL, "max_sweeps must be >= 1", "");
  if (o.precision == QF_DF64 || o.precision == QF_C64_REFINE_DF)
    return qf_internal_set_error(QF_EINVAL, "the batched kernel takes QF_C128, QF_C64 or QF_C64_REFINE64", "");
  if (o.precision != QF_C128 && o.precision != QF_C64 && o.precision != QF_C64_REFINE64)
    return qf_internal_set_error(QF_EINVAL, "unknown precision", "");
  if (!(o.beta >= 0.0 && o.beta <= 1.0))
    return qf_internal_set_error(QF_EINVAL, "beta outside [0, 1]", "");
  if (o.long_diff_count < 0 || o.long_diff_count >= kRing)
    return qf_internal_set_error(QF_EINVAL, "long_diff_count must be in [0, 127] here", "");
  // sizes and offsets (host arrays)
  std::vector<BatchInst> inst(n_instances);
  long long loc_total = 0;
  for (int i = 0; i < n_instances; ++i) {
    const int n = n_qubits[i], p = n_gates[i];
    if (n < QF_MIN_QUBITS || n > QF_BATCH_MAX_QUBITS)
      return qf_internal_set_error(QF_EINVAL, "an instance's qubit count is outside [2, QF_BATCH_MAX_QUBITS]", "");
    if (p < 1) return qf_internal_set_error(QF_EINVAL, "an instance has no gates", "");
    loc_total += p;
  }
  // locations to the host for validation
  std::vector<qf_loc> hl(kmode ? 0 : loc_total);
  std::vector<qf_gate_loc> hk(kmode ? loc_total : 0);
  {
    void* dst = kmode ? (void*)hk.data() : (void*)hl.data();
    const void* src = kmode ? (const void*)klocations : (const void*)locations;
    const size_t bytes = (kmode ? sizeof(qf_gate_loc) : sizeof(qf_loc)) * loc_total;
    if (is_dev(src)) {
      if (cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
        return qf_internal_set_error(QF_ECUDA, "copying locations failed", "");
    } else {
      memcpy(dst, src, bytes);
    }
  }
  std::vector<int4> hgk(kmode ? loc_total : 0);
  std::vector<int> hgoff(kmode ? loc_total : 0), hge(n_instances);
  long long tgt_total = 0, gate_total = 0, lo = 0;
  int nmax = 0;
  for (int i = 0; i < n_instances; ++i) {
    const int n = n_qubits[i], p = n_gates[i];
    int ge = 0;
    for (int k = 0; k < p; ++k) {
      if (kmode) {
        const qf_gate_loc l = hk[lo + k];
        if (l.k != 2 && l.k != 3)
          return qf_internal_set_error(QF_EINVAL, "the batched call takes gates of 2 or 3 qubits", "");
        for (int a = 0; a < l.k; ++a) {
          if (l.q[a] < 0 || l.q[a] >= n)
            return qf_internal_set_error(QF_EINVAL, "an instance has an invalid location", "");
          for (int b = 0; b < a; ++b)
            if (l.q[a] == l.q[b])
              return qf_internal_set_error(QF_EINVAL, "an instance has a repeated qubit", "");
        }
        if (l.k > n) return qf_internal_set_error(QF_EINVAL, "a gate has more qubits than its instance", "");
        hgk[lo + k] = make_int4(l.k, l.q[0], l.q[1], l.k == 3 ? l.q[2] : 0);
        hgoff[lo + k] = ge;
        ge += 1 << (2 * l.k);
      } else {
        const qf_loc l = hl[lo + k];
        if (l.a < 0 || l.a >= n || l.b < 0 || l.b >= n || l.a == l.b)
          return qf_internal_set_error(QF_EINVAL, "an instance has an invalid location", "");
        ge += 16;
      }
    }
    hge[i] = ge;
    inst[i] = BatchInst{n, p, lo, tgt_total, gate_total};
    lo += p;
    tgt_total += 1ll << (2 * n);
    gate_total += (long long)n_starts * ge;
    if (n > nmax) nmax = n;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const long long problems = (long long)n_instances * n_starts;
  // device buffers
  // hand out the biggest instances first (work ~ 4^n * p per sweep), so the
  // last warps to finish hold short problems
  std::vector<int> order(n_instances);
  for (int i = 0; i < n_instances; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return ((long long)hge[x] << (2 * inst[x].n)) > ((long long)hge[y] << (2 * inst[y].n));
  });
  DevMem d_inst, d_order, d_locs, d_tgt, d_gates, d_yprev, d_cost, d_sw, d_c64, d_reason, d_flags,
      d_hist, d_gk, d_goff, d_ge;
  const size_t hist_row = (size_t)o.max_sweeps + 1;
  const size_t hist_bytes = sizeof(double) * (size_t)problems * hist_row;
  double* hist_dev = nullptr;  // where the kernel writes the cost history
  if (o.cost_history) {
    if (is_dev(o.cost_history)) {
      hist_dev = o.cost_history;
    } else {
      if (d_hist.alloc(hist_bytes) != cudaSuccess) {
        cudaGetLastError();
        return qf_internal_set_error(QF_ENOMEM, "device allocation for the cost history failed", "");
      }
      hist_dev = (double*)d_hist.p;
    }
  }
  if (d_inst.alloc(sizeof(BatchInst) * n_instances) != cudaSuccess ||
      d_order.alloc(sizeof(int) * n_instances) != cudaSuccess ||
      d_locs.alloc(kmode ? 16 : sizeof(qf_loc) * loc_total) != cudaSuccess ||
      d_gk.alloc(kmode ? sizeof(int4) * loc_total : 16) != cudaSuccess ||
      d_goff.alloc(kmode ? sizeof(int) * loc_total : 16) != cudaSuccess ||
      d_ge.alloc(kmode ? sizeof(int) * n_instances : 16) != cudaSuccess ||
      d_tgt.alloc(sizeof(double2) * tgt_total) != cudaSuccess ||
      d_gates.alloc(sizeof(double2) * gate_total) != cudaSuccess ||
      d_yprev.alloc(sizeof(float2) * gate_total) != cudaSuccess ||
      d_cost.alloc(sizeof(double) * problems) != cudaSuccess ||
      d_sw.alloc(sizeof(int) * problems) != cudaSuccess ||
      d_c64.alloc(sizeof(int) * problems) != cudaSuccess ||
      d_reason.alloc(sizeof(int) * problems) != cudaSuccess ||
      d_flags.alloc(sizeof(int) * (2 * (size_t)n_instances + 2)) != cudaSuccess) {
    cudaGetLastError();
    return qf_internal_set_error(QF_ENOMEM, "device allocation for the batch failed", "");
  }
  cudaError_t e = cudaMemcpyAsync(d_inst.p, inst.data(), sizeof(BatchInst) * n_instances,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_order.p, order.data(), sizeof(int) * n_instances, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !kmode)
    e = cudaMemcpyAsync(d_locs.p, hl.data(), sizeof(qf_loc) * loc_total, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && kmode)
    e = cudaMemcpyAsync(d_gk.p, hgk.data(), sizeof(int4) * loc_total, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && kmode)
    e = cudaMemcpyAsync(d_goff.p, hgoff.data(), sizeof(int) * loc_total, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && kmode)
    e = cudaMemcpyAsync(d_ge.p, hge.data(), sizeof(int) * n_instances, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_tgt.p, targets, sizeof(double2) * tgt_total, cudaMemcpyDefault, st);
  if (e != cudaSuccess)
    return qf_internal_set_error(QF_ECUDA, "copying the batch inputs failed", cudaGetErrorString(e));

  BatchParams bp;
  bp.inst = (const BatchInst*)d_inst.p;
  bp.order = (const int*)d_order.p;
  bp.n_inst = n_instances;
  bp.S = n_starts;
  bp.locs = (const int2*)d_locs.p;
  bp.targets = (const double2*)d_tgt.p;
  bp.gates = (double2*)d_gates.p;
  bp.yprev = (float2*)d_yprev.p;
  bp.cost_out = (double*)d_cost.p;
  bp.sweeps_out = (int*)d_sw.p;
  bp.c64_out = (int*)d_c64.p;
  bp.reason_out = (int*)d_reason.p;
  int* flags = (int*)d_flags.p;
  bp.conv_flag = flags;
  bp.plat_count = flags + n_instances;
  bp.status = flags + 2 * n_instances;
  bp.work = (unsigned*)(flags + 2 * n_instances + 1);
  bp.dist_tol = o.dist_tol;
  bp.diff_a = o.diff_tol_a;
  bp.diff_r = o.diff_tol_r;
  bp.long_r = o.long_diff_r;
  bp.beta = o.beta;
  bp.switch_tol = o.switch_tol;
  bp.max_sweeps = o.max_sweeps;
  bp.min_sweeps = o.min_sweeps;
  bp.reset_iter = o.reset_iter;
  bp.long_L = o.long_diff_count;
  bp.precision = o.precision;
  bp.max_c64 = o.max_c64_sweeps;
  bp.hist = hist_dev;
  bp.hist_row = (int)hist_row;
  bp.tmax_bytes = (1 << (2 * nmax)) * 16;
  // after the tensor: operators, scratch and the cost ring (the mixed kernel
  // also keeps 8x8 operators and the 8x8 polar's scratch)
  bp.warp_bytes = ((bp.tmax_bytes + (kmode ? 4352 : 768) + kRing * 8) + 255) & ~255;
  BatchParamsK pk;
  pk.gk = (const int4*)d_gk.p;
  pk.goff = (const int*)d_goff.p;
  pk.inst_ge = (const int*)d_ge.p;
  const size_t flag_bytes = sizeof(int) * (2 * (size_t)n_instances + 2);

  int dev = 0, smem_optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int max_wpc = smem_optin / bp.warp_bytes;
  if (max_wpc < 1)
    return qf_internal_set_error(QF_EINVAL, "the largest instance does not fit in shared memory", "");
  const auto launch = [&](const BatchParams& b, int wpc_, cudaStream_t s_, int* ctas_) {
    if (!kmode) return launch_batch(b, wpc_, smem_optin, s_, ctas_);
    pk.b = b;
    return launch_batch_k(pk, wpc_, smem_optin, s_, ctas_);
  };

  // choose warps per CTA
  int wpc = 0;
  const auto key = std::make_tuple(nmax | (kmode ? 256 : 0), o.precision, dev);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) wpc = it->second;
  }
  if (wpc == 0 || wpc > max_wpc) {
    float best_ms = 1e30f;
    BatchParams tp = bp;
    tp.max_sweeps = 2;
    tp.hist = nullptr;
    tp.n_inst = (int)std::min<long long>(n_instances, std::max<long long>(1, 4096 / n_starts));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int cand : {1, 2, 4, 8}) {
      if (cand > max_wpc) break;
      e = cudaMemcpyAsync(d_gates.p, initial_gates, sizeof(double2) * gate_total, cudaMemcpyDefault, st);
      if (e == cudaSuccess) e = cudaMemsetAsync(d_flags.p, 0, flag_bytes, st);
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      if (e == cudaSuccess) e = launch(tp, cand, st, nullptr);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) break;
      if (ms < best_ms) {
        best_ms = ms;
        wpc = cand;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess)
      return qf_internal_set_error(QF_ECUDA, "autotuning launch failed", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tuned[key] = wpc;
  }

  // the run: reset, then one persistent launch, captured as a CUDA graph
  nvtxRangePushA("qf batched run");
  struct PopAtExit {
    ~PopAtExit() { nvtxRangePop(); }
  } pop_at_exit;
  e = cudaMemcpyAsync(d_gates.p, initial_gates, sizeof(double2) * gate_total, cudaMemcpyDefault, st);
  if (e != cudaSuccess)
    return qf_internal_set_error(QF_ECUDA, "copying the initial gates failed", cudaGetErrorString(e));
  cudaStream_t cap = nullptr;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
    return qf_internal_set_error(QF_ECUDA, "stream creation failed", "");
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int ctas = 0;
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e1 = cudaMemsetAsync(d_flags.p, 0, flag_bytes, cap);
    // all-ones bytes are a NaN: entries after a start's last sweep
    if (e1 == cudaSuccess && hist_dev) e1 = cudaMemsetAsync(hist_dev, 0xff, hist_bytes, cap);
    cudaError_t e2 = e1 == cudaSuccess ? launch(bp, wpc, cap, &ctas) : e1;
    e = cudaStreamEndCapture(cap, &graph);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  cudaEvent_t k0 = nullptr, k1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&k0);
  if (e == cudaSuccess) e = cudaEventCreate(&k1);
  if (e == cudaSuccess) e = cudaEventRecord(k0, st);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
  if (e == cudaSuccess) e = cudaEventRecord(k1, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float kms = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&kms, k0, k1);
  if (k0) cudaEventDestroy(k0);
  if (k1) cudaEventDestroy(k1);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess)
    return qf_internal_set_error(QF_ECUDA, "batched launch failed", cudaGetErrorString(e));

  // outputs
  std::vector<int> hsw(problems), hreason(problems), hc64(problems);
  int hstatus = 0;
  e = cudaMemcpy(out_costs, d_cost.p, sizeof(double) * problems, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(hsw.data(), d_sw.p, sizeof(int) * problems, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(&hstatus, bp.status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(hc64.data(), d_c64.p, sizeof(int) * problems, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(out_gates, d_gates.p, sizeof(double2) * gate_total, cudaMemcpyDefault);
  if (e == cudaSuccess && hist_dev && hist_dev != o.cost_history)
    e = cudaMemcpy(o.cost_history, hist_dev, hist_bytes, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess)
    return qf_internal_set_error(QF_ECUDA, "copying the batch results failed", cudaGetErrorString(e));
  if (out_sweeps)
    for (long long q = 0; q < problems; ++q) out_sweeps[q] = hsw[q];
  if (out_best)
    for (int i = 0; i < n_instances; ++i) {
      int b = 0;
      for (int s = 1; s < n_starts; ++s)
        if (out_costs[(long long)i * n_starts + s] < out_costs[(long long)i * n_starts + b]) b = s;
      out_best[i] = b;
    }
  if (stats) {
    stats->warps_per_cta = wpc;
    stats->ctas = ctas;
    stats->kernel_ms = kms;
    long long c64 = 0, sw = 0;
    for (long long q = 0; q < problems; ++q) {
      c64 += hc64[q];
      sw += hsw[q];
    }
    stats->total_sweeps = sw;
    stats->total_c64_sweeps = c64;
  }
  if (hstatus != 0)
    return qf_internal_set_error(QF_ENONFINITE, "an environment or update was not finite", "");
  return QF_OK;
}

}  // namespace

extern "C" int qf_instantiate_batched(int n_instances, const int32_t* n_qubits,
                                      const int32_t* n_gates, const qf_loc* locations,
                                      const qf_c128* targets, int n_starts,
                                      const qf_c128* initial_gates, const qf_options* opts,
                                      qf_c128* out_gates, double* out_costs, int32_t* out_sweeps,
                                      int32_t* out_best, qf_batch_stats* stats, void* stream) {
  if (!locations) return qf_internal_set_error(QF_EINVAL, "NULL argument", "");
  return batched_impl(n_instances, n_qubits, n_gates, locations, nullptr, targets, n_starts,
                      initial_gates, opts, out_gates, out_costs, out_sweeps, out_best, stats, stream);
}

extern "C" int qf_instantiate_batched_k(int n_instances, const int32_t* n_qubits,
                                        const int32_t* n_gates, const qf_gate_loc* locations,
                                        const qf_c128* targets, int n_starts,
                                        const qf_c128* initial_gates, const qf_options* opts,
                                        qf_c128* out_gates, double* out_costs, int32_t* out_sweeps,
                                        int32_t* out_best, qf_batch_stats* stats, void* stream) {
  if (!locations) return qf_internal_set_error(QF_EINVAL, "NULL argument", "");
  return batched_impl(n_instances, n_qubits, n_gates, nullptr, locations, targets, n_starts,
                      initial_gates, opts, out_gates, out_costs, out_sweeps, out_best, stats, stream);
}
