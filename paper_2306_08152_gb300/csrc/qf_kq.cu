// Three-qubit gates (k = 3) for the QFactor sweep on sm_103a: the fused
// pass, the environment with its 8x8 update, and the 8x8 polar.
//
// The paper states the method for two-qubit gates and notes that it extends
// to k-qubit unitaries, whose environment is 2^k x 2^k (Sec. III).  A gate
// on qubits (q0, q1, q2) touches bit positions p_i = n-1-q_i of the row and
// column index; its local index is 4*bit(p0) + 2*bit(p1) + bit(p2).  The 64
// entries that share every other row and column bit form an 8x8 block B,
// and the fused update of Alg. 1 is B <- L B R, exactly as for 4x4 blocks.

#include <string.h>

#include <type_traits>

#include "qf_device.cuh"
#include "qf_internal.h"
#include "qf_warp8.cuh"

namespace qf {
namespace {

using namespace dev;

// The warp 8x8 math (lane layout, products, Jacobi, warp polar) is in
// qf_warp8.cuh.
using namespace w8;

// ------------------------------------------------------------------ pass
//
// B <- L B R on every 8x8 block.  A warp handles 4 blocks; lane 4x + b holds
// row x of block b (consecutive blocks take consecutive column rest
// indices, so a warp access covers 4 adjacent columns of 8 rows).  R acts
// along the row in registers; the rows then go through a padded per-warp
// shared buffer so that lane 4y + b takes column y for L, and writes it.
// Used for complex128 and df64, whose arithmetic bounds the pass; complex64
// takes pass8a_kernel or pass8f_kernel (below).

// Offset of local index v of a gate on bit positions (p0, p1, p2).
__device__ __forceinline__ unsigned off8(int v, int p0, int p1, int p2) {
  return (((unsigned)v >> 2) & 1u) << p0 | (((unsigned)v >> 1) & 1u) << p1 | ((unsigned)v & 1u) << p2;
}

constexpr int kPass8Threads = 256;
constexpr int kBlkStride = 8 * 9 + 4;  // padded 8x8 block in the transpose buffer

template <typename R, bool HL, bool HR>
__global__ void __launch_bounds__(kPass8Threads)
pass8_kernel(typename Cplx<R>::T* __restrict__ T, int n, int p0, int p1, int p2,
             const double2* __restrict__ L, long long Ls, const double2* __restrict__ Rm,
             long long Rs) {
  typedef typename Cplx<R>::T C;
  __shared__ C sL[64], sR[64];
  __shared__ C buf[kPass8Threads / 32][4 * kBlkStride];
  const int s = blockIdx.y;
  if (threadIdx.x < 64) {
    if (HL) sL[threadIdx.x] = cmake(L[s * Ls + threadIdx.x], R());
    if (HR) sR[threadIdx.x] = cmake(Rm[s * Rs + threadIdx.x], R());
  }
  __syncthreads();
  const unsigned N = 1u << n;
  int q[3] = {p0, p1, p2};  // ascending for the deposit
  if (q[0] > q[1]) { const int t = q[0]; q[0] = q[1]; q[1] = t; }
  if (q[1] > q[2]) { const int t = q[1]; q[1] = q[2]; q[2] = t; }
  if (q[0] > q[1]) { const int t = q[0]; q[0] = q[1]; q[1] = t; }
  unsigned off[8];  // constant indices only (a lane-dependent index would move it to local memory)
#pragma unroll
  for (int x = 0; x < 8; ++x) off[x] = off8(x, p0, p1, p2);
  const int lnc = n - 3;
  const unsigned cmask = (1u << lnc) - 1u;
  const unsigned nblk = 1u << (2 * lnc);
  C* __restrict__ Ts = T + (size_t)s * N * N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = lane & 3, x = lane >> 2;
  const unsigned offx = off8(x, p0, p1, p2);
  C* wb = buf[w];
  const unsigned warps = gridDim.x * (kPass8Threads / 32);
  for (unsigned grp = blockIdx.x * (kPass8Threads / 32) + w; grp * 4u < nblk; grp += warps) {
    const unsigned blk = grp * 4u + (unsigned)b;
    const bool valid = blk < nblk;
    const unsigned r0 = dep1(dep1(dep1(blk >> lnc, q[0]), q[1]), q[2]);
    const unsigned c0 = dep1(dep1(dep1(blk & cmask, q[0]), q[1]), q[2]);
    C row[8];
    if (valid) {
      const C* src = Ts + (size_t)(r0 | offx) * N + c0;
#pragma unroll
      for (int y = 0; y < 8; ++y) row[y] = src[off[y]];
    } else {
#pragma unroll
      for (int y = 0; y < 8; ++y) row[y] = czero<C>();
    }
    if (HR) {  // row <- row R
      C t[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        C acc = czero<C>();
#pragma unroll
        for (int k = 0; k < 8; ++k) acc = cfma(row[k], sR[k * 8 + c], acc);
        t[c] = cfinish(acc);
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) row[c] = t[c];
    }
    if (HL) {
#pragma unroll
      for (int y = 0; y < 8; ++y) wb[b * kBlkStride + x * 9 + y] = row[y];
      __syncwarp();
      const int y = x;  // this lane now takes column y of block b
      C col[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) col[k] = wb[b * kBlkStride + k * 9 + y];
      __syncwarp();  // the buffer is rewritten by the next group
      if (valid) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          C acc = czero<C>();
#pragma unroll
          for (int k = 0; k < 8; ++k) acc = cfma(sL[r * 8 + k], col[k], acc);
          Ts[(size_t)(r0 | off[r]) * N + (c0 | offx)] = cfinish(acc);
        }
      }
    } else if (valid) {
      C* dst = Ts + (size_t)(r0 | offx) * N + c0;
#pragma unroll
      for (int y = 0; y < 8; ++y) dst[off[y]] = row[y];
    }
  }
}

// complex64 version for the FP32 pipe.  The old layout spends one broadcast
// shared load of an operator entry per complex multiply-add, which puts the
// shared-memory pipe near its limit; here a lane takes row x of two blocks
// (b and b + 4 of an 8-block group), so every operator entry loaded serves
// two rows.  The R stage writes each output column straight to the
// transpose buffer and the L stage each output row straight to global
// memory, so a lane holds only its two input rows (80 registers: three
// CTAs of eight warps per SM).  Without L the lane reads its own rows back
// from the buffer.  (Loading the next group's rows ahead of the arithmetic
// needs 123 registers, two CTAs per SM, and ran slower.)
constexpr int kPass8fBlocks = 8;  // blocks per warp and group

struct Grp8 {  // one block of a group: its row and column rest offsets
  unsigned r0, c0;
  bool valid;
};

constexpr int kPass8fCtasPerSm = 3;

template <bool HL, bool HR>
__global__ void __launch_bounds__(kPass8Threads, kPass8fCtasPerSm)
pass8f_kernel(float2* __restrict__ T, int n, int p0, int p1, int p2, const double2* __restrict__ L,
              long long Ls, const double2* __restrict__ Rm, long long Rs) {
  __shared__ float2 sL[64], sR[64];
  __shared__ float2 buf[kPass8Threads / 32][kPass8fBlocks * kBlkStride];
  const int s = blockIdx.y;
  if (threadIdx.x < 64) {
    if (HL) sL[threadIdx.x] = cmake(L[s * Ls + threadIdx.x], 0.f);
    if (HR) sR[threadIdx.x] = cmake(Rm[s * Rs + threadIdx.x], 0.f);
  }
  __syncthreads();
  const unsigned N = 1u << n;
  int q[3] = {p0, p1, p2};  // ascending for the deposit
  if (q[0] > q[1]) { const int t = q[0]; q[0] = q[1]; q[1] = t; }
  if (q[1] > q[2]) { const int t = q[1]; q[1] = q[2]; q[2] = t; }
  if (q[0] > q[1]) { const int t = q[0]; q[0] = q[1]; q[1] = t; }
  const unsigned m0 = 1u << p0, m1 = 1u << p1, m2 = 1u << p2;
  // offset of local index v (a compile-time constant at every use)
  auto off = [&](int v) { return ((v & 4) ? m0 : 0u) | ((v & 2) ? m1 : 0u) | ((v & 1) ? m2 : 0u); };
  const int lnc = n - 3;
  const unsigned cmask = (1u << lnc) - 1u;
  const unsigned nblk = 1u << (2 * lnc);
  float2* __restrict__ Ts = T + (size_t)s * N * N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = lane & 3, x = lane >> 2;
  const unsigned offx = off8(x, p0, p1, p2);  // offset of this lane's row (R stage) / column (L stage)
  float2* wb = buf[w];
  const unsigned warps = gridDim.x * (kPass8Threads / 32);
  auto locate = [&](unsigned grp, int h) {
    const unsigned blk = grp * kPass8fBlocks + (unsigned)(b + 4 * h);
    Grp8 g;
    g.valid = blk < nblk;
    g.r0 = dep1(dep1(dep1(blk >> lnc, q[0]), q[1]), q[2]);
    g.c0 = dep1(dep1(dep1(blk & cmask, q[0]), q[1]), q[2]);
    return g;
  };
  auto load = [&](const Grp8& g, float2* row) {
    if (g.valid) {
      const float2* src = Ts + (size_t)(g.r0 | offx) * N + g.c0;
#pragma unroll
      for (int y = 0; y < 8; ++y) row[y] = src[off(y)];
    } else {
#pragma unroll
      for (int y = 0; y < 8; ++y) row[y] = make_float2(0.f, 0.f);
    }
  };
  unsigned grp = blockIdx.x * (kPass8Threads / 32) + w;
  for (; grp * kPass8fBlocks < nblk; grp += warps) {
    const Grp8 cg[2] = {locate(grp, 0), locate(grp, 1)};
    float2 row[2][8];
    load(cg[0], row[0]);
    load(cg[1], row[1]);
    // R stage (or the plain row) into the transpose buffer, column by column
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      float2 a0 = row[0][c], a1 = row[1][c];
      if (HR) {
        a0 = a1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float2 r = sR[k * 8 + c];
          a0 = cfma(row[0][k], r, a0);
          a1 = cfma(row[1][k], r, a1);
        }
      }
      wb[b * kBlkStride + x * 9 + c] = a0;
      wb[(b + 4) * kBlkStride + x * 9 + c] = a1;
    }
    __syncwarp();
    if (HL) {  // L stage: this lane takes column x of blocks b and b + 4
      float2 col[2][8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        col[0][k] = wb[b * kBlkStride + k * 9 + x];
        col[1][k] = wb[(b + 4) * kBlkStride + k * 9 + x];
      }
      __syncwarp();  // the buffer is rewritten by the next group
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        float2 a0 = make_float2(0.f, 0.f), a1 = a0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float2 l = sL[r * 8 + k];
          a0 = cfma(l, col[0][k], a0);
          a1 = cfma(l, col[1][k], a1);
        }
        if (cg[0].valid) Ts[(size_t)(cg[0].r0 | off(r)) * N + (cg[0].c0 | offx)] = a0;
        if (cg[1].valid) Ts[(size_t)(cg[1].r0 | off(r)) * N + (cg[1].c0 | offx)] = a1;
      }
    } else {  // R only: the lane reads its own output rows back and writes them
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float2 o[8];
#pragma unroll
        for (int y = 0; y < 8; ++y) o[y] = wb[(b + 4 * h) * kBlkStride + x * 9 + y];
        if (cg[h].valid) {
          float2* dst = Ts + (size_t)(cg[h].r0 | offx) * N + cg[h].c0;
#pragma unroll
          for (int y = 0; y < 8; ++y) dst[off(y)] = o[y];
        }
      }
      __syncwarp();  // the buffer is rewritten by the next group
    }
  }
}

// complex64 pass for n >= 7, used when every gate bit is >= 2.  A warp
// takes 16 blocks (lane b) with the same rest row and 16 consecutive rest
// columns, and a lane the rows x = xh, xh + 2, xh + 4, xh + 6 (xh = lane /
// 16).  With every gate bit >= 4 the low four column bits are rest bits, so
// the 16 columns a warp access takes in one row are 16 adjacent entries (a
// whole 128-byte line); with the lowest gate bit at 2 or 3 they fall in runs
// of 4 or 8 adjacent entries.  (Gates on bit 0 or 1 leave runs of one or two
// entries; those take pass8c_kernel, or pass8f_kernel with a bit above 5.)
// Every broadcast operator entry serves four rows.  The R stage (the identity without R)
// writes each output column to the transpose buffer; the L stage reads
// columns y = xh + 2j back and writes each output row to global memory.
// The buffer pads each block to 65 slots, so both the column writes and the
// column reads of a warp hit every bank pair exactly twice.  (Used with L;
// the R-only pass goes to pass8f_kernel.)
constexpr int kPass8aThreads = 128;
constexpr int kPass8aCtasPerSm = 4;
constexpr int kBlkA = 65;

// Operators as pairs of adjacent entries for 16-byte shared loads (each
// load serves two output columns or rows): R2[k][c/2] = (R[k][c], R[k][c+1]),
// LT2[k][r/2] = (L[r][k], L[r+1][k]).  Threads 0..31 fill entry t of each.
__device__ __forceinline__ void load_op_pairs8(float4* R2, float4* LT2, const double2* L,
                                               const double2* Rm, bool hr) {
  const int t = threadIdx.x;
  if (t < 32) {
    const int k = t >> 2, c2 = (t & 3) * 2;
    const double2 l0 = L[c2 * 8 + k], l1 = L[(c2 + 1) * 8 + k];
    LT2[t] = make_float4((float)l0.x, (float)l0.y, (float)l1.x, (float)l1.y);
    if (hr) {
      const double2 r0 = Rm[k * 8 + c2], r1 = Rm[k * 8 + c2 + 1];
      R2[t] = make_float4((float)r0.x, (float)r0.y, (float)r1.x, (float)r1.y);
    }
  }
}

template <bool HR>
__global__ void __launch_bounds__(kPass8aThreads, kPass8aCtasPerSm)
pass8a_kernel(float2* __restrict__ T, int n, int p0, int p1, int p2, const double2* __restrict__ L,
              long long Ls, const double2* __restrict__ Rm, long long Rs) {
  __shared__ float4 sR2[32], sLT2[32];
  __shared__ float2 buf[kPass8aThreads / 32][16 * kBlkA];
  const int s = blockIdx.y;
  load_op_pairs8(sR2, sLT2, L + s * Ls, HR ? Rm + s * Rs : nullptr, HR);
  __syncthreads();
  const unsigned N = 1u << n;
  int q[3] = {p0, p1, p2};  // ascending for the deposit
  if (q[0] > q[1]) { const int t = q[0]; q[0] = q[1]; q[1] = t; }
  if (q[1] > q[2]) { const int t = q[1]; q[1] = q[2]; q[2] = t; }
  if (q[0] > q[1]) { const int t = q[0]; q[0] = q[1]; q[1] = t; }
  const unsigned m0 = 1u << p0, m1 = 1u << p1, m2 = 1u << p2;
  auto off = [&](int v) { return ((v & 4) ? m0 : 0u) | ((v & 2) ? m1 : 0u) | ((v & 1) ? m2 : 0u); };
  const int cgb = n - 7;  // bits of the 16-column group index within a rest row
  const unsigned ngrp = 1u << (2 * (n - 3) - 4);
  float2* __restrict__ Ts = T + (size_t)s * N * N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = lane & 15, xh = lane >> 4;
  const unsigned ox = xh ? m2 : 0u;  // off(xh + 2i) = ox | off(2i)
  float2* wb = buf[w] + b * kBlkA;
  for (unsigned g = blockIdx.x * (kPass8aThreads / 32) + w; g < ngrp;
       g += gridDim.x * (kPass8aThreads / 32)) {
    const unsigned rr = g >> cgb, cc = ((g & ((1u << cgb) - 1u)) << 4) | (unsigned)b;
    const unsigned r0 = dep1(dep1(dep1(rr, q[0]), q[1]), q[2]);
    const unsigned c0 = dep1(dep1(dep1(cc, q[0]), q[1]), q[2]);
    float2 v[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int y = 0; y < 8; ++y) v[i][y] = Ts[(size_t)(r0 | ox | off(2 * i)) * N + (c0 | off(y))];
    if (HR) {  // kept rolled: the fully unrolled group body overflows the instruction cache
#pragma unroll 1
      for (int c = 0; c < 8; c += 2) {
        float2 a[4], b2[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = b2[i] = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float4 r = sR2[k * 4 + c / 2];
          const float2 r0 = make_float2(r.x, r.y), r1 = make_float2(r.z, r.w);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            a[i] = cfma(v[i][k], r0, a[i]);
            b2[i] = cfma(v[i][k], r1, b2[i]);
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          wb[(xh + 2 * i) * 8 + c] = a[i];
          wb[(xh + 2 * i) * 8 + c + 1] = b2[i];
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int i = 0; i < 4; ++i) wb[(xh + 2 * i) * 8 + c] = v[i][c];
    }
    {
      __syncwarp();
      float2 col[4][8];
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int k = 0; k < 8; ++k) col[j][k] = wb[k * 8 + xh + 2 * j];
      __syncwarp();  // the buffer is rewritten by the next group
#pragma unroll 1
      for (int r = 0; r < 8; r += 2) {
        float2 a[4], b2[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) a[j] = b2[j] = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float4 l = sLT2[k * 4 + r / 2];
          const float2 l0 = make_float2(l.x, l.y), l1 = make_float2(l.z, l.w);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            a[j] = cfma(l0, col[j][k], a[j]);
            b2[j] = cfma(l1, col[j][k], b2[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          Ts[(size_t)(r0 | off(r)) * N + (c0 | ox | off(2 * j))] = a[j];
          Ts[(size_t)(r0 | off(r + 1)) * N + (c0 | ox | off(2 * j))] = b2[j];
        }
      }
    }
  }
}

// complex64 pass for gates with every bit <= 5 (n >= 6) that pass8a_kernel
// does not take: a bit at 0 or 1, where the layouts above touch 8-16 lines
// per warp access, or n = 6.  A warp
// takes a tile of the 8 row variants of one rest row and 64 adjacent
// columns (8 blocks: the tile holds every column variant of 8 rest
// columns), loads and stores it with 16-byte accesses of whole lines (lane
// l: columns 2l, 2l+1), and moves it through shared memory:
//   R stage  lane (j, xa) = (l & 7, l >> 3) takes rows xa and xa + 4 of
//            block j, in place;
//   L stage  lane l takes columns 2l and 2l+1 of every row and writes the
//            output rows to global memory.
// Each broadcast operator entry serves two rows or two columns.  The
// shared tile is XOR-swizzled per launch: slot(x, c) = 64x + (c & 48) +
// ((c & 15) ^ phi), phi = Px(x & 3) ^ Qh(c >> 4), with (P, Q) GF(2)-linear
// and chosen on the host so that every warp access above (fixed y in the R
// stage, fixed row in the others) hits each 8-byte bank pair exactly twice
// (pass8c_swizzle).
constexpr int kPass8cThreads = 128;
constexpr int kPass8cCtasPerSm = 4;

template <bool HR>
__global__ void __launch_bounds__(kPass8cThreads, kPass8cCtasPerSm)
pass8c_kernel(float2* __restrict__ T, int n, int p0, int p1, int p2, const double2* __restrict__ L,
              long long Ls, const double2* __restrict__ Rm, long long Rs, unsigned phx, unsigned phh) {
  __shared__ float4 sR2[32], sLT2[32];
  __shared__ float2 buf[kPass8cThreads / 32][512];
  const int s = blockIdx.y;
  load_op_pairs8(sR2, sLT2, L + s * Ls, HR ? Rm + s * Rs : nullptr, HR);
  __syncthreads();
  const unsigned N = 1u << n;
  int q[3] = {p0, p1, p2};  // ascending for the deposit
  if (q[0] > q[1]) { const int t = q[0]; q[0] = q[1]; q[1] = t; }
  if (q[1] > q[2]) { const int t = q[1]; q[1] = q[2]; q[2] = t; }
  if (q[0] > q[1]) { const int t = q[0]; q[0] = q[1]; q[1] = t; }
  const unsigned m0 = 1u << p0, m1 = 1u << p1, m2 = 1u << p2;
  auto off = [&](int v) { return ((v & 4) ? m0 : 0u) | ((v & 2) ? m1 : 0u) | ((v & 1) ? m2 : 0u); };
  auto slot = [&](int x, unsigned c) {
    const unsigned phi = ((phx >> (4 * (x & 3))) ^ (phh >> (4 * (c >> 4)))) & 15u;
    return x * 64 + (int)(c & 48u) + (int)((c & 15u) ^ phi);
  };
  const int ctb = n - 6;  // bits of the 64-column tile index
  const unsigned ntiles = 1u << (2 * n - 9);
  float2* __restrict__ Ts = T + (size_t)s * N * N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float2* tb = buf[w];
  const int j = lane & 7, xa = lane >> 3;
  const unsigned cj = dep1(dep1(dep1((unsigned)j, q[0]), q[1]), q[2]);  // block j's rest bits
  for (unsigned g = blockIdx.x * (kPass8cThreads / 32) + w; g < ntiles;
       g += gridDim.x * (kPass8cThreads / 32)) {
    const unsigned rr = g >> ctb, t = g & ((1u << ctb) - 1u);
    const unsigned r0 = dep1(dep1(dep1(rr, q[0]), q[1]), q[2]);
    const size_t cb = (size_t)t * 64 + 2 * lane;
    {  // load: rows x, columns 2 lane and 2 lane + 1
      float4 v[8];
#pragma unroll
      for (int x = 0; x < 8; ++x) v[x] = *reinterpret_cast<const float4*>(Ts + (size_t)(r0 | off(x)) * N + cb);
#pragma unroll
      for (int x = 0; x < 8; ++x) {
        tb[slot(x, 2u * lane)] = make_float2(v[x].x, v[x].y);
        tb[slot(x, 2u * lane + 1u)] = make_float2(v[x].z, v[x].w);
      }
    }
    __syncwarp();
    if (HR) {  // rows xa and xa + 4 of block j <- row R; every slot here is this lane's
      float2 ia[8], ib[8];
#pragma unroll
      for (int y = 0; y < 8; ++y) {
        const unsigned c = cj | off(y);
        ia[y] = tb[slot(xa, c)];
        ib[y] = tb[slot(xa + 4, c)];
      }
#pragma unroll 1
      for (int c = 0; c < 8; c += 2) {
        float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
#pragma unroll
        for (int y = 0; y < 8; ++y) {
          const float4 r = sR2[y * 4 + c / 2];
          const float2 r0 = make_float2(r.x, r.y), r1 = make_float2(r.z, r.w);
          a0 = cfma(ia[y], r0, a0);
          a1 = cfma(ia[y], r1, a1);
          b0 = cfma(ib[y], r0, b0);
          b1 = cfma(ib[y], r1, b1);
        }
        const unsigned cc0 = cj | off(c), cc1 = cj | off(c + 1);
        tb[slot(xa, cc0)] = a0;
        tb[slot(xa, cc1)] = a1;
        tb[slot(xa + 4, cc0)] = b0;
        tb[slot(xa + 4, cc1)] = b1;
      }
      __syncwarp();
    }
    float2 ce[8], co[8];  // columns 2 lane and 2 lane + 1 of every row
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      ce[k] = tb[slot(k, 2u * lane)];
      co[k] = tb[slot(k, 2u * lane + 1u)];
    }
    __syncwarp();  // the buffer is rewritten by the next tile
#pragma unroll 1
    for (int r = 0; r < 8; r += 2) {
      float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float4 l = sLT2[k * 4 + r / 2];
        const float2 l0 = make_float2(l.x, l.y), l1 = make_float2(l.z, l.w);
        a0 = cfma(l0, ce[k], a0);
        b0 = cfma(l0, co[k], b0);
        a1 = cfma(l1, ce[k], a1);
        b1 = cfma(l1, co[k], b1);
      }
      *reinterpret_cast<float4*>(Ts + (size_t)(r0 | off(r)) * N + cb) = make_float4(a0.x, a0.y, b0.x, b0.y);
      *reinterpret_cast<float4*>(Ts + (size_t)(r0 | off(r + 1)) * N + cb) = make_float4(a1.x, a1.y, b1.x, b1.y);
    }
  }
}

// The swizzle of pass8c_kernel for gate bits (p0, p1, p2), all <= 5: the
// first (P, Q) in a fixed order such that (a) some column-tile bit (c >> 4)
// flips bank bit 0, which spreads a row's even (or odd) columns over all 16
// banks, and (b) the map from (block j, row xa & 3) to banks in the R stage
// has rank 4 over GF(2), i.e. hits each bank exactly twice.  Returned as
// nibble tables: phx = Px(x) for x = 0..3, phh = Qh(h) for h = 0..3.
bool pass8c_swizzle(int p0, int p1, int p2, unsigned* phx, unsigned* phh) {
  int rest[3], nr = 0;
  for (int b = 0; b < 6; ++b)
    if (b != p0 && b != p1 && b != p2 && nr < 3) rest[nr++] = b;
  if (nr != 3) return false;
  for (unsigned P0 = 0; P0 < 16; ++P0)
    for (unsigned P1 = 0; P1 < 16; ++P1)
      for (unsigned Q0 = 0; Q0 < 16; ++Q0)
        for (unsigned Q1 = 0; Q1 < 16; ++Q1) {
          if (!((Q0 | Q1) & 1u)) continue;
          const unsigned Qc[2] = {Q0, Q1};
          unsigned cols[5];
          for (int i = 0; i < 3; ++i) cols[i] = rest[i] < 4 ? 1u << rest[i] : Qc[rest[i] - 4];
          cols[3] = P0;
          cols[4] = P1;
          unsigned basis[4];
          int rank = 0;
          for (int i = 0; i < 5; ++i) {
            unsigned v = cols[i];
            for (int k = 0; k < rank; ++k) v = (v ^ basis[k]) < v ? v ^ basis[k] : v;
            if (v) basis[rank++] = v;
          }
          if (rank != 4) continue;
          *phx = 0u;
          *phh = 0u;
          for (unsigned x = 0; x < 4; ++x)
            *phx |= (((x & 1u) ? P0 : 0u) ^ ((x & 2u) ? P1 : 0u)) << (4 * x);
          for (unsigned h = 0; h < 4; ++h)
            *phh |= (((h & 1u) ? Q0 : 0u) ^ ((h & 2u) ? Q1 : 0u)) << (4 * h);
          return true;
        }
  return false;
}

// pass8c_swizzle for every bit triple, computed once; false if a bit is
// above 5 (or the triple has no swizzle, which the search does not meet).
bool pass8c_tables(int p0, int p1, int p2, unsigned* phx, unsigned* phh) {
  struct Tab {
    unsigned x[6][6][6], h[6][6][6];
    bool ok[6][6][6];
  };
  static const Tab tab = [] {
    Tab t{};
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 6; ++b)
        for (int c = 0; c < 6; ++c)
          t.ok[a][b][c] = a != b && a != c && b != c && pass8c_swizzle(a, b, c, &t.x[a][b][c], &t.h[a][b][c]);
    return t;
  }();
  if (p0 < 0 || p1 < 0 || p2 < 0 || p0 > 5 || p1 > 5 || p2 > 5 || !tab.ok[p0][p1][p2]) return false;
  *phx = tab.x[p0][p1][p2];
  *phh = tab.h[p0][p1][p2];
  return true;
}

// ------------------------------------------------------------ environment
//
// P[x][y] = sum over the 2^(n-3) rests r of T[(r, x), (r, y)], from the
// tensor before the gate's removal (E = P u^dagger backward, u^dagger P
// forward), as for two-qubit gates.  Items are (rest, x); a thread sums its
// items' 8 entries y in the tensor's accumulation precision, the warp folds
// its 4 rests per x with two shuffles, the CTA adds its warps in order and
// writes 128 partial sums; the last CTA of the start (atomic ticket) adds
// the CTAs' partials in a fixed order and runs the 8x8 update on one warp.

constexpr int kEnv8Threads = 128;

template <typename R>
__global__ void __launch_bounds__(kEnv8Threads)
env8_kernel(const typename Cplx<R>::T* __restrict__ T, int n, int p0, int p1, int p2, int mode,
            double2* __restrict__ gates_k, long long gstride, double beta, double2* __restrict__ LR,
            double2* __restrict__ out, long long out_stride, double* __restrict__ sigma_out,
            int* __restrict__ status, double* __restrict__ part, unsigned* __restrict__ counters) {
  using CT = typename Cplx<R>::T;
  using Ar = typename Acc<R>::T;
  __shared__ double red[kEnv8Threads / 32][8][16];
  __shared__ double2 sm[160];  // P, then the polar's scratch
  __shared__ bool is_last;
  const int s = blockIdx.y, B = gridDim.x, bb = blockIdx.x;
  const unsigned N = 1u << n;
  int q[3] = {p0, p1, p2};
  if (q[0] > q[1]) { const int t = q[0]; q[0] = q[1]; q[1] = t; }
  if (q[1] > q[2]) { const int t = q[1]; q[1] = q[2]; q[2] = t; }
  if (q[0] > q[1]) { const int t = q[0]; q[0] = q[1]; q[1] = t; }
  unsigned off[8];  // constant indices only
#pragma unroll
  for (int x = 0; x < 8; ++x) off[x] = off8(x, p0, p1, p2);
  const unsigned items = N;  // 2^(n-3) rests x 8 rows
  const unsigned chunk = ((items / 8u + B - 1) / B) * 8u;  // whole rests per CTA
  const unsigned i_beg = bb * chunk;
  const unsigned i_end = min(items, i_beg + chunk);
  const CT* Ts = T + (size_t)s * N * N;
  Ar v[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = Ar(0);
  const int x = threadIdx.x & 7;  // blockDim and chunk are multiples of 8
  const unsigned offx = off8(x, p0, p1, p2);
  for (unsigned it = i_beg + threadIdx.x; it < i_end; it += blockDim.x) {
    const unsigned d = dep1(dep1(dep1(it >> 3, q[0]), q[1]), q[2]);
    const CT* rowp = Ts + (size_t)(d | offx) * N + d;
#pragma unroll
    for (int y = 0; y < 8; ++y) {
      const auto e = to_acc(rowp[off[y]]);
      v[2 * y] += e.x;
      v[2 * y + 1] += e.y;
    }
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    v[i] += __shfl_xor_sync(kFull, v[i], 8);
    v[i] += __shfl_xor_sync(kFull, v[i], 16);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane < 8)
#pragma unroll
    for (int i = 0; i < 16; ++i) red[wid][lane][i] = (double)v[i];
  __syncthreads();
  if (threadIdx.x < 128) {
    const int xx = threadIdx.x >> 4, c = threadIdx.x & 15;
    double acc = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) acc += red[k][xx][c];
    part[((size_t)s * B + bb) * 128 + threadIdx.x] = acc;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned ticket = atomicAdd(&counters[s], 1u);
    is_last = (ticket == (unsigned)B - 1u);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  if (threadIdx.x < 128) {  // P[x][y] component c = 2y (+1 for the imaginary part)
    double acc = 0.0;
    for (int k = 0; k < B; ++k) acc += __ldcg(&part[((size_t)s * B + k) * 128 + threadIdx.x]);
    reinterpret_cast<double*>(sm)[threadIdx.x] = acc;
  }
  if (threadIdx.x == 0) counters[s] = 0u;
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const L8 L;
  const double2 P0 = sm[L.g * 8 + L.j], P1 = sm[(L.g + 4) * 8 + L.j];
  __syncwarp();
  if (mode == kTraceOnly) {
    out[s * out_stride + L.g * 8 + L.j] = P0;
    out[s * out_stride + (L.g + 4) * 8 + L.j] = P1;
    return;
  }
  double2 u0 = gates_k[s * gstride + L.g * 8 + L.j], u1 = gates_k[s * gstride + (L.g + 4) * 8 + L.j];
  double2 E0, E1;
  if (mode == kForward)
    mm8_dn(L, u0, u1, P0, P1, E0, E1);  // u^dagger P
  else
    mm8_nd(L, P0, P1, u0, u1, E0, E1);  // P u^dagger
  if (out) {
    out[s * out_stride + L.g * 8 + L.j] = E0;
    out[s * out_stride + (L.g + 4) * 8 + L.j] = E1;
  }
  double2 ud0 = u0, ud1 = u1;
  dag8(L, ud0, ud1);
  double2* lr = LR + (size_t)s * 128;
  if (mode == kEnvOnly) {
    lr[L.g * 8 + L.j] = u0;
    lr[(L.g + 4) * 8 + L.j] = u1;
    lr[64 + L.g * 8 + L.j] = ud0;
    lr[64 + (L.g + 4) * 8 + L.j] = ud1;
    return;
  }
  double2 A0 = E0, A1 = E1;
  if (beta != 0.0) {
    A0 = make_double2((1.0 - beta) * E0.x + beta * ud0.x, (1.0 - beta) * E0.y + beta * ud0.y);
    A1 = make_double2((1.0 - beta) * E1.x + beta * ud1.x, (1.0 - beta) * E1.y + beta * ud1.y);
  }
  double2 n0, n1;
  double sg = 0.0;
  if (!warp_polar8(A0, A1, sm, &n0, &n1, &sg)) {
    if (L.l == 0) atomicCAS(status, 0, -4);
    n0 = u0;  // keep the old gate: the tensor stays consistent
    n1 = u1;
    sg = 0.0;
  }
  gates_k[s * gstride + L.g * 8 + L.j] = n0;
  gates_k[s * gstride + (L.g + 4) * 8 + L.j] = n1;
  const bool bwd = mode == kBackward;
  lr[L.g * 8 + L.j] = bwd ? n0 : ud0;
  lr[(L.g + 4) * 8 + L.j] = bwd ? n1 : ud1;
  lr[64 + L.g * 8 + L.j] = bwd ? ud0 : n0;
  lr[64 + (L.g + 4) * 8 + L.j] = bwd ? ud1 : n1;
  if (sigma_out && L.l == 0) sigma_out[s] = sg;
}

// One warp per 8x8 matrix.
__global__ void __launch_bounds__(128) optimize8_kernel(const double2* __restrict__ E,
                                                        const double2* __restrict__ u_old,
                                                        double beta, int count,
                                                        double2* __restrict__ u_out,
                                                        double* __restrict__ sigma_out) {
  __shared__ double2 sm[4][128];
  const int wid = threadIdx.x >> 5;
  const int m = blockIdx.x * 4 + wid;
  if (m >= count) return;  // whole warps leave together
  const L8 L;
  const double2* e = E + (size_t)m * 64;
  double2 a0 = e[L.g * 8 + L.j], a1 = e[(L.g + 4) * 8 + L.j];
  if (beta != 0.0) {
    double2 d0 = u_old[(size_t)m * 64 + L.g * 8 + L.j], d1 = u_old[(size_t)m * 64 + (L.g + 4) * 8 + L.j];
    dag8(L, d0, d1);
    a0 = make_double2((1.0 - beta) * a0.x + beta * d0.x, (1.0 - beta) * a0.y + beta * d0.y);
    a1 = make_double2((1.0 - beta) * a1.x + beta * d1.x, (1.0 - beta) * a1.y + beta * d1.y);
  }
  double2 u0, u1;
  double sg;
  if (!warp_polar8(a0, a1, sm[wid], &u0, &u1, &sg)) {
    u0 = u1 = make_double2(NAN, NAN);
    sg = NAN;
  }
  u_out[(size_t)m * 64 + L.g * 8 + L.j] = u0;
  u_out[(size_t)m * 64 + (L.g + 4) * 8 + L.j] = u1;
  if (sigma_out && L.l == 0) sigma_out[m] = sg;
}

// Three FP64 Newton-Schulz steps u <- u (3I - u^dagger u) / 2 per 8x8 gate.
__global__ void __launch_bounds__(128) reunitarize8_kernel(double2* __restrict__ gates, int count) {
  const int m = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (m >= count) return;
  const L8 L;
  double2* gp = gates + (size_t)m * 64;
  double2 u0 = gp[L.g * 8 + L.j], u1 = gp[(L.g + 4) * 8 + L.j];
  for (int step = 0; step < 3; ++step) {
    double2 P0, P1;
    mm8_dn(L, u0, u1, u0, u1, P0, P1);
    const double2 Q0 = make_double2((L.g == L.j ? 1.5 : 0.0) - 0.5 * P0.x, -0.5 * P0.y);
    const double2 Q1 = make_double2((L.g + 4 == L.j ? 1.5 : 0.0) - 0.5 * P1.x, -0.5 * P1.y);
    mm8(L, u0, u1, Q0, Q1, u0, u1);
  }
  gp[L.g * 8 + L.j] = u0;
  gp[(L.g + 4) * 8 + L.j] = u1;
}

// Re-unitarisation of a circuit with 4x4 and 8x8 gates: warp m takes gate
// m % p of start m / p; desc[k] = (size, entry offset); three FP64
// Newton-Schulz steps each.
__global__ void __launch_bounds__(128) reunitarize_mixed_kernel(double2* __restrict__ gates, long long gsz,
                                                                const int2* __restrict__ desc, int p,
                                                                int count) {
  const int m = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (m >= count) return;  // whole warps leave together
  const int s = m / p, k = m % p;
  const int2 d = desc[k];
  if (d.x == 4) return;  // 16x16 gates: reunitarize16_kernel
  double2* gp = gates + (size_t)s * gsz + d.y;
  if (d.x == 3) {
    const L8 L;
    double2 u0 = gp[L.g * 8 + L.j], u1 = gp[(L.g + 4) * 8 + L.j];
    for (int step = 0; step < 3; ++step) {
      double2 P0, P1;
      mm8_dn(L, u0, u1, u0, u1, P0, P1);
      const double2 Q0 = make_double2((L.g == L.j ? 1.5 : 0.0) - 0.5 * P0.x, -0.5 * P0.y);
      const double2 Q1 = make_double2((L.g + 4 == L.j ? 1.5 : 0.0) - 0.5 * P1.x, -0.5 * P1.y);
      mm8(L, u0, u1, Q0, Q1, u0, u1);
    }
    gp[L.g * 8 + L.j] = u0;
    gp[(L.g + 4) * 8 + L.j] = u1;
  } else {
    const Lane L;
    const int e = L.l & 15;
    double2 u = gp[e];
    for (int step = 0; step < 3; ++step) {
      const double2 P = wmm_dn(L, u, u);
      const double2 Q = make_double2((L.i == L.j ? 1.5 : 0.0) - 0.5 * P.x, -0.5 * P.y);
      u = wmm(L, u, Q);
    }
    if (L.l < 16) gp[e] = u;
  }
}

// Grids of the complex64 passes: kPass8Waves times the resident CTAs, so
// that CTAs retire throughout the pass and a higher-priority environment
// kernel of the other start group finds SM room while the pass runs.
constexpr int kPass8Waves = 8;

template <typename R, bool HL, bool HR>
void pass8_launch(void* T, int n, int S, int p0, int p1, int p2, const double2* L, long long Ls,
                  const double2* Rm, long long Rs, cudaStream_t st) {
  typedef typename Cplx<R>::T C;
  const long long groups = ((1ll << (2 * (n - 3))) + 3) / 4;
  const long long want = (groups + 7) / 8;
  long long cap = ((long long)sm_count() * 4 + S - 1) / S;
  if (cap < 1) cap = 1;
  dim3 grid((unsigned)(want < cap ? want : cap), S);
  if constexpr (std::is_same<R, float>::value) {
    unsigned phx = 0, phh = 0;
    if (HL && n >= 7 && p0 >= 2 && p1 >= 2 && p2 >= 2) {
      const long long agroups = 1ll << (2 * (n - 3) - 4);
      const long long awant = (agroups + 3) / 4;
      long long acap = ((long long)sm_count() * kPass8aCtasPerSm * kPass8Waves + S - 1) / S;
      if (acap < 1) acap = 1;
      dim3 agrid((unsigned)(awant < acap ? awant : acap), S);
      pass8a_kernel<HR><<<agrid, kPass8aThreads, 0, st>>>((float2*)T, n, p0, p1, p2, L, Ls, Rm, Rs);
    } else if (HL && n >= 6 && pass8c_tables(p0, p1, p2, &phx, &phh)) {
      const long long ctiles = 1ll << (2 * n - 9);
      const long long cwant = (ctiles + 3) / 4;
      long long ccap = ((long long)sm_count() * kPass8cCtasPerSm * kPass8Waves + S - 1) / S;
      if (ccap < 1) ccap = 1;
      dim3 cgrid((unsigned)(cwant < ccap ? cwant : ccap), S);
      pass8c_kernel<HR><<<cgrid, kPass8cThreads, 0, st>>>((float2*)T, n, p0, p1, p2, L, Ls, Rm, Rs, phx, phh);
    } else {
      const long long fgroups = ((1ll << (2 * (n - 3))) + kPass8fBlocks - 1) / kPass8fBlocks;
      const long long fwant = (fgroups + 7) / 8;
      long long fcap = ((long long)sm_count() * kPass8fCtasPerSm * kPass8Waves + S - 1) / S;
      if (fcap < 1) fcap = 1;
      dim3 fgrid((unsigned)(fwant < fcap ? fwant : fcap), S);
      pass8f_kernel<HL, HR><<<fgrid, kPass8Threads, 0, st>>>((float2*)T, n, p0, p1, p2, L, Ls, Rm, Rs);
    }
  } else
    pass8_kernel<R, HL, HR><<<grid, kPass8Threads, 0, st>>>((C*)T, n, p0, p1, p2, L, Ls, Rm, Rs);
}

template <typename R>
void pass8_ops(void* T, int n, int S, int p0, int p1, int p2, const double2* L, long long Ls,
               const double2* Rm, long long Rs, cudaStream_t st) {
  if (L && Rm)
    pass8_launch<R, true, true>(T, n, S, p0, p1, p2, L, Ls, Rm, Rs, st);
  else if (L)
    pass8_launch<R, true, false>(T, n, S, p0, p1, p2, L, Ls, Rm, Rs, st);
  else if (Rm)
    pass8_launch<R, false, true>(T, n, S, p0, p1, p2, L, Ls, Rm, Rs, st);
}

}  // namespace

// ================================================================ launchers

cudaError_t launch_pass8(void* T, int n, int S, const int* q, const double2* L, long long Ls,
                         const double2* R, long long Rs, int prec, cudaStream_t st) {
  if (!L && !R) return cudaSuccess;
  const int p0 = qubit_bit(n, q[0]), p1 = qubit_bit(n, q[1]), p2 = qubit_bit(n, q[2]);
  if (prec == 0)
    pass8_ops<double>(T, n, S, p0, p1, p2, L, Ls, R, Rs, st);
  else if (prec == 2)
    pass8_ops<DF>(T, n, S, p0, p1, p2, L, Ls, R, Rs, st);
  else
    pass8_ops<float>(T, n, S, p0, p1, p2, L, Ls, R, Rs, st);
  return cudaGetLastError();
}

cudaError_t launch_update8(const void* T, int n, int S, const int* q, double2* gates_k,
                           long long gstride, int mode, double beta, double2* LR, double2* out,
                           long long out_stride, double* sigma_out, int* status, double* part,
                           unsigned* counters, int prec, cudaStream_t st) {
  const int p0 = qubit_bit(n, q[0]), p1 = qubit_bit(n, q[1]), p2 = qubit_bit(n, q[2]);
  dim3 grid(env_ctas(n), S);
  if (prec == 0)
    env8_kernel<double><<<grid, kEnv8Threads, 0, st>>>((const double2*)T, n, p0, p1, p2, mode, gates_k,
                                                       gstride, beta, LR, out, out_stride, sigma_out,
                                                       status, part, counters);
  else if (prec == 2)
    env8_kernel<DF><<<grid, kEnv8Threads, 0, st>>>((const dfc*)T, n, p0, p1, p2, mode, gates_k, gstride,
                                                   beta, LR, out, out_stride, sigma_out, status, part,
                                                   counters);
  else
    env8_kernel<float><<<grid, kEnv8Threads, 0, st>>>((const float2*)T, n, p0, p1, p2, mode, gates_k,
                                                      gstride, beta, LR, out, out_stride, sigma_out,
                                                      status, part, counters);
  return cudaGetLastError();
}

cudaError_t launch_optimize8(const double2* E, const double2* u_old, double beta, int count,
                             double2* u_out, double* sigma_out, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  optimize8_kernel<<<(count + 3) / 4, 128, 0, st>>>(E, u_old, beta, count, u_out, sigma_out);
  return cudaGetLastError();
}

cudaError_t launch_reunitarize_mixed(double2* gates, long long gsz, const int2* desc, int p, int S,
                                     cudaStream_t st) {
  const int count = p * S;
  if (count <= 0) return cudaSuccess;
  reunitarize_mixed_kernel<<<(count + 3) / 4, 128, 0, st>>>(gates, gsz, desc, p, count);
  return cudaGetLastError();
}

cudaError_t launch_reunitarize8(double2* gates, int count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  reunitarize8_kernel<<<(count + 3) / 4, 128, 0, st>>>(gates, count);
  return cudaGetLastError();
}

}  // namespace qf
