// Gate-application kernels of the QFactor sweep for sm_103a: the initial
// conjugate transpose, the fused pass B <- L B R, the trace, and helpers.
//
// Layout: a circuit tensor T is N x N row-major (N = 2^n), interleaved
// complex (float2 for complex64, double2 for complex128); start s occupies
// entries [s*N*N, (s+1)*N*N).  Qubit q is bit n-1-q of a row index and of a
// column index, so a gate on (a, b) touches row bits {pa, pb} and column bits
// {pa, pb} with pa = n-1-a, pb = n-1-b; its local index is 2*bit_pa + bit_pb.
//
// Every 16 entries that share all non-gate row and column bits form one 4x4
// block B (rows x = local row index, columns y = local column index).  The
// fused update of Alg. 1 (remove the old gate on one side, apply the new one
// on the other) is B <- L B R for every block: one read and one write of T.
// The 4x4 work is far too small to be a dense contraction worth tensor
// cores (32 complex FMAs per 16 entries): the complex64 pass is bound by HBM
// and the complex128 pass by the FP64 pipe.

#include <string.h>

#include "qf_device.cuh"
#include "qf_internal.h"

namespace qf {
namespace {

using namespace dev;

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
  for (int j = threadIdx.y; j < 32; j += 8) {
    int r = by + j, c = bx + threadIdx.x;
    if (r < N && c < N) tile[j][threadIdx.x] = V[(size_t)r * N + c];
  }
  __syncthreads();
  typename Cplx<R>::T* Ts = T + (size_t)s * N * N;
  for (int j = threadIdx.y; j < 32; j += 8) {
    int r = bx + j, c = by + threadIdx.x;
    if (r < N && c < N) {
      double2 v = tile[threadIdx.x][j];
      v.y = -v.y;
      Ts[(size_t)r * N + c] = cmake(v, R());
    }
  }
}

constexpr int kPassThreads = 256;

// Resident CTAs per SM the pass kernels are built for: complex64 passes are
// memory-bound and want many bytes in flight, complex128 ones are bound by
// the FP64 pipe at any occupancy, df64 ones need warps to hide the latency
// of their dependent TwoSum chains.  WIDE: the window mapping's larger
// per-thread state.
template <typename R, bool WIDE> struct PassOcc { static constexpr int v = 1; };
template <> struct PassOcc<float, false> { static constexpr int v = 3; };
template <> struct PassOcc<float, true> { static constexpr int v = 2; };
template <> struct PassOcc<DF, false> { static constexpr int v = 1; };
template <> struct PassOcc<DF, true> { static constexpr int v = 1; };

template <typename R, bool HL, bool HR>
__device__ __forceinline__ void load_ops(typename Cplx<R>::T* sL, typename Cplx<R>::T* sR,
                                         const double2* __restrict__ L, long long Ls,
                                         const double2* __restrict__ Rm, long long Rs, int s) {
  if (threadIdx.x < 16) {
    if (HL) sL[threadIdx.x] = cmake(L[s * Ls + threadIdx.x], R());
    if (HR) sR[threadIdx.x] = cmake(Rm[s * Rs + threadIdx.x], R());
  }
  __syncthreads();
}

// ------------------------------------------------------------- the pass
//
// Block mapping: one thread owns one 4x4 block per loop trip, consecutive
// threads taking consecutive values of the column rest index.  Every warp
// load then reads 32 entries that are contiguous, or made of runs of at
// least 4 entries (full 32-byte sectors), whenever the gate's lower column
// bit is bit 2 or above.

template <typename R, bool HL, bool HR>
__global__ void __launch_bounds__(kPassThreads, (PassOcc<R, false>::v))
pass_block_kernel(typename Cplx<R>::T* __restrict__ T, int n, int plo, int phi, int pa, int pb,
                  const double2* __restrict__ L, long long Ls, const double2* __restrict__ Rm,
                  long long Rs) {
  typedef typename Cplx<R>::T C;
  __shared__ C sL[16], sR[16];
  const int s = blockIdx.y;
  load_ops<R, HL, HR>(sL, sR, L, Ls, Rm, Rs, s);

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
        for (int y = 0; y < 4; ++y) t[y] = czero<C>();
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int y = 0; y < 4; ++y) t[y] = cfma(bm[x][k], sR[k * 4 + y], t[y]);
#pragma unroll
        for (int y = 0; y < 4; ++y) bm[x][y] = cfinish(t[y]);
      }
    }
    if (HL) {  // B <- L B, one column at a time
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        C t[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          C acc = czero<C>();
#pragma unroll
          for (int k = 0; k < 4; ++k) acc = cfma(sL[x * 4 + k], bm[k][y], acc);
          t[x] = cfinish(acc);
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

// Half-block mapping (df64): two adjacent lanes share one 4x4 block, the
// even lane holding rows 0-1 and the odd lane rows 2-3.  Each applies R to
// its two rows; one exchange of four entries through shuffles leaves the
// even lane with columns 0-1 and the odd lane with columns 2-3 of all four
// rows, and each applies L to its two columns.  Half the per-thread state of
// the block mapping, so twice the resident warps for the long dependent
// chains of double-FP32 arithmetic.  Blocks are ordered as in the block
// mapping (consecutive lane pairs take consecutive column rest indices).

template <typename R, bool HL, bool HR>
__global__ void __launch_bounds__(kPassThreads, 2)
pass_half_kernel(typename Cplx<R>::T* __restrict__ T, int n, int plo, int phi, int pa, int pb,
                 const double2* __restrict__ L, long long Ls, const double2* __restrict__ Rm,
                 long long Rs) {
  typedef typename Cplx<R>::T C;
  __shared__ C sL[16], sR[16];
  const int s = blockIdx.y;
  load_ops<R, HL, HR>(sL, sR, L, Ls, Rm, Rs, s);

  const unsigned N = 1u << n;
  const int lnc = n - 2;
  const unsigned cmask = (1u << lnc) - 1u;
  const unsigned units = 2u << (2 * lnc);  // two lanes per block: a multiple of 32 (n >= 4)
  C* __restrict__ Ts = T + (size_t)s * N * N;
  const unsigned o1 = 1u << pb, o2 = 1u << pa;
  const unsigned off[4] = {0u, o1, o2, o1 | o2};  // constant indices only
  const int h = threadIdx.x & 1;  // the row pair {2h, 2h+1}
  // off[2h + i] without a lane-dependent index (which would put the arrays
  // in local memory)
  const unsigned oh = h ? o2 : 0u;

  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < units;
       t += gridDim.x * blockDim.x) {
    const unsigned blk = t >> 1;
    const unsigned r0 = dep2(blk >> lnc, plo, phi);
    const unsigned c0 = dep2(blk & cmask, plo, phi);
    C e[2][4];  // rows 2h, 2h+1
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const unsigned rb = (r0 | oh | (i ? o1 : 0u)) * N;
#pragma unroll
      for (int y = 0; y < 4; ++y) e[i][y] = Ts[rb + (c0 | off[y])];
    }
    if (HR) {  // rows <- rows R
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        C t4[4];
#pragma unroll
        for (int y = 0; y < 4; ++y) t4[y] = czero<C>();
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int y = 0; y < 4; ++y) t4[y] = cfma(e[i][k], sR[k * 4 + y], t4[y]);
#pragma unroll
        for (int y = 0; y < 4; ++y) e[i][y] = cfinish(t4[y]);
      }
    }
    if (HL) {
      // exchange: the even lane gives columns 2-3 of its rows and takes
      // columns 0-1 of rows 2-3; the odd lane the mirror image
      C col[4][2];  // all four rows of columns {2h, 2h+1}
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const C give = h ? e[i][j] : e[i][2 + j];
          const C keep = h ? e[i][2 + j] : e[i][j];
          const C got = shfl(give, (int)(threadIdx.x & 31) ^ 1);
          col[i][j] = h ? got : keep;      // row i
          col[2 + i][j] = h ? keep : got;  // row 2 + i
        }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        C t4[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          C acc = czero<C>();
#pragma unroll
          for (int k = 0; k < 4; ++k) acc = cfma(sL[x * 4 + k], col[k][j], acc);
          t4[x] = cfinish(acc);
        }
#pragma unroll
        for (int x = 0; x < 4; ++x) Ts[(r0 | off[x]) * N + (c0 | oh | (j ? o1 : 0u))] = t4[x];
      }
    } else {
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const unsigned rb = (r0 | oh | (i ? o1 : 0u)) * N;
#pragma unroll
        for (int y = 0; y < 4; ++y) Ts[rb + (c0 | off[y])] = e[i][y];
      }
    }
  }
}

// Lane mapping, for gates whose lower column bit is bit 0 or 1 (there the
// block mapping would leave half of every sector to another instruction).
// Lanes own 32 consecutive columns of one row, so every warp load and store
// is one contiguous run.  A thread holds, for its column c and the 4 rows of
// its row block, the entries at c and (MODE 1) at c with the gate's upper
// column bit set; the block partners that differ in a gate column bit
// below 5 live in other lanes and are fetched with shuffles.
//   MODE 1: one gate column bit (lb) below 5, the other (tb) at 5 or above.
//   MODE 2: both gate column bits below 5.

template <typename R, int MODE, bool HL, bool HR>
__global__ void __launch_bounds__(kPassThreads, (PassOcc<R, false>::v))
pass_lane_kernel(typename Cplx<R>::T* __restrict__ T, int n, int plo, int phi, int pa, int pb,
                 const double2* __restrict__ L, long long Ls, const double2* __restrict__ Rm,
                 long long Rs) {
  typedef typename Cplx<R>::T C;
  __shared__ C sL[16], sR[16];
  const int s = blockIdx.y;
  load_ops<R, HL, HR>(sL, sR, L, Ls, Rm, Rs, s);

  const unsigned N = 1u << n;
  C* __restrict__ Ts = T + (size_t)s * N * N;
  const unsigned o1 = 1u << pb, o2 = 1u << pa;
  const unsigned off[4] = {0u, o1, o2, o1 | o2};
  const int lane = threadIdx.x & 31;
  // MODE 1: which gate column bit lives in the lane index
  const bool lb_is_a = (MODE == 1) && (pa < 5);
  const int lb = lb_is_a ? pa : pb;
  const int tb = lb_is_a ? pb : pa;
  const int lcols = (MODE == 1) ? n - 1 : n;  // log2 of column units per row block
  const unsigned units = (N >> 2) << lcols;   // a multiple of 32: whole warps

  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < units;
       t += gridDim.x * blockDim.x) {
    const unsigned tc = t & ((1u << lcols) - 1u);
    const unsigned r0 = dep2(t >> lcols, plo, phi);
    if (MODE == 2) {
      const unsigned c = tc;
      C e[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) e[x] = Ts[(r0 | off[x]) * N + c];
      if (HR) {
        const int yown = 2 * ((c >> pa) & 1) + ((c >> pb) & 1);
        const unsigned cb = (c & ~(o1 | o2)) & 31u;
        C t4[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          C acc = czero<C>();
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const C v = shfl(e[x], (int)(cb | off[k]));
            acc = cfma(v, sR[k * 4 + yown], acc);
          }
          t4[x] = cfinish(acc);
        }
#pragma unroll
        for (int x = 0; x < 4; ++x) e[x] = t4[x];
      }
      if (HL) {
        C t4[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          C acc = czero<C>();
#pragma unroll
          for (int k = 0; k < 4; ++k) acc = cfma(sL[x * 4 + k], e[k], acc);
          t4[x] = cfinish(acc);
        }
#pragma unroll
        for (int x = 0; x < 4; ++x) e[x] = t4[x];
      }
#pragma unroll
      for (int x = 0; x < 4; ++x) Ts[(r0 | off[x]) * N + c] = e[x];
    } else {
      const unsigned c = dep1(tc, tb);
      const unsigned ot = 1u << tb;
      C e[4][2];
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const unsigned rb = (r0 | off[x]) * N;
        e[x][0] = Ts[rb + c];
        e[x][1] = Ts[rb + (c | ot)];
      }
      if (HR) {
        const int lbv = (c >> lb) & 1;
        const int partner = lane ^ (1 << lb);
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const C q0 = shfl(e[x][0], partner), q1 = shfl(e[x][1], partner);
          // B[x][k] for k = 0..3: k's lane bit picks own/partner, its
          // thread bit picks the variant
          C bk[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int kl = lb_is_a ? (k >> 1) : (k & 1);
            const int kt = lb_is_a ? (k & 1) : (k >> 1);
            const C own = kt ? e[x][1] : e[x][0];
            const C oth = kt ? q1 : q0;
            bk[k] = (kl == lbv) ? own : oth;
          }
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            const int y = lb_is_a ? (2 * lbv + v) : (2 * v + lbv);
            C acc = czero<C>();
#pragma unroll
            for (int k = 0; k < 4; ++k) acc = cfma(bk[k], sR[k * 4 + y], acc);
            e[x][v] = cfinish(acc);
          }
        }
      }
      if (HL) {
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          C t4[4];
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            C acc = czero<C>();
#pragma unroll
            for (int k = 0; k < 4; ++k) acc = cfma(sL[x * 4 + k], e[k][v], acc);
            t4[x] = cfinish(acc);
          }
#pragma unroll
          for (int x = 0; x < 4; ++x) e[x][v] = t4[x];
        }
      }
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const unsigned rb = (r0 | off[x]) * N;
        Ts[rb + c] = e[x][0];
        Ts[rb + (c | ot)] = e[x][1];
      }
    }
  }
}

// Window mapping, for gates whose two column bits both lie in bits 0..2
// (the last pairs of a linear brickwork).  A thread owns, in each of the 4
// rows of its row block, the aligned window of W = 4 (bits {0,1}) or W = 8
// entries that contains the gate's column partners, i.e. 1 or 2 whole 4x4
// blocks, and moves it with 32-byte vector loads and stores: consecutive
// threads take consecutive windows, so every warp access is one contiguous
// run of full sectors and no shuffles are needed.  PA and PB are the gate's
// bit positions (pa = n-1-a, pb = n-1-b).

__device__ __forceinline__ void vld32(const float2* p, float2* v) {
  asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(v[0].x), "=f"(v[0].y), "=f"(v[1].x), "=f"(v[1].y), "=f"(v[2].x),
                 "=f"(v[2].y), "=f"(v[3].x), "=f"(v[3].y)
               : "l"(p));
}
__device__ __forceinline__ void vst32(float2* p, const float2* v) {
  asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0].x),
               "f"(v[0].y), "f"(v[1].x), "f"(v[1].y), "f"(v[2].x), "f"(v[2].y), "f"(v[3].x),
               "f"(v[3].y)
               : "memory");
}
__device__ __forceinline__ void vld32(const double2* p, double2* v) {
  asm volatile("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];"
               : "=d"(v[0].x), "=d"(v[0].y), "=d"(v[1].x), "=d"(v[1].y)
               : "l"(p));
}
__device__ __forceinline__ void vst32(double2* p, const double2* v) {
  asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(v[0].x), "d"(v[0].y),
               "d"(v[1].x), "d"(v[1].y)
               : "memory");
}

__device__ __forceinline__ void vld32(const dfc* p, dfc* v) {
  asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(v[0].h.x), "=f"(v[0].h.y), "=f"(v[0].l.x), "=f"(v[0].l.y), "=f"(v[1].h.x),
                 "=f"(v[1].h.y), "=f"(v[1].l.x), "=f"(v[1].l.y)
               : "l"(p));
}
__device__ __forceinline__ void vst32(dfc* p, const dfc* v) {
  asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0].h.x),
               "f"(v[0].h.y), "f"(v[0].l.x), "f"(v[0].l.y), "f"(v[1].h.x), "f"(v[1].h.y),
               "f"(v[1].l.x), "f"(v[1].l.y)
               : "memory");
}

template <typename R, int PA, int PB>
__global__ void __launch_bounds__(kPassThreads, (PassOcc<R, true>::v))
pass_window_kernel(typename Cplx<R>::T* __restrict__ T, int n, const double2* __restrict__ L,
                   long long Ls, const double2* __restrict__ Rm, long long Rs) {
  typedef typename Cplx<R>::T C;
  constexpr int HI = PA > PB ? PA : PB;
  constexpr int W = HI <= 1 ? 4 : 8;          // window entries
  constexpr int NBLK = W / 4;                 // 4x4 blocks per window
  constexpr int FREE = 3 - PA - PB;           // the free bit of an 8-entry window
  constexpr int PER = 32 / (int)sizeof(C);    // entries per 32-byte access
  __shared__ C sL[16], sR[16];
  const int s = blockIdx.y;
  load_ops<R, true, true>(sL, sR, L, Ls, Rm, Rs, s);
  const int lo = PA < PB ? PA : PB;
  const unsigned N = 1u << n;
  const int lw = n - (W == 4 ? 2 : 3);  // log2 windows per row
  const unsigned units = (N >> 2) << lw;
  C* __restrict__ Ts = T + (size_t)s * N * N;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < units;
       t += gridDim.x * blockDim.x) {
    const unsigned r0 = dep2(t >> lw, lo, HI);
    const unsigned cb = (t & ((1u << lw) - 1u)) * W;
    // row bits of the gate sit at the same positions as its column bits
    const unsigned roff[4] = {0u, 1u << PB, 1u << PA, (1u << PA) | (1u << PB)};
    C win[4][W];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const C* row = Ts + (r0 | roff[x]) * N + cb;
#pragma unroll
      for (int v = 0; v < W / PER; ++v) vld32(row + v * PER, &win[x][v * PER]);
    }
#pragma unroll
    for (int b = 0; b < NBLK; ++b) {
      // column position of local index y in block b
#define QF_POS(y) (((((y) >> 1) & 1) << PA) | (((y) & 1) << PB) | (NBLK == 2 ? (b << FREE) : 0))
#pragma unroll
      for (int x = 0; x < 4; ++x) {  // B <- B R
        C t4[4];
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          C acc = czero<C>();
#pragma unroll
          for (int k = 0; k < 4; ++k) acc = cfma(win[x][QF_POS(k)], sR[k * 4 + y], acc);
          t4[y] = cfinish(acc);
        }
#pragma unroll
        for (int y = 0; y < 4; ++y) win[x][QF_POS(y)] = t4[y];
      }
#pragma unroll
      for (int y = 0; y < 4; ++y) {  // B <- L B
        C t4[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          C acc = czero<C>();
#pragma unroll
          for (int k = 0; k < 4; ++k) acc = cfma(sL[x * 4 + k], win[k][QF_POS(y)], acc);
          t4[x] = cfinish(acc);
        }
#pragma unroll
        for (int x = 0; x < 4; ++x) win[x][QF_POS(y)] = t4[x];
      }
#undef QF_POS
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      C* row = Ts + (r0 | roff[x]) * N + cb;
#pragma unroll
      for (int v = 0; v < W / PER; ++v) vst32(row + v * PER, &win[x][v * PER]);
    }
  }
}

// --------------------------------------------------- two gates, one pass
//
// Look-ahead pass for two consecutive updates on disjoint qubit pairs:
// T <- (L1 (x) L2) T (R1 (x) R2), (L1, R1) on bit positions (pa1, pb1) and
// (L2, R2) on (pa2, pb2).  A CTA of 128 threads works on tiles of 16 rows
// (every value of the 4 gate row bits) x 128 columns (every value of the 4
// gate column bits and of the 3 lowest other column bits) = 2048 entries,
// 16 KB of complex64, double-buffered: while one tile is transformed the
// next streams in with 16-byte cp.async copies (bit positions 0..2 are
// always tile columns, so every copy is 16-byte aligned and covers whole
// 64-byte runs).  Four CTAs share an SM, so one CTA's barrier waits overlap
// another's arithmetic.
//   columns  each thread takes the 16 column partners of one (row, window)
//            pair and applies R1 and R2;
//   rows     each thread takes the 16 row partners of one tile column,
//            applies L1 and L2 and writes the results to global memory.
// 16 complex multiply-adds per entry for two updates against one read and
// one write; they run as packed f32x2 FMAs (acc += (b.x,b.x)(a.x,a.y) +
// (-b.y,b.y)(a.y,a.x)), each operator entry loaded once per stage and used
// for four vectors.  Shared memory holds tile columns XOR-swizzled in
// 16-byte units (bits 4..6 of the column into bits 1..3), and odd tile rows
// XOR a per-launch mask into bits 1..3 that spreads the column phase's
// half-warps (8 windows x 2 rows) over the banks.

constexpr int kPairThreads = 128;
constexpr int kPairCols = 128;
constexpr int kPairTileEntries = 16 * kPairCols;
constexpr int kPairChunks = 3;  // 8-bit chunks of the tile index (n <= 18)

// Per-launch geometry, passed by value (constant bank: every lookup below
// is warp-uniform).  Byte offsets are for complex64 entries.
struct PairParams {
  int n;
  int tile_bits;                 // 2n - 11: tiles per start = 2^tile_bits
  int tbit_pos[kPairChunks * 8]; // tile-index bit i -> row (>= 32: 32 + row bit) or column bit
  int tcol_pos[8];               // compressed tile column bit -> global column bit
  int win_cpos[4];               // window bit -> compressed tile column bit (3 used)
  int rxmask;                    // slot XOR of odd tile rows (bank spread)
  int gsw[16];                   // swizzled compressed column of column-local pair (y1, y2)
  int rsm[16];                   // shared-memory byte offset of tile row of pair (x1, x2)
  long long rglob[16];           // global byte offset of the row of pair (x1, x2)
  long long rtile[16];           // global byte offset of tile row t_r
};

__device__ __forceinline__ unsigned pswz(unsigned c) { return c ^ (((c >> 4) & 7u) << 1); }

typedef unsigned long long f32x2;  // two packed floats (x in the low word)

__device__ __forceinline__ f32x2 ffma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f32x2 pswap(f32x2 a) {  // (x, y) -> (y, x)
  float x, y;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a));
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(y), "f"(x));
  return r;
}
__device__ __forceinline__ f32x2 pk2(float x, float y) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}

// Operator entry b as two packed pairs: (b.x, b.x) and (-b.y, b.y).
struct OpE {
  f32x2 re, im;
};
__device__ __forceinline__ OpE load_op(const float4* ops, int i) {
  const float4 v = ops[i];
  return OpE{pk2(v.x, v.y), pk2(v.z, v.w)};
}
// acc += a * b
__device__ __forceinline__ f32x2 cmad2(f32x2 acc, f32x2 a, f32x2 a_sw, OpE b) {
  return ffma2(b.im, a_sw, ffma2(b.re, a, acc));
}

__device__ __forceinline__ void cp_async16(unsigned smem_addr, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// 4x4 complex matrix applied along one index of a thread's 4x4 block:
// out[c][j] = sum_k in[k][j] op[k][c] (kRight) or out[r][j] = sum_k op[r][k] in[k][j]
// (left); j is the batch index.  in[k][j] is addressed through Get, out through Put.
template <bool kRight, typename In, typename Out>
__device__ __forceinline__ void apply4(const float4* op, In in, Out out) {
  f32x2 o[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) o[i][j] = 0ull;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    f32x2 a[4], sw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      a[j] = in(k, j);
      sw[j] = pswap(a[j]);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const OpE b = load_op(op, kRight ? k * 4 + c : c * 4 + k);
#pragma unroll
      for (int j = 0; j < 4; ++j) o[c][j] = cmad2(o[c][j], a[j], sw[j], b);
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j) out(c, j, o[c][j]);
}

__global__ void __launch_bounds__(kPairThreads, 4)
pass_pair_kernel(float2* __restrict__ T, const __grid_constant__ PairParams pp,
                 const double2* __restrict__ L1, const double2* __restrict__ R1, long long s1,
                 const double2* __restrict__ L2, const double2* __restrict__ R2, long long s2) {
  extern __shared__ __align__(16) float4 pair_smem[];
  __shared__ float4 sop[4][16];  // L1, R1, L2, R2 as (b.x, b.x, -b.y, b.y)
  __shared__ long long tab[kPairChunks][256];  // tile byte offset of each 8-bit chunk value
  const int s = blockIdx.y;
  const int tid = threadIdx.x;
  const int n = pp.n;
  const long long rowbytes = 8ll << n;
  if (tid < 64) {
    const int o = tid >> 4, e = tid & 15;
    const double2* src = o == 0 ? L1 + s * s1 : o == 1 ? R1 + s * s1 : o == 2 ? L2 + s * s2 : R2 + s * s2;
    const double2 v = src[e];
    sop[o][e] = make_float4((float)v.x, (float)v.x, -(float)v.y, (float)v.y);
  }
#pragma unroll
  for (int j = 0; j < kPairChunks; ++j)
    for (int v = tid; v < 256; v += kPairThreads) {
      long long off = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int bit = j * 8 + i;
        if (bit < pp.tile_bits && ((v >> i) & 1)) {
          const int ps = pp.tbit_pos[bit];
          off += ps >= 32 ? (rowbytes << (ps - 32)) : (8ll << ps);
        }
      }
      tab[j][v] = off;
    }
  // per-thread constants: the copy column, the column-phase block and the
  // row-phase column
  unsigned ccol = 0;  // global column of this thread's copy pair
  {
    const unsigned c = (unsigned)(tid & 63) * 2u;
#pragma unroll
    for (int i = 0; i < 7; ++i) ccol |= ((c >> i) & 1u) << pp.tcol_pos[i];
  }
  unsigned rcol = 0;  // global column of this thread's row-phase tile column
#pragma unroll
  for (int i = 0; i < 7; ++i) rcol |= (((unsigned)tid >> i) & 1u) << pp.tcol_pos[i];
  unsigned wcomp = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) wcomp |= (((unsigned)tid >> i) & 1u) << pp.win_cpos[i];
  const unsigned ctr = (unsigned)tid >> 3;  // column-phase tile row
  const unsigned cblock = ctr * kPairCols + (pswz(wcomp) ^ ((ctr & 1u) ? (unsigned)pp.rxmask : 0u));
  const unsigned rsc = pswz((unsigned)tid) * 8u;  // byte offset (row slot masks are in rsm)
  const unsigned hi = (unsigned)tid >> 6;         // copies go to rows 2i + hi
  const unsigned cp_dst =
      hi * kPairCols * 8u + (pswz((unsigned)(tid & 63) * 2u) ^ (hi ? (unsigned)pp.rxmask : 0u)) * 8u;
  __syncthreads();

  const unsigned tiles = 1u << pp.tile_bits;
  char* Tb = reinterpret_cast<char*>(T + (size_t)s * ((size_t)1 << (2 * n)));
  const unsigned smem0 = (unsigned)__cvta_generic_to_shared(pair_smem);
  auto tile_off = [&](unsigned t) {
    return tab[0][t & 255u] + tab[1][(t >> 8) & 255u] + tab[2][(t >> 16) & 255u];
  };
  auto issue = [&](long long toff, unsigned buf) {
    const char* src = Tb + toff + ccol * 8u;
#pragma unroll
    for (int i = 0; i < 8; ++i)
      cp_async16(smem0 + buf * (kPairTileEntries * 8u) + cp_dst + (unsigned)i * (2u * kPairCols * 8u),
                 src + pp.rtile[2 * i + hi]);
  };

  unsigned t = blockIdx.x;
  long long toff = t < tiles ? tile_off(t) : 0;
  if (t < tiles) issue(toff, 0);
  cp_async_commit();
  unsigned cur = 0;
  for (; t < tiles; t += gridDim.x) {
    const unsigned tn = t + gridDim.x;
    const long long tnoff = tn < tiles ? tile_off(tn) : 0;
    if (tn < tiles) issue(tnoff, cur ^ 1u);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    f32x2* tile = reinterpret_cast<f32x2*>(pair_smem) + cur * kPairTileEntries;
    char* tileb = reinterpret_cast<char*>(tile);
    {  // columns: B <- B (R1 (x) R2) on the 16 column partners of (row, window)
      f32x2 e[4][4];  // [y1][y2]
#pragma unroll
      for (int k = 0; k < 16; ++k) e[k >> 2][k & 3] = tile[cblock ^ (unsigned)pp.gsw[k]];
      f32x2 m[4][4];
      apply4<true>(sop[1], [&](int k, int j) { return e[k][j]; },
                   [&](int c, int j, f32x2 v) { m[c][j] = v; });
      apply4<true>(sop[3], [&](int k, int j) { return m[j][k]; },
                   [&](int c, int j, f32x2 v) { tile[cblock ^ (unsigned)pp.gsw[j * 4 + c]] = v; });
    }
    __syncthreads();
    {  // rows: B <- (L1 (x) L2) B on the 16 row partners of tile column tid
      f32x2 m[4][4];
      apply4<false>(sop[0], [&](int k, int j) {
        return *reinterpret_cast<const f32x2*>(tileb + ((unsigned)pp.rsm[k * 4 + j] ^ rsc)); },
                    [&](int c, int j, f32x2 v) { m[c][j] = v; });
      char* dst = Tb + toff + rcol * 8u;
      apply4<false>(sop[2], [&](int k, int j) { return m[j][k]; },
                    [&](int c, int j, f32x2 v) {
                      *reinterpret_cast<f32x2*>(dst + pp.rglob[j * 4 + c]) = v; });
    }
    __syncthreads();  // this buffer is refilled by the next iteration's prefetch
    cur ^= 1u;
    toff = tnoff;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

}  // namespace

bool pair_pass_supported(int n, int a1, int b1, int a2, int b2, int prec) {
  if (prec != 1 || n < 8 || 2 * n - 11 > kPairChunks * 8) return false;
  return a1 != a2 && a1 != b2 && b1 != a2 && b1 != b2 && a1 != b1 && a2 != b2;
}

size_t pair_params_bytes() { return sizeof(PairParams); }

void make_pair_params(int n, int a1, int b1, int a2, int b2, void* host_out) {
  PairParams g;
  memset(&g, 0, sizeof(g));
  g.n = n;
  g.tile_bits = 2 * n - 11;
  const int pa1 = qubit_bit(n, a1), pb1 = qubit_bit(n, b1);
  const int pa2 = qubit_bit(n, a2), pb2 = qubit_bit(n, b2);
  const unsigned gmask = (1u << pa1) | (1u << pb1) | (1u << pa2) | (1u << pb2);
  // tile column bits: the 4 gate bits and the 3 lowest other bits (window)
  unsigned tmask = gmask;
  int win[3], nw = 0;
  for (int b = 0; b < n && nw < 3; ++b)
    if (!((gmask >> b) & 1u)) {
      tmask |= 1u << b;
      win[nw++] = b;
    }
  int ntb = 0;
  for (int b = 0; b < n; ++b)
    if ((tmask >> b) & 1u) g.tcol_pos[ntb++] = b;
  auto cpos = [&](int b) {
    for (int i = 0; i < 7; ++i)
      if (g.tcol_pos[i] == b) return i;
    return -1;
  };
  for (int i = 0; i < 3; ++i) g.win_cpos[i] = cpos(win[i]);
  // tile index: the n-8 non-tile column bits (low), then the n-4 non-gate row bits
  int nb = 0;
  for (int b = 0; b < n; ++b)
    if (!((tmask >> b) & 1u)) g.tbit_pos[nb++] = b;
  for (int b = 0; b < n; ++b)
    if (!((gmask >> b) & 1u)) g.tbit_pos[nb++] = 32 + b;
  // tile rows: the 4 gate bits in increasing position order
  int gs[4] = {pa1, pb1, pa2, pb2};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 3 - i; ++j)
      if (gs[j] > gs[j + 1]) {
        const int t = gs[j];
        gs[j] = gs[j + 1];
        gs[j + 1] = t;
      }
  auto rpos = [&](int b) {
    for (int i = 0; i < 4; ++i)
      if (gs[i] == b) return i;
    return -1;
  };
  const long long rowbytes = 8ll << n;
  for (int tr = 0; tr < 16; ++tr) {
    long long r = 0;
    for (int i = 0; i < 4; ++i) r |= (long long)((tr >> i) & 1) << gs[i];
    g.rtile[tr] = r * rowbytes;
  }
  unsigned gcomb[16], rcomb[16];
  for (int v1 = 0; v1 < 4; ++v1)
    for (int v2 = 0; v2 < 4; ++v2) {
      // local index 2*bit(pa) + bit(pb) for each gate
      const unsigned c = (((unsigned)(v1 >> 1) & 1u) << cpos(pa1)) | (((unsigned)v1 & 1u) << cpos(pb1)) |
                         (((unsigned)(v2 >> 1) & 1u) << cpos(pa2)) | (((unsigned)v2 & 1u) << cpos(pb2));
      // the gate bits and the window bits are disjoint and the swizzle is
      // linear over XOR, so a partner's slot is block ^ pswz(gate part)
      g.gsw[v1 * 4 + v2] = (int)(c ^ (((c >> 4) & 7u) << 1));
      gcomb[v1 * 4 + v2] = c;
      const unsigned r = (((unsigned)(v1 >> 1) & 1u) << rpos(pa1)) | (((unsigned)v1 & 1u) << rpos(pb1)) |
                         (((unsigned)(v2 >> 1) & 1u) << rpos(pa2)) | (((unsigned)v2 & 1u) << rpos(pb2));
      rcomb[v1 * 4 + v2] = r;
      g.rglob[v1 * 4 + v2] = g.rtile[r];
    }
  // slot XOR of odd rows: the mask (bits 1..3, keeping 16-byte pairs) with
  // the fewest bank conflicts in the column phase, where a half-warp reads
  // one partner of 8 windows in 2 adjacent rows
  unsigned wins[8];
  for (int w = 0; w < 8; ++w) {
    unsigned c = 0;
    for (int i = 0; i < 3; ++i) c |= ((unsigned)(w >> i) & 1u) << g.win_cpos[i];
    wins[w] = c;
  }
  auto sw = [](unsigned c) { return c ^ (((c >> 4) & 7u) << 1); };
  int best = 99;
  for (unsigned mask = 0; mask < 16; mask += 2) {
    int worst = 1;
    for (int k = 0; k < 16; ++k)
      for (int h = 0; h < 8; ++h) {
        int cnt[16] = {0};
        for (int rr = 0; rr < 2; ++rr)
          for (int w = 0; w < 8; ++w) {
            const unsigned tr = 2 * h + rr;
            const unsigned slot = sw(wins[w] | gcomb[k]) ^ ((tr & 1u) ? mask : 0u);
            const int b = (int)(slot & 15u);
            if (++cnt[b] > worst) worst = cnt[b];
          }
      }
    if (worst < best) {
      best = worst;
      g.rxmask = (int)mask;
    }
  }
  for (int k = 0; k < 16; ++k)
    g.rsm[k] = (int)((rcomb[k] * kPairCols + ((rcomb[k] & 1u) ? (unsigned)g.rxmask : 0u)) * 8u);
  memcpy(host_out, &g, sizeof(g));
}

cudaError_t launch_pair_pass(void* T, int n, int S, const void* params, const double2* L1,
                             const double2* R1, long long s1, const double2* L2,
                             const double2* R2, long long s2, cudaStream_t st) {
  const size_t smem = 2 * kPairTileEntries * sizeof(float2);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(pass_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  PairParams pp;
  memcpy(&pp, params, sizeof(pp));
  const unsigned tiles = 1u << (2 * n - 11);
  long long cap = ((long long)sm_count() * 4 + S - 1) / S;
  if (cap < 1) cap = 1;
  dim3 grid((unsigned)((long long)tiles < cap ? tiles : cap), S);
  pass_pair_kernel<<<grid, kPairThreads, smem, st>>>((float2*)T, pp, L1, R1, s1, L2, R2, s2);
  return cudaGetLastError();
}

namespace {

// ----------------------------------------------------------------- trace

// ------------------------------------------------ one-pass InitCircuitTensor
//
// After T_s <- V^dagger, every gate of Alg. 1's InitCircuitTensor acts on
// the column index only (T <- T (u_k on (a_k, b_k))), so each row of T_s can
// take all p gates in order on its own.  A CTA loads a row (N entries) into
// shared memory once, applies the gates there and writes the row back: one
// read and one write of T instead of p.  The gate list is cut into steps of
// one gate, or of two consecutive gates on four distinct qubits (they
// commute, so one step applies both); each step is one barrier.
//   two-gate step: a thread owns a 16-entry block (the 4 gate bits) and
//                  applies the first gate along its 2 bits, then the second;
//   one-gate step: a thread owns four 4-entry tuples and applies the gate to
//                  each.
// Packed f32x2 FMAs as in the pair pass; the row is XOR-swizzled in shared
// memory (bits 4..7 of a column into bits 0..3), which keeps the 16 lanes of
// a half-warp on distinct banks when the gate bits are the lowest ones.
// Used for complex64, where the per-gate passes are bound by HBM.  128
// threads and 4 CTAs per SM (128 registers, ~50 KB of shared memory each at
// 12 qubits): 256-thread CTAs took 138 registers and fit once per SM
// (9.1 ms against 7.2 ms for 8 starts at 12 qubits and 66 gates).

constexpr int kBuildThreads = 128;  // 4 CTAs per SM (registers and shared memory)
constexpr int kBuildMaxSteps = 960;

struct BuildParams {
  int n, steps;
  // per step: bit positions (pa1 | pb1 << 4, pa2 | pb2 << 4) and the first
  // gate's index; bit 15 of `gate` marks a two-gate step (gates k, k+1)
  unsigned char bits[kBuildMaxSteps][2];
  unsigned short gate[kBuildMaxSteps];
};

__device__ __forceinline__ unsigned bswz(unsigned c) { return c ^ ((c >> 4) & 15u); }

__global__ void __launch_bounds__(kBuildThreads, 4)
build_rows_kernel(float2* __restrict__ T, const __grid_constant__ BuildParams bp,
                  const double2* __restrict__ gates, long long gstride, int p) {
  extern __shared__ __align__(16) unsigned char build_smem[];
  const int n = bp.n;
  const unsigned N = 1u << n;
  float4* ops = reinterpret_cast<float4*>(build_smem);     // p x 16: (u.x, u.x, -u.y, u.y)
  f32x2* row = reinterpret_cast<f32x2*>(ops + p * 16);     // N entries, swizzled
  const int s = blockIdx.y;
  const double2* g = gates + s * gstride;
  for (int i = threadIdx.x; i < p * 16; i += blockDim.x) {
    const double2 v = g[i];
    ops[i] = make_float4((float)v.x, (float)v.x, -(float)v.y, (float)v.y);
  }
  f32x2* __restrict__ Ts = reinterpret_cast<f32x2*>(T + (size_t)s * N * N);
  const unsigned items = N >> 4;  // 16-entry blocks, or 4 tuples of 4
  for (unsigned r = blockIdx.x; r < N; r += gridDim.x) {
    f32x2* src = Ts + (size_t)r * N;
    for (unsigned i = threadIdx.x; i < N; i += blockDim.x) row[bswz(i)] = src[i];
    __syncthreads();
    for (int st = 0; st < bp.steps; ++st) {
      const unsigned b0 = bp.bits[st][0], b1 = bp.bits[st][1];
      const unsigned gk = bp.gate[st];
      const int k = (int)(gk & 0x7fffu);
      const int pa1 = b0 & 15, pb1 = b0 >> 4;
      if (gk & 0x8000u) {
        const int pa2 = b1 & 15, pb2 = b1 >> 4;
        // the 4 gate bits in ascending order, for the block base
        int q[4] = {pa1, pb1, pa2, pb2};
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3 - i; ++j)
            if (q[j] > q[j + 1]) {
              const int t = q[j];
              q[j] = q[j + 1];
              q[j + 1] = t;
            }
        unsigned off[16];  // swizzled offset of entry (x1, x2)
#pragma unroll
        for (int x1 = 0; x1 < 4; ++x1)
#pragma unroll
          for (int x2 = 0; x2 < 4; ++x2)
            off[x1 * 4 + x2] = bswz((((unsigned)x1 >> 1) << pa1) | (((unsigned)x1 & 1u) << pb1) |
                                    (((unsigned)x2 >> 1) << pa2) | (((unsigned)x2 & 1u) << pb2));
        for (unsigned t = threadIdx.x; t < items; t += blockDim.x) {
          const unsigned base = bswz(dep1(dep1(dep1(dep1(t, q[0]), q[1]), q[2]), q[3]));
          f32x2 m[4][4];
          apply4<true>(ops + k * 16, [&](int kk, int j) { return row[base ^ off[kk * 4 + j]]; },
                       [&](int c, int j, f32x2 v) { m[c][j] = v; });
          apply4<true>(ops + (k + 1) * 16, [&](int kk, int j) { return m[j][kk]; },
                       [&](int c, int j, f32x2 v) { row[base ^ off[j * 4 + c]] = v; });
        }
      } else {
        const int plo = pa1 < pb1 ? pa1 : pb1, phi = pa1 < pb1 ? pb1 : pa1;
        const unsigned o[4] = {0u, bswz(1u << pb1), bswz(1u << pa1), bswz((1u << pa1) | (1u << pb1))};
        for (unsigned t = threadIdx.x; t < items; t += blockDim.x) {
          unsigned base[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) base[j] = bswz(dep2(t + (unsigned)j * items, plo, phi));
          apply4<true>(ops + k * 16, [&](int kk, int j) { return row[base[j] ^ o[kk]]; },
                       [&](int c, int j, f32x2 v) { row[base[j] ^ o[c]] = v; });
        }
      }
      __syncthreads();
    }
    for (unsigned i = threadIdx.x; i < N; i += blockDim.x) src[i] = row[bswz(i)];
    __syncthreads();
  }
}

// status <- QF_ENONFINITE (-4) if any of the `count` doubles is NaN or Inf
// and no earlier error is recorded there.
__global__ void __launch_bounds__(256) check_finite_kernel(const double* __restrict__ x, size_t count,
                                                           int* __restrict__ status) {
  bool bad = false;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicCAS(status, 0, -4);
}

// Entry-wise conversion between tensor precisions through FP64 (exact from
// complex64 and df64; complex128 -> df64 keeps about 48 bits).
template <typename RS, typename RD>
__global__ void __launch_bounds__(256) convert_kernel(const typename Cplx<RS>::T* __restrict__ src,
                                                      typename Cplx<RD>::T* __restrict__ dst,
                                                      size_t count) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = cmake(to_d2(src[i]), RD());
}

template <typename RS>
void convert_from(const void* src, void* dst, int dp, size_t count, cudaStream_t st) {
  size_t blocks = (count + 255) / 256;
  const size_t cap = (size_t)sm_count() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  typedef typename Cplx<RS>::T CS;
  if (dp == 0)
    convert_kernel<RS, double><<<(unsigned)blocks, 256, 0, st>>>((const CS*)src, (double2*)dst, count);
  else if (dp == 2)
    convert_kernel<RS, DF><<<(unsigned)blocks, 256, 0, st>>>((const CS*)src, (dfc*)dst, count);
  else
    convert_kernel<RS, float><<<(unsigned)blocks, 256, 0, st>>>((const CS*)src, (float2*)dst, count);
}

constexpr int kTraceThreads = 256;

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
    re += __shfl_xor_sync(kFull, re, h);
    im += __shfl_xor_sync(kFull, im, h);
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

// ------------------------------------------------------------- dispatch

template <typename R, bool HL, bool HR>
void launch_block(void* T, int n, int S, int plo, int phi, int pa, int pb, const double2* L,
                  long long Ls, const double2* Rm, long long Rs, cudaStream_t st) {
  typedef typename Cplx<R>::T C;
  const unsigned nblk = 1u << (2 * (n - 2));
  const int per_sm = PassOcc<R, false>::v;
  long long want = (nblk + kPassThreads - 1) / kPassThreads;
  long long cap = ((long long)sm_count() * per_sm + S - 1) / S;
  if (cap < 1) cap = 1;
  dim3 grid((unsigned)(want < cap ? want : cap), S);
  pass_block_kernel<R, HL, HR><<<grid, kPassThreads, 0, st>>>((C*)T, n, plo, phi, pa, pb, L, Ls,
                                                              Rm, Rs);
}

template <typename R, int MODE, bool HL, bool HR>
void launch_lane(void* T, int n, int S, int plo, int phi, int pa, int pb, const double2* L,
                 long long Ls, const double2* Rm, long long Rs, cudaStream_t st) {
  typedef typename Cplx<R>::T C;
  const int lcols = MODE == 1 ? n - 1 : n;
  const unsigned units = (1u << (n - 2)) << lcols;
  const int per_sm = PassOcc<R, false>::v;
  long long want = (units + kPassThreads - 1) / kPassThreads;
  long long cap = ((long long)sm_count() * per_sm + S - 1) / S;
  if (cap < 1) cap = 1;
  dim3 grid((unsigned)(want < cap ? want : cap), S);
  pass_lane_kernel<R, MODE, HL, HR><<<grid, kPassThreads, 0, st>>>((C*)T, n, plo, phi, pa, pb,
                                                                   L, Ls, Rm, Rs);
}

template <typename R, int PA, int PB>
void launch_window(void* T, int n, int S, const double2* L, long long Ls, const double2* Rm,
                   long long Rs, cudaStream_t st) {
  typedef typename Cplx<R>::T C;
  constexpr int W = (PA > PB ? PA : PB) <= 1 ? 4 : 8;
  const unsigned units = (1u << (n - 2)) << (n - (W == 4 ? 2 : 3));
  const int per_sm = PassOcc<R, true>::v;
  long long want = (units + kPassThreads - 1) / kPassThreads;
  long long cap = ((long long)sm_count() * per_sm + S - 1) / S;
  if (cap < 1) cap = 1;
  dim3 grid((unsigned)(want < cap ? want : cap), S);
  pass_window_kernel<R, PA, PB><<<grid, kPassThreads, 0, st>>>((C*)T, n, L, Ls, Rm, Rs);
}

template <typename R>
bool try_window(void* T, int n, int S, int pa, int pb, const double2* L, long long Ls,
                const double2* Rm, long long Rs, cudaStream_t st) {
  if (n < 3 || pa > 2 || pb > 2) return false;
  // df64 is bound by the FP32 pipe; a window's 4 x 8 entries of 16 bytes
  // per thread leave too few warps to hide its arithmetic latency, so the
  // lane and half-block mappings take these gates
  if (sizeof(R) == 1) return false;
#define QF_W(A, B)                                                \
  if (pa == A && pb == B) {                                       \
    launch_window<R, A, B>(T, n, S, L, Ls, Rm, Rs, st);           \
    return true;                                                  \
  }
  QF_W(1, 0) QF_W(0, 1) QF_W(2, 1) QF_W(1, 2) QF_W(2, 0) QF_W(0, 2)
#undef QF_W
  return false;
}

template <typename R, bool HL, bool HR>
void launch_half(void* T, int n, int S, int plo, int phi, int pa, int pb, const double2* L,
                 long long Ls, const double2* Rm, long long Rs, cudaStream_t st) {
  typedef typename Cplx<R>::T C;
  const long long units = 2ll << (2 * (n - 2));
  long long want = (units + kPassThreads - 1) / kPassThreads;
  long long cap = ((long long)sm_count() * 2 + S - 1) / S;
  if (cap < 1) cap = 1;
  dim3 grid((unsigned)(want < cap ? want : cap), S);
  pass_half_kernel<R, HL, HR><<<grid, kPassThreads, 0, st>>>((C*)T, n, plo, phi, pa, pb, L, Ls, Rm,
                                                              Rs);
}

template <typename R, bool HL, bool HR>
void pass_dispatch(void* T, int n, int S, int pa, int pb, const double2* L, long long Ls,
                   const double2* Rm, long long Rs, cudaStream_t st) {
  const int plo = pa < pb ? pa : pb, phi = pa < pb ? pb : pa;
  if (HL && HR && try_window<R>(T, n, S, pa, pb, L, Ls, Rm, Rs, st)) return;
  if (n >= 6 && plo <= 1) {
    if (phi < 5)
      launch_lane<R, 2, HL, HR>(T, n, S, plo, phi, pa, pb, L, Ls, Rm, Rs, st);
    else
      launch_lane<R, 1, HL, HR>(T, n, S, plo, phi, pa, pb, L, Ls, Rm, Rs, st);
  } else {
    if constexpr (sizeof(R) == 1) {  // df64
      // the half-block kernel's shuffles need whole warps: 2^(2n-3) units
      // are a multiple of 32 from n = 4 on
      if (n >= 4) {
        launch_half<R, HL, HR>(T, n, S, plo, phi, pa, pb, L, Ls, Rm, Rs, st);
        return;
      }
    }
    launch_block<R, HL, HR>(T, n, S, plo, phi, pa, pb, L, Ls, Rm, Rs, st);
  }
}

template <typename R>
void pass_ops(void* T, int n, int S, int pa, int pb, const double2* L, long long Ls,
              const double2* Rm, long long Rs, cudaStream_t st) {
  if (L && Rm)
    pass_dispatch<R, true, true>(T, n, S, pa, pb, L, Ls, Rm, Rs, st);
  else if (L)
    pass_dispatch<R, true, false>(T, n, S, pa, pb, L, Ls, Rm, Rs, st);
  else if (Rm)
    pass_dispatch<R, false, true>(T, n, S, pa, pb, L, Ls, Rm, Rs, st);
}

}  // namespace

// ================================================================ launchers

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

cudaError_t launch_set_identity(double2* M, int n, cudaStream_t st) {
  const size_t NN = (size_t)1 << (2 * n);
  size_t blocks = (NN + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  set_identity_kernel<<<(unsigned)blocks, 256, 0, st>>>(M, n);
  return cudaGetLastError();
}

cudaError_t launch_conj_transpose(const double2* V, void* T, int n, int S, int prec,
                                  cudaStream_t st) {
  const int N = 1 << n;
  dim3 grid((N + 31) / 32, (N + 31) / 32, S), block(32, 8);
  if (prec == 0)
    conj_transpose_kernel<double><<<grid, block, 0, st>>>(V, (double2*)T, N);
  else if (prec == 2)
    conj_transpose_kernel<DF><<<grid, block, 0, st>>>(V, (dfc*)T, N);
  else
    conj_transpose_kernel<float><<<grid, block, 0, st>>>(V, (float2*)T, N);
  return cudaGetLastError();
}

cudaError_t launch_pass(void* T, int n, int S, int a, int b, const double2* L,
                        long long Lstride, const double2* R, long long Rstride, int prec,
                        cudaStream_t st) {
  if (!L && !R) return cudaSuccess;
  const int pa = qubit_bit(n, a), pb = qubit_bit(n, b);
  if (prec == 0)
    pass_ops<double>(T, n, S, pa, pb, L, Lstride, R, Rstride, st);
  else if (prec == 2)
    pass_ops<DF>(T, n, S, pa, pb, L, Lstride, R, Rstride, st);
  else
    pass_ops<float>(T, n, S, pa, pb, L, Lstride, R, Rstride, st);
  return cudaGetLastError();
}

cudaError_t launch_check_finite(const double* x, size_t count, int* status, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  size_t blocks = (count + 255) / 256;
  const size_t cap = (size_t)sm_count() * 8;
  if (blocks > cap) blocks = cap;
  check_finite_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, count, status);
  return cudaGetLastError();
}

bool build_rows_supported(int n, int p, int prec) {
  if (prec != 1 || n < 10 || n > 15 || p > kBuildMaxSteps) return false;
  const size_t smem = ((size_t)1 << n) * sizeof(float2) + (size_t)p * 16 * sizeof(float4);
  return smem <= 200 * 1024;
}

cudaError_t launch_build_rows(void* T, int n, int S, int p, const int* pa, const int* pb,
                              const double2* gates, long long gstride, cudaStream_t st) {
  BuildParams bp;
  memset(&bp, 0, sizeof(bp));
  bp.n = n;
  int steps = 0;
  for (int k = 0; k < p;) {
    bp.bits[steps][0] = (unsigned char)(pa[k] | (pb[k] << 4));
    const bool pair = k + 1 < p && pa[k + 1] != pa[k] && pa[k + 1] != pb[k] && pb[k + 1] != pa[k] &&
                      pb[k + 1] != pb[k];
    if (pair) {
      bp.bits[steps][1] = (unsigned char)(pa[k + 1] | (pb[k + 1] << 4));
      bp.gate[steps] = (unsigned short)(k | 0x8000);
      k += 2;
    } else {
      bp.gate[steps] = (unsigned short)k;
      k += 1;
    }
    ++steps;
  }
  bp.steps = steps;
  const size_t smem = ((size_t)1 << n) * sizeof(float2) + (size_t)p * 16 * sizeof(float4);
  static size_t attr = 0;
  if (smem > attr) {
    const cudaError_t e = cudaFuncSetAttribute(build_rows_kernel,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = smem;
  }
  int per_sm = (int)((224 * 1024) / (smem + 1024));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 8) per_sm = 8;
  long long cap = ((long long)sm_count() * per_sm + S - 1) / S;
  const long long rows = 1ll << n;
  const unsigned threads = (unsigned)(((1u << n) >> 4) < (unsigned)kBuildThreads ? ((1u << n) >> 4)
                                                                                  : kBuildThreads);
  dim3 grid((unsigned)(rows < cap ? rows : cap), S);
  build_rows_kernel<<<grid, threads, smem, st>>>((float2*)T, bp, gates, gstride, p);
  return cudaGetLastError();
}

cudaError_t launch_convert(const void* src, int sp, void* dst, int dp, size_t count, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  if (sp == 0)
    convert_from<double>(src, dst, dp, count, st);
  else if (sp == 2)
    convert_from<DF>(src, dst, dp, count, st);
  else
    convert_from<float>(src, dst, dp, count, st);
  return cudaGetLastError();
}

cudaError_t launch_trace(const void* T, int n, int S, double2* tr, int prec, cudaStream_t st) {
  if (prec == 0)
    trace_kernel<double><<<S, kTraceThreads, 0, st>>>((const double2*)T, n, tr);
  else if (prec == 2)
    trace_kernel<DF><<<S, kTraceThreads, 0, st>>>((const dfc*)T, n, tr);
  else
    trace_kernel<float><<<S, kTraceThreads, 0, st>>>((const float2*)T, n, tr);
  return cudaGetLastError();
}

}  // namespace qf
