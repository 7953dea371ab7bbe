// V-cycle (Fig. mgalgorithm) with CheapSIMPLE smoothing (Algorithm 4, Sec. 5.2), the fine-level
// saddle apply, and the FP64 helpers of the setup (dot products, lambda_max power iteration).
//
// Every cycle kernel is templated on the storage and arithmetic type T: double for the FP64
// cycle, float for the FP32 cycle (FP32 storage, arithmetic and accumulation).  In both, the
// inverted nodal Schur blocks and the coarsest inverse stay FP64.
//
// GB300 retires FP64 fused multiply-adds at a small fraction of its FP32 rate, so a warp
// FP64 instruction costs many SM cycles: every kernel issues one FMA per matrix value with
// all lanes busy wherever the row structure allows, and keeps cross-lane reductions out of
// the inner loops.  Two mappings:
//  * SELL-32, one thread per block row (fine-level K and P: short rows, many rows);
//  * one warp per block row, one lane per block, BR partial sums per lane reduced once at the
//    end (restriction and coarse levels: long rows or few rows).
#include "amgc_internal.cuh"

#include <algorithm>
#include <cmath>

namespace amgc {

constexpr int kRowWarps = 8;   // warps per block of the warp-per-row kernels

template <class T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }
template <class T>
__device__ __forceinline__ T ldcs(const T* p) { return __ldcs(p); }

// MODE 0: y  = A1 x1 + A2 x2
// MODE 1: y += A1 x1
// MODE 2: y  = b - A1 x1 - A2 x2                        (residual)
// MODE 3: y  = x0 + omega * dinv * (b - A1 x1 - A2 x2)    (damped Jacobi, out of place)
// MODE 4: y  = dinv * (A1 x1 + A2 x2)                     (power step on D^-1 K)
template <int MODE, class T>
__device__ __forceinline__ void store_row(T* __restrict__ y, const T* __restrict__ b, const T* __restrict__ x0,
                                          const T* __restrict__ dinv, T omega, int64_t o, T s) {
  if (MODE == 0) y[o] = s;
  else if (MODE == 1) y[o] += s;
  else if (MODE == 2) y[o] = b[o] - s;
  else if (MODE == 3) y[o] = x0[o] + omega * dinv[o] * (b[o] - s);
  else y[o] = dinv[o] * s;
}

// lane-per-block accumulation of one block row: acc[r] += sum_c A[b][r][c] x[col[b]][c]
template <int BR, int BC, class T>
__device__ __forceinline__ void lane_blocks(int64_t b0, int64_t b1, const int* __restrict__ col,
                                            const T* __restrict__ val, const T* __restrict__ x, int lane,
                                            T (&acc)[BR]) {
  for (int64_t b = b0 + lane; b < b1; b += 32) {
    const T* xc = x + (int64_t)__ldg(col + b) * BC;
    T xv[BC];
#pragma unroll
    for (int c = 0; c < BC; ++c) xv[c] = ldg(xc + c);
    const T* v = val + b * (BR * BC);
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int c = 0; c < BC; ++c) acc[r] = fma(ldg(v + r * BC + c), xv[c], acc[r]);
  }
}

template <int BR, int BC1, int BC2, int MODE, class T>
__global__ void __launch_bounds__(kRowWarps * 32)
k_rowop(int nbr, const int* __restrict__ rp1, const int* __restrict__ c1, const T* __restrict__ v1,
        const T* __restrict__ x1, const int* __restrict__ rp2, const int* __restrict__ c2, const T* __restrict__ v2,
        const T* __restrict__ x2, const T* __restrict__ b, const T* __restrict__ x0, const T* __restrict__ dinv,
        T omega, T* __restrict__ y) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int row = blockIdx.x * kRowWarps + wid;
  if (row >= nbr) return;
  T acc[BR];
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = T(0);
  lane_blocks<BR, BC1, T>(rp1[row], rp1[row + 1], c1, v1, x1, lane, acc);
  if (rp2 != nullptr) lane_blocks<BR, BC2, T>(rp2[row], rp2[row + 1], c2, v2, x2, lane, acc);
  T out = T(0);
#pragma unroll
  for (int r = 0; r < BR; ++r) {
    const T t = warp_sum(acc[r]);
    if (lane == r) out = t;
  }
  if (lane < BR) store_row<MODE, T>(y, b, x0, dinv, omega, (int64_t)row * BR + lane, out);
}

// Warp per block row for 6-row blocks: lane 6s + r (s = 0..4, r = 0..5) owns block row r of
// every fifth block of the row starting at slot s, so the six lanes of a slot read one block's
// 6 x BC values contiguously and share the x gather; lanes 30 and 31 idle.  The five partial
// sums of each block row are then added across slots (lanes r, r+6, ..., r+24).
// acc += sum_c v[c] x[c] over one block row (c in order); VEC (BC = 6): the six values of v and of x
// in three two-element loads each (both 8 * sizeof(T)-aligned: checked by the launcher), half the
// load instructions of the scalar form and the same arithmetic
template <class T>
struct Pair;
template <>
struct Pair<double> { using type = double2; };
template <>
struct Pair<float> { using type = float2; };
template <int BC, bool VEC, class T>
__device__ __forceinline__ T block_row_dot(const T* __restrict__ v, const T* __restrict__ x, T acc) {
  if constexpr (VEC && BC == 6) {
    using P2 = typename Pair<T>::type;
    const P2* vp = reinterpret_cast<const P2*>(v);
    const P2* xp = reinterpret_cast<const P2*>(x);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const P2 a = __ldg(vp + k), y = __ldg(xp + k);
      acc = fma(a.x, y.x, acc);
      acc = fma(a.y, y.y, acc);
    }
  } else {
#pragma unroll
    for (int c = 0; c < BC; ++c) acc = fma(ldg(v + c), ldg(x + c), acc);
  }
  return acc;
}
template <int BC, bool VEC, class T>
__device__ __forceinline__ void slot_blocks6(int b0, int b1, const int* __restrict__ col, const T* __restrict__ val,
                                             const T* __restrict__ x, int s, int r, T& acc) {
  if (s >= 5) return;
#pragma unroll 2
  for (int b = b0 + s; b < b1; b += 5) {
    const T* xc = x + (int64_t)__ldg(col + b) * BC;
    const T* v = val + (int64_t)b * (6 * BC) + r * BC;
    acc = block_row_dot<BC, VEC, T>(v, xc, acc);
  }
}
template <int BC1, int BC2, int MODE, class T, bool VEC>
__global__ void __launch_bounds__(kRowWarps * 32)
k_rowop6(int nbr, const int* __restrict__ rp1, const int* __restrict__ c1, const T* __restrict__ v1,
         const T* __restrict__ x1, const int* __restrict__ rp2, const int* __restrict__ c2, const T* __restrict__ v2,
         const T* __restrict__ x2, const T* __restrict__ b, const T* __restrict__ x0, const T* __restrict__ dinv,
         T omega, T* __restrict__ y) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int row = blockIdx.x * kRowWarps + wid;
  if (row >= nbr) return;
  const int s = lane / 6, r = lane - 6 * (lane / 6);
  T acc = T(0);
  slot_blocks6<BC1, VEC, T>(rp1[row], rp1[row + 1], c1, v1, x1, s, r, acc);
  if (rp2 != nullptr) slot_blocks6<BC2, false, T>(rp2[row], rp2[row + 1], c2, v2, x2, s, r, acc);
  const T a1 = acc + __shfl_down_sync(0xffffffffu, acc, 6);
  const T a2 = a1 + __shfl_down_sync(0xffffffffu, a1, 12);
  const T out = a2 + __shfl_down_sync(0xffffffffu, acc, 24);
  if (lane < 6) store_row<MODE, T>(y, b, x0, dinv, omega, (int64_t)row * 6 + lane, out);
}

// CTA of W warps per block row for long rows of 6-row blocks (the restrictions between coarse
// levels, several hundred blocks per row, with W = 8; the coarse K, about 40 blocks per row, with
// W = 2; the restriction from a 3-DOF level has its own kernel, k_rowop63_long, unless its values
// are not aligned for paired loads).  Warp w takes slots 5w .. 5w+4 of every
// group of 5 W consecutive blocks with the lane mapping of k_rowop6; the warps' row sums are
// added in warp order (deterministic).
template <int W, int BC1, int BC2, int MODE, class T, bool VEC>
__global__ void __launch_bounds__(W * 32)
k_rowop6_long(int nbr, const int* __restrict__ rp1, const int* __restrict__ c1, const T* __restrict__ v1,
              const T* __restrict__ x1, const int* __restrict__ rp2, const int* __restrict__ c2,
              const T* __restrict__ v2, const T* __restrict__ x2, const T* __restrict__ b, const T* __restrict__ x0,
              const T* __restrict__ dinv, T omega, T* __restrict__ y) {
  constexpr int kLongWarps = W;
  __shared__ T part[kLongWarps][6];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int row = blockIdx.x;
  if (row >= nbr) return;
  const int s = lane / 6, r = lane - 6 * (lane / 6);
  T acc = T(0);
  if (s < 5) {
    const int stride = 5 * kLongWarps;
#pragma unroll 2
    for (int blk = rp1[row] + 5 * wid + s; blk < rp1[row + 1]; blk += stride) {
      const T* xc = x1 + (int64_t)__ldg(c1 + blk) * BC1;
      const T* v = v1 + (int64_t)blk * (6 * BC1) + r * BC1;
      acc = block_row_dot<BC1, VEC, T>(v, xc, acc);
    }
    if (rp2 != nullptr) {
      for (int blk = rp2[row] + 5 * wid + s; blk < rp2[row + 1]; blk += stride) {
        const T* xc = x2 + (int64_t)__ldg(c2 + blk) * BC2;
        const T* v = v2 + (int64_t)blk * (6 * BC2) + r * BC2;
#pragma unroll
        for (int c = 0; c < BC2; ++c) acc = fma(ldg(v + c), ldg(xc + c), acc);
      }
    }
  }
  const T a1 = acc + __shfl_down_sync(0xffffffffu, acc, 6);
  const T a2 = a1 + __shfl_down_sync(0xffffffffu, a1, 12);
  const T w = a2 + __shfl_down_sync(0xffffffffu, acc, 24);
  if (lane < 6) part[wid][lane] = w;
  __syncthreads();
  if (threadIdx.x < 6) {
    T out = T(0);
#pragma unroll
    for (int q = 0; q < kLongWarps; ++q) out += part[q][threadIdx.x];
    store_row<MODE, T>(y, b, x0, dinv, omega, (int64_t)row * 6 + threadIdx.x, out);
  }
}

// The restriction from a 3-DOF level (6 x 3 blocks, about 190 per row on the finest level): one
// block per lane, its 18 values in nine paired loads and its three x values, six running sums
// per lane (a third of the load instructions of the lane-per-block-row mapping and all 32 lanes
// busy); the six sums are reduced over the warp by a reduce-scatter butterfly (nine shuffles:
// after the rounds on lane bits 4, 3 and 2 lane L holds the partial of row 4 b4 + 2 b3 + b2 of
// its eight-lane set, rounds on bits 1 and 0 finish it), then over the CTA's warps in order.
template <int W, int MODE, class T>
__global__ void __launch_bounds__(W * 32)
k_rowop63_long(int nbr, const int* __restrict__ rp, const int* __restrict__ col, const T* __restrict__ val,
               const T* __restrict__ x, const T* __restrict__ b, const T* __restrict__ x0,
               const T* __restrict__ dinv, T omega, T* __restrict__ y) {
  using P2 = typename Pair<T>::type;
  __shared__ T part[W][6];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int row = blockIdx.x;
  if (row >= nbr) return;
  T a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = T(0);
  const int e1 = rp[row + 1];
#pragma unroll 2
  for (int blk = rp[row] + wid * 32 + lane; blk < e1; blk += W * 32) {
    const T* xc = x + (int64_t)__ldg(col + blk) * 3;
    const T xa = ldg(xc), xb = ldg(xc + 1), xd = ldg(xc + 2);
    const P2* vp = reinterpret_cast<const P2*>(val + (int64_t)blk * 18);
    T v[18];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const P2 q = __ldg(vp + k);
      v[2 * k] = q.x;
      v[2 * k + 1] = q.y;
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      a[r] = fma(v[3 * r], xa, a[r]);
      a[r] = fma(v[3 * r + 1], xb, a[r]);
      a[r] = fma(v[3 * r + 2], xd, a[r]);
    }
  }
  {   // lane bit 4: keep rows 0..3 (bit clear) or 4..7 (set)
    const bool hi = lane & 16;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const T send = hi ? a[k] : a[k + 4], keep = hi ? a[k + 4] : a[k];
      a[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
  }
  {   // lane bit 3: of those four, keep two
    const bool hi = lane & 8;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const T send = hi ? a[k] : a[k + 2], keep = hi ? a[k + 2] : a[k];
      a[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
  }
  {   // lane bit 2: keep one
    const bool hi = lane & 4;
    const T send = hi ? a[0] : a[1], keep = hi ? a[1] : a[0];
    a[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  a[0] += __shfl_xor_sync(0xffffffffu, a[0], 2);
  a[0] += __shfl_xor_sync(0xffffffffu, a[0], 1);
  const int r = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
  if ((lane & 3) == 0 && r < 6) part[wid][r] = a[0];
  __syncthreads();
  if (threadIdx.x < 6) {
    T out = T(0);
#pragma unroll
    for (int q = 0; q < W; ++q) out += part[q][threadIdx.x];
    store_row<MODE, T>(y, b, x0, dinv, omega, (int64_t)row * 6 + threadIdx.x, out);
  }
}

template <int BR, int BC1, int BC2, int MODE, class T>
static int launch_rowop(const BsrV<T>& A1, const T* x1, const BsrV<T>* A2, const T* x2, const T* b, const T* x0,
                        const T* dinv, double omega, T* y, cudaStream_t s) {
  if (A1.nbr == 0) return AMGC_OK;
  // six-column blocks: the paired loads need both operands aligned to two elements
  const size_t pair = 2 * sizeof(T);
  if (BR == 6 && BC1 == 3 && A2 == nullptr && A1.nbr < (1 << 16) && A1.nnzb > 24 * (int64_t)A1.nbr &&
      reinterpret_cast<uintptr_t>(A1.val) % pair == 0) {
    // FP32 (memory-bound): eight warps per row keep more loads in flight; FP64 (bound by the FMA
    // rate): two, so that the row's blocks fill the lanes over several passes
    if (sizeof(T) == 4 && A1.nnzb > 96 * (int64_t)A1.nbr)
      AMGC_LAUNCH(k_rowop63_long<8, MODE, T><<<A1.nbr, 8 * 32, 0, s>>>(A1.nbr, A1.rp, A1.col, A1.val, x1, b, x0, dinv,
                                                                      (T)omega, y));
    else
      AMGC_LAUNCH(k_rowop63_long<2, MODE, T><<<A1.nbr, 2 * 32, 0, s>>>(A1.nbr, A1.rp, A1.col, A1.val, x1, b, x0, dinv,
                                                                      (T)omega, y));
    AMGC_CUDA_TRY(cudaGetLastError());
    return AMGC_OK;
  }
  const bool vec = BC1 == 6 && reinterpret_cast<uintptr_t>(A1.val) % pair == 0 &&
                   reinterpret_cast<uintptr_t>(x1) % pair == 0;
  // long rows of 6-row blocks: a CTA of 8 (more than 96 blocks per row) or 2 (more than 24)
  // warps per row, so that the SMs hold enough warps
  if (BR == 6 && A1.nbr < (1 << 16) && A1.nnzb > 24 * (int64_t)A1.nbr) {
    const int* r2 = A2 ? A2->rp : nullptr;
    const int* k2 = A2 ? A2->col : nullptr;
    const T* w2 = A2 ? A2->val : nullptr;
    if (A1.nnzb > 96 * (int64_t)A1.nbr) {
      if (vec)
        AMGC_LAUNCH(k_rowop6_long<8, BC1, BC2, MODE, T, true><<<A1.nbr, 8 * 32, 0, s>>>(
            A1.nbr, A1.rp, A1.col, A1.val, x1, r2, k2, w2, x2, b, x0, dinv, (T)omega, y));
      else
        AMGC_LAUNCH(k_rowop6_long<8, BC1, BC2, MODE, T, false><<<A1.nbr, 8 * 32, 0, s>>>(
            A1.nbr, A1.rp, A1.col, A1.val, x1, r2, k2, w2, x2, b, x0, dinv, (T)omega, y));
    } else {
      if (vec)
        AMGC_LAUNCH(k_rowop6_long<2, BC1, BC2, MODE, T, true><<<A1.nbr, 2 * 32, 0, s>>>(
            A1.nbr, A1.rp, A1.col, A1.val, x1, r2, k2, w2, x2, b, x0, dinv, (T)omega, y));
      else
        AMGC_LAUNCH(k_rowop6_long<2, BC1, BC2, MODE, T, false><<<A1.nbr, 2 * 32, 0, s>>>(
            A1.nbr, A1.rp, A1.col, A1.val, x1, r2, k2, w2, x2, b, x0, dinv, (T)omega, y));
    }
    AMGC_CUDA_TRY(cudaGetLastError());
    return AMGC_OK;
  }
  if (BR == 6 && BC1 == 6) {
    if (vec)
      AMGC_LAUNCH(k_rowop6<BC1, BC2, MODE, T, true><<<div_up(A1.nbr, kRowWarps), kRowWarps * 32, 0, s>>>(
          A1.nbr, A1.rp, A1.col, A1.val, x1, A2 ? A2->rp : nullptr, A2 ? A2->col : nullptr, A2 ? A2->val : nullptr,
          x2, b, x0, dinv, (T)omega, y));
    else
      AMGC_LAUNCH(k_rowop6<BC1, BC2, MODE, T, false><<<div_up(A1.nbr, kRowWarps), kRowWarps * 32, 0, s>>>(
          A1.nbr, A1.rp, A1.col, A1.val, x1, A2 ? A2->rp : nullptr, A2 ? A2->col : nullptr, A2 ? A2->val : nullptr,
          x2, b, x0, dinv, (T)omega, y));
    AMGC_CUDA_TRY(cudaGetLastError());
    return AMGC_OK;
  }
  AMGC_LAUNCH(k_rowop<BR, BC1, BC2, MODE, T><<<div_up(A1.nbr, kRowWarps), kRowWarps * 32, 0, s>>>(
      A1.nbr, A1.rp, A1.col, A1.val, x1, A2 ? A2->rp : nullptr, A2 ? A2->col : nullptr, A2 ? A2->val : nullptr, x2,
      b, x0, dinv, (T)omega, y));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

template <int MODE, class T>
static int rowop(const BsrV<T>& A1, const T* x1, const BsrV<T>* A2, const T* x2, const T* b, const T* x0,
                 const T* dinv, double omega, T* y, cudaStream_t s) {
  const int br = A1.br, bc1 = A1.bc, bc2 = A2 ? A2->bc : 3;
#define AMGC_ROWOP_CASE(R, C1, C2) \
  if (br == R && bc1 == C1 && bc2 == C2) return launch_rowop<R, C1, C2, MODE, T>(A1, x1, A2, x2, b, x0, dinv, omega, y, s);
  AMGC_ROWOP_CASE(3, 3, 3)
  AMGC_ROWOP_CASE(6, 6, 3)
  AMGC_ROWOP_CASE(3, 6, 3)
  AMGC_ROWOP_CASE(6, 3, 3)
#undef AMGC_ROWOP_CASE
  set_error("rowop: unsupported block shape");
  return AMGC_EINVAL;
}

static BsrV<double> view_of(const DBsr& A) {
  BsrV<double> v;
  v.nbr = A.nbr; v.nbc = A.nbc; v.br = A.br; v.bc = A.bc; v.nnzb = A.nnzb;
  v.rp = A.rowptr.p; v.col = A.col.p; v.val = A.val.p;
  return v;
}

int bsr_spmv(const DBsr& A, const double* x, double* y, double alpha, double beta, cudaStream_t s) {
  (void)alpha;
  (void)beta;
  const BsrV<double> v = view_of(A);
  return rowop<0, double>(v, x, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, y, s);
}

// ------------------------------------------------------------------ SELL-32 row apply
// TPR threads per block row (1 or 2).  With TPR = 2 a warp covers 16 rows of a 32-row slice,
// lanes 0-15 take the even slots and lanes 16-31 the odd slots (each half-warp load is 16
// consecutive values) and one shuffle adds the halves: twice the loads in flight for the
// HBM-bound FP32 cycle.  The FP64 kernel is bound by the FP64 FMA rate and runs one thread
// per row (no extra instructions).  Value k of a block is one load and one FMA; matrix data
// is streamed (evict-first) so the vectors stay cached.  An optional second matrix A2 (the B1
// block, few rows) is added from its BSR rows.
constexpr int kSellThreads = 128;

template <int BR, int BC, int MODE, class T, int TPR>
__global__ void __launch_bounds__(kSellThreads)
k_sell(int nbr, const int* __restrict__ soff, const int* __restrict__ slen, const int* __restrict__ scol,
       const T* __restrict__ sval, const T* __restrict__ x, const int* __restrict__ rp2, const int* __restrict__ c2,
       const T* __restrict__ v2, const T* __restrict__ x2, const T* __restrict__ b, const T* __restrict__ x0,
       const T* __restrict__ dinv, T omega, T* __restrict__ y, const int* __restrict__ perm) {
  constexpr int BS = BR * BC;
  constexpr int RPW = 32 / TPR;                                // rows per warp
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int part = lane / RPW;                                 // slot residue handled by this lane
  const int pos = (gt >> 5) * RPW + (lane % RPW);              // SELL position
  const bool live = pos < nbr;
  const int r = live ? pos : nbr - 1;                          // dead lanes mirror a valid position
  const int sl = r >> 5, ls = r & 31;
  const int row = perm ? __ldg(perm + r) : r;                  // the block row at that position
  const int64_t o = soff[sl];
  const int L = slen[sl];
  const int* cp = scol + o * 32 + ls;
  const T* vp = sval + o * (BS * 32) + ls;
  T acc[BR];
#pragma unroll
  for (int q = 0; q < BR; ++q) acc[q] = T(0);
#pragma unroll 3
  for (int t = part; t < L; t += TPR) {
    const T* xc = x + (int64_t)__ldcs(cp + t * 32) * BC;
    T xv[BC];
#pragma unroll
    for (int c = 0; c < BC; ++c) xv[c] = ldg(xc + c);
    const T* v = vp + (int64_t)t * (BS * 32);
#pragma unroll
    for (int q = 0; q < BR; ++q)
#pragma unroll
      for (int c = 0; c < BC; ++c) acc[q] = fma(ldcs(v + (q * BC + c) * 32), xv[c], acc[q]);
  }
  if (TPR == 2) {
#pragma unroll
    for (int q = 0; q < BR; ++q) acc[q] += __shfl_down_sync(0xffffffffu, acc[q], 16);
  }
  if (part != 0 || !live) return;
  if (rp2 != nullptr) {
    for (int e = rp2[row]; e < rp2[row + 1]; ++e) {
      const T* blk = v2 + (int64_t)e * BR * 3;
      const T* d = x2 + 3 * (int64_t)c2[e];
      const T d0 = d[0], d1 = d[1], d2 = d[2];
#pragma unroll
      for (int q = 0; q < BR; ++q) acc[q] = fma(blk[3 * q], d0, fma(blk[3 * q + 1], d1, fma(blk[3 * q + 2], d2, acc[q])));
    }
  }
#pragma unroll
  for (int q = 0; q < BR; ++q) store_row<MODE, T>(y, b, x0, dinv, omega, (int64_t)row * BR + q, acc[q]);
}

template <int BR, int BC, int MODE, class T, int TPR>
static void launch_sell(const SellV<T>& S, int nbr, const int* rp2, const int* c2, const T* v2, const T* x,
                        const T* x2, const T* b, const T* x0, const T* dinv, double omega, T* y, cudaStream_t s) {
  // FP64 is bound by each SM's FMA rate and all CTAs fit at once: two-warp CTAs spread the row
  // groups over the SMs more evenly than four-warp ones
  const int threads = sizeof(T) == 8 ? kSellThreads / 2 : kSellThreads;
  const int g = div_up((int64_t)nbr * TPR, threads);
  AMGC_LAUNCH(k_sell<BR, BC, MODE, T, TPR><<<g, threads, 0, s>>>(nbr, S.off, S.len, S.col, S.val, x, rp2, c2, v2, x2,
                                                                 b, x0, dinv, (T)omega, y, S.perm));
}

// ---------------------------------------------------------------- TMA-staged FP32 fine-level apply
// The FP32 cycle's fine-level K apply streams 200 MB per launch and is bound by memory latency
// when every lane loads its own values.  Here each warp owns whole 32-row slices and a
// kTmaStages-deep shared-memory pipeline: lane 0 moves the next chunks of kTmaChunk slots of the
// slice (values and block columns, contiguous in the SELL layout) with one bulk asynchronous copy
// per array, completing on an mbarrier, while the warp computes the current chunk from shared
// memory.  Only the x gathers go to global memory.  Every wait is bounded by `polls` tests of the
// mbarrier (a kernel argument, kTmaSpin by default; 0 makes every wait give up without a test, which
// exercises the give-up path deterministically): when any lane of a warp gives up, the whole warp
// gives up (the decision is a warp vote, so the lanes never diverge), sets ST_TIMEOUT, waits for its
// copies still in flight with the full kTmaSpin limit, and returns.
constexpr int kTmaChunk = 4;                       // slots per stage
constexpr int kTmaStages = 3;                      // stages per warp (copies run two chunks ahead)
constexpr int kTmaWarps = 6;                       // warps per CTA
constexpr int kTmaStageBytes = kTmaChunk * 9 * 32 * 4 + kTmaChunk * 32 * 4;   // 3x3 FP32 values + columns
constexpr int kTmaSmem = kTmaWarps * kTmaStages * kTmaStageBytes;
constexpr unsigned kTmaSpin = 1u << 26;           // default polls before a wait gives up

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// true once the phase with the given parity has completed; false after `limit` polls (the
// non-blocking test, so that the limit bounds the time: about a second at most for kTmaSpin)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned limit) {
  for (unsigned it = 0; it < limit; ++it) {
    unsigned done;
    asm volatile(
        "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

struct TmaMeta {
  int valid, s, t0, n, last;
};

// y = op(K x [+ B1 lam]) over the FP32 SELL copy of a 3x3-block matrix (op as in store_row);
// slices are taken in order from the counter *ctr (zero at launch) by lane 0 of each warp.
template <int MODE>
__global__ void __launch_bounds__(kTmaWarps * 32)
k_sell_tma(int nbr, int nslice, const int* __restrict__ soff, const int* __restrict__ slen,
           const int* __restrict__ scol, const float* __restrict__ sval, const float* __restrict__ x,
           const int* __restrict__ rp2, const int* __restrict__ c2, const float* __restrict__ v2,
           const float* __restrict__ x2, const float* __restrict__ b, const float* __restrict__ x0,
           const float* __restrict__ dinv, float omega, float* __restrict__ y, unsigned* __restrict__ ctr,
           int* __restrict__ st, unsigned polls) {
  extern __shared__ __align__(128) unsigned char tma_sh[];
  __shared__ uint64_t bars[kTmaWarps][kTmaStages];
  __shared__ TmaMeta meta[kTmaWarps][kTmaStages];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned char* stage_base = tma_sh + (size_t)wid * kTmaStages * kTmaStageBytes;
  uint64_t* bar = bars[wid];
  TmaMeta* mt = meta[wid];
  // issue state (lane 0 only)
  int is_s = 0, is_t0 = 0, is_len = 0;
  bool is_have = false;
  auto fetch = [&]() {
    const int s = (int)atomicAdd(ctr, 1u);
    is_have = s < nslice;
    if (is_have) {
      is_s = s;
      is_t0 = 0;
      is_len = slen[s];
    }
  };
  auto issue = [&](int stg) {
    TmaMeta m{0, 0, 0, 0, 0};
    if (is_have) {
      const int n = min(kTmaChunk, is_len - is_t0);
      m = TmaMeta{1, is_s, is_t0, n, is_t0 + n >= is_len ? 1 : 0};
      const int64_t g = (int64_t)soff[is_s] + is_t0;
      unsigned char* dv = stage_base + (size_t)stg * kTmaStageBytes;
      unsigned char* dc = dv + kTmaChunk * 9 * 32 * 4;
      const unsigned bv = (unsigned)n * 9u * 32u * 4u, bc = (unsigned)n * 32u * 4u;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&bar[stg], bv + bc);
      if (n > 0) {
        bulk_g2s(dv, sval + g * 288, bv, &bar[stg]);
        bulk_g2s(dc, scol + g * 32, bc, &bar[stg]);
      }
      is_t0 += n;
      if (is_t0 >= is_len) fetch();
    }
    mt[stg] = m;
  };
  if (lane == 0) {
    for (int q = 0; q < kTmaStages; ++q) mbar_init(&bar[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fetch();
    for (int q = 0; q + 1 < kTmaStages; ++q) issue(q);
  }
  __syncwarp();
  unsigned phase = 0u;   // bit q: parity of the next phase of stage q
  float acc[3] = {0.f, 0.f, 0.f};
  for (int k = 0;; ++k) {
    const int stg = k % kTmaStages;
    const TmaMeta m = mt[stg];
    if (!m.valid) break;
    if (lane == 0) issue((k + kTmaStages - 1) % kTmaStages);   // the stage chunk k-1 used
    __syncwarp();
    // every lane tests the barrier (each lane reads the copied data), the warp acts on the vote
    const bool landed = mbar_wait(&bar[stg], (phase >> stg) & 1u, polls);
    if (!__all_sync(0xffffffffu, landed)) {
      // give up, as one warp: record it, wait for this warp's copies still in flight (bounded by
      // the full limit, so that no copy lands after the CTA has left), leave
      if (lane == 0) {
        atomicOr(st, ST_TIMEOUT);
        for (int q = 0; q < kTmaStages; ++q)
          if (mt[q].valid) mbar_wait(&bar[q], (phase >> q) & 1u, kTmaSpin);
      }
      __syncwarp();
      return;
    }
    phase ^= 1u << stg;
    const float* vs = reinterpret_cast<const float*>(stage_base + (size_t)stg * kTmaStageBytes);
    const int* cs = reinterpret_cast<const int*>(vs + kTmaChunk * 9 * 32);
    // all x gathers of the chunk first (slots past n read x[0..2], never used), then the FMAs
    float xr[kTmaChunk][3];
#pragma unroll
    for (int t = 0; t < kTmaChunk; ++t) {
      const float* xc = x + 3 * (int64_t)(t < m.n ? cs[t * 32 + lane] : 0);
      xr[t][0] = __ldg(xc);
      xr[t][1] = __ldg(xc + 1);
      xr[t][2] = __ldg(xc + 2);
    }
#pragma unroll
    for (int t = 0; t < kTmaChunk; ++t) {
      if (t < m.n) {
        const float* v = vs + t * 288 + lane;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          acc[q] = fmaf(v[(3 * q) * 32], xr[t][0], acc[q]);
          acc[q] = fmaf(v[(3 * q + 1) * 32], xr[t][1], acc[q]);
          acc[q] = fmaf(v[(3 * q + 2) * 32], xr[t][2], acc[q]);
        }
      }
    }
    if (m.last) {
      const int row = m.s * 32 + lane;
      if (row < nbr) {
        if (rp2 != nullptr) {
          for (int e = rp2[row]; e < rp2[row + 1]; ++e) {
            const float* blk = v2 + (int64_t)e * 9;
            const float* d = x2 + 3 * (int64_t)c2[e];
            const float d0 = d[0], d1 = d[1], dd2 = d[2];
#pragma unroll
            for (int q = 0; q < 3; ++q) acc[q] = fmaf(blk[3 * q], d0, fmaf(blk[3 * q + 1], d1, fmaf(blk[3 * q + 2], dd2, acc[q])));
          }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) store_row<MODE, float>(y, b, x0, dinv, omega, (int64_t)row * 3 + q, acc[q]);
      }
      acc[0] = acc[1] = acc[2] = 0.f;
    }
    __syncwarp();
  }
}

template <int MODE>
static int launch_sell_tma(const SellV<float>& S, int nbr, const BsrV<float>* A2, const float* x, const float* x2,
                           const float* b, const float* x0, const float* dinv, double omega, float* y,
                           cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  AMGC_CUDA_TRY(cudaGetDevice(&dev));
  AMGC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  AMGC_CUDA_TRY(cudaFuncSetAttribute(k_sell_tma<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTmaSmem));
  AMGC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sell_tma<MODE>, kTmaWarps * 32, kTmaSmem));
  const int grid = std::max(1, std::min(div_up(S.nslice, kTmaWarps), sms * std::max(per_sm, 1)));
  AMGC_CUDA_TRY(cudaMemsetAsync(S.ctr, 0, sizeof(unsigned), s));
  AMGC_LAUNCH(k_sell_tma<MODE><<<grid, kTmaWarps * 32, kTmaSmem, s>>>(
      nbr, S.nslice, S.off, S.len, S.col, S.val, x, A2 ? A2->rp : nullptr, A2 ? A2->col : nullptr,
      A2 ? A2->val : nullptr, x2, b, x0, dinv, (float)omega, y, S.ctr, S.st, S.polls < 0 ? kTmaSpin : (unsigned)S.polls));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

// tpr <= 0: the default (one thread per row in FP64, which is FMA-bound; two in FP32)
template <int MODE, class T>
static int sell_apply(const SellV<T>& S, int nbr, const BsrV<T>* A2, const T* x, const T* x2, const T* b, const T* x0,
                      const T* dinv, double omega, T* y, cudaStream_t s, int tpr = 0) {
  if (tpr <= 0) tpr = sizeof(T) == 8 ? 1 : 2;
  const int* rp2 = A2 ? A2->rp : nullptr;
  const int* c2 = A2 ? A2->col : nullptr;
  const T* v2 = A2 ? A2->val : nullptr;
  if (nbr == 0) return AMGC_OK;
#define AMGC_SELL_CASE(R, C)                                                                         \
  if (S.br == R && S.bc == C) {                                                                      \
    if (tpr == 1) launch_sell<R, C, MODE, T, 1>(S, nbr, rp2, c2, v2, x, x2, b, x0, dinv, omega, y, s); \
    else launch_sell<R, C, MODE, T, 2>(S, nbr, rp2, c2, v2, x, x2, b, x0, dinv, omega, y, s);          \
    AMGC_CUDA_TRY(cudaGetLastError());                                                               \
    return AMGC_OK;                                                                                  \
  }
  AMGC_SELL_CASE(3, 3)
  AMGC_SELL_CASE(3, 6)
  AMGC_SELL_CASE(6, 3)
  AMGC_SELL_CASE(6, 6)
#undef AMGC_SELL_CASE
  set_error("sell_apply: unsupported block shape");
  return AMGC_EINVAL;
}

// Applies of K (with the multiplier coupling A2), P and R with the level's chosen row mapping.
template <int MODE, class T>
static int mapped_apply(const BsrV<T>& A, const SellV<T>& S, int map, const BsrV<T>* A2, const T* x, const T* x2,
                        const T* b, const T* x0, const T* dinv, double omega, T* y, cudaStream_t s) {
  // map 3: the staged kernel for the FP32 fine-level 3x3 K (an autotuner candidate)
  if constexpr (sizeof(T) == 4 && MODE != 1 && MODE != 4) {
    if (map == 3 && S.ctr != nullptr && S.nslice > 0 && S.br == 3 && S.bc == 3 && S.perm == nullptr)
      return launch_sell_tma<MODE>(S, A.nbr, A2, x, x2, b, x0, dinv, omega, y, s);
  }
  if (map == 3) map = -1;
  if (S.nslice > 0 && map != 0) return sell_apply<MODE, T>(S, A.nbr, A2, x, x2, b, x0, dinv, omega, y, s, map);
  return rowop<MODE, T>(A, x, A2, x2, b, x0, dinv, omega, y, s);
}

// ------------------------------------------------------------------ multiplier-node kernels
// One warp per multiplier node.
// MODE 0: out_l = g_l - (B2 u)_l + Z_l lam_l                       (residual)
// MODE 1: d = -Sinv_l (g_l - (B2 u)_l + Z_l lam_l); lam_l += alpha d; out_l = d  (corrector)
// MODE 2: out_l = (B2 u)_l - Z_l lam_l                             (saddle apply)
// Lanes per multiplier node (and per B1 row) of the multiplier-row kernels: a group of G lanes
// shares a row's blocks (lane-per-block in strides of G), the group sum is an xor butterfly (every
// lane of the group ends with the same bits: IEEE addition commutes), and the per-component
// epilogue runs on lanes 0 .. 2 (0 .. BU-1) of the group, so that a warp serves 32 / G rows and
// the FP64 epilogue costs one warp instruction per step for all of them.
template <int BU>
struct RowGroup {
  static constexpr int G = BU <= 4 ? 4 : 8;
};
template <int G, class T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
  return v;
}
template <int BR, int BC, int G, class T>
__device__ __forceinline__ void group_blocks(int64_t b0, int64_t b1, const int* __restrict__ col,
                                             const T* __restrict__ val, const T* __restrict__ x, int gl,
                                             T (&acc)[BR]) {
#pragma unroll 2
  for (int64_t b = b0 + gl; b < b1; b += G) {
    const T* xc = x + (int64_t)__ldg(col + b) * BC;
    T xv[BC];
#pragma unroll
    for (int c = 0; c < BC; ++c) xv[c] = ldg(xc + c);
    const T* v = val + b * (BR * BC);
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int c = 0; c < BC; ++c) acc[r] = fma(ldg(v + r * BC + c), xv[c], acc[r]);
  }
}
// one multiplier node l per group of G lanes (gl: lane in the group); every lane of the warp calls
// it (the group sums and the exchange of the residual components are warp shuffles), `valid`
// false for the groups past the last node
template <int G, int BU, int MODE, class T>
__device__ __forceinline__ void lm_node(int l, bool valid, int gl, const int* __restrict__ rp,
                                        const int* __restrict__ col, const T* __restrict__ val,
                                        const T* __restrict__ u, const T* __restrict__ Z, const T* __restrict__ g,
                                        T* __restrict__ lam, const double* __restrict__ Sinv, double alpha,
                                        T* __restrict__ out) {
  // the loads that do not depend on the row's blocks go first, so that their latencies overlap
  const int c = gl < 3 ? gl : 0;   // lanes 3 .. G-1 of a group mirror component 0 and store nothing
  const bool st = valid && gl < 3;
  int b0 = 0, b1 = 0;
  T z0 = T(0), z1 = T(0), z2 = T(0), l0 = T(0), l1 = T(0), l2 = T(0), gc = T(0);
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  if (valid) {
    b0 = rp[l];
    b1 = rp[l + 1];
    const T* z = Z + (int64_t)l * 9 + 3 * c;
    z0 = z[0];
    z1 = z[1];
    z2 = z[2];
    l0 = lam[3 * (int64_t)l];
    l1 = lam[3 * (int64_t)l + 1];
    l2 = lam[3 * (int64_t)l + 2];
    if (MODE != 2) gc = g[3 * (int64_t)l + c];
    if (MODE == 1) {
      const double* S = Sinv + (int64_t)l * 9 + 3 * c;   // FP64 Schur-block inverse, row c
      s0 = S[0];
      s1 = S[1];
      s2 = S[2];
    }
  }
  T acc[3] = {T(0), T(0), T(0)};
  if (valid) group_blocks<3, BU, G, T>(b0, b1, col, val, u, gl, acc);
  const T bu0 = group_sum<G>(acc[0]), bu1 = group_sum<G>(acc[1]), bu2 = group_sum<G>(acc[2]);
  const T buc = c == 0 ? bu0 : (c == 1 ? bu1 : bu2);
  const T zl = z0 * l0 + z1 * l1 + z2 * l2;
  const T lc = c == 0 ? l0 : (c == 1 ? l1 : l2);
  if (MODE == 2) {
    if (st) out[3 * (int64_t)l + c] = buc - zl;
    return;
  }
  const T rc = gc - buc + zl;
  if (MODE == 0) {
    if (st) out[3 * (int64_t)l + c] = rc;
    return;
  }
  const int g0 = (threadIdx.x & 31) & ~(G - 1);   // first lane of the group
  const T r0 = __shfl_sync(0xffffffffu, rc, g0), r1 = __shfl_sync(0xffffffffu, rc, g0 + 1),
          r2 = __shfl_sync(0xffffffffu, rc, g0 + 2);
  if (!st) return;
  const double d = -(s0 * r0 + s1 * r1 + s2 * r2);
  lam[3 * (int64_t)l + c] = (T)(lc + alpha * d);
  out[3 * (int64_t)l + c] = (T)d;
}

template <int BU, int MODE, class T, int G>
__global__ void __launch_bounds__(128)
k_lm(int nl, const int* __restrict__ rp, const int* __restrict__ col, const T* __restrict__ val,
     const T* __restrict__ u, const T* __restrict__ Z, const T* __restrict__ g, T* __restrict__ lam,
     const double* __restrict__ Sinv, double alpha, T* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int first = (int)((gt >> 5) * (32 / G));   // the warp's first node
  if (first >= nl) return;                         // whole warps only: the groups shuffle
  const int l = first + lane / G;
  lm_node<G, BU, MODE, T>(l, l < nl, lane & (G - 1), rp, col, val, u, Z, g, lam, Sinv, alpha, out);
}
// grid of the group-per-row kernels: 32 / G rows per warp, 128-thread blocks
template <int BU>
static int group_grid(int64_t rows) {
  return (int)div_up(rows * RowGroup<BU>::G, 128);
}
// Lanes per row of the corrector, multiplier-residual and B1-update launches.  Few rows (under
// kGroupRowsFP64 in FP64, any count in FP32) leave these launches bound by the chain of dependent
// loads of a row: the smallest of 8, 16, 32 lanes that covers the rows' mean length, so that a
// row takes one pass of its group.  Many FP64 rows make the FP64 pipe the limit, where every
// group-sum round costs a warp instruction whatever the group's width: 4 lanes per row (8 for
// six-DOF B1 rows, which need six), a few passes per row and two rounds per sum.
constexpr int64_t kGroupRowsFP64 = 4096;
static int pick_group(int64_t nnzb, int64_t rows, bool fp64, int bu) {
  if (fp64 && rows >= kGroupRowsFP64) return bu <= 4 ? 4 : 8;
  const double mean = rows > 0 ? (double)nnzb / (double)rows : 0.0;
  return mean <= 8.0 ? 8 : (mean <= 16.0 ? 16 : 32);
}
// the same with 4 lanes allowed (three-DOF rows)
#define AMGC_GROUP_DISPATCH3(gsel, LAUNCH) \
  do {                                     \
    if ((gsel) == 4) {                     \
      constexpr int G_ = 4;                \
      LAUNCH;                              \
    } else {                               \
      AMGC_GROUP_DISPATCH(gsel, LAUNCH);   \
    }                                      \
  } while (0)
#define AMGC_GROUP_DISPATCH(gsel, LAUNCH) \
  do {                                    \
    if ((gsel) == 8) {                    \
      constexpr int G_ = 8;               \
      LAUNCH;                             \
    } else if ((gsel) == 16) {            \
      constexpr int G_ = 16;              \
      LAUNCH;                             \
    } else {                              \
      constexpr int G_ = 32;              \
      LAUNCH;                             \
    }                                     \
  } while (0)

template <int MODE, class T>
static int lm_op(const LevelV<T>& L, const T* u, const T* g, T* lam, double alpha, T* out, cudaStream_t s,
                 bool transposed = false) {
  if (L.nl == 0) return AMGC_OK;
  const int th = 128;
  const BsrV<T>& B = transposed ? L.B1T : L.B2;   // multiplier rows of A: B2; of A^T: B1^T
  const T* Z = transposed ? L.ZT : L.Z;
  const int gs = pick_group(B.nnzb, L.nl, sizeof(T) == 8, L.bu);
  const int grid = (int)div_up((int64_t)L.nl * gs, th);
  if (L.bu == 3)
    AMGC_GROUP_DISPATCH3(gs, AMGC_LAUNCH((k_lm<3, MODE, T, G_><<<grid, th, 0, s>>>(L.nl, B.rp, B.col, B.val, u, Z, g,
                                                                                 lam, L.Sinv, alpha, out))));
  else
    AMGC_GROUP_DISPATCH(gs, AMGC_LAUNCH((k_lm<6, MODE, T, G_><<<grid, th, 0, s>>>(L.nl, B.rp, B.col, B.val, u, Z, g,
                                                                                 lam, L.Sinv, alpha, out))));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

template <class T>
__global__ void k_copy(int64_t n, const T* __restrict__ a, T* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = a[i];
}
template <class Tb>
__device__ __forceinline__ Tb convert_to(double v) { return (Tb)v; }
template <>
__device__ __forceinline__ float convert_to<float>(double v) { return f64_to_f32_rn(v); }
template <class Tb>
__device__ __forceinline__ Tb convert_to(float v) { return (Tb)v; }
template <class Ta, class Tb>
__global__ void k_convert(int64_t n, const Ta* __restrict__ a, Tb* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = convert_to<Tb>(a[i]);
}
template <class T>
__global__ void k_zero(int64_t n, T* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = T(0);
}
// Jacobi sweep from a zero guess, y = omega D^-1 f, with the multipliers' zero guess (lam = 0)
// set in the same launch
template <class T>
__global__ void k_jacobi_zero(int64_t n, int64_t nlam, const T* __restrict__ f, const T* __restrict__ dinv, T omega,
                              T* __restrict__ y, T* __restrict__ lam) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = omega * dinv[i] * f[i];
  if (i < nlam) lam[i] = T(0);
}
// u_i = uin_i - alpha atinv_i (B1 dlam)_i for row i of B1 (one group of G lanes, see lm_node),
// with uin = u for the update in place
template <int G, int BU, class T>
__device__ __forceinline__ void b1_row(int i, bool valid, int gl, const int* __restrict__ rp,
                                       const int* __restrict__ col, const T* __restrict__ val,
                                       const T* __restrict__ dlam, const T* __restrict__ atinv, T alpha,
                                       const T* uin, T* u) {
  const bool st = valid && gl < BU;
  int b0 = 0, b1 = 0;
  T ui = T(0), ai = T(0);
  if (valid) {
    b0 = rp[i];
    b1 = rp[i + 1];
  }
  if (st) {   // independent of the row's blocks: issued before them
    ui = uin[(int64_t)i * BU + gl];
    ai = atinv[(int64_t)i * BU + gl];
  }
  T acc[BU];
#pragma unroll
  for (int r = 0; r < BU; ++r) acc[r] = T(0);
  if (valid) group_blocks<BU, 3, G, T>(b0, b1, col, val, dlam, gl, acc);
  T out = T(0);
#pragma unroll
  for (int r = 0; r < BU; ++r) {
    const T v = group_sum<G>(acc[r]);
    if (gl == r) out = v;
  }
  if (st) {
    ui -= alpha * ai * out;
    u[(int64_t)i * BU + gl] = ui;
  }
}
// the same over the rows of B1 with entries, in place, 32 / G rows per warp
template <int BU, class T, int G>
__global__ void __launch_bounds__(128)
k_b1_update(int nrows, const int* __restrict__ rows, const int* __restrict__ rp, const int* __restrict__ col,
            const T* __restrict__ val, const T* __restrict__ dlam, const T* __restrict__ atinv, T alpha, T* u) {
  static_assert(G >= BU, "a B1 row's update needs BU lanes of its group");
  const int lane = threadIdx.x & 31;
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int first = (int)((gt >> 5) * (32 / G));
  if (first >= nrows) return;
  const int t = first + lane / G;
  const bool valid = t < nrows;
  b1_row<G, BU, T>(valid ? rows[t] : 0, valid, lane & (G - 1), rp, col, val, dlam, atinv, alpha, u, u);
}
template <class T>
static int b1_update(int bu, int nrows, const int* rows, const BsrV<T>& B, const T* dlam, const T* atinv, T alpha, T* u,
                     cudaStream_t s) {
  if (nrows == 0) return AMGC_OK;
  const int gs = pick_group(B.nnzb, nrows, sizeof(T) == 8, bu);   // the rows listed hold all of B's blocks
  const int grid = (int)div_up((int64_t)nrows * gs, 128);
  if (bu == 3)
    AMGC_GROUP_DISPATCH3(gs, AMGC_LAUNCH((k_b1_update<3, T, G_><<<grid, 128, 0, s>>>(nrows, rows, B.rp, B.col, B.val,
                                                                                   dlam, atinv, alpha, u))));
  else
    AMGC_GROUP_DISPATCH(gs, AMGC_LAUNCH((k_b1_update<6, T, G_><<<grid, 128, 0, s>>>(nrows, rows, B.rp, B.col, B.val,
                                                                                   dlam, atinv, alpha, u))));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}
// Split sweep (smoother form 2).  The corrector reads the Jacobi iterate only on the interface rows
// (B2's columns) and the B1 update writes only there (B1's rows), so those rows take their Jacobi
// step into a compact vector uI on a second stream, where the corrector follows at once, while
// the Jacobi step of all rows runs on the main stream; after the join the B1 update writes the
// interface rows' final values over the main step's output.  The arithmetic per row is that of
// the sequential sweep, the K row's sum in lane-per-block order.
// uI_t = x_i + omega dinv_i (f_i - K_i x - B1_i lam) for interface row i = rows[t] (one warp)
template <int BU, class T>
__global__ void __launch_bounds__(128)
k_ir_jacobi(int n, const int* __restrict__ rows, const int* __restrict__ krp, const int* __restrict__ kcol,
            const T* __restrict__ kval, const T* __restrict__ x, const int* __restrict__ brp,
            const int* __restrict__ bcol, const T* __restrict__ bval, const T* __restrict__ lam,
            const T* __restrict__ f, const T* __restrict__ dinv, T omega, T* __restrict__ uI) {
  const int lane = threadIdx.x & 31;
  const int t = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (t >= n) return;
  const int i = rows[t];
  T acc[BU];
#pragma unroll
  for (int r = 0; r < BU; ++r) acc[r] = T(0);
  lane_blocks<BU, BU, T>(krp[i], krp[i + 1], kcol, kval, x, lane, acc);
  lane_blocks<BU, 3, T>(brp[i], brp[i + 1], bcol, bval, lam, lane, acc);
  T out = T(0);
#pragma unroll
  for (int r = 0; r < BU; ++r) {
    const T v = warp_sum(acc[r]);
    if (lane == r) out = v;
  }
  if (lane < BU) {
    const int64_t o = (int64_t)i * BU + lane;
    uI[(int64_t)t * BU + lane] = x[o] + omega * dinv[o] * (f[o] - out);
  }
}
// u_i = uI_t - alpha atinv_i (B1 dlam)_i for interface row i = rows[t] (groups of G lanes, as
// k_b1_update)
template <int BU, class T>
__global__ void __launch_bounds__(128)
k_ir_b1(int n, const int* __restrict__ rows, const int* __restrict__ rp, const int* __restrict__ col,
        const T* __restrict__ val, const T* __restrict__ dlam, const T* __restrict__ atinv, T alpha,
        const T* __restrict__ uI, T* __restrict__ u) {
  constexpr int G = RowGroup<BU>::G;
  const int lane = threadIdx.x & 31, gl = lane & (G - 1);
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int first = (int)((gt >> 5) * (32 / G));
  if (first >= n) return;
  const int t = first + lane / G;
  const bool valid = t < n;
  const int i = valid ? rows[t] : 0;
  T acc[BU];
#pragma unroll
  for (int r = 0; r < BU; ++r) acc[r] = T(0);
  if (valid) group_blocks<BU, 3, G, T>(rp[i], rp[i + 1], col, val, dlam, gl, acc);
  T out = T(0);
#pragma unroll
  for (int r = 0; r < BU; ++r) {
    const T v = group_sum<G>(acc[r]);
    if (gl == r) out = v;
  }
  if (valid && gl < BU) {
    T ui = uI[(int64_t)t * BU + gl];
    ui -= alpha * atinv[(int64_t)i * BU + gl] * out;
    u[(int64_t)i * BU + gl] = ui;
  }
}
// Fused corrector and B1 update of a CheapSIMPLE sweep in one CTA: the multiplier corrector on
// every node (as k_lm MODE 1), a block barrier, then the B1 update of every row of B1 with entries
// (as k_b1_update); the same arithmetic as the two launches, in one launch.  One CTA, so it pays
// only where a level's multiplier rows are few (the autotuner decides per level).
constexpr int kFuseThreads = 1024;
constexpr int kFuseMaxNodes = 2048;   // largest level the autotuner tries the single-CTA form on
template <int BU, class T, int GL, int GB>
__global__ void __launch_bounds__(kFuseThreads)
k_corrector_b1_fused(int nl, const int* __restrict__ rp2, const int* __restrict__ c2, const T* __restrict__ v2,
                     const T* u_in, const T* __restrict__ Z, const T* __restrict__ g,
                     T* __restrict__ lam, const double* __restrict__ Sinv, double alpha, T* __restrict__ dlam,
                     int nrows, const int* __restrict__ rows, const int* __restrict__ rp1, const int* __restrict__ c1,
                     const T* __restrict__ v1, const T* __restrict__ atinv, T* u) {
  // u_in and u are the same iterate: read by the corrector, updated after the barrier; GL and GB
  // lanes per row, as the two launches choose them (the same arithmetic, the same bits)
  constexpr int RL = 32 / GL, RB = 32 / GB;   // rows per warp
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int f = wid * RL; f < nl; f += nw * RL) {   // warp-uniform bounds: the groups shuffle
    const int l = f + lane / GL;
    lm_node<GL, BU, 1, T>(l, l < nl, lane & (GL - 1), rp2, c2, v2, u_in, Z, g, lam, Sinv, alpha, dlam);
  }
  __syncthreads();
  for (int f = wid * RB; f < nrows; f += nw * RB) {
    const int t = f + lane / GB;
    const bool valid = t < nrows;
    b1_row<GB, BU, T>(valid ? rows[t] : 0, valid, lane & (GB - 1), rp1, c1, v1, dlam, atinv, (T)alpha, u, u);
  }
}
template <int BU, class T, int GL>
static void launch_fused(const LevelV<T>& L, int gb, T* u, const T* g, T* lam, double alpha, cudaStream_t s) {
#define AMGC_FUSED_LAUNCH                                                                            \
  AMGC_LAUNCH((k_corrector_b1_fused<BU, T, GL, G_><<<1, kFuseThreads, 0, s>>>(                       \
      L.nl, L.B2.rp, L.B2.col, L.B2.val, u, L.Z, g, lam, L.Sinv, alpha, L.dlam, L.n_b1_rows, L.b1_rows, \
      L.B1.rp, L.B1.col, L.B1.val, L.atinv, u)))
  if constexpr (BU == 3) AMGC_GROUP_DISPATCH3(gb, AMGC_FUSED_LAUNCH);
  else AMGC_GROUP_DISPATCH(gb, AMGC_FUSED_LAUNCH);
#undef AMGC_FUSED_LAUNCH
}
template <class T>
static int corrector_b1_fused(const LevelV<T>& L, T* u, const T* g, T* lam, double alpha, cudaStream_t s) {
  // the lane groups of the two launches (lm_op, b1_update), so that the bits are theirs
  const bool fp64 = sizeof(T) == 8;
  const int gl = pick_group(L.B2.nnzb, L.nl, fp64, L.bu), gb = pick_group(L.B1.nnzb, L.n_b1_rows, fp64, L.bu);
  if (L.bu == 3)
    AMGC_GROUP_DISPATCH3(gl, (launch_fused<3, T, G_>(L, gb, u, g, lam, alpha, s)));
  else
    AMGC_GROUP_DISPATCH(gl, (launch_fused<6, T, G_>(L, gb, u, g, lam, alpha, s)));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

// u = uh - alpha atinv (B1 dlam) in one launch: blocks below ncopy copy uh into u on the rows
// without B1 entries (one thread per DOF), the others update the rows of B1 as k_b1_update does,
// reading uh
template <int BU, class T>
__global__ void __launch_bounds__(128)
k_copy_b1(int64_t nu, int ncopy, const T* __restrict__ uh, int nrows, const int* __restrict__ rows,
          const int* __restrict__ rp, const int* __restrict__ col, const T* __restrict__ val,
          const T* __restrict__ dlam, const T* __restrict__ atinv, T alpha, T* __restrict__ u) {
  if ((int)blockIdx.x < ncopy) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nu) return;
    const int64_t node = i / BU;
    if (rp[node + 1] == rp[node]) u[i] = uh[i];
    return;
  }
  const int lane = threadIdx.x & 31;
  const int t = (int)(((blockIdx.x - ncopy) * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (t >= nrows) return;
  const int i = rows[t];
  T acc[BU];
#pragma unroll
  for (int r = 0; r < BU; ++r) acc[r] = T(0);
  lane_blocks<BU, 3, T>(rp[i], rp[i + 1], col, val, dlam, lane, acc);
  T out = T(0);
#pragma unroll
  for (int r = 0; r < BU; ++r) {
    const T v = warp_sum(acc[r]);
    if (lane == r) out = v;
  }
  if (lane < BU) u[(int64_t)i * BU + lane] = uh[(int64_t)i * BU + lane] - alpha * atinv[(int64_t)i * BU + lane] * out;
}
// multiplier restriction / prolongation through P-hat^lambda (weights w_l, aggregate lagg_l)
// (restriction: one warp per coarse multiplier node, the lanes over its members)
template <class T>
__global__ void k_restrict_lm(int nlc, const int* __restrict__ ptr, const int* __restrict__ idx, const T* __restrict__ w,
                              const T* __restrict__ r, T* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int L = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (L >= nlc) return;
  T s0 = 0, s1 = 0, s2 = 0;
  for (int e = ptr[L] + lane; e < ptr[L + 1]; e += 32) {
    const int l = idx[e];
    const T wl = w[l];
    s0 += wl * r[3 * l];
    s1 += wl * r[3 * l + 1];
    s2 += wl * r[3 * l + 2];
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  if (lane == 0) {
    out[3 * L] = s0;
    out[3 * L + 1] = s1;
    out[3 * L + 2] = s2;
  }
}
template <class T>
__global__ void k_prolong_lm(int nl, const int* __restrict__ lagg, const T* __restrict__ w, const T* __restrict__ c,
                             T* __restrict__ lam) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nl) return;
  const int L = lagg[l];
  const T wl = w[l];
  lam[3 * l] += wl * c[3 * L];
  lam[3 * l + 1] += wl * c[3 * L + 1];
  lam[3 * l + 2] += wl * c[3 * L + 2];
}
// coarsest solve: y = A^{-1} x with the FP64 inverse (row-major), one warp per row
template <class T>
__global__ void k_gemv(int n, const double* __restrict__ A, const T* __restrict__ x, T* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  const double* a = A + (int64_t)row * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s = fma(a[j], (double)x[j], s);
  s = warp_sum(s);
  if (lane == 0) y[row] = (T)s;
}

// batched coarsest solve: y_g = sum_t A_q[loc(g)][t] x[glob_q(t)], q the instance of row g
template <class T>
__global__ void k_gemv_batched(int n, const int* __restrict__ inst, const int* __restrict__ loc,
                               const int* __restrict__ glob, const int* __restrict__ goff,
                               const int64_t* __restrict__ doff, const double* __restrict__ A,
                               const T* __restrict__ x, T* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  const int q = inst[row];
  const int g0 = goff[q], nq = goff[q + 1] - g0;
  const double* a = A + doff[q] + (int64_t)loc[row] * nq;
  double s = 0.0;
  for (int j = lane; j < nq; j += 32) s = fma(a[j], (double)x[glob[g0 + j]], s);
  s = warp_sum(s);
  if (lane == 0) y[row] = (T)s;
}

// ------------------------------------------------------------------ level operations
// Algorithmic bytes of one fine-level K-apply launch: K and B1 values and indices once, x and
// lambda once, the output once, plus `extra_vecs` further length-nu vectors.
template <class T>
static double k_apply_bytes(const LevelV<T>& L, int extra_vecs) {
  const double s = sizeof(T);
  double b = (double)L.K.nnzb * (L.bu * L.bu * s + 4.0) + 4.0 * (L.nn + 1);
  b += (double)L.B1.nnzb * (L.bu * 3 * s + 4.0) + (L.nl ? 4.0 * (L.nn + 1) + 3.0 * L.nl * s : 0.0);
  b += (2.0 + extra_vecs) * L.nu() * s;
  return b;
}

// K apply of level l (MODE of k_rowop), timed when the level is the finest one.
// Without `with_b1` the multiplier coupling is left out (the split sweep, whose interface rows,
// the only rows of B1, are recomputed beside it).
template <int MODE, class T>
static int k_apply(amgc_hierarchy* h, const LevelV<T>& L, int l, const T* x1, const T* lam, const T* b, const T* x0,
                   T* y, bool transposed = false, bool with_b1 = true) {
  const bool t = l == 0;
  const int kind = sizeof(T) == 8 ? 1 : 2;
  if (t) AMGC_TRY(prof_begin(h, kind));
  // K is symmetric on every level (elasticity and Galerkin products), so A^T shares it;
  // the multiplier coupling of the u rows is B1 for A and B2^T for A^T.
  const BsrV<T>* B1 = (L.nl && with_b1) ? (transposed ? &L.B2T : &L.B1) : nullptr;
  AMGC_TRY((mapped_apply<MODE, T>(L.K, L.Ks, L.kmap, B1, x1, lam, b, x0, L.dinv, L.omega_j, y, h->stream)));
  if (t)
    AMGC_TRY(prof_end(h, kind, k_apply_bytes(L, MODE == 3 ? 3 : (MODE == 2 ? 1 : 0)),
                      2.0 * ((double)L.K.nnzb * L.bu * L.bu + (double)L.B1.nnzb * L.bu * 3)));
  return AMGC_OK;
}

// Runs side(stream) on the hierarchy's side stream beside main() on its stream: a fork and a
// join through events, which a stream capture records as two parallel graph branches.  Used
// where a short kernel on the multiplier rows and a long one on the displacement rows read the
// same inputs and write disjoint outputs.
template <class FMain, class FSide>
static int fork_join(amgc_hierarchy* h, FMain&& main_fn, FSide&& side_fn) {
  if (!h->side_stream) {
    // the side stream's short kernels get the highest priority, so that their blocks start as soon
    // as blocks of the long kernel beside them retire
    int least = 0, greatest = 0;
    AMGC_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    AMGC_CUDA_TRY(cudaStreamCreateWithPriority(&h->side_stream, cudaStreamNonBlocking, greatest));
    AMGC_CUDA_TRY(cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
    AMGC_CUDA_TRY(cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming));
  }
  AMGC_CUDA_TRY(cudaEventRecord(h->fork_ev, h->stream));
  AMGC_CUDA_TRY(cudaStreamWaitEvent(h->side_stream, h->fork_ev, 0));
  AMGC_TRY(side_fn(h->side_stream));
  AMGC_CUDA_TRY(cudaEventRecord(h->join_ev, h->side_stream));
  AMGC_TRY(main_fn());
  AMGC_CUDA_TRY(cudaStreamWaitEvent(h->stream, h->join_ev, 0));
  return AMGC_OK;
}

static int block_smooth(amgc_hierarchy* h, int l, const double* b, double* x, bool zero_guess);

// `sweeps` CheapSIMPLE sweeps on [u; lambda] = x (Algorithm 4 in its cheap form), each: J damped
// Jacobi steps on the displacements, the multiplier corrector dlam = -S_bd^-1 (g - B2 u_h + Z lam),
// lam += alpha dlam, and u = u_h - alpha A~^-1 B1 dlam.  A Jacobi step reads its iterate at the
// neighbours, so it writes the other of the two displacement buffers (u and the level's t); the
// corrector and the B1 update then work in place on the buffer that holds the iterate.  From a zero
// guess the first step needs no product and its buffer is chosen so that the last step ends in u;
// from the iterate in u the steps alternate t, u, ..., and an odd count ends with one copy into u.
template <class T>
static int smooth_sweeps(amgc_hierarchy* h, const LevelV<T>& L, int l, const T* b, T* x, int sweeps, bool zero_guess) {
  if constexpr (sizeof(T) == 8) {
    if (h->smoother_kind != 0) {
      for (int k = 0; k < sweeps; ++k) AMGC_TRY(block_smooth(h, l, b, x, zero_guess && k == 0));
      return AMGC_OK;
    }
  }
  cudaStream_t s = h->stream;
  const int nu = L.nu();
  const T* f = b;
  const T* g = b + nu;
  T* u = x;
  T* lam = x + nu;
  T* t = L.t;
  const int th = 256;
  const int J = h->opts.jacobi_sweeps;
  const int steps = sweeps * J;
  T* cur = u;
  int step = 0;
  const bool split = L.fuse == 2 && L.nl > 0 && L.n_ir > 0;
  for (int k = 0; k < sweeps; ++k) {
    bool corrected = false;
    for (int j = 0; j < J; ++j, ++step) {
      if (split && j == J - 1 && !(zero_guess && step == 0)) {
        // the last Jacobi step of the sweep with the corrector and B1 update split off (form 2)
        T* dst = cur == u ? t : u;
        const T* src = cur;
        const T alpha = (T)h->opts.simple_alpha;
        AMGC_TRY(fork_join(
            h, [&]() { return k_apply<3, T>(h, L, l, src, lam, f, src, dst, false, false); },
            [&](cudaStream_t ss) -> int {
              const int gi = div_up((int64_t)L.n_ir * 32, 128);
              if (L.bu == 3)
                AMGC_LAUNCH(k_ir_jacobi<3, T><<<gi, 128, 0, ss>>>(L.n_ir, L.ir_rows, L.K.rp, L.K.col, L.K.val, src,
                                                                  L.B1.rp, L.B1.col, L.B1.val, lam, f, L.dinv,
                                                                  (T)L.omega_j, L.ir_u));
              else
                AMGC_LAUNCH(k_ir_jacobi<6, T><<<gi, 128, 0, ss>>>(L.n_ir, L.ir_rows, L.K.rp, L.K.col, L.K.val, src,
                                                                  L.B1.rp, L.B1.col, L.B1.val, lam, f, L.dinv,
                                                                  (T)L.omega_j, L.ir_u));
              AMGC_CUDA_TRY(cudaGetLastError());
              LevelV<T> Li = L;   // B2 with its columns numbered among the interface rows
              Li.B2.col = L.ir_b2c;
              return lm_op<1, T>(Li, L.ir_u, g, lam, h->opts.simple_alpha, L.dlam, ss);
            }));
        if (L.bu == 3)
          AMGC_LAUNCH(k_ir_b1<3, T><<<group_grid<3>(L.n_ir), 128, 0, s>>>(L.n_ir, L.ir_rows, L.B1.rp, L.B1.col, L.B1.val, L.dlam,
                                                       L.atinv, alpha, L.ir_u, dst));
        else
          AMGC_LAUNCH(k_ir_b1<6, T><<<group_grid<6>(L.n_ir), 128, 0, s>>>(L.n_ir, L.ir_rows, L.B1.rp, L.B1.col, L.B1.val, L.dlam,
                                                       L.atinv, alpha, L.ir_u, dst));
        AMGC_CUDA_TRY(cudaGetLastError());
        cur = dst;
        corrected = true;
      } else if (zero_guess && step == 0) {
        T* dst = ((steps - 1) % 2 == 0) ? u : t;
        const int64_t nlam = 3 * (int64_t)L.nl;
        AMGC_LAUNCH(k_jacobi_zero<T><<<div_up(std::max<int64_t>(nu, nlam), th), th, 0, s>>>(nu, nlam, f, L.dinv,
                                                                                        (T)L.omega_j, dst, lam));
        AMGC_CUDA_TRY(cudaGetLastError());
        cur = dst;
      } else {
        T* dst = cur == u ? t : u;
        AMGC_TRY((k_apply<3, T>(h, L, l, cur, lam, f, cur, dst)));
        cur = dst;
      }
    }
    if (corrected) continue;
    // corrector on the multipliers and the B1 update of the displacements, in place on cur: one
    // fused single-CTA launch where the autotuner found it faster, else two launches
    if (L.fuse == 1 && L.nl > 0) {
      AMGC_TRY(corrector_b1_fused<T>(L, cur, g, lam, h->opts.simple_alpha, s));
      continue;
    }
    AMGC_TRY((lm_op<1, T>(L, cur, g, lam, h->opts.simple_alpha, L.dlam, s)));
    AMGC_TRY(b1_update<T>(L.bu, L.n_b1_rows, L.b1_rows, L.B1, L.dlam, L.atinv, (T)h->opts.simple_alpha, cur, s));
  }
  if (cur != u) {
    AMGC_LAUNCH(k_copy<T><<<div_up(nu, th), th, 0, s>>>(nu, cur, u));
    AMGC_CUDA_TRY(cudaGetLastError());
  }
  return AMGC_OK;
}

// ------------------------------------------------------------------ block smoothers (Sec. 5.1, 5.2)
// Uzawa (Algorithm 2), Braess-Sarazin (Algorithm 3) and SIMPLE (Algorithm 4) in the cheap forms:
// K solves by damped symmetric block Gauss-Seidel in colour order, Schur solves by the block ILU(0)
// factors of the assembled approximation (set up in blocksmooth.cu).  FP64, one sweep per call.

// x_i += omega K_ii^-1 (b_i - sum_j K_ij x_j) for the nodes of one colour (one warp per node; the
// nodes of a colour do not couple, so they update x in place together)
template <int BU>
__global__ void __launch_bounds__(128)
k_cbsgs(int cnt, const int* __restrict__ nodes, const int* __restrict__ rp, const int* __restrict__ col,
        const double* __restrict__ val, const double* __restrict__ kdinv, const double* __restrict__ b,
        double* __restrict__ x, double omega) {
  const int lane = threadIdx.x & 31;
  const int t = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (t >= cnt) return;
  const int i = nodes[t];
  double acc[BU];
#pragma unroll
  for (int r = 0; r < BU; ++r) acc[r] = 0.0;
  lane_blocks<BU, BU, double>(rp[i], rp[i + 1], col, val, x, lane, acc);
#pragma unroll
  for (int r = 0; r < BU; ++r) acc[r] = warp_sum(acc[r]);
  if (lane != 0) return;
  double res[BU];
#pragma unroll
  for (int r = 0; r < BU; ++r) res[r] = b[(int64_t)i * BU + r] - acc[r];
  const double* D = kdinv + (int64_t)i * BU * BU;
#pragma unroll
  for (int r = 0; r < BU; ++r) {
    double d = 0.0;
#pragma unroll
    for (int c = 0; c < BU; ++c) d = fma(D[r * BU + c], res[c], d);
    x[(int64_t)i * BU + r] += omega * d;
  }
}

// x = U^-1 L^-1 r with the block ILU(0) factors, by levels in one CTA: forward y_i = r_i - sum_{j<i}
// L_ij y_j, then backward x_i = U_ii^-1 (y_i - sum_{j>i} U_ij x_j), in place in x; one warp per row
// of a level, a CTA barrier between levels (rows of a level read only rows of earlier levels)
constexpr int kIluThreads = 1024;
__global__ void __launch_bounds__(kIluThreads)
k_ilu_solve(const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
            const int* __restrict__ diag, const double* __restrict__ uinv, int nlev_l, const int* __restrict__ lptr,
            const int* __restrict__ lrows, int nlev_u, const int* __restrict__ uptr, const int* __restrict__ urows,
            const double* __restrict__ r, double* x) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int v = 0; v < nlev_l; ++v) {
    for (int t = lptr[v] + wid; t < lptr[v + 1]; t += nw) {
      const int i = lrows[t];
      double a0 = 0.0, a1 = 0.0, a2 = 0.0;
      for (int e = rp[i] + lane; e < diag[i]; e += 32) {
        const double* m = val + (int64_t)e * 9;
        const double* y = x + 3 * (int64_t)col[e];
        a0 += m[0] * y[0] + m[1] * y[1] + m[2] * y[2];
        a1 += m[3] * y[0] + m[4] * y[1] + m[5] * y[2];
        a2 += m[6] * y[0] + m[7] * y[1] + m[8] * y[2];
      }
      a0 = warp_sum(a0);
      a1 = warp_sum(a1);
      a2 = warp_sum(a2);
      if (lane == 0) {
        x[3 * (int64_t)i] = r[3 * (int64_t)i] - a0;
        x[3 * (int64_t)i + 1] = r[3 * (int64_t)i + 1] - a1;
        x[3 * (int64_t)i + 2] = r[3 * (int64_t)i + 2] - a2;
      }
    }
    __syncthreads();
  }
  for (int v = 0; v < nlev_u; ++v) {
    for (int t = uptr[v] + wid; t < uptr[v + 1]; t += nw) {
      const int i = urows[t];
      double a0 = 0.0, a1 = 0.0, a2 = 0.0;
      for (int e = diag[i] + 1 + lane; e < rp[i + 1]; e += 32) {
        const double* m = val + (int64_t)e * 9;
        const double* y = x + 3 * (int64_t)col[e];
        a0 += m[0] * y[0] + m[1] * y[1] + m[2] * y[2];
        a1 += m[3] * y[0] + m[4] * y[1] + m[5] * y[2];
        a2 += m[6] * y[0] + m[7] * y[1] + m[8] * y[2];
      }
      a0 = warp_sum(a0);
      a1 = warp_sum(a1);
      a2 = warp_sum(a2);
      if (lane == 0) {
        const double t0 = x[3 * (int64_t)i] - a0, t1 = x[3 * (int64_t)i + 1] - a1, t2 = x[3 * (int64_t)i + 2] - a2;
        const double* U = uinv + (int64_t)i * 9;
        x[3 * (int64_t)i] = U[0] * t0 + U[1] * t1 + U[2] * t2;
        x[3 * (int64_t)i + 1] = U[3] * t0 + U[4] * t1 + U[5] * t2;
        x[3 * (int64_t)i + 2] = U[6] * t0 + U[7] * t1 + U[8] * t2;
      }
    }
    __syncthreads();
  }
}

__global__ void k_add_vec(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = a[i] + b[i];
}
__global__ void k_axpy2(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

// `sweeps` damped symmetric block Gauss-Seidel sweeps on K x = b from the x given, colours
// ascending then descending
static int colored_sgs(amgc_hierarchy* h, const Level& L, const LevelV<double>& V, const double* b, double* x) {
  cudaStream_t s = h->stream;
  for (int sw = 0; sw < h->sgs_sweeps; ++sw)
    for (int k = 0; k < 2 * L.ncolor; ++k) {
      const int c = k < L.ncolor ? k : 2 * L.ncolor - 1 - k;
      const int cnt = L.h_col_ptr[c + 1] - L.h_col_ptr[c];
      if (cnt == 0) continue;
      const int* nodes = L.col_nodes.p + L.h_col_ptr[c];
      if (L.bu == 3)
        AMGC_LAUNCH(k_cbsgs<3><<<div_up((int64_t)cnt * 32, 128), 128, 0, s>>>(cnt, nodes, V.K.rp, V.K.col, V.K.val,
                                                                             L.kdblk_inv.p, b, x, h->sgs_omega));
      else
        AMGC_LAUNCH(k_cbsgs<6><<<div_up((int64_t)cnt * 32, 128), 128, 0, s>>>(cnt, nodes, V.K.rp, V.K.col, V.K.val,
                                                                             L.kdblk_inv.p, b, x, h->sgs_omega));
    }
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

static int ilu_apply(amgc_hierarchy* h, const Level& L, const double* r, double* x) {
  AMGC_LAUNCH(k_ilu_solve<<<1, kIluThreads, 0, h->stream>>>(L.S.rowptr.p, L.S.col.p, L.S.val.p, L.s_diag.p,
                                                          L.s_uinv.p, L.s_nlev_l, L.s_lptr.p, L.s_lrows.p,
                                                          L.s_nlev_u, L.s_uptr.p, L.s_urows.p, r, x));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

// u = uh - alpha A~^-1 B1 dlam over all displacement rows
static int b1_correct(amgc_hierarchy* h, const LevelV<double>& V, const double* uh, const double* dlam, double alpha,
                      double* u) {
  const int nu = V.nu();
  const int nc = div_up(nu, 128);
  const int gb = div_up((int64_t)V.n_b1_rows * 32, 128);
  if (V.bu == 3)
    AMGC_LAUNCH(k_copy_b1<3, double><<<nc + gb, 128, 0, h->stream>>>(nu, nc, uh, V.n_b1_rows, V.b1_rows, V.B1.rp,
                                                                    V.B1.col, V.B1.val, dlam, V.atinv, alpha, u));
  else
    AMGC_LAUNCH(k_copy_b1<6, double><<<nc + gb, 128, 0, h->stream>>>(nu, nc, uh, V.n_b1_rows, V.b1_rows, V.B1.rp,
                                                                    V.B1.col, V.B1.val, dlam, V.atinv, alpha, u));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

// one sweep of the level's block smoother on [u; lam] (zero_guess: from u = 0, lam = 0)
static int block_smooth(amgc_hierarchy* h, int l, const double* b, double* x, bool zero_guess) {
  const LevelV<double>& V = h->v64[l];
  const Level& L = h->L[l];
  cudaStream_t s = h->stream;
  const int th = 256;
  const int nu = V.nu(), nl3 = 3 * V.nl;
  const double* f = b;
  const double* g = b + nu;
  double* u = x;
  double* lam = x + nu;
  double* w = L.bs_w.p;
  double* d = L.bs_d.p;
  double* rl = L.bs_l.p;
  double* sm = L.bs_m.p;
  const double om = h->block_omega;
  const BsrV<double>* B1 = V.nl ? &V.B1 : nullptr;
  if (zero_guess) AMGC_LAUNCH(k_zero<double><<<div_up(V.rows(), th), th, 0, s>>>(V.rows(), x));
  if (h->smoother_kind == 1) {                      // Uzawa
    AMGC_TRY((mapped_apply<2, double>(V.K, V.Ks, V.kmap, B1, u, lam, f, nullptr, nullptr, 0.0, w, s)));
    AMGC_LAUNCH(k_zero<double><<<div_up(nu, th), th, 0, s>>>(nu, d));
    AMGC_TRY(colored_sgs(h, L, V, w, d));                                       // du ~ K^-1 (f - K u - B1 lam)
    if (V.nl > 0) {
      AMGC_LAUNCH(k_add_vec<<<div_up(nu, th), th, 0, s>>>(nu, u, d, w));        // u + du
      AMGC_TRY((lm_op<0, double>(V, w, g, lam, 0.0, rl, s)));                   // g - B2 (u + du) + Z lam
      AMGC_TRY(ilu_apply(h, L, rl, sm));                                         // dlam = -sm
      AMGC_LAUNCH(k_axpy2<<<div_up(nl3, th), th, 0, s>>>(nl3, -om, sm, lam));
    }
    AMGC_LAUNCH(k_axpy2<<<div_up(nu, th), th, 0, s>>>(nu, om, d, u));
  } else if (h->smoother_kind == 2) {               // Braess-Sarazin
    AMGC_TRY((mapped_apply<3, double>(V.K, V.Ks, V.kmap, B1, u, lam, f, u, V.atinv, 1.0 / om, w, s)));   // u_h
    if (V.nl > 0) {
      AMGC_TRY((lm_op<0, double>(V, w, g, lam, 0.0, rl, s)));                   // g + Z lam - B2 u_h
      AMGC_TRY(ilu_apply(h, L, rl, sm));                                         // dlam = -sm
      AMGC_LAUNCH(k_axpy2<<<div_up(nl3, th), th, 0, s>>>(nl3, -1.0, sm, lam));
      AMGC_TRY(b1_correct(h, V, w, sm, -1.0 / om, u));                           // u = u_h - A~^-1 B1 dlam / omega
    } else {
      AMGC_LAUNCH(k_copy<double><<<div_up(nu, th), th, 0, s>>>(nu, w, u));
    }
  } else {                                          // SIMPLE with the SGS predictor
    if (V.nl > 0) AMGC_TRY((rowop<2, double>(V.B1, lam, nullptr, nullptr, f, nullptr, nullptr, 0.0, w, s)));   // f - B1 lam
    else AMGC_LAUNCH(k_copy<double><<<div_up(nu, th), th, 0, s>>>(nu, f, w));
    AMGC_LAUNCH(k_copy<double><<<div_up(nu, th), th, 0, s>>>(nu, u, d));
    AMGC_TRY(colored_sgs(h, L, V, w, d));                                       // u_h ~ K^-1 (f - B1 lam) from u
    if (V.nl > 0) {
      AMGC_TRY((lm_op<0, double>(V, d, g, lam, 0.0, rl, s)));                   // g + Z lam - B2 u_h
      AMGC_TRY(ilu_apply(h, L, rl, sm));                                         // dlam = -sm
      AMGC_LAUNCH(k_axpy2<<<div_up(nl3, th), th, 0, s>>>(nl3, -om, sm, lam));
      AMGC_TRY(b1_correct(h, V, d, sm, -om, u));                                 // u = u_h - omega A~^-1 B1 dlam
    } else {
      AMGC_LAUNCH(k_copy<double><<<div_up(nu, th), th, 0, s>>>(nu, d, u));
    }
  }
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

template <class T>
static int residual(amgc_hierarchy* h, const LevelV<T>& L, int l, const T* b, const T* x, T* r) {
  const int nu = L.nu();
  return fork_join(
      h, [&]() { return k_apply<2, T>(h, L, l, x, x + nu, b, nullptr, r); },
      [&](cudaStream_t ss) { return lm_op<0, T>(L, x, b + nu, const_cast<T*>(x + nu), 0.0, r + nu, ss); });
}

template <class T>
static int vcycle_t(amgc_hierarchy* h, std::vector<LevelV<T>>& V, int l, const T* b, T* x) {
  const LevelV<T>& L = V[l];
  cudaStream_t s = h->stream;
  const int th = 256;
  if (l == (int)V.size() - 1 && h->opts.coarse_solver == 1 && l > 0) {
    // coarsest level without a merged matrix: the level smoother's sweeps from a zero guess
    const int sweeps = h->opts.smoother_sweeps;
    if (sweeps == 0) {
      AMGC_LAUNCH(k_zero<T><<<div_up(L.rows(), th), th, 0, s>>>(L.rows(), x));
      AMGC_CUDA_TRY(cudaGetLastError());
    }
    AMGC_TRY(smooth_sweeps<T>(h, L, l, b, x, sweeps, true));
    return AMGC_OK;
  }
  if (l == (int)V.size() - 1) {
    const int n = L.rows();
    if (L.c_inst)
      AMGC_LAUNCH(k_gemv_batched<T><<<div_up((int64_t)n * 32, th), th, 0, s>>>(n, L.c_inst, L.c_loc, L.c_glob, L.c_goff,
                                                                             L.c_doff, L.Ainv, b, x));
    else
      AMGC_LAUNCH(k_gemv<T><<<div_up((int64_t)n * 32, th), th, 0, s>>>(n, L.Ainv, b, x));
    AMGC_CUDA_TRY(cudaGetLastError());
    return AMGC_OK;
  }
  const int nu = L.nu();
  const LevelV<T>& C = V[l + 1];
  const int sweeps = h->opts.smoother_sweeps;
  if (sweeps == 0) {
    AMGC_LAUNCH(k_zero<T><<<div_up(L.rows(), th), th, 0, s>>>(L.rows(), x));
    AMGC_CUDA_TRY(cudaGetLastError());
  }
  AMGC_TRY(smooth_sweeps<T>(h, L, l, b, x, sweeps, true));
  AMGC_TRY(residual<T>(h, L, l, b, x, L.r));
  // restrict: C.b = [R r_u ; R^lambda r_lambda] (the multiplier part beside the displacement part)
  AMGC_TRY(fork_join(
      h, [&]() { return mapped_apply<0, T>(L.R, L.Rs, L.rmap, nullptr, L.r, nullptr, nullptr, nullptr, nullptr, 0.0, C.b, s); },
      [&](cudaStream_t ss) -> int {
        if (C.nl > 0) {
          AMGC_LAUNCH(k_restrict_lm<T><<<div_up((int64_t)C.nl * 32, 128), 128, 0, ss>>>(C.nl, L.rl_ptr, L.rl_idx, L.pl_w,
                                                                                       L.r + nu, C.b + C.nu()));
          AMGC_CUDA_TRY(cudaGetLastError());
        }
        return AMGC_OK;
      }));
  AMGC_TRY(vcycle_t<T>(h, V, l + 1, C.b, C.x));
  // prolongate and add (the multiplier part beside the displacement part)
  AMGC_TRY(fork_join(
      h, [&]() { return mapped_apply<1, T>(L.P, L.Ps, L.pmap, nullptr, C.x, nullptr, nullptr, nullptr, nullptr, 0.0, x, s); },
      [&](cudaStream_t ss) -> int {
        if (L.nl > 0) {
          AMGC_LAUNCH(k_prolong_lm<T><<<div_up(L.nl, 128), 128, 0, ss>>>(L.nl, L.lagg, L.pl_w, C.x + C.nu(), x + nu));
          AMGC_CUDA_TRY(cudaGetLastError());
        }
        return AMGC_OK;
      }));
  AMGC_TRY(smooth_sweeps<T>(h, L, l, b, x, sweeps, false));
  return AMGC_OK;
}

// ------------------------------------------------------------------ transposed cycle (adjoint)
// The cycle operator is M = (I - Q A) [Q + P M_c R (I - A Q)] + Q for one sweep each side, Q the
// CheapSIMPLE sweep operator; its transpose is the same V-cycle on A^T with the sweep Q^T, the
// transfers R = P^T and P unchanged, and the transposed coarsest inverse.  From the residual
// e = y - A^T x of a transposed sweep:
//   w   = -alpha S^-T (e_lambda - B1^T A~^-1 e_u),  lambda += w
//   u  += J_k^T (e_u - B2^T w)
// with J_k = sum_{i<k} (I - omega D^-1 K)^i omega D^-1 the k-step Jacobi predictor in residual form
// (J_1 = omega D^-1); the order of the multiplier and displacement updates is reversed with
// respect to Q.

// w_l = -alpha S^-T_l (e_l - sum_i B1T[l,i] (atinv_i e_u,i)); lam_l += w_l; out_l = w_l
template <int BU, int G>
__global__ void __launch_bounds__(128)
k_lm_tsweep(int nl, const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
            const double* __restrict__ eu, const double* __restrict__ atinv, const double* __restrict__ el,
            const double* __restrict__ SinvT, double alpha, double* __restrict__ lam, double* __restrict__ out) {
  // one node per group of G lanes, as k_lm
  const int lane = threadIdx.x & 31, gl = lane & (G - 1);
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int first = (int)((gt >> 5) * (32 / G));
  if (first >= nl) return;
  const int l = first + lane / G;
  const bool valid = l < nl;
  const int c = gl < 3 ? gl : 0;
  const bool st = valid && gl < 3;
  int b0 = 0, b1 = 0;
  double elc = 0.0, s0 = 0.0, s1 = 0.0, s2 = 0.0;
  if (valid) {
    b0 = rp[l];
    b1 = rp[l + 1];
    elc = el[3 * (int64_t)l + c];
    const double* S = SinvT + (int64_t)l * 9 + 3 * c;
    s0 = S[0];
    s1 = S[1];
    s2 = S[2];
  }
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t b = b0 + gl; b < b1; b += G) {
    const int64_t c0 = (int64_t)col[b] * BU;
    const double* v = val + b * (3 * BU);
#pragma unroll
    for (int cc = 0; cc < BU; ++cc) {
      const double xv = atinv[c0 + cc] * eu[c0 + cc];
      acc[0] = fma(v[cc], xv, acc[0]);
      acc[1] = fma(v[BU + cc], xv, acc[1]);
      acc[2] = fma(v[2 * BU + cc], xv, acc[2]);
    }
  }
  const double a0 = group_sum<G>(acc[0]), a1 = group_sum<G>(acc[1]), a2 = group_sum<G>(acc[2]);
  const double rc = elc - (c == 0 ? a0 : (c == 1 ? a1 : a2));
  const int g0 = lane & ~(G - 1);
  const double r0 = __shfl_sync(0xffffffffu, rc, g0), r1 = __shfl_sync(0xffffffffu, rc, g0 + 1),
               r2 = __shfl_sync(0xffffffffu, rc, g0 + 2);
  if (!st) return;
  const double w = -alpha * (s0 * r0 + s1 * r1 + s2 * r2);
  lam[3 * (int64_t)l + c] += w;
  out[3 * (int64_t)l + c] = w;
}
__global__ void k_axpy_dinv(int64_t n, const double* __restrict__ e, const double* __restrict__ dinv, double omega,
                            double* __restrict__ u) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) u[i] += omega * dinv[i] * e[i];
}

// s = omega D^-1 v (the folded Jacobi diagonal), u += s
__global__ void k_tjacobi_step(int64_t n, const double* __restrict__ v, const double* __restrict__ jdinv,
                               double* __restrict__ sv, double* __restrict__ u) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double si = jdinv[i] * v[i];
  sv[i] = si;
  u[i] += si;
}

template <class T>
static int tsmooth(amgc_hierarchy* h, const LevelV<double>& L, int l, const double* y, double* x, bool zero_guess) {
  cudaStream_t s = h->stream;
  const int nu = L.nu();
  const int th = 256;
  double* e = L.r;
  if (zero_guess) {
    AMGC_LAUNCH(k_zero<double><<<div_up(L.rows(), th), th, 0, s>>>(L.rows(), x));
    AMGC_LAUNCH(k_copy<double><<<div_up(L.rows(), th), th, 0, s>>>(L.rows(), y, e));
  } else {
    AMGC_TRY((k_apply<2, double>(h, L, l, x, x + nu, y, nullptr, e, true)));
    AMGC_TRY((lm_op<0, double>(L, x, y + nu, x + nu, 0.0, e + nu, s, true)));
  }
  if (L.nl > 0) {
    const int gs = pick_group(L.B1T.nnzb, L.nl, true, L.bu);
    const int grid = (int)div_up((int64_t)L.nl * gs, 128);
    if (L.bu == 3)
      AMGC_GROUP_DISPATCH3(gs, AMGC_LAUNCH((k_lm_tsweep<3, G_><<<grid, 128, 0, s>>>(
                                  L.nl, L.B1T.rp, L.B1T.col, L.B1T.val, e, L.atinv, e + nu, L.SinvT,
                                  h->opts.simple_alpha, x + nu, L.dlam))));
    else
      AMGC_GROUP_DISPATCH(gs, AMGC_LAUNCH((k_lm_tsweep<6, G_><<<grid, 128, 0, s>>>(
                                  L.nl, L.B1T.rp, L.B1T.col, L.B1T.val, e, L.atinv, e + nu, L.SinvT,
                                  h->opts.simple_alpha, x + nu, L.dlam))));
  }
  const int J = h->opts.jacobi_sweeps;
  if (J > 1) {
    // u += J_k^T (e_u - B2^T w), J_k^T = sum_{i<k} omega D^-1 (I - omega K D^-1)^i (K symmetric):
    // v = e_u - B2^T w; then k times: s = omega D^-1 v, u += s, v <- v - K s (the last skipped)
    double* v = L.t;
    double* sv = L.tsw;
    double* vn = L.tsw + nu;
    if (L.nl > 0) AMGC_TRY((rowop<2, double>(L.B2T, L.dlam, nullptr, nullptr, e, nullptr, nullptr, 0.0, v, s)));
    else AMGC_LAUNCH(k_copy<double><<<div_up(nu, th), th, 0, s>>>(nu, e, v));
    for (int i = 0; i < J; ++i) {
      AMGC_LAUNCH(k_tjacobi_step<<<div_up(nu, th), th, 0, s>>>(nu, v, L.dinv, sv, x));
      if (i + 1 < J) {
        AMGC_TRY((mapped_apply<2, double>(L.K, L.Ks, L.kmap, nullptr, sv, nullptr, v, nullptr, nullptr, 0.0, vn, s)));
        std::swap(v, vn);
      }
    }
    AMGC_CUDA_TRY(cudaGetLastError());
    return AMGC_OK;
  }
  AMGC_LAUNCH(k_axpy_dinv<<<div_up(nu, th), th, 0, s>>>(nu, e, L.dinv, L.omega_j, x));
  AMGC_CUDA_TRY(cudaGetLastError());
  return b1_update<double>(L.bu, L.n_b2t_rows, L.b2t_rows, L.B2T, L.dlam, L.dinv, L.omega_j, x, s);
}

static int vcycle_transposed(amgc_hierarchy* h, int l, const double* y, double* x) {
  std::vector<LevelV<double>>& V = h->v64;
  const LevelV<double>& L = V[l];
  cudaStream_t s = h->stream;
  const int th = 256;
  if (l == (int)V.size() - 1) {
    const int n = L.rows();
    AMGC_LAUNCH(k_gemv<double><<<div_up((int64_t)n * 32, th), th, 0, s>>>(n, L.AinvT, y, x));
    AMGC_CUDA_TRY(cudaGetLastError());
    return AMGC_OK;
  }
  const int nu = L.nu();
  const LevelV<double>& C = V[l + 1];
  const int sweeps = h->opts.smoother_sweeps;
  if (sweeps == 0) AMGC_LAUNCH(k_zero<double><<<div_up(L.rows(), th), th, 0, s>>>(L.rows(), x));
  for (int k = 0; k < sweeps; ++k) AMGC_TRY(tsmooth<double>(h, L, l, y, x, k == 0));
  // residual with A^T, then the same restriction as the forward cycle
  AMGC_TRY((k_apply<2, double>(h, L, l, x, x + nu, y, nullptr, L.r, true)));
  AMGC_TRY((lm_op<0, double>(L, x, y + nu, x + nu, 0.0, L.r + nu, s, true)));
  AMGC_TRY((rowop<0, double>(L.R, L.r, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, C.b, s)));
  if (C.nl > 0)
    AMGC_LAUNCH(k_restrict_lm<double><<<div_up((int64_t)C.nl * 32, 128), 128, 0, s>>>(C.nl, L.rl_ptr, L.rl_idx, L.pl_w, L.r + nu,
                                                                        C.b + C.nu()));
  AMGC_TRY(vcycle_transposed(h, l + 1, C.b, C.x));
  if (L.Ps.nslice > 0)
    AMGC_TRY((sell_apply<1, double>(L.Ps, L.nn, nullptr, C.x, nullptr, nullptr, nullptr, nullptr, 0.0, x, s)));
  else
    AMGC_TRY((rowop<1, double>(L.P, C.x, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, x, s)));
  if (L.nl > 0)
    AMGC_LAUNCH(k_prolong_lm<double><<<div_up(L.nl, 128), 128, 0, s>>>(L.nl, L.lagg, L.pl_w, C.x + C.nu(), x + nu));
  for (int k = 0; k < sweeps; ++k) AMGC_TRY(tsmooth<double>(h, L, l, y, x, false));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

// y = A x, or y = A^T x while the hierarchy is in transposed mode
int saddle_apply(amgc_hierarchy* h, int l, const double* x, double* y) {
  const LevelV<double>& L = h->v64[l];
  const int nu = L.nu();
  const bool tr = h->transposed;
  return fork_join(
      h, [&]() { return k_apply<0, double>(h, L, l, x, x + nu, nullptr, nullptr, y, tr); },
      [&](cudaStream_t ss) { return lm_op<2, double>(L, x, nullptr, const_cast<double*>(x + nu), 0.0, y + nu, ss, tr); });
}

// One V-cycle with FP64 input and output; the FP32 cycle converts at entry and exit.
// Captures the forward cycle core (fixed input and output buffers) into a CUDA graph on a
// private stream; the caller's stream then replays it with one launch.
static int capture_cycle(amgc_hierarchy* h, int idx) {
  if (!h->capture_stream) AMGC_CUDA_TRY(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
  const int64_t n = h->L[0].rows();
  if (idx == 0 && h->cyc_in.n == 0) {
    AMGC_TRY(h->cyc_in.alloc(n));
    AMGC_TRY(h->cyc_out.alloc(n));
  }
  cudaStream_t saved = h->stream;
  h->stream = h->capture_stream;
  const long long k0 = g_launches.load();
  cudaGraph_t graph = nullptr;
  AMGC_CUDA_TRY(cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
  int st = idx == 0 ? vcycle_t<double>(h, h->v64, 0, h->cyc_in.p, h->cyc_out.p)
                    : vcycle_t<float>(h, h->v32, 0, h->L[0].f.b.p, h->L[0].f.x.p);
  cudaError_t e = cudaStreamEndCapture(h->capture_stream, &graph);
  h->stream = saved;
  if (st != AMGC_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) {
    set_error(std::string("cycle capture: ") + cudaGetErrorString(e));
    return AMGC_ECUDA;
  }
  e = cudaGraphInstantiate(&h->cycle_graph[idx], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    h->cycle_graph[idx] = nullptr;
    set_error(std::string("cycle graph instantiation: ") + cudaGetErrorString(e));
    return AMGC_ECUDA;
  }
  h->cycle_graph_kernels[idx] = g_launches.load() - k0;
  return AMGC_OK;
}

static int replay_cycle(amgc_hierarchy* h, int idx) {
  if (!h->cycle_graph[idx]) AMGC_TRY(capture_cycle(h, idx));
  AMGC_CUDA_TRY(cudaGraphLaunch(h->cycle_graph[idx], h->stream));
  g_launches.fetch_add(h->cycle_graph_kernels[idx], std::memory_order_relaxed);
  return AMGC_OK;
}

// ------------------------------------------------------------------ nested multigrid (Sec. 3.2)
// The comparison preconditioner of Sec. 3.2 (Fig. mgmphmodelsA): the displacement-multiplier
// coupling is treated on the finest level only, by outer SIMPLE sweeps (Algorithm 4) whose
// predictor is one single-field AMG V-cycle on K:
//     u_h = u + V_K (f - K u - B1 lam)
//     dlam = -S_hat^-1 (g + Z lam - B2 u_h),   S_hat = Z + B2 A~^-1 B1 (exact, dense)
//     lam += omega dlam,   u = u_h - omega A~^-1 B1 dlam
// The K hierarchy is the displacement part of the coupled one: the same aggregates, transfers,
// Galerkin K_c, lambda_max and omega_J D^-1; V_K smooths with damped Jacobi (smoother_sweeps pre and
// post) and solves the coarsest K_c with its dense inverse.  FP64.

// dense S_hat rows of multiplier node l (one thread per node, which owns its three rows)
__global__ void k_dense_schur(int nl, const int* __restrict__ rp2, const int* __restrict__ c2,
                              const double* __restrict__ v2, const int* __restrict__ rp1, const int* __restrict__ c1,
                              const double* __restrict__ v1, const double* __restrict__ atinv,
                              const double* __restrict__ Z, double* __restrict__ A) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nl) return;
  const int64_t n = 3 * (int64_t)nl;
  for (int e = rp2[l]; e < rp2[l + 1]; ++e) {
    const int i = c2[e];
    const double* b2 = v2 + (int64_t)e * 9;
    double ba[9];
    for (int r = 0; r < 3; ++r)
      for (int k = 0; k < 3; ++k) ba[r * 3 + k] = b2[r * 3 + k] * atinv[3 * (int64_t)i + k];
    for (int q = rp1[i]; q < rp1[i + 1]; ++q) {
      const int m = c1[q];
      const double* b1 = v1 + (int64_t)q * 9;
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
          double acc = A[(3 * (int64_t)l + r) * n + 3 * (int64_t)m + c];
          for (int k = 0; k < 3; ++k) acc = fma(ba[r * 3 + k], b1[k * 3 + c], acc);
          A[(3 * (int64_t)l + r) * n + 3 * (int64_t)m + c] = acc;
        }
    }
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) A[(3 * (int64_t)l + r) * n + 3 * (int64_t)l + c] += Z[(int64_t)l * 9 + r * 3 + c];
}
// dense copy of a BR x BR block matrix (one warp per block row)
template <int BR>
__global__ void k_dense_blocks(int nbr, const int* __restrict__ rp, const int* __restrict__ col,
                               const double* __restrict__ val, double* __restrict__ A) {
  constexpr int NQ = BR * BR;
  const int lane = threadIdx.x & 31;
  const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (i >= nbr) return;
  const int64_t n = (int64_t)nbr * BR;
  const int e0 = rp[i], nq = (rp[i + 1] - e0) * NQ;
  for (int q = lane; q < nq; q += 32) {
    const int eb = q / NQ, w = q - eb * NQ;
    const int r = w / BR, c = w - r * BR;
    A[(int64_t)(i * BR + r) * n + (int64_t)col[e0 + eb] * BR + c] = val[(int64_t)e0 * NQ + q];
  }
}
__global__ void k_axpy(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

int nested_setup(amgc_hierarchy* h) {
  cudaStream_t s = h->stream;
  const int nlev = (int)h->L.size();
  const Level& Lc = h->L[nlev - 1];
  const Level& L0 = h->L[0];
  const int nk = Lc.nu();
  const int nsch = 3 * L0.nl;
  constexpr int kMaxDense = 16384;
  if (nk > kMaxDense || nsch > kMaxDense) {
    set_error("nested multigrid: the coarsest K (" + std::to_string(nk) + " rows) or S_hat (" + std::to_string(nsch) +
              " rows) exceeds the dense limit of " + std::to_string(kMaxDense));
    return AMGC_EINVAL;
  }
  for (int l = 0; l + 1 < nlev; ++l)
    if (!h->L[l].jdinv.p) {
      set_error("nested multigrid: level without Jacobi data");
      return AMGC_EINVAL;
    }
  AMGC_TRY(h->nest_Kinv.alloc((size_t)nk * nk));
  AMGC_CUDA_TRY(cudaMemsetAsync(h->nest_Kinv.p, 0, (size_t)nk * nk * sizeof(double), s));
  if (Lc.bu == 3)
    AMGC_LAUNCH(k_dense_blocks<3><<<div_up((int64_t)Lc.nn * 32, 128), 128, 0, s>>>(Lc.nn, Lc.K.rowptr.p, Lc.K.col.p,
                                                                                 Lc.K.val.p, h->nest_Kinv.p));
  else
    AMGC_LAUNCH(k_dense_blocks<6><<<div_up((int64_t)Lc.nn * 32, 128), 128, 0, s>>>(Lc.nn, Lc.K.rowptr.p, Lc.K.col.p,
                                                                                 Lc.K.val.p, h->nest_Kinv.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  AMGC_TRY(dense_inverse(h, h->nest_Kinv.p, nk));
  AMGC_TRY(h->nest_Sinv.alloc((size_t)std::max(nsch, 1) * std::max(nsch, 1)));
  if (nsch > 0) {
    AMGC_CUDA_TRY(cudaMemsetAsync(h->nest_Sinv.p, 0, (size_t)nsch * nsch * sizeof(double), s));
    AMGC_LAUNCH(k_dense_schur<<<div_up(L0.nl, 128), 128, 0, s>>>(L0.nl, L0.B2.rowptr.p, L0.B2.col.p, L0.B2.val.p,
                                                                L0.B1.rowptr.p, L0.B1.col.p, L0.B1.val.p, L0.atinv.p,
                                                                L0.Z.p, h->nest_Sinv.p));
    AMGC_CUDA_TRY(cudaGetLastError());
    AMGC_TRY(dense_inverse(h, h->nest_Sinv.p, nsch));
  }
  AMGC_TRY(check_status(h, "nested multigrid: dense inverses"));
  h->nest.clear();
  h->nest.resize(nlev);
  for (int l = 0; l < nlev; ++l) {
    const size_t n = (size_t)std::max(h->L[l].nu(), 1);
    amgc_hierarchy::NestBufs& B = h->nest[l];
    AMGC_TRY(B.x.alloc(n));
    AMGC_TRY(B.b.alloc(n));
    AMGC_TRY(B.r.alloc(n));
    AMGC_TRY(B.t.alloc(n));
  }
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  return AMGC_OK;
}

// x = V_K(b) on level l of the K hierarchy (zero initial guess)
static int kcycle(amgc_hierarchy* h, int l, const double* b, double* x) {
  const std::vector<LevelV<double>>& V = h->v64;
  const LevelV<double>& L = V[l];
  cudaStream_t s = h->stream;
  const int th = 256;
  const int nu = L.nu();
  if (l == (int)V.size() - 1) {
    AMGC_LAUNCH(k_gemv<double><<<div_up((int64_t)nu * 32, th), th, 0, s>>>(nu, h->nest_Kinv.p, b, x));
    AMGC_CUDA_TRY(cudaGetLastError());
    return AMGC_OK;
  }
  amgc_hierarchy::NestBufs& B = h->nest[l];
  amgc_hierarchy::NestBufs& C = h->nest[l + 1];
  const int J = h->opts.smoother_sweeps;
  // J damped Jacobi sweeps, each out of place (it gathers its input at the neighbours): they
  // alternate between x and B.t.  From a zero guess the first sweep needs no product and its
  // buffer is chosen so that the last one ends in x; from the iterate in x the first goes to B.t
  // and a copy brings an odd count's result back.
  auto sweeps = [&](bool zero_guess) -> int {
    double* cur = x;
    for (int j = 0; j < J; ++j) {
      double* dst = zero_guess ? (((J - 1 - j) % 2 == 0) ? x : B.t.p) : (cur == x ? B.t.p : x);
      if (zero_guess && j == 0) {
        AMGC_LAUNCH(k_jacobi_zero<double><<<div_up(nu, th), th, 0, s>>>(nu, 0, b, L.dinv, 1.0, dst, nullptr));
        AMGC_CUDA_TRY(cudaGetLastError());
      } else {
        AMGC_TRY((mapped_apply<3, double>(L.K, L.Ks, L.kmap, nullptr, cur, nullptr, b, cur, L.dinv, L.omega_j, dst, s)));
      }
      cur = dst;
    }
    if (cur != x) AMGC_LAUNCH(k_copy<double><<<div_up(nu, th), th, 0, s>>>(nu, cur, x));
    return AMGC_OK;
  };
  if (J == 0) AMGC_LAUNCH(k_zero<double><<<div_up(nu, th), th, 0, s>>>(nu, x));
  else AMGC_TRY(sweeps(true));
  AMGC_TRY((mapped_apply<2, double>(L.K, L.Ks, L.kmap, nullptr, x, nullptr, b, nullptr, nullptr, 0.0, B.r.p, s)));
  AMGC_TRY((mapped_apply<0, double>(L.R, L.Rs, L.rmap, nullptr, B.r.p, nullptr, nullptr, nullptr, nullptr, 0.0, C.b.p, s)));
  AMGC_TRY(kcycle(h, l + 1, C.b.p, C.x.p));
  AMGC_TRY((mapped_apply<1, double>(L.P, L.Ps, L.pmap, nullptr, C.x.p, nullptr, nullptr, nullptr, nullptr, 0.0, x, s)));
  if (J > 0) AMGC_TRY(sweeps(false));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

// z = the nested preconditioner applied to r (FP64, device vectors of the finest saddle rows)
static int nested_apply(amgc_hierarchy* h, const double* r, double* z) {
  const LevelV<double>& L = h->v64[0];
  cudaStream_t s = h->stream;
  const int th = 256;
  const int nu = L.nu();
  const int nl3 = 3 * L.nl;
  const double* f = r;
  const double* g = r + nu;
  double* u = z;
  double* lam = z + nu;
  amgc_hierarchy::NestBufs& B = h->nest[0];
  double* rl = L.r + nu;          // the multiplier residual (the coupled cycle's scratch)
  double* w = L.dlam;             // S_hat^-1 r_lambda
  const double om = h->nest_omega;
  for (int k = 0; k < h->nest_sweeps; ++k) {
    if (k == 0) {
      AMGC_TRY(kcycle(h, 0, f, u));                                            // u_h = V_K f
      AMGC_LAUNCH(k_zero<double><<<div_up(std::max(nl3, 1), th), th, 0, s>>>(nl3, lam));
    } else {
      AMGC_TRY((mapped_apply<2, double>(L.K, L.Ks, L.kmap, L.nl ? &L.B1 : nullptr, u, lam, f, nullptr, nullptr, 0.0,
                                        B.b.p, s)));                          // f - K u - B1 lam
      AMGC_TRY(kcycle(h, 0, B.b.p, B.x.p));
      AMGC_LAUNCH(k_axpy<<<div_up(nu, th), th, 0, s>>>(nu, 1.0, B.x.p, u));     // u_h = u + V_K(...)
    }
    if (L.nl == 0) continue;
    AMGC_TRY((lm_op<0, double>(L, u, g, lam, 0.0, rl, s)));                   // g - B2 u_h + Z lam
    AMGC_LAUNCH(k_gemv<double><<<div_up((int64_t)nl3 * 32, th), th, 0, s>>>(nl3, h->nest_Sinv.p, rl, w));
    AMGC_LAUNCH(k_axpy<<<div_up(nl3, th), th, 0, s>>>(nl3, -om, w, lam));     // lam += omega dlam, dlam = -w
    AMGC_CUDA_TRY(cudaGetLastError());                                         // u = u_h + omega A~^-1 B1 w
    AMGC_TRY(b1_update<double>(3, L.n_b1_rows, L.b1_rows, L.B1, w, L.atinv, -om, u, s));
  }
  return AMGC_OK;
}

// One V-cycle with FP64 input and output; the FP32 cycle converts at entry and exit.  Outside
// kernel timing the cycle core runs as a captured CUDA graph.
int precond_apply(amgc_hierarchy* h, const double* r, double* z) {
  if (h->transposed) return vcycle_transposed(h, 0, r, z);
  if (h->prec_kind == 1) return nested_apply(h, r, z);
  const bool graph = h->prof == 0;
  const int64_t n = h->L[0].rows();
  const int th = 256;
  if (h->opts.precision == 32) {
    float* bf = h->L[0].f.b.p;
    float* xf = h->L[0].f.x.p;
    AMGC_LAUNCH((k_convert<double, float><<<div_up(n, th), th, 0, h->stream>>>(n, r, bf)));
    if (graph) AMGC_TRY(replay_cycle(h, 1));
    else AMGC_TRY(vcycle_t<float>(h, h->v32, 0, bf, xf));
    AMGC_LAUNCH((k_convert<float, double><<<div_up(n, th), th, 0, h->stream>>>(n, xf, z)));
    AMGC_CUDA_TRY(cudaGetLastError());
    return AMGC_OK;
  }
  if (!graph) return vcycle_t<double>(h, h->v64, 0, r, z);
  if (!h->cycle_graph[0]) AMGC_TRY(capture_cycle(h, 0));
  AMGC_CUDA_TRY(cudaMemcpyAsync(h->cyc_in.p, r, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  AMGC_TRY(replay_cycle(h, 0));
  AMGC_CUDA_TRY(cudaMemcpyAsync(z, h->cyc_out.p, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  return AMGC_OK;
}

// ------------------------------------------------------------------ views and FP32 mirrors
int convert_f64_f32(int64_t n, const double* x, float* y, cudaStream_t s) {
  if (n == 0) return AMGC_OK;
  AMGC_LAUNCH((k_convert<double, float><<<div_up(n, 256), 256, 0, s>>>(n, x, y)));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

static int to_f32(amgc_hierarchy* h, const double* src, size_t n, DBuf<float>& dst) {
  AMGC_TRY(dst.alloc(std::max<size_t>(n, 1)));
  if (n == 0) return AMGC_OK;
  AMGC_LAUNCH((k_convert<double, float><<<div_up((int64_t)n, 256), 256, 0, h->stream>>>((int64_t)n, src, dst.p)));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

template <class T>
static BsrV<T> bview(const DBsr& A, const T* val) {
  BsrV<T> v;
  v.nbr = A.nbr; v.nbc = A.nbc; v.br = A.br; v.bc = A.bc; v.nnzb = A.nnzb;
  v.rp = A.rowptr.p; v.col = A.col.p; v.val = val;
  return v;
}
template <class T>
static SellV<T> sview(const Sell& S, const T* val) {
  SellV<T> v;
  v.br = S.br; v.bc = S.bc; v.nslice = S.nslice;
  v.off = S.off.p; v.len = S.len.p; v.col = S.col.p; v.val = val; v.perm = S.perm.p;
  return v;
}

template <class T>
static LevelV<T> common_view(const Level& L) {
  LevelV<T> v;
  // the Jacobi damping is folded into the dinv view (omega_J D^-1, per instance when batched)
  v.nn = L.nn; v.bu = L.bu; v.nl = L.nl; v.omega_j = 1.0;
  v.Sinv = L.Sinv.p; v.lagg = L.lagg.p; v.rl_ptr = L.rl_ptr.p; v.rl_idx = L.rl_idx.p;
  v.b1_rows = L.b1_rows.p; v.n_b1_rows = L.n_b1_rows; v.Ainv = L.Ainv.p;
  v.ir_rows = L.ir_rows.p; v.ir_b2c = L.ir_b2c.p; v.n_ir = L.n_ir;
  v.c_inst = L.c_inst.p; v.c_loc = L.c_loc.p; v.c_glob = L.c_glob.p; v.c_goff = L.c_goff.p; v.c_doff = L.c_doff.p;
  return v;
}

// Interface rows of a level (see Level::ir_rows): flags on B1's rows with entries and on B2's
// block columns, an exclusive scan for the positions, the ascending list and B2's columns mapped
// to positions.
__global__ void k_ir_mark_rows(int nn, const int* __restrict__ rp, int* __restrict__ mark) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nn) mark[i] = rp[i + 1] > rp[i] ? 1 : 0;
}
__global__ void k_ir_mark_cols(int64_t nnzb, const int* __restrict__ col, int* __restrict__ mark) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < nnzb) mark[col[e]] = 1;
}
__global__ void k_ir_list(int nn, const int* __restrict__ mark, const int* __restrict__ pos, int* __restrict__ rows) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nn && mark[i]) rows[pos[i]] = i;
}
__global__ void k_ir_remap(int64_t nnzb, const int* __restrict__ col, const int* __restrict__ pos, int* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < nnzb) out[e] = pos[col[e]];
}
static int ir_setup(amgc_hierarchy* h, Level& L) {
  cudaStream_t s = h->stream;
  L.n_ir = 0;
  if (L.nl == 0 || L.nn == 0) return AMGC_OK;
  DBuf<int> mark, pos;
  AMGC_TRY(mark.alloc(L.nn));
  AMGC_TRY(pos.alloc(L.nn));
  AMGC_LAUNCH(k_ir_mark_rows<<<div_up(L.nn, 256), 256, 0, s>>>(L.nn, L.B1.rowptr.p, mark.p));
  if (L.B2.nnzb > 0)
    AMGC_LAUNCH(k_ir_mark_cols<<<div_up(L.B2.nnzb, 256), 256, 0, s>>>(L.B2.nnzb, L.B2.col.p, mark.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  int n = 0;
  AMGC_TRY(exclusive_scan(mark.p, pos.p, L.nn, s, &n));
  AMGC_TRY(L.ir_rows.alloc(std::max(n, 1)));
  AMGC_TRY(L.ir_b2c.alloc(std::max<int64_t>(L.B2.nnzb, 1)));
  AMGC_LAUNCH(k_ir_list<<<div_up(L.nn, 256), 256, 0, s>>>(L.nn, mark.p, pos.p, L.ir_rows.p));
  if (L.B2.nnzb > 0)
    AMGC_LAUNCH(k_ir_remap<<<div_up(L.B2.nnzb, 256), 256, 0, s>>>(L.B2.nnzb, L.B2.col.p, pos.p, L.ir_b2c.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  AMGC_TRY(L.ir_u.alloc((size_t)std::max(n, 1) * L.bu));
  L.n_ir = n;
  return AMGC_OK;
}
// The smoother form a view runs: the level's setting, by default two launches.  (On the large
// two-block workload the split sweep does not pay by default once the multiplier-row kernels run on
// lane groups: the FP64 step beside it shares the FP64 FMA rate, and the FP32 step gains less than
// the fork and join cost; nor does the fused form on the coarse levels.  The autotuner times the
// forms per level.)
static int resolve_form(int f) { return f >= 0 ? f : 0; }

int make_views(amgc_hierarchy* h) {
  drop_cycle_graphs(h);   // captured cycles hold the pointers of the views rebuilt here
  h->v64.clear();
  h->v32.clear();
  const int nlev = (int)h->L.size();
  for (int l = 0; l < nlev; ++l) {
    Level& L = h->L[l];
    AMGC_TRY(ir_setup(h, L));
    LevelV<double> v = common_view<double>(L);
    v.K = bview<double>(L.K, L.K.val.p);
    v.B1 = bview<double>(L.B1, L.B1.val.p);
    v.B2 = bview<double>(L.B2, L.B2.val.p);
    v.P = bview<double>(L.P, L.P.val.p);
    v.R = bview<double>(L.R, L.R.val.p);
    v.Ks = sview<double>(L.Ks, L.Ks.val.p);
    v.Ps = sview<double>(L.Ps, L.Ps.val.p);
    v.Rs = sview<double>(L.Rs, L.Rs.val.p);
    v.kmap = L.kmap[0]; v.pmap = L.pmap[0]; v.rmap = L.rmap[0]; v.fuse = resolve_form(L.fuse[0]);
    v.ir_u = L.ir_u.p;
    v.Z = L.Z.p; v.dinv = L.jdinv.p; v.atinv = L.atinv.p; v.pl_w = L.pl_w.p;
    v.x = L.x.p; v.b = L.b.p; v.r = L.r.p; v.t = L.t.p; v.dlam = L.dlam.p; v.tsw = L.tsw.p;
    if (L.has_transposed) {
      v.B1T = bview<double>(L.B1T, L.B1T.val.p);
      v.B2T = bview<double>(L.B2T, L.B2T.val.p);
      v.ZT = L.ZT.p; v.SinvT = L.SinvT.p; v.AinvT = L.AinvT.p;
      v.b2t_rows = L.b2t_rows.p; v.n_b2t_rows = L.n_b2t_rows;
    }
    h->v64.push_back(v);
  }
  if (h->opts.precision != 32) return AMGC_OK;
  for (int l = 0; l < nlev; ++l) {
    Level& L = h->L[l];
    LevelF32& F = L.f;
    const bool last = l == nlev - 1;
    const bool smoothed = !last || (h->opts.coarse_solver == 1 && l > 0);   // the level is smoothed
    AMGC_TRY(to_f32(h, L.K.val.p, (size_t)L.K.nnzb * L.bu * L.bu, F.K));
    AMGC_TRY(to_f32(h, L.B1.val.p, (size_t)L.B1.nnzb * L.bu * 3, F.B1));
    AMGC_TRY(to_f32(h, L.B2.val.p, (size_t)L.B2.nnzb * 3 * L.bu, F.B2));
    AMGC_TRY(to_f32(h, L.Z.p, (size_t)L.nl * 9, F.Z));
    if (!last) {
      AMGC_TRY(to_f32(h, L.P.val.p, (size_t)L.P.nnzb * L.P.br * L.P.bc, F.P));
      AMGC_TRY(to_f32(h, L.R.val.p, (size_t)L.R.nnzb * L.R.br * L.R.bc, F.R));
      AMGC_TRY(to_f32(h, L.pl_w.p, (size_t)L.nl, F.pl_w));
    }
    if (smoothed) {
      AMGC_TRY(to_f32(h, L.jdinv.p, (size_t)L.nu(), F.jdinv));
      AMGC_TRY(to_f32(h, L.atinv.p, (size_t)L.nu(), F.atinv));
    }
    if (L.Ks.nslice > 0) AMGC_TRY(to_f32(h, L.Ks.val.p, L.Ks.val.n, F.Ks));
    if (L.Ps.nslice > 0) AMGC_TRY(to_f32(h, L.Ps.val.p, L.Ps.val.n, F.Ps));
    if (L.Rs.nslice > 0) AMGC_TRY(to_f32(h, L.Rs.val.p, L.Rs.val.n, F.Rs));
    const size_t n = std::max(L.rows(), 1);
    AMGC_TRY(F.x.alloc(n));
    AMGC_TRY(F.b.alloc(n));
    AMGC_TRY(F.r.alloc(n));
    AMGC_TRY(F.t.alloc(n));
    AMGC_TRY(F.dlam.alloc(std::max(3 * L.nl, 1)));
    AMGC_TRY(F.ir_u.alloc((size_t)std::max(L.n_ir, 1) * L.bu));
    LevelV<float> v = common_view<float>(L);
    v.K = bview<float>(L.K, F.K.p);
    v.B1 = bview<float>(L.B1, F.B1.p);
    v.B2 = bview<float>(L.B2, F.B2.p);
    v.P = bview<float>(L.P, F.P.p);
    v.R = bview<float>(L.R, F.R.p);
    v.Ks = sview<float>(L.Ks, F.Ks.p);
    if (l == 0 && L.Ks.nslice > 0 && L.Ks.br == 3 && L.Ks.bc == 3) {
      if (!h->tma_ctr.p) AMGC_TRY(h->tma_ctr.alloc(1));
      v.Ks.ctr = h->tma_ctr.p;
      v.Ks.st = h->status.p;
      v.Ks.polls = h->wait_polls;
    }
    v.Ps = sview<float>(L.Ps, F.Ps.p);
    v.Rs = sview<float>(L.Rs, F.Rs.p);
    v.kmap = L.kmap[1]; v.pmap = L.pmap[1]; v.rmap = L.rmap[1]; v.fuse = resolve_form(L.fuse[1]);
    v.ir_u = F.ir_u.p;
    v.Z = F.Z.p; v.dinv = F.jdinv.p; v.atinv = F.atinv.p; v.pl_w = F.pl_w.p;
    v.x = F.x.p; v.b = F.b.p; v.r = F.r.p; v.t = F.t.p; v.dlam = F.dlam.p;
    h->v32.push_back(v);
  }
  AMGC_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return AMGC_OK;
}

// ------------------------------------------------------------------ mapping overrides, wait limit
bool staged_apply_in_use(const amgc_hierarchy* h) {
  return h->opts.precision == 32 && !h->v32.empty() && h->v32[0].kmap == 3;
}

void drop_cycle_graphs(amgc_hierarchy* h) {
  for (int i = 0; i < 2; ++i) {
    if (h->cycle_graph[i]) cudaGraphExecDestroy(h->cycle_graph[i]);
    h->cycle_graph[i] = nullptr;
    h->cycle_graph_kernels[i] = 0;
  }
}

// matrix 0 = K, 1 = P, 2 = R of `level`; precision 64 or 32; mapping -1 (default), 0 (warp per
// row), 1 / 2 (SELL, one / two threads per row), 3 (the staged FP32 kernel: level-0 K only)
int set_row_mapping(amgc_hierarchy* h, int level, int matrix, int precision, int mapping) {
  const int nlev = (int)h->L.size();
  if (level < 0 || level >= nlev || matrix < 0 || matrix > 3 || (precision != 64 && precision != 32) ||
      mapping < -1 || mapping > 3 || (matrix > 0 && matrix < 3 && level == nlev - 1) || (matrix == 3 && mapping > 2)) {
    set_error("amgc_set_row_mapping: invalid level, matrix, precision or mapping");
    return AMGC_EINVAL;
  }
  if (matrix == 3) {   // the smoother form of the level: -1 default, 0 two launches, 1 fused, 2 split
    if (precision == 32 && h->opts.precision != 32) {
      set_error("amgc_set_row_mapping: the hierarchy has no FP32 cycle (precision 64)");
      return AMGC_EINVAL;
    }
    Level& L = h->L[level];
    L.fuse[precision == 32 ? 1 : 0] = mapping;
    const int f = resolve_form(mapping);
    if (precision == 64) h->v64[level].fuse = f;
    else h->v32[level].fuse = f;
    drop_cycle_graphs(h);
    return AMGC_OK;
  }
  if (precision == 32 && h->opts.precision != 32) {
    set_error("amgc_set_row_mapping: the hierarchy has no FP32 cycle (precision 64)");
    return AMGC_EINVAL;
  }
  if (mapping == 3 && !(level == 0 && matrix == 0 && precision == 32)) {
    set_error("amgc_set_row_mapping: the staged kernel applies the FP32 fine-level K only");
    return AMGC_EINVAL;
  }
  Level& L = h->L[level];
  Sell& S = matrix == 0 ? L.Ks : (matrix == 1 ? L.Ps : L.Rs);
  const DBsr& A = matrix == 0 ? L.K : (matrix == 1 ? L.P : L.R);
  const int pidx = precision == 32 ? 1 : 0;
  int* slot = matrix == 0 ? &L.kmap[pidx] : (matrix == 1 ? &L.pmap[pidx] : &L.rmap[pidx]);
  if (mapping >= 1 && S.nslice == 0) {
    AMGC_TRY(build_sell_of(h, A, S));
    *slot = mapping;
    AMGC_TRY(make_views(h));     // the views of the new SELL copy (and its FP32 mirror)
  } else {
    *slot = mapping;
    LevelV<double>& v = h->v64[level];
    if (precision == 64) (matrix == 0 ? v.kmap : (matrix == 1 ? v.pmap : v.rmap)) = mapping;
    else {
      LevelV<float>& w = h->v32[level];
      (matrix == 0 ? w.kmap : (matrix == 1 ? w.pmap : w.rmap)) = mapping;
    }
  }
  if (mapping == 3 && (h->v32.empty() || h->v32[0].Ks.ctr == nullptr)) {
    *slot = -1;
    AMGC_TRY(make_views(h));
    set_error("amgc_set_row_mapping: the fine-level K has no staged FP32 form (not 3x3 SELL)");
    return AMGC_EINVAL;
  }
  drop_cycle_graphs(h);
  return AMGC_OK;
}

int set_wait_limit(amgc_hierarchy* h, long long polls) {
  h->wait_polls = polls;
  if (!h->v32.empty()) h->v32[0].Ks.polls = polls;
  drop_cycle_graphs(h);
  return AMGC_OK;
}

// ------------------------------------------------------------------ row-mapping autotuner
// Times every candidate row mapping of one apply (1 warm-up launch, 3 timed, CUDA events on
// the hierarchy's stream) and returns the fastest: 0 warp per row, 1/2 SELL threads per row,
// 3 the staged FP32 kernel (fine-level 3x3 K only).
template <int MODE, class T>
static int tune_one(amgc_hierarchy* h, const BsrV<T>& A, const SellV<T>& S, const BsrV<T>* A2, const T* x,
                    const T* x2, const T* b, const T* dinv, T* y, int* best) {
  cudaEvent_t e0, e1;
  AMGC_CUDA_TRY(cudaEventCreate(&e0));
  AMGC_CUDA_TRY(cudaEventCreate(&e1));
  float best_ms = 1e30f;
  *best = 0;
  for (int cand = 0; cand < 4; ++cand) {
    if (cand > 0 && S.nslice == 0) break;
    if (cand == 3 && S.ctr == nullptr) break;
    for (int rep = 0; rep < 4; ++rep) {
      if (rep == 1) AMGC_CUDA_TRY(cudaEventRecord(e0, h->stream));
      AMGC_TRY((mapped_apply<MODE, T>(A, S, cand, A2, x, x2, b, x, dinv, 1.0, y, h->stream)));
    }
    AMGC_CUDA_TRY(cudaEventRecord(e1, h->stream));
    AMGC_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    AMGC_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_ms) {
      best_ms = ms;
      *best = cand;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return AMGC_OK;
}

// Times one CheapSIMPLE sweep of the level in each smoother form it has (0: two launches after
// the Jacobi step; 1: the fused single-CTA launch, tried on levels with few multiplier rows; 2:
// the split sweep, where the level has interface rows) with 1 warm-up and 3 timed sweeps (CUDA
// events on the hierarchy's stream) and keeps the fastest.  The work vectors hold finite values;
// the results are not used.
template <class T>
static int tune_form(amgc_hierarchy* h, const LevelV<T>& L, int l, int* form) {
  *form = 0;
  if (L.nl == 0 || h->smoother_kind != 0) return AMGC_OK;
  // one CTA walks every multiplier node and B1 row: beyond a few thousand of them the grid-wide
  // forms always win, and timing the single-CTA form would only lengthen the setup
  const bool small = L.nl <= kFuseMaxNodes && L.n_b1_rows <= 4 * kFuseMaxNodes;
  cudaStream_t s = h->stream;
  cudaEvent_t e0, e1;
  AMGC_CUDA_TRY(cudaEventCreate(&e0));
  AMGC_CUDA_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int cand = 0; cand < 3; ++cand) {
    if ((cand == 1 && !small) || (cand == 2 && L.n_ir == 0)) continue;
    LevelV<T> Lc = L;
    Lc.fuse = cand;
    for (int rep = 0; rep < 4; ++rep) {
      if (rep == 1) AMGC_CUDA_TRY(cudaEventRecord(e0, s));
      AMGC_TRY(smooth_sweeps<T>(h, Lc, l, L.b, L.x, 1, false));
    }
    AMGC_CUDA_TRY(cudaEventRecord(e1, s));
    AMGC_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    AMGC_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) {
      best = ms;
      *form = cand;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return AMGC_OK;
}

// fine_k_only: only the finest K (the Krylov operator apply) is tuned; the other maps keep
// their defaults (the FP64 views of a hierarchy whose cycle runs in FP32)
template <class T>
static int tune_views(amgc_hierarchy* h, std::vector<LevelV<T>>& V, int pidx, bool fine_k_only) {
  for (int l = 0; l + 1 < (int)V.size(); ++l) {
    LevelV<T>& L = V[l];
    const LevelV<T>& C = V[l + 1];
    const BsrV<T>* B1 = L.nl ? &L.B1 : nullptr;
    Level& LL = h->L[l];
    int km = LL.kmap[pidx], pm = LL.pmap[pidx], rm = LL.rmap[pidx];
    AMGC_TRY((tune_one<2, T>(h, L.K, L.Ks, B1, L.x, L.x + L.nu(), L.b, L.dinv, L.r, &km)));
    if (!fine_k_only) {
      AMGC_TRY((tune_one<1, T>(h, L.P, L.Ps, nullptr, C.x, nullptr, nullptr, nullptr, L.t, &pm)));
      AMGC_TRY((tune_one<0, T>(h, L.R, L.Rs, nullptr, L.r, nullptr, nullptr, nullptr, C.b, &rm)));
    }
    L.kmap = km; L.pmap = pm; L.rmap = rm;
    if (!fine_k_only) {   // the sweep's form, timed with the K mapping just chosen
      int form = 0;
      AMGC_TRY(tune_form<T>(h, L, l, &form));
      LL.fuse[pidx] = form;
      L.fuse = form;
    }
    LL.kmap[pidx] = km; LL.pmap[pidx] = pm; LL.rmap[pidx] = rm;
    if (fine_k_only) break;
  }
  return AMGC_OK;
}

// Builds SELL copies of K, P, R on every level that has a next one, then times the mappings.
int autotune(amgc_hierarchy* h) {
  const int nlev = (int)h->L.size();
  for (int l = 0; l + 1 < nlev; ++l) {
    Level& L = h->L[l];
    if (L.Ks.nslice == 0) AMGC_TRY(build_sell_of(h, L.K, L.Ks));
    if (L.Ps.nslice == 0) AMGC_TRY(build_sell_of(h, L.P, L.Ps));
    if (L.Rs.nslice == 0) AMGC_TRY(build_sell_of(h, L.R, L.Rs));
  }
  AMGC_TRY(make_views(h));
  const int64_t n0 = h->L[0].rows();
  (void)n0;
  // zero the work vectors the timings read (values do not matter, finiteness does)
  for (int l = 0; l < nlev; ++l) {
    Level& L = h->L[l];
    AMGC_CUDA_TRY(cudaMemsetAsync(L.x.p, 0, L.x.bytes(), h->stream));
    AMGC_CUDA_TRY(cudaMemsetAsync(L.b.p, 0, L.b.bytes(), h->stream));
    AMGC_CUDA_TRY(cudaMemsetAsync(L.r.p, 0, L.r.bytes(), h->stream));
    if (h->opts.precision == 32) {
      AMGC_CUDA_TRY(cudaMemsetAsync(L.f.x.p, 0, L.f.x.bytes(), h->stream));
      AMGC_CUDA_TRY(cudaMemsetAsync(L.f.b.p, 0, L.f.b.bytes(), h->stream));
      AMGC_CUDA_TRY(cudaMemsetAsync(L.f.r.p, 0, L.f.r.bytes(), h->stream));
    }
  }
  // an FP32 cycle uses the FP64 views for the Krylov operator apply only
  AMGC_TRY(tune_views<double>(h, h->v64, 0, h->opts.precision == 32));
  if (h->opts.precision == 32) AMGC_TRY(tune_views<float>(h, h->v32, 1, false));
  AMGC_CUDA_TRY(cudaStreamSynchronize(h->stream));
  return make_views(h);
}

// ------------------------------------------------------------------ dot products, lambda_max
__global__ void k_scale_dinv(int64_t n, const double* __restrict__ dinv, double* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] *= dinv[i];
}
__global__ void k_fill(int64_t n, double v, double* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = v;
}
// Deterministic two-stage dot products: stage 1 writes one partial per block.
constexpr int kDotThreads = 256;
constexpr int kDotBlocks = 1024;
__global__ void k_dot_partial(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                              const double* __restrict__ wgt, double* __restrict__ part) {
  __shared__ double sh[kDotThreads / 32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kDotThreads)
    s = fma(a[i] * (wgt ? wgt[i] : 1.0), b[i], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kDotThreads / 32 ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}
__global__ void k_dot_final(int nparts, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (int)(blockDim.x / 32) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) *out = v;
  }
}
// y = src / sqrt(*nrm2), the reciprocal formed once per block
__global__ void k_normalize(int64_t n, const double* __restrict__ nrm2, const double* __restrict__ src,
                            double* __restrict__ y) {
  __shared__ double inv;
  if (threadIdx.x == 0) inv = 1.0 / sqrt(*nrm2);
  __syncthreads();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = src[i] * inv;
}

int dot(amgc_hierarchy* h, int64_t n, const double* a, const double* b, const double* wgt, double* out_dev) {
  cudaStream_t s = h->stream;
  int blocks = (int)std::min<int64_t>(kDotBlocks, std::max<int64_t>(1, div_up(n, kDotThreads)));
  AMGC_LAUNCH(k_dot_partial<<<blocks, kDotThreads, 0, s>>>(n, a, b, wgt, h->partial.p));
  AMGC_LAUNCH(k_dot_final<<<1, 1024, 0, s>>>(blocks, h->partial.p, out_dev));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

// Per-instance dot products of a batched level: out[q] = sum over instance q's DOFs
// [bu*nptr[q], bu*nptr[q+1]) of a*wgt*b, one block per instance (fixed order).
__global__ void k_segdot(int ni, int bu, const int* __restrict__ nptr, const double* __restrict__ a,
                         const double* __restrict__ b, const double* __restrict__ wgt, double* __restrict__ out) {
  __shared__ double sh[32];
  const int q = blockIdx.x;
  if (q >= ni) return;
  const int64_t i0 = (int64_t)bu * nptr[q], i1 = (int64_t)bu * nptr[q + 1];
  double s = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) s = fma(a[i] * (wgt ? wgt[i] : 1.0), b[i], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (int)(blockDim.x / 32) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) out[q] = v;
  }
}
// y_i = src_i / sqrt(nrm2[inst(i)])
__global__ void k_segnormalize(int ni, int bu, const int* __restrict__ nptr, const double* __restrict__ nrm2,
                               const double* __restrict__ src, double* __restrict__ y) {
  const int q = blockIdx.y;
  const int64_t i0 = (int64_t)bu * nptr[q], i1 = (int64_t)bu * nptr[q + 1];
  const double inv = 1.0 / sqrt(nrm2[q]);
  for (int64_t i = i0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < i1; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = src[i] * inv;
}

// y = D^-1 K x (scaled) or y = K x, on the level's SELL copy when it has one, else on its BSR rows
static int power_apply(const Level& L, bool scaled, const double* x, double* y, cudaStream_t s) {
  if (L.Ks.nslice > 0) {
    const SellV<double> sv = sview<double>(L.Ks, L.Ks.val.p);
    return scaled ? sell_apply<4, double>(sv, L.nn, nullptr, x, nullptr, nullptr, nullptr, L.dinv.p, 0.0, y, s)
                  : sell_apply<0, double>(sv, L.nn, nullptr, x, nullptr, nullptr, nullptr, nullptr, 0.0, y, s);
  }
  const BsrV<double> kv = view_of(L.K);
  return scaled ? rowop<4, double>(kv, x, nullptr, nullptr, nullptr, nullptr, L.dinv.p, 0.0, y, s)
                : rowop<0, double>(kv, x, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, y, s);
}

// The same power iteration per instance of a batched level: lam[q] for every instance.  The
// instances are decoupled blocks of D^-1 K, so each instance's part of the iterate keeps its own
// direction under any per-instance scaling: the iterate is normalised per instance after steps
// 10 and 20 only, as in the single-instance iteration.
int lambda_max_instances(amgc_hierarchy* h, Level& L, std::vector<double>& lam) {
  cudaStream_t s = h->stream;
  const int ni = h->n_inst;
  const int64_t n = L.nu();
  const int th = 256;
  DBuf<double> xb, yb, sc;
  DBuf<int> dptr;
  AMGC_TRY(xb.alloc(n));
  AMGC_TRY(yb.alloc(n));
  AMGC_TRY(sc.alloc(2 * ni));
  AMGC_TRY(dptr.alloc(ni + 1));
  AMGC_CUDA_TRY(cudaMemcpyAsync(dptr.p, L.nptr.data(), (ni + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  double* xv = xb.p;
  double* yv = yb.p;
  const dim3 gs(64, ni);
  AMGC_LAUNCH(k_fill<<<div_up(n, th), th, 0, s>>>(n, 1.0, xv));
  AMGC_LAUNCH(k_segdot<<<ni, 512, 0, s>>>(ni, L.bu, dptr.p, xv, xv, nullptr, sc.p));
  AMGC_LAUNCH(k_segnormalize<<<gs, th, 0, s>>>(ni, L.bu, dptr.p, sc.p, xv, xv));
  for (int it = 0; it < 20; ++it) {
    AMGC_TRY(power_apply(L, true, xv, yv, s));
    if (it == 9 || it == 19) {
      AMGC_LAUNCH(k_segdot<<<ni, 512, 0, s>>>(ni, L.bu, dptr.p, yv, yv, nullptr, sc.p));
      AMGC_LAUNCH(k_segnormalize<<<gs, th, 0, s>>>(ni, L.bu, dptr.p, sc.p, yv, xv));
    } else {
      std::swap(xv, yv);
    }
  }
  AMGC_TRY(power_apply(L, false, xv, yv, s));
  AMGC_LAUNCH(k_segdot<<<ni, 512, 0, s>>>(ni, L.bu, dptr.p, xv, yv, nullptr, sc.p));
  AMGC_LAUNCH(k_segdot<<<ni, 512, 0, s>>>(ni, L.bu, dptr.p, xv, xv, L.kdiag.p, sc.p + ni));
  AMGC_CUDA_TRY(cudaGetLastError());
  std::vector<double> hs(2 * ni);
  AMGC_CUDA_TRY(cudaMemcpyAsync(hs.data(), sc.p, 2 * ni * sizeof(double), cudaMemcpyDeviceToHost, s));
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  lam.resize(ni);
  for (int q = 0; q < ni; ++q) {
    lam[q] = hs[ni + q] > 0.0 ? hs[q] / hs[ni + q] : 0.0;
    if (!(lam[q] > 0.0) || !std::isfinite(lam[q])) {
      set_error("lambda_max: non-positive or non-finite Rayleigh quotient on an instance");
      return AMGC_ESINGULAR;
    }
  }
  return AMGC_OK;
}

// ---------------------------------------------------------------- Schur-step damping
// One step of the power iteration on S_bd^-1 S_hat, S_hat = Z + B2 A~^-1 B1 (the operator whose
// block-diagonal approximation the CheapSIMPLE corrector inverts, Sec. 5.2).
// First t_i = A~^-1_i (B1 x)_i on the displacement rows that hold B1 blocks.
template <int BU>
__global__ void k_schur_b1(int nrows, const int* __restrict__ rows, const int* __restrict__ rp,
                           const int* __restrict__ col, const double* __restrict__ val,
                           const double* __restrict__ atinv, const double* __restrict__ x, double* __restrict__ t) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nrows) return;
  const int i = rows[k];
  double acc[BU];
#pragma unroll
  for (int m = 0; m < BU; ++m) acc[m] = 0.0;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const int l = col[e];
    const double* b = val + (int64_t)e * BU * 3;
    const double x0 = x[3 * (int64_t)l], x1 = x[3 * (int64_t)l + 1], x2 = x[3 * (int64_t)l + 2];
#pragma unroll
    for (int m = 0; m < BU; ++m) acc[m] = fma(b[m * 3], x0, fma(b[m * 3 + 1], x1, fma(b[m * 3 + 2], x2, acc[m])));
  }
#pragma unroll
  for (int m = 0; m < BU; ++m) t[(int64_t)i * BU + m] = atinv[(int64_t)i * BU + m] * acc[m];
}
// then y_l = S_bd,l^-1 (Z_l x_l + sum_i B2_li t_i) per multiplier node l
template <int BU>
__global__ void k_schur_apply(int nl, const int* __restrict__ rp, const int* __restrict__ col,
                              const double* __restrict__ val, const double* __restrict__ t, const double* __restrict__ Z,
                              const double* __restrict__ Sinv, const double* __restrict__ x, double* __restrict__ y) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nl) return;
  const double* z = Z + (int64_t)l * 9;
  const double x0 = x[3 * (int64_t)l], x1 = x[3 * (int64_t)l + 1], x2 = x[3 * (int64_t)l + 2];
  double r[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) r[a] = fma(z[a * 3], x0, fma(z[a * 3 + 1], x1, z[a * 3 + 2] * x2));
  for (int e = rp[l]; e < rp[l + 1]; ++e) {
    const int i = col[e];
    const double* b = val + (int64_t)e * 3 * BU;
#pragma unroll
    for (int m = 0; m < BU; ++m) {
      const double tv = t[(int64_t)i * BU + m];
#pragma unroll
      for (int a = 0; a < 3; ++a) r[a] = fma(b[a * BU + m], tv, r[a]);
    }
  }
  const double* si = Sinv + (int64_t)l * 9;
#pragma unroll
  for (int a = 0; a < 3; ++a) y[3 * (int64_t)l + a] = fma(si[a * 3], r[0], fma(si[a * 3 + 1], r[1], si[a * 3 + 2] * r[2]));
}
// Sinv_l *= f[l]
__global__ void k_scale_sinv(int nl, const double* __restrict__ f, double* __restrict__ Sinv) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nl * 9) return;
  Sinv[t] *= f[t / 9];
}

// rho_q of S_bd^-1 S_hat per instance q: 30 power steps from the normalised ones vector (per
// instance), rho = the norm of the last product.  The multiplier correction of instance q is then
// damped by alpha_q = min(alpha, (4/3)/rho_q), applied by scaling its inverted Schur blocks by
// alpha_q / alpha (the sweep kernels keep multiplying by alpha).
int schur_damping_setup(amgc_hierarchy* h, Level& L) {
  cudaStream_t s = h->stream;
  const int ni = h->n_inst;
  const int nl = L.nl;
  const int64_t n = 3 * (int64_t)nl;
  const int th = 256;
  std::vector<int> lp = ni > 1 ? L.lptr : std::vector<int>{0, nl};
  DBuf<double> xv, yv, tv, sc;
  DBuf<int> dptr;
  AMGC_TRY(xv.alloc(n));
  AMGC_TRY(yv.alloc(n));
  AMGC_TRY(tv.alloc((size_t)std::max(L.nu(), 1)));
  AMGC_TRY(sc.alloc(ni));
  AMGC_TRY(dptr.alloc(ni + 1));
  AMGC_CUDA_TRY(cudaMemcpyAsync(dptr.p, lp.data(), (ni + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  AMGC_CUDA_TRY(cudaMemsetAsync(tv.p, 0, (size_t)std::max(L.nu(), 1) * sizeof(double), s));
  AMGC_LAUNCH(k_fill<<<div_up(n, th), th, 0, s>>>(n, 1.0, xv.p));
  AMGC_LAUNCH(k_segdot<<<ni, 512, 0, s>>>(ni, 3, dptr.p, xv.p, xv.p, nullptr, sc.p));
  const dim3 gs(16, ni);
  AMGC_LAUNCH(k_segnormalize<<<gs, th, 0, s>>>(ni, 3, dptr.p, sc.p, xv.p, xv.p));
  for (int it = 0; it < 30; ++it) {
    if (L.n_b1_rows > 0) {
      if (L.bu == 3)
        AMGC_LAUNCH(k_schur_b1<3><<<div_up(L.n_b1_rows, 128), 128, 0, s>>>(L.n_b1_rows, L.b1_rows.p, L.B1.rowptr.p,
                                                                          L.B1.col.p, L.B1.val.p, L.atinv.p, xv.p, tv.p));
      else
        AMGC_LAUNCH(k_schur_b1<6><<<div_up(L.n_b1_rows, 128), 128, 0, s>>>(L.n_b1_rows, L.b1_rows.p, L.B1.rowptr.p,
                                                                          L.B1.col.p, L.B1.val.p, L.atinv.p, xv.p, tv.p));
    }
    if (L.bu == 3)
      AMGC_LAUNCH(k_schur_apply<3><<<div_up(nl, 128), 128, 0, s>>>(nl, L.B2.rowptr.p, L.B2.col.p, L.B2.val.p, tv.p,
                                                                   L.Z.p, L.Sinv.p, xv.p, yv.p));
    else
      AMGC_LAUNCH(k_schur_apply<6><<<div_up(nl, 128), 128, 0, s>>>(nl, L.B2.rowptr.p, L.B2.col.p, L.B2.val.p, tv.p,
                                                                   L.Z.p, L.Sinv.p, xv.p, yv.p));
    AMGC_LAUNCH(k_segdot<<<ni, 512, 0, s>>>(ni, 3, dptr.p, yv.p, yv.p, nullptr, sc.p));
    if (it < 29) AMGC_LAUNCH(k_segnormalize<<<gs, th, 0, s>>>(ni, 3, dptr.p, sc.p, yv.p, xv.p));
  }
  AMGC_CUDA_TRY(cudaGetLastError());
  std::vector<double> hs(ni);
  AMGC_CUDA_TRY(cudaMemcpyAsync(hs.data(), sc.p, ni * sizeof(double), cudaMemcpyDeviceToHost, s));
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  const double alpha = h->opts.simple_alpha;
  L.schur_rho.assign(ni, 0.0);
  std::vector<double> f(nl, 1.0);
  for (int q = 0; q < ni; ++q) {
    const double rho = std::sqrt(hs[q]);
    if (!(rho > 0.0) || !std::isfinite(rho)) {
      set_error("schur_damping: power iteration on S_bd^-1 S_hat broke down");
      return AMGC_ESINGULAR;
    }
    L.schur_rho[q] = rho;
    const double fq = alpha > 0.0 ? std::min(alpha, (4.0 / 3.0) / rho) / alpha : 1.0;
    for (int l = lp[q]; l < lp[q + 1]; ++l) f[l] = fq;
  }
  AMGC_CUDA_TRY(cudaMemcpyAsync(yv.p, f.data(), nl * sizeof(double), cudaMemcpyHostToDevice, s));
  AMGC_LAUNCH(k_scale_sinv<<<div_up((int64_t)nl * 9, th), th, 0, s>>>(nl, yv.p, L.Sinv.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  return AMGC_OK;
}

static int dot_on(cudaStream_t s, double* part, int64_t n, const double* a, const double* b, const double* wgt,
                  double* out_dev) {
  int blocks = (int)std::min<int64_t>(kDotBlocks, std::max<int64_t>(1, div_up(n, kDotThreads)));
  AMGC_LAUNCH(k_dot_partial<<<blocks, kDotThreads, 0, s>>>(n, a, b, wgt, part));
  AMGC_LAUNCH(k_dot_final<<<1, 1024, 0, s>>>(blocks, part, out_dev));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

// lambda_max(D^{-1} K): 20 power steps from the normalised ones vector, then the generalised
// Rayleigh quotient (x^T K x)/(x^T D x) with D the pointwise diagonal of K (kdiag).  Started on
// the auxiliary stream after the level's diagonal is ready (lambda_max_start), so that it runs
// beside the aggregation and the tentative transfers; lambda_max_finish joins it.
int lambda_max_start(amgc_hierarchy* h, Level& L) {
  const int64_t n = L.nu();
  const int th = 256;
  if (!h->aux_stream) AMGC_CUDA_TRY(cudaStreamCreateWithFlags(&h->aux_stream, cudaStreamNonBlocking));
  cudaStream_t s = h->aux_stream;
  AMGC_TRY(L.lmx_x.alloc(n));
  AMGC_TRY(L.lmx_y.alloc(n));
  AMGC_TRY(L.lmx_sc.alloc(4));
  AMGC_TRY(L.lmx_part.alloc(kDotBlocks));
  cudaEvent_t ready;
  AMGC_CUDA_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  AMGC_CUDA_TRY(cudaEventRecord(ready, h->stream));   // diagonal, SELL copy and buffers in place
  AMGC_CUDA_TRY(cudaStreamWaitEvent(s, ready, 0));
  cudaEventDestroy(ready);
  double* xv = L.lmx_x.p;
  double* yv = L.lmx_y.p;
  double* sc = L.lmx_sc.p;
  double* part = L.lmx_part.p;
  AMGC_LAUNCH(k_fill<<<div_up(n, th), th, 0, s>>>(n, 1.0 / sqrt((double)n), xv));
  AMGC_CUDA_TRY(cudaGetLastError());
  // y = D^-1 K x in one launch; the iterate is normalised after steps 10 and 20 only (the
  // direction, and with it the Rayleigh quotient, does not depend on the intermediate scaling,
  // and 10 steps cannot overflow for any lambda_max below 1e30)
  for (int it = 0; it < 20; ++it) {
    AMGC_TRY(power_apply(L, true, xv, yv, s));
    if (it == 9 || it == 19) {
      AMGC_TRY(dot_on(s, part, n, yv, yv, nullptr, sc));
      AMGC_LAUNCH(k_normalize<<<div_up(n, th), th, 0, s>>>(n, sc, yv, xv));
    } else {
      std::swap(xv, yv);
    }
    AMGC_CUDA_TRY(cudaGetLastError());
  }
  AMGC_TRY(power_apply(L, false, xv, yv, s));
  AMGC_TRY(dot_on(s, part, n, xv, yv, nullptr, sc));             // x^T K x
  AMGC_TRY(dot_on(s, part, n, xv, xv, L.kdiag.p, sc + 1));       // x^T D x
  if (!L.lmx_done) AMGC_CUDA_TRY(cudaEventCreateWithFlags(&L.lmx_done, cudaEventDisableTiming));
  AMGC_CUDA_TRY(cudaEventRecord(L.lmx_done, s));
  return AMGC_OK;
}

int lambda_max_finish(amgc_hierarchy* h, Level& L, double* out) {
  cudaStream_t s = h->stream;
  AMGC_CUDA_TRY(cudaStreamWaitEvent(s, L.lmx_done, 0));
  double hs[2] = {0.0, 0.0};
  AMGC_CUDA_TRY(cudaMemcpyAsync(hs, L.lmx_sc.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  // the buffers are released in order on the main stream, after the join
  L.lmx_x.release();
  L.lmx_y.release();
  L.lmx_sc.release();
  L.lmx_part.release();
  if (!(hs[1] > 0.0) || !std::isfinite(hs[0] / hs[1])) {
    set_error("lambda_max: non-positive or non-finite Rayleigh quotient");
    return AMGC_ESINGULAR;
  }
  *out = hs[0] / hs[1];
  return AMGC_OK;
}

int lambda_max_estimate(amgc_hierarchy* h, Level& L, double* out) {
  AMGC_TRY(lambda_max_start(h, L));
  return lambda_max_finish(h, L, out);
}

}  // namespace amgc
