// Multi-column V-cycle of batched hierarchies: the right-hand sides of amgc_solve_batched go through
// one cycle together (Fig. mgalgorithm with CheapSIMPLE smoothing, Algorithm 4), so that every
// matrix value of every level is read once for all NC columns: the sparse products are sparse
// matrix times NC vectors, everything else runs per column in the same launch (grid y = column).
//
// Column c of a level-l vector sits at p + c * rows(l) (column-major, as the batched FGMRES keeps
// its vectors), so the finest level reads the solver's vectors in place.  Same arithmetic, in the
// same order per column, as the single-column cycle of cycle.cu, hence the same results.
#include "amgc_internal.cuh"

#include <algorithm>

namespace amgc {

namespace {

template <class T>
__device__ __forceinline__ T cvt(double v) { return (T)v; }
template <>
__device__ __forceinline__ float cvt<float>(double v) { return f64_to_f32_rn(v); }

// MODE 0: y = s; 1: y += s; 2: y = b - s; 3: y = x0 + omega dinv (b - s)   (as cycle.cu's store_row)
template <int MODE, class T>
__device__ __forceinline__ void mc_store(T* y, const T* b, const T* x0, const T* dinv, T omega, int64_t o,
                                         int64_t oc, T s) {
  if (MODE == 0) y[oc] = s;
  else if (MODE == 1) y[oc] += s;
  else if (MODE == 2) y[oc] = b[oc] - s;
  else y[oc] = x0[oc] + omega * dinv[o] * (b[oc] - s);
}

// SELL-32, one thread per block row, NC columns: each stored value is loaded once and used for
// every column (x, x2 with column stride ldx; y, b, x0 with ldy)
template <int BR, int BC, int MODE, class T, int NC>
__global__ void __launch_bounds__(128)
k_mc_sell(int nbr, const int* __restrict__ soff, const int* __restrict__ slen, const int* __restrict__ scol,
          const T* __restrict__ sval, const T* __restrict__ x, int64_t ldx, const int* __restrict__ rp2,
          const int* __restrict__ c2, const T* __restrict__ v2, const T* __restrict__ x2, const T* __restrict__ b,
          const T* __restrict__ x0, const T* __restrict__ dinv, T omega, T* __restrict__ y, int64_t ldy,
          const int* __restrict__ rinst, const int* __restrict__ live, const int* __restrict__ perm) {
  constexpr int BS = BR * BC;
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;   // SELL position
  if (pos >= nbr) return;
  const int row = perm ? perm[pos] : pos;                  // its block row
  if (live && !live[rinst[row]]) return;
  const int sl = pos >> 5, ls = pos & 31;
  const int64_t o = soff[sl];
  const int L = slen[sl];
  const int* cp = scol + o * 32 + ls;
  const T* vp = sval + o * (BS * 32) + ls;
  T acc[NC][BR];
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int q = 0; q < BR; ++q) acc[c][q] = T(0);
  for (int t = 0; t < L; ++t) {
    const int64_t xc = (int64_t)__ldcs(cp + t * 32) * BC;
    T xv[NC][BC];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int k = 0; k < BC; ++k) xv[c][k] = __ldg(x + c * ldx + xc + k);
    const T* v = vp + (int64_t)t * (BS * 32);
#pragma unroll
    for (int q = 0; q < BR; ++q)
#pragma unroll
      for (int k = 0; k < BC; ++k) {
        const T a = __ldcs(v + (q * BC + k) * 32);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c][q] = fma(a, xv[c][k], acc[c][q]);
      }
  }
  if (rp2 != nullptr) {
    for (int e = rp2[row]; e < rp2[row + 1]; ++e) {
      const T* blk = v2 + (int64_t)e * BR * 3;
      const int64_t d = 3 * (int64_t)c2[e];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T d0 = x2[c * ldx + d], d1 = x2[c * ldx + d + 1], d2 = x2[c * ldx + d + 2];
#pragma unroll
        for (int q = 0; q < BR; ++q)
          acc[c][q] = fma(blk[3 * q], d0, fma(blk[3 * q + 1], d1, fma(blk[3 * q + 2], d2, acc[c][q])));
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int q = 0; q < BR; ++q) {
      const int64_t o1 = (int64_t)row * BR + q;
      mc_store<MODE, T>(y, b, x0, dinv, omega, o1, o1 + c * ldy, acc[c][q]);
    }
}

// W warps per block row (1: eight rows per CTA), one lane per block, NC columns; the warps' sums
// are added in warp order
template <int BR, int BC1, int BC2, int MODE, class T, int NC, int W>
__global__ void __launch_bounds__(256)
k_mc_rows(int nbr, const int* __restrict__ rp1, const int* __restrict__ c1, const T* __restrict__ v1,
          const T* __restrict__ x1, int64_t ldx, const int* __restrict__ rp2, const int* __restrict__ c2,
          const T* __restrict__ v2, const T* __restrict__ x2, const T* __restrict__ b, const T* __restrict__ x0,
          const T* __restrict__ dinv, T omega, T* __restrict__ y, int64_t ldy, const int* __restrict__ rinst,
          const int* __restrict__ live) {
  __shared__ T part[W > 1 ? W : 1][NC * BR];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int row = W > 1 ? (int)blockIdx.x : (int)blockIdx.x * (blockDim.x >> 5) + wid;
  if (row >= nbr || (live && !live[rinst[row]])) return;   // uniform over the row's warps
  const int w = W > 1 ? wid : 0;
  T acc[NC][BR];
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int q = 0; q < BR; ++q) acc[c][q] = T(0);
  for (int e = rp1[row] + w * 32 + lane; e < rp1[row + 1]; e += 32 * W) {
    const int64_t xc = (int64_t)__ldg(c1 + e) * BC1;
    const T* v = v1 + (int64_t)e * (BR * BC1);
#pragma unroll
    for (int k = 0; k < BC1; ++k) {
      T xv[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) xv[c] = __ldg(x1 + c * ldx + xc + k);
#pragma unroll
      for (int q = 0; q < BR; ++q) {
        const T a = __ldg(v + q * BC1 + k);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c][q] = fma(a, xv[c], acc[c][q]);
      }
    }
  }
  if (rp2 != nullptr) {
    for (int e = rp2[row] + w * 32 + lane; e < rp2[row + 1]; e += 32 * W) {
      const int64_t xc = (int64_t)__ldg(c2 + e) * BC2;
      const T* v = v2 + (int64_t)e * (BR * BC2);
#pragma unroll
      for (int k = 0; k < BC2; ++k) {
        T xv[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) xv[c] = __ldg(x2 + c * ldx + xc + k);
#pragma unroll
        for (int q = 0; q < BR; ++q) {
          const T a = __ldg(v + q * BC2 + k);
#pragma unroll
          for (int c = 0; c < NC; ++c) acc[c][q] = fma(a, xv[c], acc[c][q]);
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int q = 0; q < BR; ++q) acc[c][q] = warp_sum(acc[c][q]);
  if (W > 1) {
    if (lane == 0)
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int q = 0; q < BR; ++q) part[w][c * BR + q] = acc[c][q];
    __syncthreads();
    if (threadIdx.x >= NC * BR) return;
    const int c = threadIdx.x / BR, q = threadIdx.x - (threadIdx.x / BR) * BR;
    T s = T(0);
#pragma unroll
    for (int k = 0; k < W; ++k) s += part[k][threadIdx.x];
    const int64_t o1 = (int64_t)row * BR + q;
    mc_store<MODE, T>(y, b, x0, dinv, omega, o1, o1 + c * ldy, s);
    return;
  }
  if (lane != 0) return;
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int q = 0; q < BR; ++q) {
      const int64_t o1 = (int64_t)row * BR + q;
      mc_store<MODE, T>(y, b, x0, dinv, omega, o1, o1 + c * ldy, acc[c][q]);
    }
}

// multiplier rows (one warp per node, grid y = column), as cycle.cu's k_lm:
// MODE 0 residual, 1 corrector (lam updated, correction in out), 2 saddle apply
template <int BU, int MODE, class T>
__global__ void __launch_bounds__(128)
k_mc_lm(int nl, const int* __restrict__ rp, const int* __restrict__ col, const T* __restrict__ val,
        const T* __restrict__ u, const T* __restrict__ Z, const T* __restrict__ g, T* __restrict__ lam,
        const double* __restrict__ Sinv, double alpha, T* __restrict__ out, int64_t ld, const int* __restrict__ linst,
        const int* __restrict__ live) {
  const int lane = threadIdx.x & 31;
  const int l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (l >= nl || (live && !live[linst[l]])) return;
  const int64_t co = blockIdx.y * ld;
  u += co;
  lam += co;
  out += co;
  if (g) g += co;
  T acc[3] = {T(0), T(0), T(0)};
  for (int64_t e = rp[l] + lane; e < rp[l + 1]; e += 32) {
    const T* xc = u + (int64_t)__ldg(col + e) * BU;
    const T* v = val + e * (3 * BU);
#pragma unroll
    for (int k = 0; k < BU; ++k) {
      const T xv = __ldg(xc + k);
#pragma unroll
      for (int q = 0; q < 3; ++q) acc[q] = fma(__ldg(v + q * BU + k), xv, acc[q]);
    }
  }
  const T bu0 = warp_sum(acc[0]), bu1 = warp_sum(acc[1]), bu2 = warp_sum(acc[2]);
  if (lane != 0) return;
  const T* z = Z + (int64_t)l * 9;
  const T l0 = lam[3 * l], l1 = lam[3 * l + 1], l2 = lam[3 * l + 2];
  const T zl0 = z[0] * l0 + z[1] * l1 + z[2] * l2;
  const T zl1 = z[3] * l0 + z[4] * l1 + z[5] * l2;
  const T zl2 = z[6] * l0 + z[7] * l1 + z[8] * l2;
  if (MODE == 2) {
    out[3 * l] = bu0 - zl0;
    out[3 * l + 1] = bu1 - zl1;
    out[3 * l + 2] = bu2 - zl2;
    return;
  }
  const T r0 = g[3 * l] - bu0 + zl0, r1 = g[3 * l + 1] - bu1 + zl1, r2 = g[3 * l + 2] - bu2 + zl2;
  if (MODE == 0) {
    out[3 * l] = r0;
    out[3 * l + 1] = r1;
    out[3 * l + 2] = r2;
    return;
  }
  const double* S = Sinv + (int64_t)l * 9;
  const double d0 = -(S[0] * r0 + S[1] * r1 + S[2] * r2);
  const double d1 = -(S[3] * r0 + S[4] * r1 + S[5] * r2);
  const double d2 = -(S[6] * r0 + S[7] * r1 + S[8] * r2);
  lam[3 * l] = (T)(l0 + alpha * d0);
  lam[3 * l + 1] = (T)(l1 + alpha * d1);
  lam[3 * l + 2] = (T)(l2 + alpha * d2);
  out[3 * l] = (T)d0;
  out[3 * l + 1] = (T)d1;
  out[3 * l + 2] = (T)d2;
}

// u -= alpha atinv (B1 dlam) on the rows of B1 with entries (one warp per row, grid y = column)
template <int BU, class T>
__global__ void __launch_bounds__(128)
k_mc_b1_update(int nrows, const int* __restrict__ rows, const int* __restrict__ rp, const int* __restrict__ col,
               const T* __restrict__ val, const T* __restrict__ dlam, const T* __restrict__ atinv, T alpha,
               T* __restrict__ u, int64_t ld, const int* __restrict__ ninst, const int* __restrict__ live) {
  const int lane = threadIdx.x & 31;
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (t >= nrows) return;
  const int64_t co = blockIdx.y * ld;
  dlam += co;
  u += co;
  const int i = rows[t];
  if (live && !live[ninst[i]]) return;
  T acc[BU];
#pragma unroll
  for (int r = 0; r < BU; ++r) acc[r] = T(0);
  for (int64_t b = rp[i] + lane; b < rp[i + 1]; b += 32) {
    const T* xc = dlam + (int64_t)__ldg(col + b) * 3;
    const T x0 = __ldg(xc), x1 = __ldg(xc + 1), x2 = __ldg(xc + 2);
    const T* v = val + b * (BU * 3);
#pragma unroll
    for (int r = 0; r < BU; ++r) acc[r] = fma(v[r * 3], x0, fma(v[r * 3 + 1], x1, fma(v[r * 3 + 2], x2, acc[r])));
  }
  T out = T(0);
#pragma unroll
  for (int r = 0; r < BU; ++r) {
    const T v = warp_sum(acc[r]);
    if (lane == r) out = v;
  }
  if (lane < BU) u[(int64_t)i * BU + lane] -= alpha * atinv[(int64_t)i * BU + lane] * out;
}

// (masked: the DOFs of node i / bu and the multiplier entries of node i / 3 of finished instances)
template <class T>
__global__ void k_mc_jacobi_zero(int64_t n, int64_t nlam, const T* __restrict__ f, const T* __restrict__ dinv, T omega,
                                 T* __restrict__ y, T* __restrict__ lam, int64_t ld, int bu, const int* __restrict__ ninst,
                                 const int* __restrict__ linst, const int* __restrict__ live) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t co = blockIdx.y * ld;
  if (i < n && (!live || live[ninst[i / bu]])) y[co + i] = omega * dinv[i] * f[co + i];
  if (i < nlam && (!live || live[linst[i / 3]])) lam[co + i] = T(0);
}
template <class T>
__global__ void k_mc_copy(int64_t n, const T* __restrict__ a, int64_t lda, T* __restrict__ y, int64_t ldy, int bu,
                          const int* __restrict__ ninst, const int* __restrict__ live) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && (!live || live[ninst[i / bu]])) y[blockIdx.y * ldy + i] = a[blockIdx.y * lda + i];
}
template <class T>
__global__ void k_mc_zero(int64_t n, T* __restrict__ y, int64_t ld) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[blockIdx.y * ld + i] = T(0);
}
template <class Ta, class Tb>
__global__ void k_mc_convert(int64_t n, const Ta* __restrict__ a, int64_t lda, Tb* __restrict__ y, int64_t ldy) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[blockIdx.y * ldy + i] = cvt<Tb>((double)a[blockIdx.y * lda + i]);
}
// multiplier restriction (one warp per coarse node) and prolongation through P-hat^lambda
template <class T>
__global__ void k_mc_restrict_lm(int nlc, const int* __restrict__ ptr, const int* __restrict__ idx,
                                 const T* __restrict__ w, const T* __restrict__ r, int64_t ldr, T* __restrict__ out,
                                 int64_t ldo, const int* __restrict__ linst_c, const int* __restrict__ live) {
  const int lane = threadIdx.x & 31;
  const int L = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (L >= nlc || (live && !live[linst_c[L]])) return;
  r += blockIdx.y * ldr;
  out += blockIdx.y * ldo;
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
__global__ void k_mc_prolong_lm(int nl, const int* __restrict__ lagg, const T* __restrict__ w, const T* __restrict__ c,
                                int64_t ldc, T* __restrict__ lam, int64_t ldl, const int* __restrict__ linst,
                                const int* __restrict__ live) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nl || (live && !live[linst[l]])) return;
  c += blockIdx.y * ldc;
  lam += blockIdx.y * ldl;
  const int L = lagg[l];
  const T wl = w[l];
  lam[3 * l] += wl * c[3 * L];
  lam[3 * l + 1] += wl * c[3 * L + 1];
  lam[3 * l + 2] += wl * c[3 * L + 2];
}
// batched coarsest solve, NC columns: each instance's dense inverse row read once
template <class T, int NC>
__global__ void k_mc_gemv_batched(int n, const int* __restrict__ inst, const int* __restrict__ loc,
                                  const int* __restrict__ glob, const int* __restrict__ goff,
                                  const int64_t* __restrict__ doff, const double* __restrict__ A,
                                  const T* __restrict__ x, T* __restrict__ y, int64_t ld, const int* __restrict__ live) {
  const int lane = threadIdx.x & 31;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  const int q = inst[row];
  if (live && !live[q]) return;
  const int g0 = goff[q], nq = goff[q + 1] - g0;
  const double* a = A + doff[q] + (int64_t)loc[row] * nq;
  double s[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) s[c] = 0.0;
  for (int j = lane; j < nq; j += 32) {
    const double aj = a[j];
    const int gj = glob[g0 + j];
#pragma unroll
    for (int c = 0; c < NC; ++c) s[c] = fma(aj, (double)x[c * ld + gj], s[c]);
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const double v = warp_sum(s[c]);
    if (lane == 0) y[c * ld + row] = (T)v;
  }
}

// ------------------------------------------------------------------ host side
template <class T>
struct McBufs {
  DBuf<T> x, b, r, t, dl;
};

// y (ldy) = op(A x (ldx) [+ A2 x2]) for NC columns; SELL when the matrix has a 3-row SELL copy,
// else W warps per row by the mean row length (as the single-column kernels choose).  Rows whose
// instance is finished (live[rinst[row]] == 0) are skipped when live is given.
template <int MODE, class T, int NC>
int mc_apply(const BsrV<T>& A, const SellV<T>& S, const BsrV<T>* A2, const T* x, const T* x2, int64_t ldx,
             const T* b, const T* x0, const T* dinv, double omega, T* y, int64_t ldy, const int* rinst,
             const int* live, cudaStream_t s) {
  if (A.nbr == 0) return AMGC_OK;
  const int* r2 = A2 ? A2->rp : nullptr;
  const int* k2 = A2 ? A2->col : nullptr;
  const T* w2 = A2 ? A2->val : nullptr;
  if (S.nslice > 0 && S.br == 3) {
    const int g = div_up(A.nbr, 128);
    if (S.bc == 3)
      AMGC_LAUNCH(k_mc_sell<3, 3, MODE, T, NC><<<g, 128, 0, s>>>(A.nbr, S.off, S.len, S.col, S.val, x, ldx, r2, k2,
                                                                w2, x2, b, x0, dinv, (T)omega, y, ldy, rinst, live, S.perm));
    else if (S.bc == 6)
      AMGC_LAUNCH(k_mc_sell<3, 6, MODE, T, NC><<<g, 128, 0, s>>>(A.nbr, S.off, S.len, S.col, S.val, x, ldx, r2, k2,
                                                                w2, x2, b, x0, dinv, (T)omega, y, ldy, rinst, live, S.perm));
    else {
      set_error("multi-column apply: unsupported SELL block shape");
      return AMGC_EINVAL;
    }
    AMGC_CUDA_TRY(cudaGetLastError());
    return AMGC_OK;
  }
  const double mean = A.nbr ? (double)A.nnzb / A.nbr : 0.0;
  const int bc2 = A2 ? A2->bc : 3;
#define AMGC_MC_ROWS(BR_, BC1_)                                                                                 \
  if (A.br == BR_ && A.bc == BC1_ && bc2 == 3) {                                                                \
    if (mean > 96)                                                                                              \
      AMGC_LAUNCH(k_mc_rows<BR_, BC1_, 3, MODE, T, NC, 8><<<A.nbr, 256, 0, s>>>(                                  \
          A.nbr, A.rp, A.col, A.val, x, ldx, r2, k2, w2, x2, b, x0, dinv, (T)omega, y, ldy, rinst, live));        \
    else if (mean > 24)                                                                                         \
      AMGC_LAUNCH(k_mc_rows<BR_, BC1_, 3, MODE, T, NC, 2><<<A.nbr, 64, 0, s>>>(                                   \
          A.nbr, A.rp, A.col, A.val, x, ldx, r2, k2, w2, x2, b, x0, dinv, (T)omega, y, ldy, rinst, live));        \
    else                                                                                                        \
      AMGC_LAUNCH(k_mc_rows<BR_, BC1_, 3, MODE, T, NC, 1><<<div_up(A.nbr, 8), 256, 0, s>>>(                     \
          A.nbr, A.rp, A.col, A.val, x, ldx, r2, k2, w2, x2, b, x0, dinv, (T)omega, y, ldy, rinst, live));        \
    AMGC_CUDA_TRY(cudaGetLastError());                                                                          \
    return AMGC_OK;                                                                                             \
  }
  AMGC_MC_ROWS(3, 3)
  AMGC_MC_ROWS(6, 6)
  AMGC_MC_ROWS(3, 6)
  AMGC_MC_ROWS(6, 3)
#undef AMGC_MC_ROWS
  set_error("multi-column apply: unsupported block shape");
  return AMGC_EINVAL;
}

// instance of every displacement node and multiplier node of every level (masks)
struct McMaps {
  std::vector<DBuf<int>> node, lm;
};

template <class T, int NC>
struct McCycle {
  amgc_hierarchy* h;
  std::vector<LevelV<T>>& V;
  std::vector<McBufs<T>>& B;
  const McMaps& maps;
  const int* live;      // instance flags (null: every instance)
  cudaStream_t s;
  static constexpr int th = 256;

  const int* ni(int l) const { return maps.node[l].p; }
  const int* li(int l) const { return maps.lm[l].p; }

  int lm(int l, int mode, const T* u, const T* g, T* lam, double alpha, T* out, int64_t ld) {
    const LevelV<T>& L = V[l];
    if (L.nl == 0) return AMGC_OK;
    const dim3 grid(div_up((int64_t)L.nl * 32, 128), NC);
#define AMGC_MC_LM(BU_, M_)                                                                                       \
  AMGC_LAUNCH(k_mc_lm<BU_, M_, T><<<grid, 128, 0, s>>>(L.nl, L.B2.rp, L.B2.col, L.B2.val, u, L.Z, g, lam, L.Sinv, \
                                                        alpha, out, ld, li(l), live))
    if (L.bu == 3) {
      if (mode == 0) AMGC_MC_LM(3, 0);
      else if (mode == 1) AMGC_MC_LM(3, 1);
      else AMGC_MC_LM(3, 2);
    } else {
      if (mode == 0) AMGC_MC_LM(6, 0);
      else if (mode == 1) AMGC_MC_LM(6, 1);
      else AMGC_MC_LM(6, 2);
    }
#undef AMGC_MC_LM
    AMGC_CUDA_TRY(cudaGetLastError());
    return AMGC_OK;
  }

  // `sweeps` CheapSIMPLE sweeps (as cycle.cu's smooth_sweeps), every column at once
  int smooth(int l, McBufs<T>& W, const T* b, T* x, int sweeps, bool zero_guess) {
    const LevelV<T>& L = V[l];
    const int nu = L.nu();
    const int64_t ld = L.rows();
    const T* f = b;
    const T* g = b + nu;
    T* u = x;
    T* lam = x + nu;
    T* t = W.t.p;
    const int J = h->opts.jacobi_sweeps;
    const int steps = sweeps * J;
    const BsrV<T>* B1 = L.nl ? &L.B1 : nullptr;
    T* cur = u;
    int step = 0;
    for (int k = 0; k < sweeps; ++k) {
      for (int j = 0; j < J; ++j, ++step) {
        if (zero_guess && step == 0) {
          T* dst = ((steps - 1) % 2 == 0) ? u : t;
          const int64_t nlam = 3 * (int64_t)L.nl;
          AMGC_LAUNCH(k_mc_jacobi_zero<T><<<dim3(div_up(std::max<int64_t>(nu, nlam), th), NC), th, 0, s>>>(
              nu, nlam, f, L.dinv, (T)L.omega_j, dst, lam, ld, L.bu, ni(l), li(l), live));
          AMGC_CUDA_TRY(cudaGetLastError());
          cur = dst;
        } else {
          T* dst = cur == u ? t : u;
          AMGC_TRY((mc_apply<3, T, NC>(L.K, L.Ks, B1, cur, lam, ld, f, cur, L.dinv, L.omega_j, dst, ld, ni(l), live, s)));
          cur = dst;
        }
      }
      AMGC_TRY(lm(l, 1, cur, g, lam, h->opts.simple_alpha, W.dl.p, ld));
      if (L.n_b1_rows > 0) {
        const dim3 gb(div_up((int64_t)L.n_b1_rows * 32, 128), NC);
        if (L.bu == 3)
          AMGC_LAUNCH(k_mc_b1_update<3, T><<<gb, 128, 0, s>>>(L.n_b1_rows, L.b1_rows, L.B1.rp, L.B1.col, L.B1.val,
                                                              W.dl.p, L.atinv, (T)h->opts.simple_alpha, cur, ld, ni(l),
                                                              live));
        else
          AMGC_LAUNCH(k_mc_b1_update<6, T><<<gb, 128, 0, s>>>(L.n_b1_rows, L.b1_rows, L.B1.rp, L.B1.col, L.B1.val,
                                                              W.dl.p, L.atinv, (T)h->opts.simple_alpha, cur, ld, ni(l),
                                                              live));
        AMGC_CUDA_TRY(cudaGetLastError());
      }
    }
    if (cur != u) {
      AMGC_LAUNCH(k_mc_copy<T><<<dim3(div_up(nu, th), NC), th, 0, s>>>(nu, cur, ld, u, ld, L.bu, ni(l), live));
      AMGC_CUDA_TRY(cudaGetLastError());
    }
    return AMGC_OK;
  }

  int cycle(int l, const T* b, T* x) {
    const LevelV<T>& L = V[l];
    McBufs<T>& W = B[l];
    const int64_t ld = L.rows();
    if (l == (int)V.size() - 1) {
      const int n = L.rows();
      AMGC_LAUNCH(k_mc_gemv_batched<T, NC><<<div_up((int64_t)n * 32, th), th, 0, s>>>(
          n, L.c_inst, L.c_loc, L.c_glob, L.c_goff, L.c_doff, L.Ainv, b, x, ld, live));
      AMGC_CUDA_TRY(cudaGetLastError());
      return AMGC_OK;
    }
    const int nu = L.nu();
    const LevelV<T>& C = V[l + 1];
    McBufs<T>& CW = B[l + 1];
    const int64_t ldc = C.rows();
    const int sweeps = h->opts.smoother_sweeps;
    if (sweeps == 0) AMGC_LAUNCH(k_mc_zero<T><<<dim3(div_up(L.rows(), th), NC), th, 0, s>>>(L.rows(), x, ld));
    AMGC_TRY(smooth(l, W, b, x, sweeps, true));
    // residual, restriction (the rows of R are the coarse level's nodes)
    const BsrV<T>* B1 = L.nl ? &L.B1 : nullptr;
    AMGC_TRY((mc_apply<2, T, NC>(L.K, L.Ks, B1, x, x + nu, ld, b, nullptr, nullptr, 0.0, W.r.p, ld, ni(l), live, s)));
    AMGC_TRY(lm(l, 0, x, b + nu, x + nu, 0.0, W.r.p + nu, ld));
    AMGC_TRY((mc_apply<0, T, NC>(L.R, L.Rs, nullptr, W.r.p, nullptr, ld, nullptr, nullptr, nullptr, 0.0, CW.b.p, ldc,
                                 ni(l + 1), live, s)));
    if (C.nl > 0) {
      AMGC_LAUNCH(k_mc_restrict_lm<T><<<dim3(div_up((int64_t)C.nl * 32, 128), NC), 128, 0, s>>>(
          C.nl, L.rl_ptr, L.rl_idx, L.pl_w, W.r.p + nu, ld, CW.b.p + C.nu(), ldc, li(l + 1), live));
      AMGC_CUDA_TRY(cudaGetLastError());
    }
    AMGC_TRY(cycle(l + 1, CW.b.p, CW.x.p));
    // prolongation
    AMGC_TRY((mc_apply<1, T, NC>(L.P, L.Ps, nullptr, CW.x.p, nullptr, ldc, nullptr, nullptr, nullptr, 0.0, x, ld, ni(l),
                                 live, s)));
    if (L.nl > 0) {
      AMGC_LAUNCH(k_mc_prolong_lm<T><<<dim3(div_up(L.nl, 128), NC), 128, 0, s>>>(L.nl, L.lagg, L.pl_w, CW.x.p + C.nu(),
                                                                                 ldc, x + nu, ld, li(l), live));
      AMGC_CUDA_TRY(cudaGetLastError());
    }
    AMGC_TRY(smooth(l, W, b, x, sweeps, false));
    return AMGC_OK;
  }
};

template <class T>
int alloc_mc(amgc_hierarchy* h, std::vector<McBufs<T>>& B, int nc) {
  const int nlev = (int)h->L.size();
  if ((int)B.size() == nlev && B[0].x.n >= (size_t)nc * std::max(h->L[0].rows(), 1)) return AMGC_OK;
  B.clear();
  B.resize(nlev);
  for (int l = 0; l < nlev; ++l) {
    const size_t n = (size_t)nc * std::max(h->L[l].rows(), 1);
    AMGC_TRY(B[l].x.alloc(n));
    AMGC_TRY(B[l].b.alloc(n));
    AMGC_TRY(B[l].r.alloc(n));
    AMGC_TRY(B[l].t.alloc(n));
    AMGC_TRY(B[l].dl.alloc(n));
  }
  return AMGC_OK;
}

// node -> instance and multiplier node -> instance of every level, from the instance ranges
int build_maps(amgc_hierarchy* h, McMaps& M) {
  const int nlev = (int)h->L.size();
  if ((int)M.node.size() == nlev) return AMGC_OK;
  M.node.clear();
  M.lm.clear();
  M.node.resize(nlev);
  M.lm.resize(nlev);
  cudaStream_t s = h->stream;
  for (int l = 0; l < nlev; ++l) {
    const Level& L = h->L[l];
    std::vector<int> a(std::max(L.nn, 1), 0), b(std::max(L.nl, 1), 0);
    if (h->n_inst > 1 && (int)L.nptr.size() == h->n_inst + 1 && (int)L.lptr.size() == h->n_inst + 1) {
      for (int q = 0; q < h->n_inst; ++q) {
        for (int i = L.nptr[q]; i < L.nptr[q + 1]; ++i) a[i] = q;
        for (int i = L.lptr[q]; i < L.lptr[q + 1]; ++i) b[i] = q;
      }
    }
    AMGC_TRY(M.node[l].alloc(a.size()));
    AMGC_TRY(M.lm[l].alloc(b.size()));
    AMGC_CUDA_TRY(cudaMemcpyAsync(M.node[l].p, a.data(), a.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    AMGC_CUDA_TRY(cudaMemcpyAsync(M.lm[l].p, b.data(), b.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  }
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  return AMGC_OK;
}

}  // namespace

// Work buffers and instance maps of the multi-column cycle, kept by the hierarchy between calls.
struct McState {
  std::vector<McBufs<double>> b64;
  std::vector<McBufs<float>> b32;
  DBuf<float> in32, out32;
  McMaps maps;
};

void mc_state_free(McState* st) { delete st; }

// z = V-cycle(r) for kMcCols columns at once (column stride rows[0], FP64 in and out), skipping the
// rows of instances with live[q] == 0 when live is given; the FP32 cycle converts at entry and exit
int precond_apply_cols(amgc_hierarchy* h, const double* r, double* z, const int* live) {
  constexpr int NC = kMcCols;
  if (!h->mc) h->mc = new McState();
  McState& M = *h->mc;
  AMGC_TRY(build_maps(h, M.maps));
  const int64_t n = h->L[0].rows();
  cudaStream_t s = h->stream;
  if (h->opts.precision == 32) {
    AMGC_TRY(alloc_mc<float>(h, M.b32, NC));
    if (M.in32.n < (size_t)NC * n) {
      AMGC_TRY(M.in32.alloc((size_t)NC * n));
      AMGC_TRY(M.out32.alloc((size_t)NC * n));
    }
    AMGC_LAUNCH((k_mc_convert<double, float><<<dim3(div_up(n, 256), NC), 256, 0, s>>>(n, r, n, M.in32.p, n)));
    McCycle<float, NC> c{h, h->v32, M.b32, M.maps, live, s};
    AMGC_TRY(c.cycle(0, M.in32.p, M.out32.p));
    AMGC_LAUNCH((k_mc_convert<float, double><<<dim3(div_up(n, 256), NC), 256, 0, s>>>(n, M.out32.p, n, z, n)));
    AMGC_CUDA_TRY(cudaGetLastError());
    return AMGC_OK;
  }
  AMGC_TRY(alloc_mc<double>(h, M.b64, NC));
  McCycle<double, NC> c{h, h->v64, M.b64, M.maps, live, s};
  return c.cycle(0, r, z);
}

// y = A x for kMcCols columns (FP64, column stride rows[0]): the fine K (with B1) read once; rows of
// instances with live[q] == 0 skipped when live is given
int saddle_apply_cols(amgc_hierarchy* h, const double* x, double* y, const int* live) {
  constexpr int NC = kMcCols;
  if (!h->mc) h->mc = new McState();
  AMGC_TRY(build_maps(h, h->mc->maps));
  const McMaps& maps = h->mc->maps;
  const LevelV<double>& L = h->v64[0];
  const int nu = L.nu();
  const int64_t ld = L.rows();
  cudaStream_t s = h->stream;
  const BsrV<double>* B1 = L.nl ? &L.B1 : nullptr;
  AMGC_TRY((mc_apply<0, double, NC>(L.K, L.Ks, B1, x, x + nu, ld, nullptr, nullptr, nullptr, 0.0, y, ld,
                                    maps.node[0].p, live, s)));
  if (L.nl > 0) {
    AMGC_LAUNCH(k_mc_lm<3, 2, double><<<dim3(div_up((int64_t)L.nl * 32, 128), NC), 128, 0, s>>>(
        L.nl, L.B2.rp, L.B2.col, L.B2.val, x, L.Z, nullptr, const_cast<double*>(x + nu), L.Sinv, 0.0, y + nu, ld,
        maps.lm[0].p, live));
    AMGC_CUDA_TRY(cudaGetLastError());
  }
  return AMGC_OK;
}

}  // namespace amgc
