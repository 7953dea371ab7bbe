// Block-sparse row operations of the V-cycle and of FGMRES (FP64).
//
// Mapping: one warp per block row.  A lane keeps the same value slot w (and so the same
// block-row index w / BC) for every block it visits, so each matrix value costs exactly one
// fused multiply-add; the per-row outputs are summed once at the end through shared memory.
// GB300 issues FP64 FMAs at a small fraction of its FP32 rate, so avoiding redundant FP64
// arithmetic matters as much as coalescing here.
#include "amgc_internal.cuh"

#include <algorithm>
#include <cmath>

namespace amgc {

constexpr int kRowWarps = 8;   // warps per block of the row kernels

// Accumulates sum_b A[row, b] x[col[b]] for one block row into the lane's slots.
template <int BR, int BC>
struct RowMap {
  static constexpr int BS = BR * BC;
  static constexpr int KB = BS <= 32 ? 32 / BS : 1;      // blocks per warp step
  static constexpr int NW = BS <= 32 ? 1 : (BS + 31) / 32;  // values per lane per block
};

template <int BR, int BC>
__device__ __forceinline__ void row_accumulate(int64_t b0, int64_t b1, const int* __restrict__ col,
                                               const double* __restrict__ val, const double* __restrict__ x,
                                               int lane, double (&acc)[RowMap<BR, BC>::NW]) {
  using RM = RowMap<BR, BC>;
  if (RM::BS <= 32) {
    const int slot = lane / RM::BS;
    const int w = lane - slot * RM::BS;
    const int c = w % BC;
    if (lane < RM::KB * RM::BS) {
      for (int64_t b = b0 + slot; b < b1; b += RM::KB) {
        const int j = __ldg(col + b);
        acc[0] = fma(__ldg(val + b * RM::BS + w), __ldg(x + (int64_t)j * BC + c), acc[0]);
      }
    }
  } else {
    for (int64_t b = b0; b < b1; ++b) {
      const int j = __ldg(col + b);
#pragma unroll
      for (int k = 0; k < RM::NW; ++k) {
        const int w = lane + 32 * k;
        if (w < RM::BS) acc[k] = fma(__ldg(val + b * RM::BS + w), __ldg(x + (int64_t)j * BC + (w % BC)), acc[k]);
      }
    }
  }
}

// Sums the lane slots of one warp into the BR row outputs; valid in lanes < BR.
template <int BR, int BC>
__device__ __forceinline__ double row_reduce(double* sh, int lane, const double (&acc)[RowMap<BR, BC>::NW]) {
  using RM = RowMap<BR, BC>;
#pragma unroll
  for (int k = 0; k < RM::NW; ++k) sh[lane + 32 * k] = acc[k];
  __syncwarp();
  double s = 0.0;
  if (lane < BR) {
    for (int slot = 0; slot < RM::KB; ++slot)
#pragma unroll
      for (int c = 0; c < BC; ++c) s += sh[slot * RM::BS + lane * BC + c];
  }
  __syncwarp();
  return s;
}

// MODE 0: y  = A1 x1 + A2 x2
// MODE 1: y += A1 x1
// MODE 2: y  = b - A1 x1 - A2 x2                        (residual)
// MODE 3: y  = x0 + omega * dinv * (b - A1 x1 - A2 x2)    (damped Jacobi, out of place)
template <int BR, int BC1, int BC2, int MODE>
__global__ void __launch_bounds__(kRowWarps * 32)
k_rowop(int nbr, const int* __restrict__ rp1, const int* __restrict__ c1, const double* __restrict__ v1,
        const double* __restrict__ x1, const int* __restrict__ rp2, const int* __restrict__ c2,
        const double* __restrict__ v2, const double* __restrict__ x2, const double* __restrict__ b,
        const double* __restrict__ x0, const double* __restrict__ dinv, double omega, double* __restrict__ y) {
  constexpr int NS = (RowMap<BR, BC1>::NW > RowMap<BR, BC2>::NW ? RowMap<BR, BC1>::NW : RowMap<BR, BC2>::NW) * 32;
  __shared__ double sh[kRowWarps][NS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int row = blockIdx.x * kRowWarps + wid;
  if (row >= nbr) return;
  double acc1[RowMap<BR, BC1>::NW];
#pragma unroll
  for (int k = 0; k < RowMap<BR, BC1>::NW; ++k) acc1[k] = 0.0;
  row_accumulate<BR, BC1>(rp1[row], rp1[row + 1], c1, v1, x1, lane, acc1);
  double s = row_reduce<BR, BC1>(sh[wid], lane, acc1);
  if (rp2 != nullptr) {
    const int64_t e0 = rp2[row], e1 = rp2[row + 1];
    if (e1 > e0) {
      double acc2[RowMap<BR, BC2>::NW];
#pragma unroll
      for (int k = 0; k < RowMap<BR, BC2>::NW; ++k) acc2[k] = 0.0;
      row_accumulate<BR, BC2>(e0, e1, c2, v2, x2, lane, acc2);
      s += row_reduce<BR, BC2>(sh[wid], lane, acc2);
    }
  }
  if (lane < BR) {
    const int64_t o = (int64_t)row * BR + lane;
    if (MODE == 0) y[o] = s;
    else if (MODE == 1) y[o] += s;
    else if (MODE == 2) y[o] = b[o] - s;
    else y[o] = x0[o] + omega * dinv[o] * (b[o] - s);
  }
}

template <int BR, int BC1, int BC2, int MODE>
static int launch_rowop(int nbr, const DBsr& A1, const double* x1, const DBsr* A2, const double* x2,
                        const double* b, const double* x0, const double* dinv, double omega, double* y,
                        cudaStream_t s) {
  if (nbr == 0) return AMGC_OK;
  AMGC_LAUNCH(k_rowop<BR, BC1, BC2, MODE><<<div_up(nbr, kRowWarps), kRowWarps * 32, 0, s>>>(
      nbr, A1.rowptr.p, A1.col.p, A1.val.p, x1, A2 ? A2->rowptr.p : nullptr, A2 ? A2->col.p : nullptr,
      A2 ? A2->val.p : nullptr, x2, b, x0, dinv, omega, y));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

// Dispatch on (BR, BC1, BC2) for the shapes the hierarchy uses.
template <int MODE>
static int rowop(const DBsr& A1, const double* x1, const DBsr* A2, const double* x2, const double* b,
                 const double* x0, const double* dinv, double omega, double* y, cudaStream_t s) {
  const int br = A1.br, bc1 = A1.bc, bc2 = A2 ? A2->bc : 3;
  const int n = A1.nbr;
#define AMGC_ROWOP_CASE(R, C1, C2)                                                          \
  if (br == R && bc1 == C1 && bc2 == C2)                                                    \
    return launch_rowop<R, C1, C2, MODE>(n, A1, x1, A2, x2, b, x0, dinv, omega, y, s);
  AMGC_ROWOP_CASE(3, 3, 3)
  AMGC_ROWOP_CASE(6, 6, 3)
  AMGC_ROWOP_CASE(3, 6, 3)
  AMGC_ROWOP_CASE(6, 3, 3)
#undef AMGC_ROWOP_CASE
  set_error("rowop: unsupported block shape");
  return AMGC_EINVAL;
}

int bsr_spmv(const DBsr& A, const double* x, double* y, double alpha, double beta, cudaStream_t s) {
  (void)alpha;
  (void)beta;
  return rowop<0>(A, x, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, y, s);
}

// ------------------------------------------------------------------ multiplier-node kernels
// r_l = g_l - (B2 u)_l + Z_l lam_l  (MODE 0: store residual into out)
// MODE 1: corrector of CheapSIMPLE: d = -Sinv_l r_l; lam_l += alpha d; dlam_l = d
// MODE 2: y_l = (B2 u)_l - Z_l lam_l  (saddle apply)
template <int BU, int MODE>
__global__ void k_lm(int nl, const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
                     const double* __restrict__ u, const double* __restrict__ Z, const double* __restrict__ g,
                     double* __restrict__ lam, const double* __restrict__ Sinv, double alpha,
                     double* __restrict__ out) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nl) return;
  double bu0 = 0, bu1 = 0, bu2 = 0;
  for (int e = rp[l]; e < rp[l + 1]; ++e) {
    const double* blk = val + (int64_t)e * 3 * BU;
    const double* uj = u + (int64_t)col[e] * BU;
#pragma unroll
    for (int c = 0; c < BU; ++c) {
      const double x = uj[c];
      bu0 = fma(blk[c], x, bu0);
      bu1 = fma(blk[BU + c], x, bu1);
      bu2 = fma(blk[2 * BU + c], x, bu2);
    }
  }
  const double* z = Z + (int64_t)l * 9;
  const double l0 = lam[3 * l], l1 = lam[3 * l + 1], l2 = lam[3 * l + 2];
  const double zl0 = z[0] * l0 + z[1] * l1 + z[2] * l2;
  const double zl1 = z[3] * l0 + z[4] * l1 + z[5] * l2;
  const double zl2 = z[6] * l0 + z[7] * l1 + z[8] * l2;
  if (MODE == 2) {
    out[3 * l] = bu0 - zl0;
    out[3 * l + 1] = bu1 - zl1;
    out[3 * l + 2] = bu2 - zl2;
    return;
  }
  const double r0 = g[3 * l] - bu0 + zl0, r1 = g[3 * l + 1] - bu1 + zl1, r2 = g[3 * l + 2] - bu2 + zl2;
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
  lam[3 * l] = l0 + alpha * d0;
  lam[3 * l + 1] = l1 + alpha * d1;
  lam[3 * l + 2] = l2 + alpha * d2;
  out[3 * l] = d0;
  out[3 * l + 1] = d1;
  out[3 * l + 2] = d2;
}

template <int MODE>
static int lm_op(const Level& L, const double* u, const double* g, double* lam, double alpha, double* out,
                 cudaStream_t s) {
  if (L.nl == 0) return AMGC_OK;
  const int th = 128;
  if (L.bu == 3)
    AMGC_LAUNCH(k_lm<3, MODE><<<div_up(L.nl, th), th, 0, s>>>(L.nl, L.B2.rowptr.p, L.B2.col.p, L.B2.val.p, u, L.Z.p, g, lam,
                                                  L.Sinv.p, alpha, out));
  else
    AMGC_LAUNCH(k_lm<6, MODE><<<div_up(L.nl, th), th, 0, s>>>(L.nl, L.B2.rowptr.p, L.B2.col.p, L.B2.val.p, u, L.Z.p, g, lam,
                                                  L.Sinv.p, alpha, out));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

// x_u = uh - alpha * atinv * (B1 dlam)   over all displacement DOFs (B1 rows listed in b1_rows)
__global__ void k_copy(int64_t n, const double* __restrict__ a, double* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = a[i];
}
__global__ void k_zero(int64_t n, double* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = 0.0;
}
__global__ void k_jacobi_zero(int64_t n, const double* __restrict__ f, const double* __restrict__ dinv, double omega,
                              double* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = omega * dinv[i] * f[i];
}
template <int BU>
__global__ void k_b1_update(int nrows, const int* __restrict__ rows, const int* __restrict__ rp,
                            const int* __restrict__ col, const double* __restrict__ val, const double* __restrict__ dlam,
                            const double* __restrict__ atinv, double alpha, double* __restrict__ u) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nrows) return;
  const int i = rows[t];
  double acc[BU];
#pragma unroll
  for (int r = 0; r < BU; ++r) acc[r] = 0.0;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const double* blk = val + (int64_t)e * BU * 3;
    const double* d = dlam + (int64_t)col[e] * 3;
#pragma unroll
    for (int r = 0; r < BU; ++r) acc[r] += blk[3 * r] * d[0] + blk[3 * r + 1] * d[1] + blk[3 * r + 2] * d[2];
  }
#pragma unroll
  for (int r = 0; r < BU; ++r) u[(int64_t)i * BU + r] -= alpha * atinv[(int64_t)i * BU + r] * acc[r];
}

// lambda restriction / prolongation through P-hat^lambda (weights w_l, aggregate lagg_l)
__global__ void k_restrict_lm(int nlc, const int* __restrict__ ptr, const int* __restrict__ idx,
                              const double* __restrict__ w, const double* __restrict__ r, double* __restrict__ out) {
  const int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= nlc) return;
  double s0 = 0, s1 = 0, s2 = 0;
  for (int e = ptr[L]; e < ptr[L + 1]; ++e) {
    const int l = idx[e];
    const double wl = w[l];
    s0 += wl * r[3 * l];
    s1 += wl * r[3 * l + 1];
    s2 += wl * r[3 * l + 2];
  }
  out[3 * L] = s0;
  out[3 * L + 1] = s1;
  out[3 * L + 2] = s2;
}
__global__ void k_prolong_lm(int nl, const int* __restrict__ lagg, const double* __restrict__ w,
                             const double* __restrict__ c, double* __restrict__ lam) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nl) return;
  const int L = lagg[l];
  const double wl = w[l];
  lam[3 * l] += wl * c[3 * L];
  lam[3 * l + 1] += wl * c[3 * L + 1];
  lam[3 * l + 2] += wl * c[3 * L + 2];
}

// dense y = A x, A row-major n x n (coarsest solve with the explicit inverse)
__global__ void k_gemv(int n, const double* __restrict__ A, const double* __restrict__ x, double* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  const double* a = A + (int64_t)row * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s = fma(a[j], x[j], s);
  s = warp_sum(s);
  if (lane == 0) y[row] = s;
}

// ------------------------------------------------------------------ level operations
// Algorithmic bytes of one K-apply launch on level L: K and B1 values and indices once,
// x and lambda once, the output once, plus `extra_vecs` further length-nu vectors.
static double k_apply_bytes(const Level& L, int extra_vecs) {
  const double s = 8.0;
  double b = (double)L.K.nnzb * (L.bu * L.bu * s + 4.0) + 4.0 * (L.nn + 1);
  b += (double)L.B1.nnzb * (L.bu * 3 * s + 4.0) + (L.nl ? 4.0 * (L.nn + 1) + 3.0 * L.nl * s : 0.0);
  b += (2.0 + extra_vecs) * L.nu() * s;
  return b;
}

// K apply of level l through rowop<MODE>, timed when the level is the finest one.
template <int MODE>
static int k_apply(amgc_hierarchy* h, int l, const double* x1, const double* lam, const double* b, const double* x0,
                   double* y) {
  Level& L = h->L[l];
  const bool t = l == 0;
  if (t) AMGC_TRY(prof_begin(h));
  AMGC_TRY(rowop<MODE>(L.K, x1, L.nl ? &L.B1 : nullptr, lam, b, x0, L.dinv.p, L.omega_j, y, h->stream));
  if (t) AMGC_TRY(prof_end(h, k_apply_bytes(L, MODE == 3 ? 3 : (MODE == 2 ? 1 : 0))));
  return AMGC_OK;
}
static int smooth(amgc_hierarchy* h, int l, const double* b, double* x, bool zero_guess) {
  Level& L = h->L[l];
  cudaStream_t s = h->stream;
  const int nu = L.nu();
  const double* f = b;
  const double* g = b + nu;
  double* u = x;
  double* lam = x + nu;
  double* t = L.t.p;   // u_half
  const int th = 256;
  for (int j = 0; j < h->opts.jacobi_sweeps; ++j) {
    double* src = (j % 2 == 0) ? u : t;
    double* dst = (j % 2 == 0) ? t : u;
    if (zero_guess && j == 0) {
      AMGC_LAUNCH(k_zero<<<div_up(3 * (int64_t)L.nl, th), th, 0, s>>>(3 * (int64_t)L.nl, lam));
      AMGC_LAUNCH(k_jacobi_zero<<<div_up(nu, th), th, 0, s>>>(nu, f, L.dinv.p, L.omega_j, dst));
      AMGC_CUDA_TRY(cudaGetLastError());
    } else {
      AMGC_TRY(k_apply<3>(h, l, src, lam, f, src, dst));
    }
  }
  double* uh = (h->opts.jacobi_sweeps % 2 == 1) ? t : u;
  // corrector on the multipliers: dlam = -S^-1 (g - B2 uh + Z lam), lam += alpha dlam
  AMGC_TRY(lm_op<1>(L, uh, g, lam, h->opts.simple_alpha, L.dlam.p, s));
  // u = uh - alpha A~^-1 B1 dlam
  if (uh != u) {
    AMGC_LAUNCH(k_copy<<<div_up(nu, th), th, 0, s>>>(nu, uh, u));
    AMGC_CUDA_TRY(cudaGetLastError());
  }
  if (L.n_b1_rows > 0) {
    if (L.bu == 3)
      AMGC_LAUNCH(k_b1_update<3><<<div_up(L.n_b1_rows, 128), 128, 0, s>>>(L.n_b1_rows, L.b1_rows.p, L.B1.rowptr.p, L.B1.col.p,
                                                             L.B1.val.p, L.dlam.p, L.atinv.p, h->opts.simple_alpha, u));
    else
      AMGC_LAUNCH(k_b1_update<6><<<div_up(L.n_b1_rows, 128), 128, 0, s>>>(L.n_b1_rows, L.b1_rows.p, L.B1.rowptr.p, L.B1.col.p,
                                                             L.B1.val.p, L.dlam.p, L.atinv.p, h->opts.simple_alpha, u));
    AMGC_CUDA_TRY(cudaGetLastError());
  }
  return AMGC_OK;
}

static int residual(amgc_hierarchy* h, int l, const double* b, const double* x, double* r) {
  Level& L = h->L[l];
  const int nu = L.nu();
  AMGC_TRY(k_apply<2>(h, l, x, x + nu, b, nullptr, r));
  AMGC_TRY(lm_op<0>(L, x, b + nu, const_cast<double*>(x + nu), 0.0, r + nu, h->stream));
  return AMGC_OK;
}

int saddle_apply(amgc_hierarchy* h, int l, const double* x, double* y) {
  Level& L = h->L[l];
  const int nu = L.nu();
  AMGC_TRY(k_apply<0>(h, l, x, x + nu, nullptr, nullptr, y));
  AMGC_TRY(lm_op<2>(L, x, nullptr, const_cast<double*>(x + nu), 0.0, y + nu, h->stream));
  return AMGC_OK;
}

int vcycle(amgc_hierarchy* h, int l, const double* b, double* x) {
  Level& L = h->L[l];
  cudaStream_t s = h->stream;
  const int th = 256;
  if (l == (int)h->L.size() - 1) {
    const int n = L.rows();
    AMGC_LAUNCH(k_gemv<<<div_up((int64_t)n * 32, th), th, 0, s>>>(n, L.Ainv.p, b, x));
    AMGC_CUDA_TRY(cudaGetLastError());
    return AMGC_OK;
  }
  const int nu = L.nu();
  Level& C = h->L[l + 1];
  const int sweeps = h->opts.smoother_sweeps;
  if (sweeps == 0) {
    AMGC_LAUNCH(k_zero<<<div_up(L.rows(), th), th, 0, s>>>(L.rows(), x));
    AMGC_CUDA_TRY(cudaGetLastError());
  }
  for (int k = 0; k < sweeps; ++k) AMGC_TRY(smooth(h, l, b, x, k == 0));
  AMGC_TRY(residual(h, l, b, x, L.r.p));
  // restrict: C.b = [R r_u ; R^lambda r_lambda]
  AMGC_TRY(rowop<0>(L.R, L.r.p, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, C.b.p, s));
  if (C.nl > 0) {
    AMGC_LAUNCH(k_restrict_lm<<<div_up(C.nl, 128), 128, 0, s>>>(C.nl, L.rl_ptr.p, L.rl_idx.p, L.pl_w.p, L.r.p + nu,
                                                    C.b.p + C.nu()));
    AMGC_CUDA_TRY(cudaGetLastError());
  }
  AMGC_TRY(vcycle(h, l + 1, C.b.p, C.x.p));
  // prolongate and add
  AMGC_TRY(rowop<1>(L.P, C.x.p, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, x, s));
  if (L.nl > 0) {
    AMGC_LAUNCH(k_prolong_lm<<<div_up(L.nl, 128), 128, 0, s>>>(L.nl, L.lagg.p, L.pl_w.p, C.x.p + C.nu(), x + nu));
    AMGC_CUDA_TRY(cudaGetLastError());
  }
  for (int k = 0; k < sweeps; ++k) AMGC_TRY(smooth(h, l, b, x, false));
  return AMGC_OK;
}

// ------------------------------------------------------------------ lambda_max by power iteration
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
// y /= sqrt(*nrm2)
__global__ void k_normalize(int64_t n, const double* __restrict__ nrm2, const double* __restrict__ src,
                            double* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = src[i] / sqrt(*nrm2);
}

int dot(amgc_hierarchy* h, int64_t n, const double* a, const double* b, const double* wgt, double* out_dev) {
  cudaStream_t s = h->stream;
  int blocks = (int)std::min<int64_t>(kDotBlocks, std::max<int64_t>(1, div_up(n, kDotThreads)));
  AMGC_LAUNCH(k_dot_partial<<<blocks, kDotThreads, 0, s>>>(n, a, b, wgt, h->partial.p));
  AMGC_LAUNCH(k_dot_final<<<1, 1024, 0, s>>>(blocks, h->partial.p, out_dev));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

// lambda_max(D^{-1} K): 20 power steps from the normalised ones vector, then the generalised
// Rayleigh quotient (x^T K x)/(x^T D x) with D the pointwise diagonal of K (kdiag).
int lambda_max_estimate(amgc_hierarchy* h, Level& L, double* out) {
  cudaStream_t s = h->stream;
  const int64_t n = L.nu();
  const int th = 256;
  DBuf<double> xv, yv, sc;
  AMGC_TRY(xv.alloc(n));
  AMGC_TRY(yv.alloc(n));
  AMGC_TRY(sc.alloc(4));
  AMGC_LAUNCH(k_fill<<<div_up(n, th), th, 0, s>>>(n, 1.0 / sqrt((double)n), xv.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  for (int it = 0; it < 20; ++it) {
    AMGC_TRY(bsr_spmv(L.K, xv.p, yv.p, 1.0, 0.0, s));
    AMGC_LAUNCH(k_scale_dinv<<<div_up(n, th), th, 0, s>>>(n, L.dinv.p, yv.p));
    AMGC_TRY(dot(h, n, yv.p, yv.p, nullptr, sc.p));
    AMGC_LAUNCH(k_normalize<<<div_up(n, th), th, 0, s>>>(n, sc.p, yv.p, xv.p));
    AMGC_CUDA_TRY(cudaGetLastError());
  }
  AMGC_TRY(bsr_spmv(L.K, xv.p, yv.p, 1.0, 0.0, s));
  AMGC_TRY(dot(h, n, xv.p, yv.p, nullptr, sc.p));             // x^T K x
  AMGC_TRY(dot(h, n, xv.p, xv.p, L.kdiag.p, sc.p + 1));       // x^T D x
  double hs[2] = {0.0, 0.0};
  AMGC_CUDA_TRY(cudaMemcpyAsync(hs, sc.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  if (!(hs[1] > 0.0) || !std::isfinite(hs[0] / hs[1])) {
    set_error("lambda_max: non-positive or non-finite Rayleigh quotient");
    return AMGC_ESINGULAR;
  }
  *out = hs[0] / hs[1];
  return AMGC_OK;
}

}  // namespace amgc
