// Right-preconditioned flexible GMRES(m) with one V-cycle per iteration (Sec. 3), stopped on
// ||r_k|| / ||r_0|| < tol for the full residual [r_u; r_lambda] (Eq. ch7_linearstoppingcriterion).
// Arnoldi: classical Gram-Schmidt with one re-orthogonalisation pass (CGS2), so each pass is a
// single streaming multi-dot plus a single streaming update over the basis.  Hessenberg
// columns, Givens rotations and the residual estimate live on the device; the host reads one
// scalar per iteration to decide whether to stop.
//
// The first pass's projection coefficients h1 are taken from FP32 copies of the basis and of w
// (FP32 arithmetic, FP64 partial sums); every update w -= V h and the second projection run in
// FP64.  After the exact FP64 update w1 = w - V h1, the second pass measures what h1 missed,
// h2 = V^T w1, so the Hessenberg column h1 + h2 and the Arnoldi relation w = V (h1 + h2) + w2
// hold to FP64 rounding whatever h1's accuracy; h1 only has to be close enough for the second
// pass to finish the orthogonalisation (its error is at FP32 level).  On GB300 the FP64 pipe
// bounds every Arnoldi sweep, and the first projection then reads half the bytes and issues no
// FP64 multiply-adds.
#include "amgc_internal.cuh"

#include <algorithm>
#include <cmath>

namespace amgc {

constexpr int kMdThreads = 256;
constexpr int kMdWarps = kMdThreads / 32;
constexpr int kMdBlocks = 608;   // 4 x 152 SMs
constexpr int kUpThreads = 256;
constexpr int kMaxRestart = 256;

// part[b * nk + k] = sum over block b's row chunk of V[k][i] * w[i], k = 0..nk-1.
// Warp q of the block takes the basis vectors k = q, q + 8, ...; lanes stream the chunk.
__global__ void __launch_bounds__(kMdThreads)
k_multidot(int64_t n, int nk, const double* __restrict__ V, const double* __restrict__ w, double* __restrict__ part) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = blockIdx.x * chunk;
  const int64_t b1 = b0 + chunk < n ? b0 + chunk : n;
  for (int k = wid; k < nk; k += kMdWarps) {
    const double* v = V + (int64_t)k * n;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;   // four independent chains: 8 loads in flight
    int64_t i = b0 + lane;
    for (; i + 96 < b1; i += 128) {
      s0 = fma(v[i], w[i], s0);
      s1 = fma(v[i + 32], w[i + 32], s1);
      s2 = fma(v[i + 64], w[i + 64], s2);
      s3 = fma(v[i + 96], w[i + 96], s3);
    }
    for (; i < b1; i += 32) s0 = fma(v[i], w[i], s0);
    const double t = warp_sum((s0 + s1) + (s2 + s3));
    if (lane == 0) part[(int64_t)blockIdx.x * nk + k] = t;
  }
}
// The same partial dot products from FP32 copies of the basis and of w: FP32 products and
// per-lane FP32 sums over the block's chunk, FP64 sums across the warp.
__global__ void __launch_bounds__(kMdThreads)
k_multidot_f32(int64_t n, int nk, const float* __restrict__ V, const float* __restrict__ w, double* __restrict__ part) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = blockIdx.x * chunk;
  const int64_t b1 = b0 + chunk < n ? b0 + chunk : n;
  for (int k = wid; k < nk; k += kMdWarps) {
    const float* v = V + (int64_t)k * n;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int64_t i = b0 + lane;
    for (; i + 96 < b1; i += 128) {
      s0 = fmaf(v[i], w[i], s0);
      s1 = fmaf(v[i + 32], w[i + 32], s1);
      s2 = fmaf(v[i + 64], w[i + 64], s2);
      s3 = fmaf(v[i + 96], w[i + 96], s3);
    }
    for (; i < b1; i += 32) s0 = fmaf(v[i], w[i], s0);
    const double t = warp_sum((double)((s0 + s1) + (s2 + s3)));
    if (lane == 0) part[(int64_t)blockIdx.x * nk + k] = t;
  }
}
// y = fp32(x)
__global__ void k_to_f32(int64_t n, const double* __restrict__ x, float* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = f64_to_f32_rn(x[i]);
}
// out[k*ldo] (+)= sum_b part[b*nk + k], one warp per k (fixed order: deterministic)
__global__ void k_multidot_final(int nk, int nb, const double* __restrict__ part, double* __restrict__ out, int ldo,
                                 int accumulate, double* __restrict__ hk) {
  const int lane = threadIdx.x & 31;
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (k >= nk) return;
  double s = 0.0;
  for (int b = lane; b < nb; b += 32) s += part[(int64_t)b * nk + k];
  s = warp_sum(s);
  if (lane == 0) {
    if (hk) hk[k] = s;
    out[(int64_t)k * ldo] = accumulate ? out[(int64_t)k * ldo] + s : s;
  }
}

// w[i] -= sum_k V[k][i] h[k]; with norm != nullptr also one partial of ||w||^2 per block.
__global__ void __launch_bounds__(kUpThreads)
k_basis_update(int64_t n, int nk, const double* __restrict__ V, const double* __restrict__ h, double* __restrict__ w,
               double* __restrict__ norm) {
  __shared__ double hs[kMaxRestart + 1];
  __shared__ double red[kUpThreads / 32];
  for (int k = threadIdx.x; k < nk; k += blockDim.x) hs[k] = h[k];
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double s = 0.0;
  if (i < n) {
    s = w[i];
#pragma unroll 8
    for (int k = 0; k < nk; ++k) s = fma(-V[(int64_t)k * n + i], hs[k], s);
    w[i] = s;
  }
  if (norm == nullptr) return;
  const double t = warp_sum(s * s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0;
#pragma unroll
    for (int q = 0; q < kUpThreads / 32; ++q) u += red[q];
    norm[blockIdx.x] = u;
  }
}

// ||w||^2 from nb block partials (fixed order) into scal[2], H[j+1][j] = ||w||, then the Givens
// rotations of column j (one block; column j and the rotations are staged in shared memory so
// that the sequential part reads no global memory)
__global__ void __launch_bounds__(kUpThreads)
k_norm_givens(int nb, const double* __restrict__ part, int j, int m, double* H, double* cs, double* sn, double* g,
              double beta0, double* scal) {
  __shared__ double red[kUpThreads / 32];
  __shared__ double hc[kMaxRestart + 1], c[kMaxRestart], sv[kMaxRestart];
  double t = 0.0;
  for (int b = threadIdx.x; b < nb; b += kUpThreads) t += part[b];
  for (int i = threadIdx.x; i <= j; i += kUpThreads) hc[i] = H[(int64_t)i * m + j];
  for (int i = threadIdx.x; i < j; i += kUpThreads) {
    c[i] = cs[i];
    sv[i] = sn[i];
  }
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double nrm2 = 0.0;
#pragma unroll
    for (int q = 0; q < kUpThreads / 32; ++q) nrm2 += red[q];
    scal[2] = nrm2;
    hc[j + 1] = sqrt(nrm2);
    for (int i = 0; i < j; ++i) {
      const double a = hc[i], b = hc[i + 1];
      hc[i] = c[i] * a + sv[i] * b;
      hc[i + 1] = -sv[i] * a + c[i] * b;
    }
    const double a = hc[j], b = hc[j + 1];
    const double den = hypot(a, b);
    const double cj = den > 0.0 ? a / den : 1.0;
    const double sj = den > 0.0 ? b / den : 0.0;
    cs[j] = cj;
    sn[j] = sj;
    hc[j] = den;
    hc[j + 1] = 0.0;
    const double gj = g[j];
    g[j + 1] = -sj * gj;
    g[j] = cj * gj;
    scal[0] = fabs(g[j + 1]) / beta0;
    scal[1] = isfinite(den) && isfinite(g[j + 1]) ? 0.0 : 1.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= j + 1; i += kUpThreads) H[(int64_t)i * m + j] = hc[i];
}
// x[i] += sum_k Zs[k][i] y[k]
__global__ void k_solution_update(int64_t n, int nk, const double* __restrict__ Zs, const double* __restrict__ y,
                                  double* __restrict__ x) {
  __shared__ double ys[kMaxRestart];
  for (int k = threadIdx.x; k < nk; k += blockDim.x) ys[k] = y[k];
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = x[i];
  for (int k = 0; k < nk; ++k) s = fma(Zs[(int64_t)k * n + i], ys[k], s);
  x[i] = s;
}
// 1 / sqrt(nrm2) formed once per block (an FP64 division per element would cost more than the
// memory traffic of these kernels); 0 when nrm2 is 0
__device__ __forceinline__ double block_rsqrt(const double* nrm2) {
  __shared__ double inv;
  if (threadIdx.x == 0) {
    const double nr = sqrt(*nrm2);
    inv = nr > 0.0 ? 1.0 / nr : 0.0;
  }
  __syncthreads();
  return inv;
}
// v = w / sqrt(nrm2) (zero vector on breakdown), with its FP32 copy vf
__global__ void k_arnoldi_normalize(int64_t n, const double* __restrict__ nrm2, const double* __restrict__ w,
                                    double* __restrict__ v, float* __restrict__ vf) {
  const double inv = block_rsqrt(nrm2);
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    const double t = w[i] * inv;
    v[i] = t;
    vf[i] = f64_to_f32_rn(t);
  }
}
// start of a cycle: v0 = r / beta (and its FP32 copy), g = (beta, 0, ...)
__global__ void k_cycle_start(int64_t n, const double* __restrict__ nrm2, const double* __restrict__ r,
                              double* __restrict__ v0, float* __restrict__ v0f, double* __restrict__ g, int m) {
  const double inv = block_rsqrt(nrm2);
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    const double t = r[i] * inv;
    v0[i] = t;
    v0f[i] = f64_to_f32_rn(t);
  }
  if (i <= m) g[i] = i == 0 ? sqrt(*nrm2) : 0.0;
}
// back substitution H(0:k,0:k) y = g(0:k) (single thread)
__global__ void k_backsolve(int k, int m, const double* __restrict__ H, const double* __restrict__ g, double* __restrict__ y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int q = i + 1; q < k; ++q) s -= H[i * m + q] * y[q];
    y[i] = s / H[i * m + i];
  }
}
__global__ void k_sub(int64_t n, const double* __restrict__ a, double* __restrict__ b) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i] - b[i];
}
__global__ void k_zero_vec(int64_t n, double* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = 0.0;
}

static int ensure_workspace(amgc_hierarchy* h, int64_t n, int m) {
  if (h->m_alloc == m && h->V.n == (size_t)(m + 1) * n) return AMGC_OK;
  AMGC_TRY(h->V.alloc((size_t)(m + 1) * n));
  AMGC_TRY(h->Vf.alloc((size_t)(m + 1) * n));
  AMGC_TRY(h->Zs.alloc((size_t)m * n));
  AMGC_TRY(h->H.alloc((size_t)(m + 1) * m));
  AMGC_TRY(h->givens.alloc((size_t)2 * m));
  AMGC_TRY(h->gvec.alloc(m + 1));
  AMGC_TRY(h->y.alloc(m + 1));
  AMGC_TRY(h->wk.alloc(std::max((size_t)kMdBlocks * (m + 1), (size_t)div_up(n, kUpThreads))));
  AMGC_TRY(h->rk.alloc(n));
  AMGC_TRY(h->xk.alloc(8));
  h->m_alloc = m;
  return AMGC_OK;
}

// h = V[0..nk)^T w into H column (stride m), optionally accumulating; hk receives the new values
static int multidot(amgc_hierarchy* h, int64_t n, int nk, const double* V, const double* w, double* Hcol, int m,
                    int accumulate, double* hk) {
  cudaStream_t s = h->stream;
  AMGC_LAUNCH(k_multidot<<<kMdBlocks, kMdThreads, 0, s>>>(n, nk, V, w, h->wk.p));
  AMGC_LAUNCH(k_multidot_final<<<div_up((int64_t)nk * 32, 128), 128, 0, s>>>(nk, kMdBlocks, h->wk.p, Hcol, m, accumulate,
                                                                            hk));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

int fgmres(amgc_hierarchy* h, const double* rhs, double* x, double tol_in, int* iters_out, double* relres_out) {
  cudaStream_t s = h->stream;
  const int64_t n = h->L[0].rows();
  const int m = std::max(1, std::min(h->opts.fgmres_restart, kMaxRestart));
  const int maxit = std::max(1, h->opts.fgmres_maxit);
  const double tol = tol_in > 0.0 ? tol_in : h->opts.tol;
  AMGC_TRY(ensure_workspace(h, n, m));
  const int th = 256;
  const int gn = div_up(n, th);
  const int gu = div_up(n, kUpThreads);
  double* scal = h->xk.p;          // [0] residual estimate, [1] breakdown flag, [2] norm^2, [3] scratch
  double* hk = h->y.p;             // reuse: projection coefficients of the current pass
  DBuf<double> hbuf;
  AMGC_TRY(hbuf.alloc(m + 1));
  double* cs = h->givens.p;
  double* sn = h->givens.p + m;
  double* pin = h->h_pinned;
  // the staged FP32 apply reports a bounded wait that gave up in the status word, read with the
  // iteration's residual estimate
  const bool staged = staged_apply_in_use(h) && !h->transposed;
  int* pst = reinterpret_cast<int*>(pin + 8);

  AMGC_LAUNCH(k_zero_vec<<<gn, th, 0, s>>>(n, x));
  AMGC_TRY(dot(h, n, rhs, rhs, nullptr, scal + 2));
  AMGC_CUDA_TRY(cudaMemcpyAsync(pin, scal + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  const double beta0 = std::sqrt(pin[0]);
  if (!std::isfinite(beta0)) {
    set_error("fgmres: non-finite right-hand side");
    return AMGC_BREAKDOWN;
  }
  if (beta0 == 0.0) {
    if (iters_out) *iters_out = 0;
    if (relres_out) *relres_out = 0.0;
    return AMGC_OK;
  }
  AMGC_CUDA_TRY(cudaMemcpyAsync(h->rk.p, rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  int total = 0;
  bool converged = false;
  double relres = 1.0;
  while (total < maxit && !converged) {
    // ||r||^2 is in scal[2]
    AMGC_LAUNCH(k_cycle_start<<<div_up(std::max<int64_t>(n, m + 1), th), th, 0, s>>>(n, scal + 2, h->rk.p, h->V.p,
                                                                                   h->Vf.p, h->gvec.p, m));
    AMGC_CUDA_TRY(cudaMemsetAsync(h->H.p, 0, (size_t)(m + 1) * m * sizeof(double), s));
    int jd = 0;
    for (int j = 0; j < m && total < maxit; ++j) {
      double* vj = h->V.p + (int64_t)j * n;
      double* zj = h->Zs.p + (int64_t)j * n;
      double* w = h->V.p + (int64_t)(j + 1) * n;
      AMGC_TRY(precond_apply(h, vj, zj));
      AMGC_TRY(saddle_apply(h, 0, zj, w));
      // CGS2: first projection from the FP32 copies (w's copy in the slot of v_{j+1}), then
      // FP64 update, FP64 projection, FP64 update with the partial norms of the result
      float* wf = h->Vf.p + (int64_t)(j + 1) * n;
      AMGC_LAUNCH(k_to_f32<<<gn, th, 0, s>>>(n, w, wf));
      AMGC_LAUNCH(k_multidot_f32<<<kMdBlocks, kMdThreads, 0, s>>>(n, j + 1, h->Vf.p, wf, h->wk.p));
      AMGC_LAUNCH(k_multidot_final<<<div_up((int64_t)(j + 1) * 32, 128), 128, 0, s>>>(j + 1, kMdBlocks, h->wk.p,
                                                                                     h->H.p + j, m, 0, hbuf.p));
      AMGC_LAUNCH(k_basis_update<<<gu, kUpThreads, 0, s>>>(n, j + 1, h->V.p, hbuf.p, w, nullptr));
      AMGC_TRY(multidot(h, n, j + 1, h->V.p, w, h->H.p + j, m, 1, hbuf.p));
      AMGC_LAUNCH(k_basis_update<<<gu, kUpThreads, 0, s>>>(n, j + 1, h->V.p, hbuf.p, w, h->wk.p));
      AMGC_CUDA_TRY(cudaGetLastError());
      AMGC_LAUNCH(k_norm_givens<<<1, kUpThreads, 0, s>>>(gu, h->wk.p, j, m, h->H.p, cs, sn, h->gvec.p, beta0, scal));
      AMGC_LAUNCH(k_arnoldi_normalize<<<gn, th, 0, s>>>(n, scal + 2, w, w, wf));
      AMGC_CUDA_TRY(cudaGetLastError());
      AMGC_CUDA_TRY(cudaMemcpyAsync(pin, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      if (staged) AMGC_CUDA_TRY(cudaMemcpyAsync(pst, h->status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
      AMGC_CUDA_TRY(cudaStreamSynchronize(s));
      if (staged && *pst != 0) return check_status(h, "fgmres (FP32 V-cycle)");
      ++total;
      jd = j + 1;
      relres = pin[0];
      if (pin[1] != 0.0 || !std::isfinite(relres)) {
        set_error("fgmres: non-finite Hessenberg entry");
        return AMGC_BREAKDOWN;
      }
      if (relres < tol) {
        converged = true;
        break;
      }
    }
    AMGC_LAUNCH(k_backsolve<<<1, 32, 0, s>>>(jd, m, h->H.p, h->gvec.p, hk));
    AMGC_LAUNCH(k_solution_update<<<gn, th, 0, s>>>(n, jd, h->Zs.p, hk, x));
    // true residual r = b - A x
    AMGC_TRY(saddle_apply(h, 0, x, h->rk.p));
    AMGC_LAUNCH(k_sub<<<gn, th, 0, s>>>(n, rhs, h->rk.p));
    AMGC_CUDA_TRY(cudaGetLastError());
    AMGC_TRY(dot(h, n, h->rk.p, h->rk.p, nullptr, scal + 2));
  }
  AMGC_CUDA_TRY(cudaMemcpyAsync(pin, scal + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  const double true_rel = std::sqrt(pin[0]) / beta0;
  if (iters_out) *iters_out = total;
  if (relres_out) *relres_out = true_rel;
  h->stats.last_iters = total;
  h->stats.last_relres = true_rel;
  if (!std::isfinite(true_rel)) {
    set_error("fgmres: non-finite residual");
    return AMGC_BREAKDOWN;
  }
  if (!converged) {
    set_error("fgmres: iteration limit reached");
    return AMGC_NOT_CONVERGED;
  }
  return AMGC_OK;
}

}  // namespace amgc
