// Batched solves: n_inst independent contact systems concatenated block-diagonally, each with
// nrhs right-hand sides.  One hierarchy and one V-cycle serve every instance at once (instance
// ranges stay contiguous on every level); FGMRES keeps one Krylov space per (instance, rhs)
// system: segmented dot products over instance-aligned row chunks, per-system Hessenberg
// columns, Givens rotations, stopping test and solution update, all in lockstep.  Vectors hold
// nrhs columns of length rows[0] (column-major).
#include "amgc_internal.cuh"

#include <algorithm>
#include <cmath>

namespace amgc {

constexpr int kBChunk = 4096;     // rows per chunk (chunks never straddle an instance range)
constexpr int kBThreads = 256;

// part[(k * nrhs + r) * nchunk + c] = sum over chunk c of V[k][r][i] * w[r][i]
__global__ void __launch_bounds__(kBThreads)
k_bmultidot(int nchunk, const int* __restrict__ row0, const int* __restrict__ row1, int nrhs, int64_t n, int nk,
            const double* __restrict__ V, const double* __restrict__ w, double* __restrict__ part,
            const int* __restrict__ chunk_inst, const int* __restrict__ live) {
  const int c = blockIdx.x, r = blockIdx.y;
  if (live && !live[chunk_inst[c]]) return;   // a finished instance: its sums are not read
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t b0 = row0[c], b1 = row1[c];
  const double* wr = w + (int64_t)r * n;
  for (int k = wid; k < nk; k += kBThreads / 32) {
    const double* v = V + ((int64_t)k * nrhs + r) * n;
    double s = 0.0;
    for (int64_t i = b0 + lane; i < b1; i += 32) s = fma(v[i], wr[i], s);
    s = warp_sum(s);
    if (lane == 0) part[((int64_t)k * nrhs + r) * nchunk + c] = s;
  }
}
// out[s * os + k * ok] (+)= sum of the instance's chunks; one warp per (k, system)
__global__ void k_bmultidot_final(int nk, int ni, int nrhs, int nchunk, const int* __restrict__ cptr,
                                  const double* __restrict__ part, double* __restrict__ out, int64_t os, int64_t ok,
                                  int accumulate, double* __restrict__ hk, int ldh) {
  const int lane = threadIdx.x & 31;
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nsys = ni * nrhs;
  if (wg >= nk * nsys) return;
  const int k = wg / nsys, sys = wg - k * nsys;
  const int q = sys / nrhs, r = sys - q * nrhs;
  double s = 0.0;
  for (int c = cptr[q] + lane; c < cptr[q + 1]; c += 32) s += part[((int64_t)k * nrhs + r) * nchunk + c];
  s = warp_sum(s);
  if (lane == 0) {
    double* o = out + sys * os + k * ok;
    *o = accumulate ? *o + s : s;
    if (hk) hk[(int64_t)sys * ldh + k] = s;
  }
}
// w[r][i] -= sum_k V[k][r][i] hk[sys][k], sys = (instance of row i, r)
__global__ void k_bbasis_update(int64_t n, int nrhs, int nk, const double* __restrict__ V, const double* __restrict__ hk,
                                int ldh, const int* __restrict__ row_inst, double* __restrict__ w,
                                const int* __restrict__ live) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * nrhs) return;
  const int r = (int)(t / n);
  const int64_t i = t - (int64_t)r * n;
  if (live && !live[row_inst[i]]) return;
  const int sys = row_inst[i] * nrhs + r;
  const double* h = hk + (int64_t)sys * ldh;
  double s = w[t];
  for (int k = 0; k < nk; ++k) s = fma(-V[((int64_t)k * nrhs + r) * n + i], h[k], s);
  w[t] = s;
}
// inv[sys] = 1 / sqrt(nrm2[sys]) (0 for a zero norm), so that the vector kernels multiply
__global__ void k_brsqrt(int nsys, const double* __restrict__ nrm2, double* __restrict__ inv) {
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= nsys) return;
  const double nr = sqrt(nrm2[sys]);
  inv[sys] = nr > 0.0 ? 1.0 / nr : 0.0;
}
// v = w / sqrt(nrm2[sys]) with inv = k_brsqrt(nrm2) (0 on breakdown)
__global__ void k_bnormalize(int64_t n, int nrhs, const int* __restrict__ row_inst, const double* __restrict__ inv,
                             const double* __restrict__ w, double* __restrict__ v, const int* __restrict__ live) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * nrhs) return;
  const int r = (int)(t / n);
  const int64_t i = t - (int64_t)r * n;
  if (live && !live[row_inst[i]]) return;
  v[t] = w[t] * inv[row_inst[i] * nrhs + r];
}
// H[sys][j+1][j] = sqrt(nrm2[sys])
__global__ void k_bsubdiag(int nsys, int j, int m, const double* __restrict__ nrm2, double* __restrict__ H) {
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys < nsys) H[(int64_t)sys * (m + 1) * m + (int64_t)(j + 1) * m + j] = sqrt(nrm2[sys]);
}
// Givens update of column j of every live system; counts the live systems left
__global__ void k_bgivens(int nsys, int j, int m, double* __restrict__ H, double* __restrict__ cs,
                          double* __restrict__ sn, double* __restrict__ g, const double* __restrict__ beta0,
                          int* __restrict__ done, int* __restrict__ jd, int* __restrict__ iters, int total,
                          double tol, int* __restrict__ live, int* __restrict__ bad) {
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= nsys || done[sys]) return;
  double* Hs = H + (int64_t)sys * (m + 1) * m;
  double* c = cs + (int64_t)sys * m;
  double* sv = sn + (int64_t)sys * m;
  double* gs = g + (int64_t)sys * (m + 1);
  for (int i = 0; i < j; ++i) {
    const double a = Hs[i * m + j], b = Hs[(i + 1) * m + j];
    Hs[i * m + j] = c[i] * a + sv[i] * b;
    Hs[(i + 1) * m + j] = -sv[i] * a + c[i] * b;
  }
  const double a = Hs[j * m + j], b = Hs[(j + 1) * m + j];
  const double den = hypot(a, b);
  c[j] = den > 0.0 ? a / den : 1.0;
  sv[j] = den > 0.0 ? b / den : 0.0;
  Hs[j * m + j] = den;
  Hs[(j + 1) * m + j] = 0.0;
  const double gj = gs[j];
  gs[j + 1] = -sv[j] * gj;
  gs[j] = c[j] * gj;
  jd[sys] = j + 1;
  iters[sys] = total;
  if (!isfinite(den) || !isfinite(gs[j + 1])) {
    atomicAdd(bad, 1);
    done[sys] = 1;
    return;
  }
  if (fabs(gs[j + 1]) < tol * beta0[sys]) done[sys] = 1;
  else atomicAdd(live, 1);
}
// back substitution per system with its own number of columns jd[sys]; y[sys][k] = 0 beyond
__global__ void k_bbacksolve(int nsys, int m, const double* __restrict__ H, const double* __restrict__ g,
                             const int* __restrict__ jd, double* __restrict__ y) {
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= nsys) return;
  const double* Hs = H + (int64_t)sys * (m + 1) * m;
  const double* gs = g + (int64_t)sys * (m + 1);
  double* ys = y + (int64_t)sys * (m + 1);
  const int k = jd[sys];
  for (int i = m - 1; i >= k; --i) ys[i] = 0.0;
  for (int i = k - 1; i >= 0; --i) {
    double s = gs[i];
    for (int q = i + 1; q < k; ++q) s -= Hs[i * m + q] * ys[q];
    ys[i] = s / Hs[i * m + i];
  }
}
// x[r][i] += sum_{k < jd[sys]} Zs[k][r][i] y[sys][k]: only the columns the system's own Krylov space
// holds (the later columns of a finished instance were never written)
__global__ void k_bsolution_update(int64_t n, int nrhs, int nk, const double* __restrict__ Zs,
                                   const double* __restrict__ y, int ldy, const int* __restrict__ row_inst,
                                   const int* __restrict__ jd, double* __restrict__ x) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * nrhs) return;
  const int r = (int)(t / n);
  const int64_t i = t - (int64_t)r * n;
  const int sys = row_inst[i] * nrhs + r;
  const double* ys = y + (int64_t)sys * ldy;
  const int kk = min(nk, jd[sys]);
  double s = x[t];
  for (int k = 0; k < kk; ++k) s = fma(Zs[((int64_t)k * nrhs + r) * n + i], ys[k], s);
  x[t] = s;
}
// start of a cycle for the live systems: v0 = r / beta with inv = k_brsqrt(beta^2)
__global__ void k_bcycle_start(int64_t n, int nrhs, const int* __restrict__ row_inst, const double* __restrict__ inv,
                               const double* __restrict__ r, double* __restrict__ v0) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * nrhs) return;
  const int rr = (int)(t / n);
  const int64_t i = t - (int64_t)rr * n;
  v0[t] = r[t] * inv[row_inst[i] * nrhs + rr];
}
__global__ void k_bgvec(int nsys, int m, const double* __restrict__ nrm2, double* __restrict__ g, int* __restrict__ jd) {
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= nsys) return;
  g[(int64_t)sys * (m + 1)] = sqrt(nrm2[sys]);
  for (int k = 1; k <= m; ++k) g[(int64_t)sys * (m + 1) + k] = 0.0;
  jd[sys] = 0;
}
// live[q] = some system of instance q is still iterating
__global__ void k_binst_live(int ni, int nrhs, const int* __restrict__ done, int* __restrict__ live) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ni) return;
  int a = 0;
  for (int r = 0; r < nrhs; ++r) a |= done[q * nrhs + r] == 0;
  live[q] = a;
}
__global__ void k_bsub(int64_t n, const double* __restrict__ a, double* __restrict__ b) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i] - b[i];
}

// instance-aligned row chunks of the fine level and the row -> instance map
static int batch_tables(amgc_hierarchy* h) {
  if (h->b_nchunk > 0) return AMGC_OK;
  const Level& L = h->L[0];
  const int ni = h->n_inst;
  const int n = L.rows(), nu = L.nu();
  std::vector<int> r0, r1, cptr(ni + 1, 0), inst(n, 0);
  auto add = [&](int a, int b, int q) {
    for (int s = a; s < b; s += kBChunk) {
      r0.push_back(s);
      r1.push_back(std::min(b, s + kBChunk));
    }
    for (int i = a; i < b; ++i) inst[i] = q;
  };
  for (int q = 0; q < ni; ++q) {
    cptr[q] = (int)r0.size();
    add(3 * L.nptr[q], 3 * L.nptr[q + 1], q);
    add(nu + 3 * L.lptr[q], nu + 3 * L.lptr[q + 1], q);
  }
  cptr[ni] = (int)r0.size();
  const int nc = (int)r0.size();
  AMGC_TRY(h->b_chunk_row0.alloc(nc));
  AMGC_TRY(h->b_chunk_row1.alloc(nc));
  AMGC_TRY(h->b_chunk_ptr.alloc(ni + 1));
  AMGC_TRY(h->b_chunk_inst.alloc(nc));
  AMGC_TRY(h->b_row_inst.alloc(n));
  std::vector<int> cinst(nc, 0);
  for (int q = 0; q < ni; ++q)
    for (int c = cptr[q]; c < cptr[q + 1]; ++c) cinst[c] = q;
  cudaStream_t s = h->stream;
  AMGC_CUDA_TRY(cudaMemcpyAsync(h->b_chunk_row0.p, r0.data(), nc * sizeof(int), cudaMemcpyHostToDevice, s));
  AMGC_CUDA_TRY(cudaMemcpyAsync(h->b_chunk_row1.p, r1.data(), nc * sizeof(int), cudaMemcpyHostToDevice, s));
  AMGC_CUDA_TRY(cudaMemcpyAsync(h->b_chunk_ptr.p, cptr.data(), (ni + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  AMGC_CUDA_TRY(cudaMemcpyAsync(h->b_row_inst.p, inst.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
  AMGC_CUDA_TRY(cudaMemcpyAsync(h->b_chunk_inst.p, cinst.data(), nc * sizeof(int), cudaMemcpyHostToDevice, s));
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  h->b_nchunk = nc;
  return AMGC_OK;
}

int fgmres_batched(amgc_hierarchy* h, int nrhs, const double* rhs, double* x, int* iters_out, double* relres_out) {
  cudaStream_t s = h->stream;
  AMGC_TRY(batch_tables(h));
  const int64_t n = h->L[0].rows();
  const int ni = h->n_inst;
  const int nsys = ni * nrhs;
  const int m = std::max(1, std::min(h->opts.fgmres_restart, 256));
  const int maxit = std::max(1, h->opts.fgmres_maxit);
  const double tol = h->opts.tol;
  const int nc = h->b_nchunk;
  const int64_t nv = n * nrhs;
  const int th = 256;
  const int gv = div_up(nv, th);
  const int gs = div_up(nsys, 128);
  DBuf<double> V, Zs, H, cs, sn, g, y, hk, part, nrm2, beta0, rv, rinv;
  DBuf<int> done, jd, it, cnt, ilive;
  AMGC_TRY(V.alloc((size_t)(m + 1) * nv));
  AMGC_TRY(Zs.alloc((size_t)m * nv));
  AMGC_TRY(H.alloc((size_t)nsys * (m + 1) * m));
  AMGC_TRY(cs.alloc((size_t)nsys * m));
  AMGC_TRY(sn.alloc((size_t)nsys * m));
  AMGC_TRY(g.alloc((size_t)nsys * (m + 1)));
  AMGC_TRY(y.alloc((size_t)nsys * (m + 1)));
  AMGC_TRY(hk.alloc((size_t)nsys * (m + 1)));
  AMGC_TRY(part.alloc((size_t)(m + 1) * nrhs * nc));
  AMGC_TRY(nrm2.alloc(nsys));
  AMGC_TRY(rinv.alloc(nsys));
  AMGC_TRY(beta0.alloc(nsys));
  AMGC_TRY(rv.alloc(nv));
  AMGC_TRY(done.alloc(nsys));
  AMGC_TRY(jd.alloc(nsys));
  AMGC_TRY(it.alloc(nsys));
  AMGC_TRY(cnt.alloc(2));
  AMGC_TRY(ilive.alloc(ni));
  const int* ri = h->b_row_inst.p;
  // segmented squared norms of the nrhs columns of a -> out[sys]
  // lv: the instance flags (rows of finished instances skipped), or null for every row
  auto segnorm2 = [&](const double* a, double* out, const int* lv) -> int {
    AMGC_LAUNCH(k_bmultidot<<<dim3(nc, nrhs), kBThreads, 0, s>>>(nc, h->b_chunk_row0.p, h->b_chunk_row1.p, nrhs, n, 1,
                                                                 a, a, part.p, h->b_chunk_inst.p, lv));
    AMGC_LAUNCH(k_bmultidot_final<<<div_up((int64_t)nsys * 32, 128), 128, 0, s>>>(
        1, ni, nrhs, nc, h->b_chunk_ptr.p, part.p, out, 1, 0, 0, nullptr, 0));
    AMGC_CUDA_TRY(cudaGetLastError());
    return AMGC_OK;
  };
  // groups of kMcCols right-hand sides go through the multi-column cycle and operator apply (each
  // matrix block read once per group), the rest one column at a time
  auto apply_cols = [&](bool precond, const double* in, double* out, const int* lv) -> int {
    int r = 0;
    for (; r + kMcCols <= nrhs; r += kMcCols) {
      if (precond) AMGC_TRY(precond_apply_cols(h, in + r * n, out + r * n, lv));
      else AMGC_TRY(saddle_apply_cols(h, in + r * n, out + r * n, lv));
    }
    for (; r < nrhs; ++r) {
      if (precond) AMGC_TRY(precond_apply(h, in + r * n, out + r * n));
      else AMGC_TRY(saddle_apply(h, 0, in + r * n, out + r * n));
    }
    return AMGC_OK;
  };
  AMGC_CUDA_TRY(cudaMemsetAsync(x, 0, nv * sizeof(double), s));
  AMGC_CUDA_TRY(cudaMemsetAsync(it.p, 0, nsys * sizeof(int), s));
  AMGC_TRY(segnorm2(rhs, nrm2.p, nullptr));
  std::vector<double> hb(nsys);
  AMGC_CUDA_TRY(cudaMemcpyAsync(hb.data(), nrm2.p, nsys * sizeof(double), cudaMemcpyDeviceToHost, s));
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<int> hdone(nsys, 0);
  for (int q = 0; q < nsys; ++q) {
    hb[q] = std::sqrt(hb[q]);
    if (!std::isfinite(hb[q])) {
      set_error("fgmres_batched: non-finite right-hand side");
      return AMGC_BREAKDOWN;
    }
    if (hb[q] == 0.0) hdone[q] = 1;
  }
  AMGC_CUDA_TRY(cudaMemcpyAsync(beta0.p, hb.data(), nsys * sizeof(double), cudaMemcpyHostToDevice, s));
  AMGC_CUDA_TRY(cudaMemcpyAsync(done.p, hdone.data(), nsys * sizeof(int), cudaMemcpyHostToDevice, s));
  AMGC_LAUNCH(k_binst_live<<<div_up(ni, 128), 128, 0, s>>>(ni, nrhs, done.p, ilive.p));
  AMGC_CUDA_TRY(cudaMemcpyAsync(rv.p, rhs, nv * sizeof(double), cudaMemcpyDeviceToDevice, s));
  int total = 0, live = 0;
  for (int q = 0; q < nsys; ++q) live += hdone[q] == 0;
  while (total < maxit && live > 0) {
    // cycle start on the current residual rv
    AMGC_TRY(segnorm2(rv.p, nrm2.p, nullptr));
    AMGC_LAUNCH(k_brsqrt<<<gs, 128, 0, s>>>(nsys, nrm2.p, rinv.p));
    AMGC_LAUNCH(k_bcycle_start<<<gv, th, 0, s>>>(n, nrhs, ri, rinv.p, rv.p, V.p));
    AMGC_LAUNCH(k_bgvec<<<gs, 128, 0, s>>>(nsys, m, nrm2.p, g.p, jd.p));
    AMGC_CUDA_TRY(cudaMemsetAsync(H.p, 0, (size_t)nsys * (m + 1) * m * sizeof(double), s));
    int jmax = 0;
    for (int j = 0; j < m && total < maxit; ++j) {
      double* vj = V.p + (int64_t)j * nv;
      double* zj = Zs.p + (int64_t)j * nv;
      double* w = V.p + (int64_t)(j + 1) * nv;
      AMGC_TRY(apply_cols(true, vj, zj, ilive.p));
      AMGC_TRY(apply_cols(false, zj, w, ilive.p));
      for (int pass = 0; pass < 2; ++pass) {
        AMGC_LAUNCH(k_bmultidot<<<dim3(nc, nrhs), kBThreads, 0, s>>>(nc, h->b_chunk_row0.p, h->b_chunk_row1.p, nrhs, n,
                                                                     j + 1, V.p, w, part.p, h->b_chunk_inst.p, ilive.p));
        AMGC_LAUNCH(k_bmultidot_final<<<div_up((int64_t)(j + 1) * nsys * 32, 128), 128, 0, s>>>(
            j + 1, ni, nrhs, nc, h->b_chunk_ptr.p, part.p, H.p + j, (int64_t)(m + 1) * m, m, pass, hk.p, m + 1));
        AMGC_LAUNCH(k_bbasis_update<<<gv, th, 0, s>>>(n, nrhs, j + 1, V.p, hk.p, m + 1, ri, w, ilive.p));
      }
      AMGC_TRY(segnorm2(w, nrm2.p, ilive.p));
      AMGC_LAUNCH(k_bsubdiag<<<gs, 128, 0, s>>>(nsys, j, m, nrm2.p, H.p));
      AMGC_LAUNCH(k_brsqrt<<<gs, 128, 0, s>>>(nsys, nrm2.p, rinv.p));
      AMGC_LAUNCH(k_bnormalize<<<gv, th, 0, s>>>(n, nrhs, ri, rinv.p, w, w, ilive.p));
      ++total;
      AMGC_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, 2 * sizeof(int), s));
      AMGC_LAUNCH(k_bgivens<<<gs, 128, 0, s>>>(nsys, j, m, H.p, cs.p, sn.p, g.p, beta0.p, done.p, jd.p, it.p, total,
                                               tol, cnt.p, cnt.p + 1));
      AMGC_LAUNCH(k_binst_live<<<div_up(ni, 128), 128, 0, s>>>(ni, nrhs, done.p, ilive.p));
      AMGC_CUDA_TRY(cudaGetLastError());
      int hc[2] = {0, 0};
      AMGC_CUDA_TRY(cudaMemcpyAsync(hc, cnt.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
      AMGC_CUDA_TRY(cudaStreamSynchronize(s));
      jmax = j + 1;
      if (hc[1] > 0) {
        set_error("fgmres_batched: non-finite Hessenberg entry");
        return AMGC_BREAKDOWN;
      }
      live = hc[0];
      if (live == 0) break;
    }
    AMGC_LAUNCH(k_bbacksolve<<<gs, 128, 0, s>>>(nsys, m, H.p, g.p, jd.p, y.p));
    AMGC_LAUNCH(k_bsolution_update<<<gv, th, 0, s>>>(n, nrhs, jmax, Zs.p, y.p, m + 1, ri, jd.p, x));
    AMGC_TRY(apply_cols(false, x, rv.p, nullptr));   // every system's true residual
    AMGC_LAUNCH(k_bsub<<<gv, th, 0, s>>>(nv, rhs, rv.p));
    AMGC_CUDA_TRY(cudaGetLastError());
  }
  // true relative residuals per system
  AMGC_TRY(segnorm2(rv.p, nrm2.p, nullptr));
  std::vector<double> hr(nsys);
  std::vector<int> hi(nsys), hd(nsys);
  AMGC_CUDA_TRY(cudaMemcpyAsync(hr.data(), nrm2.p, nsys * sizeof(double), cudaMemcpyDeviceToHost, s));
  AMGC_CUDA_TRY(cudaMemcpyAsync(hi.data(), it.p, nsys * sizeof(int), cudaMemcpyDeviceToHost, s));
  AMGC_CUDA_TRY(cudaMemcpyAsync(hd.data(), done.p, nsys * sizeof(int), cudaMemcpyDeviceToHost, s));
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  bool all = true;
  for (int q = 0; q < nsys; ++q) {
    const double rr = hb[q] > 0.0 ? std::sqrt(hr[q]) / hb[q] : 0.0;
    if (relres_out) relres_out[q] = rr;
    if (iters_out) iters_out[q] = hi[q];
    if (!std::isfinite(rr)) {
      set_error("fgmres_batched: non-finite residual");
      return AMGC_BREAKDOWN;
    }
    all = all && hd[q];
  }
  h->stats.last_iters = total;
  if (h->opts.precision == 32) AMGC_TRY(check_status(h, "fgmres_batched"));   // bounded waits of the FP32 cycle
  if (!all) {
    set_error("fgmres_batched: iteration limit reached for some systems");
    return AMGC_NOT_CONVERGED;
  }
  return AMGC_OK;
}

}  // namespace amgc
