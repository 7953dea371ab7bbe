// Set-up data of the block smoothers of Sec. 5.1 besides CheapSIMPLE, in the cheap forms of
// Sec. 5.2 that the paper's experiments use (Sec. 6.1): damped symmetric Gauss-Seidel sweeps for
// the K block and an incomplete LU factorisation without fill (ILU(0)) of the assembled Schur
// approximation.
//
//  * SGS is taken over the nodal bu x bu blocks of K in the order of a Jones-Plassmann colouring of
//    K's node graph (colours ascending, then descending): the nodes of one colour do not couple,
//    so each colour is one data-parallel step.  Priorities are the MIS-2 keys
//    fmix32(i ^ seed) * 2^32 + i; in every round an uncoloured node whose key exceeds that of each
//    uncoloured neighbour takes the smallest colour none of its coloured neighbours has (the
//    picked nodes are pairwise non-adjacent, so the colours they read do not change in the round).
//  * The Schur approximation Z + s B2 A~^-1 B1 (s = 1, or 1/omega for Braess-Sarazin) is assembled
//    on the nodal 3x3 blocks of the multipliers; ILU(0) eliminates row by row on that block pattern
//    (A_ik <- A_ik A_kk^-1, A_ij <- A_ij - A_ik A_kj for the blocks of the pattern), the rows of one
//    dependency level at a time, and keeps the inverted diagonal blocks of U for the solves.
#include "amgc_internal.cuh"

#include <algorithm>
#include <cmath>

namespace amgc {

// ------------------------------------------------------------------ Jones-Plassmann colouring
__device__ __forceinline__ unsigned long long jp_key(int i, uint32_t seed) {
  return ((unsigned long long)fmix32((uint32_t)i ^ seed) << 32) | (unsigned long long)(uint32_t)i;
}

__global__ void k_jp_pick(int n, const int* __restrict__ rp, const int* __restrict__ col, uint32_t seed,
                          const int* __restrict__ color, uint8_t* __restrict__ pick) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (color[i] >= 0) {
    pick[i] = 0;
    return;
  }
  const unsigned long long ki = jp_key(i, seed);
  for (int q = rp[i]; q < rp[i + 1]; ++q) {
    const int j = col[q];
    if (j != i && color[j] < 0 && jp_key(j, seed) > ki) {
      pick[i] = 0;
      return;
    }
  }
  pick[i] = 1;
}

// picked node: the smallest colour absent among its coloured neighbours (a bit set of the first 256
// colours, a search beyond them); counts the nodes still uncoloured afterwards
__global__ void k_jp_assign(int n, const int* __restrict__ rp, const int* __restrict__ col,
                            const uint8_t* __restrict__ pick, int* __restrict__ color, int* __restrict__ left) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (!pick[i]) {
    if (color[i] < 0) atomicAdd(left, 1);
    return;
  }
  unsigned used[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  for (int q = rp[i]; q < rp[i + 1]; ++q) {
    const int j = col[q];
    const int c = j != i ? color[j] : -1;
    if (c >= 0 && c < 256) used[c >> 5] |= 1u << (c & 31);
  }
  int c = -1;
  for (int w = 0; w < 8 && c < 0; ++w)
    if (used[w] != 0xffffffffu) c = 32 * w + __ffs(~used[w]) - 1;
  if (c < 0) {   // all of the first 256 colours taken
    for (c = 256;; ++c) {
      bool taken = false;
      for (int q = rp[i]; q < rp[i + 1] && !taken; ++q) taken = col[q] != i && color[col[q]] == c;
      if (!taken) break;
    }
  }
  color[i] = c;
}

static int jp_coloring(amgc_hierarchy* h, Level& L) {
  cudaStream_t s = h->stream;
  const int n = L.nn;
  DBuf<uint8_t> pick;
  DBuf<int> left;
  AMGC_TRY(L.color.alloc(n));
  AMGC_TRY(pick.alloc(n));
  AMGC_TRY(left.alloc(1));
  AMGC_CUDA_TRY(cudaMemsetAsync(L.color.p, 0xff, (size_t)n * sizeof(int), s));   // -1: uncoloured
  int remaining = n;
  for (int round = 0; remaining > 0; ++round) {
    if (round > n) {
      set_error("colouring: no progress");
      return AMGC_EINVAL;
    }
    AMGC_LAUNCH(k_jp_pick<<<div_up(n, 256), 256, 0, s>>>(n, L.K.rowptr.p, L.K.col.p, h->opts.seed, L.color.p, pick.p));
    AMGC_CUDA_TRY(cudaMemsetAsync(left.p, 0, sizeof(int), s));
    AMGC_LAUNCH(k_jp_assign<<<div_up(n, 256), 256, 0, s>>>(n, L.K.rowptr.p, L.K.col.p, pick.p, L.color.p, left.p));
    AMGC_CUDA_TRY(cudaGetLastError());
    AMGC_CUDA_TRY(cudaMemcpyAsync(&remaining, left.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  }
  // number of colours, then the node lists per colour
  std::vector<int> hc(n);
  AMGC_CUDA_TRY(cudaMemcpyAsync(hc.data(), L.color.p, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, s));
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  L.ncolor = n ? 1 + *std::max_element(hc.begin(), hc.end()) : 0;
  AMGC_TRY(bucket_lists(n, L.color.p, L.ncolor, L.col_ptr, L.col_nodes, s));
  L.h_col_ptr.assign(L.ncolor + 1, 0);
  AMGC_CUDA_TRY(cudaMemcpyAsync(L.h_col_ptr.data(), L.col_ptr.p, (L.ncolor + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  return AMGC_OK;
}

// ------------------------------------------------------------------ small dense inverses
// in-place inverse of an n x n row-major block (n <= 6) by Gauss-Jordan with partial pivoting;
// false for a zero pivot
template <int N>
__device__ bool invert_small(double* a) {
  double m[N][2 * N];
  for (int r = 0; r < N; ++r)
    for (int c = 0; c < 2 * N; ++c) m[r][c] = c < N ? a[r * N + c] : (c - N == r ? 1.0 : 0.0);
  for (int k = 0; k < N; ++k) {
    int p = k;
    for (int r = k + 1; r < N; ++r)
      if (fabs(m[r][k]) > fabs(m[p][k])) p = r;
    if (m[p][k] == 0.0) return false;
    if (p != k)
      for (int c = 0; c < 2 * N; ++c) {
        const double t = m[k][c];
        m[k][c] = m[p][c];
        m[p][c] = t;
      }
    const double inv = 1.0 / m[k][k];
    for (int c = 0; c < 2 * N; ++c) m[k][c] *= inv;
    for (int r = 0; r < N; ++r) {
      if (r == k) continue;
      const double f = m[r][k];
      if (f != 0.0)
        for (int c = 0; c < 2 * N; ++c) m[r][c] -= f * m[k][c];
    }
  }
  for (int r = 0; r < N; ++r)
    for (int c = 0; c < N; ++c) a[r * N + c] = m[r][N + c];
  return true;
}

// inverted diagonal block of every block row of K
template <int BU>
__global__ void k_dblk_inv(int nn, const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
                           double* __restrict__ out, int* st) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  int lo = rp[i], hi = rp[i + 1] - 1, pos = -1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    if (col[mid] == i) {
      pos = mid;
      break;
    }
    if (col[mid] < i) lo = mid + 1;
    else hi = mid - 1;
  }
  double a[BU * BU];
  if (pos < 0) {
    atomicOr(st, ST_NO_DIAG);
    return;
  }
  for (int t = 0; t < BU * BU; ++t) a[t] = val[(int64_t)pos * BU * BU + t];
  if (!invert_small<BU>(a)) atomicOr(st, ST_SINGULAR);
  for (int t = 0; t < BU * BU; ++t) out[(int64_t)i * BU * BU + t] = a[t];
}

// ------------------------------------------------------------------ Schur approximation
// B1s = s A~^-1 B1 (row scaling of B1's BU x 3 blocks)
template <int BU>
__global__ void k_scale_b1(int nn, const int* __restrict__ rp, const double* __restrict__ val,
                           const double* __restrict__ atinv, double sc, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  for (int e = rp[i]; e < rp[i + 1]; ++e)
    for (int r = 0; r < BU; ++r) {
      const double a = sc * atinv[(int64_t)i * BU + r];
      for (int c = 0; c < 3; ++c) out[((int64_t)e * BU + r) * 3 + c] = a * val[((int64_t)e * BU + r) * 3 + c];
    }
}
__global__ void k_sdiag_count(int nl, const int* __restrict__ rp, const int* __restrict__ col, int* __restrict__ cnt) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nl) return;
  int has = 0;
  for (int e = rp[l]; e < rp[l + 1]; ++e) has |= col[e] == l;
  cnt[l] = rp[l + 1] - rp[l] + (has ? 0 : 1);
}
// S row l = the product row with Z_l added on the diagonal block (inserted in column order if the
// product has none there); diag[l] = its position
__global__ void k_sdiag_fill(int nl, const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
                             const double* __restrict__ Z, const int* __restrict__ srp, int* __restrict__ scol,
                             double* __restrict__ sval, int* __restrict__ diag) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nl) return;
  int o = srp[l];
  bool placed = false;
  auto put_diag = [&](const double* add) {
    scol[o] = l;
    for (int t = 0; t < 9; ++t) sval[(int64_t)o * 9 + t] = (add ? add[t] : 0.0) + Z[(int64_t)l * 9 + t];
    diag[l] = o;
    ++o;
    placed = true;
  };
  for (int e = rp[l]; e < rp[l + 1]; ++e) {
    const int c = col[e];
    if (!placed && c > l) put_diag(nullptr);
    if (c == l) {
      put_diag(val + (int64_t)e * 9);
      continue;
    }
    scol[o] = c;
    for (int t = 0; t < 9; ++t) sval[(int64_t)o * 9 + t] = val[(int64_t)e * 9 + t];
    ++o;
  }
  if (!placed) put_diag(nullptr);
}

// ------------------------------------------------------------------ block ILU(0)
// dependency levels of the forward (L) and backward (U) block substitutions, one thread: the level
// of a row is one more than the largest level of the rows it reads
__global__ void k_ilu_levels(int n, const int* __restrict__ rp, const int* __restrict__ col, int* __restrict__ lev_l,
                             int* __restrict__ lev_u, int* __restrict__ nlev) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int ml = 0, mu = 0;
  for (int i = 0; i < n; ++i) {
    int v = 0;
    for (int e = rp[i]; e < rp[i + 1] && col[e] < i; ++e) v = max(v, lev_l[col[e]] + 1);
    lev_l[i] = v;
    ml = max(ml, v);
  }
  for (int i = n - 1; i >= 0; --i) {
    int v = 0;
    for (int e = rp[i + 1] - 1; e >= rp[i] && col[e] > i; --e) v = max(v, lev_u[col[e]] + 1);
    lev_u[i] = v;
    mu = max(mu, v);
  }
  nlev[0] = n ? ml + 1 : 0;
  nlev[1] = n ? mu + 1 : 0;
}

__device__ __forceinline__ void mul33(const double* a, const double* b, double* c) {
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) c[r * 3 + q] = a[r * 3] * b[q] + a[r * 3 + 1] * b[3 + q] + a[r * 3 + 2] * b[6 + q];
}

// factorises the rows of one level (one thread per row), in place: the blocks left of the
// diagonal become L (unit diagonal implied), the others U; uinv receives the inverse of U_ii
__global__ void k_ilu_rows(int cnt, const int* __restrict__ rows, const int* __restrict__ rp, const int* __restrict__ col,
                           double* __restrict__ val, const int* __restrict__ diag, double* __restrict__ uinv, int* st) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int i = rows[t];
  const int e0 = rp[i], e1 = rp[i + 1];
  for (int p = e0; p < e1 && col[p] < i; ++p) {
    const int k = col[p];
    double a[9], m[9];
    for (int q = 0; q < 9; ++q) a[q] = val[(int64_t)p * 9 + q];
    mul33(a, uinv + (int64_t)k * 9, m);                       // A_ik <- A_ik U_kk^-1
    for (int q = 0; q < 9; ++q) val[(int64_t)p * 9 + q] = m[q];
    // A_ij -= A_ik A_kj for the blocks j > k of row k that row i has
    int pi = p + 1;
    for (int pk = diag[k] + 1; pk < rp[k + 1]; ++pk) {
      const int j = col[pk];
      while (pi < e1 && col[pi] < j) ++pi;
      if (pi == e1) break;
      if (col[pi] != j) continue;
      double d[9];
      mul33(m, val + (int64_t)pk * 9, d);
      for (int q = 0; q < 9; ++q) val[(int64_t)pi * 9 + q] -= d[q];
    }
  }
  double u[9];
  for (int q = 0; q < 9; ++q) u[q] = val[(int64_t)diag[i] * 9 + q];
  if (!invert_small<3>(u)) atomicOr(st, ST_SINGULAR);
  for (int q = 0; q < 9; ++q) uinv[(int64_t)i * 9 + q] = u[q];
}

// Schur approximation of level L (scale s on the B2 A~^-1 B1 term), factored by block ILU(0)
static int schur_ilu_setup(amgc_hierarchy* h, Level& L, double sc) {
  cudaStream_t s = h->stream;
  const int nl = L.nl;
  // B2 (s A~^-1 B1)
  DBsr B1s, P;
  B1s.nbr = L.B1.nbr; B1s.nbc = L.B1.nbc; B1s.br = L.B1.br; B1s.bc = L.B1.bc; B1s.nnzb = L.B1.nnzb;
  AMGC_TRY(B1s.rowptr.alloc(L.B1.nbr + 1));
  AMGC_TRY(B1s.col.alloc(std::max<int64_t>(L.B1.nnzb, 1)));
  AMGC_TRY(B1s.val.alloc((size_t)std::max<int64_t>(L.B1.nnzb, 1) * L.bu * 3));
  AMGC_CUDA_TRY(cudaMemcpyAsync(B1s.rowptr.p, L.B1.rowptr.p, (L.B1.nbr + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s));
  if (L.B1.nnzb > 0)
    AMGC_CUDA_TRY(cudaMemcpyAsync(B1s.col.p, L.B1.col.p, L.B1.nnzb * sizeof(int), cudaMemcpyDeviceToDevice, s));
  if (L.bu == 3)
    AMGC_LAUNCH(k_scale_b1<3><<<div_up(L.nn, 256), 256, 0, s>>>(L.nn, L.B1.rowptr.p, L.B1.val.p, L.atinv.p, sc, B1s.val.p));
  else
    AMGC_LAUNCH(k_scale_b1<6><<<div_up(L.nn, 256), 256, 0, s>>>(L.nn, L.B1.rowptr.p, L.B1.val.p, L.atinv.p, sc, B1s.val.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  AMGC_TRY(spgemm(h, L.B2, B1s, P));
  // + Z on the diagonal blocks
  DBsr& S = L.S;
  S.nbr = nl; S.nbc = nl; S.br = 3; S.bc = 3;
  AMGC_TRY(S.rowptr.alloc(nl + 1));
  AMGC_CUDA_TRY(cudaMemsetAsync(S.rowptr.p, 0, (nl + 1) * sizeof(int), s));
  AMGC_LAUNCH(k_sdiag_count<<<div_up(nl, 256), 256, 0, s>>>(nl, P.rowptr.p, P.col.p, S.rowptr.p));
  int nnzb = 0;
  AMGC_TRY(exclusive_scan(S.rowptr.p, S.rowptr.p, nl + 1, s, &nnzb));
  S.nnzb = nnzb;
  AMGC_TRY(S.col.alloc(nnzb));
  AMGC_TRY(S.val.alloc((size_t)nnzb * 9));
  AMGC_TRY(L.s_diag.alloc(nl));
  AMGC_LAUNCH(k_sdiag_fill<<<div_up(nl, 256), 256, 0, s>>>(nl, P.rowptr.p, P.col.p, P.val.p, L.Z.p, S.rowptr.p, S.col.p,
                                                          S.val.p, L.s_diag.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  // level schedules of the substitutions (the factorisation follows the forward one)
  DBuf<int> lev_l, lev_u, nlev;
  AMGC_TRY(lev_l.alloc(nl));
  AMGC_TRY(lev_u.alloc(nl));
  AMGC_TRY(nlev.alloc(2));
  AMGC_LAUNCH(k_ilu_levels<<<1, 1, 0, s>>>(nl, S.rowptr.p, S.col.p, lev_l.p, lev_u.p, nlev.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  int hn[2] = {0, 0};
  AMGC_CUDA_TRY(cudaMemcpyAsync(hn, nlev.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  L.s_nlev_l = hn[0];
  L.s_nlev_u = hn[1];
  AMGC_TRY(bucket_lists(nl, lev_l.p, hn[0], L.s_lptr, L.s_lrows, s));
  AMGC_TRY(bucket_lists(nl, lev_u.p, hn[1], L.s_uptr, L.s_urows, s));
  std::vector<int> lp(hn[0] + 1);
  AMGC_CUDA_TRY(cudaMemcpyAsync(lp.data(), L.s_lptr.p, (hn[0] + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  AMGC_TRY(L.s_uinv.alloc((size_t)nl * 9));
  for (int v = 0; v < hn[0]; ++v) {
    const int cnt = lp[v + 1] - lp[v];
    AMGC_LAUNCH(k_ilu_rows<<<div_up(cnt, 64), 64, 0, s>>>(cnt, L.s_lrows.p + lp[v], S.rowptr.p, S.col.p, S.val.p,
                                                          L.s_diag.p, L.s_uinv.p, h->status.p));
  }
  AMGC_CUDA_TRY(cudaGetLastError());
  return check_status(h, "block smoother: ILU(0) of the Schur approximation");
}

int block_smoother_setup(amgc_hierarchy* h, bool schur_only) {
  cudaStream_t s = h->stream;
  const int kind = h->smoother_kind;
  const int nlev = (int)h->L.size();
  const bool coarse_smooth = h->opts.coarse_solver == 1 && nlev > 1;
  const double sc = kind == 2 ? 1.0 / h->block_omega : 1.0;
  for (int l = 0; l < nlev; ++l) {
    Level& L = h->L[l];
    if (!(l + 1 < nlev || coarse_smooth)) continue;
    if (!schur_only) {
      if (kind == 1 || kind == 3) {
        AMGC_TRY(jp_coloring(h, L));
        AMGC_TRY(L.kdblk_inv.alloc((size_t)L.nn * L.bu * L.bu));
        if (L.bu == 3)
          AMGC_LAUNCH(k_dblk_inv<3><<<div_up(L.nn, 128), 128, 0, s>>>(L.nn, L.K.rowptr.p, L.K.col.p, L.K.val.p,
                                                                      L.kdblk_inv.p, h->status.p));
        else
          AMGC_LAUNCH(k_dblk_inv<6><<<div_up(L.nn, 128), 128, 0, s>>>(L.nn, L.K.rowptr.p, L.K.col.p, L.K.val.p,
                                                                      L.kdblk_inv.p, h->status.p));
        AMGC_CUDA_TRY(cudaGetLastError());
        AMGC_TRY(check_status(h, "block smoother: diagonal blocks of K"));
      }
      AMGC_TRY(L.bs_w.alloc(std::max(L.nu(), 1)));
      AMGC_TRY(L.bs_d.alloc(std::max(L.nu(), 1)));
      AMGC_TRY(L.bs_l.alloc(std::max(3 * L.nl, 1)));
      AMGC_TRY(L.bs_m.alloc(std::max(3 * L.nl, 1)));
    }
    if (L.nl > 0) AMGC_TRY(schur_ilu_setup(h, L, sc));
  }
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  return AMGC_OK;
}

}  // namespace amgc
